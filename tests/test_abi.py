"""The C ABI: the library builds, loads without a GPU, and exports every function the header
declares; the binding's host-side helpers behave."""
import ctypes
import os
import re

import numpy as np

from paper_1612_00474_gb300 import build, inputs, rpb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rpb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rpb_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_binding_exports():
    assert sorted(rpb.EXPORTS) == _declared()


def test_library_loads_and_exports_every_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_soa_roundtrip():
    x = np.arange(12.0).reshape(4, 3)
    s = inputs.to_soa(x)
    assert np.array_equal(s[:4], x[:, 0]) and np.array_equal(s[8:], x[:, 2])
    assert np.array_equal(inputs.from_soa(s, 4), x)


def test_monolayer_generator_properties():
    p = inputs.monolayer(500, seed=1)
    L = np.sqrt(500 * np.pi / 0.4)
    assert p.shape == (500, 3) and p[:, :2].min() >= 0 and p[:, :2].max() <= L and p[:, 2].min() >= 1.0
    d = np.linalg.norm(p[:, None, :] - p[None, :, :], axis=-1) + 1e9 * np.eye(500)
    assert d.min() >= 2.0
    assert np.array_equal(p, inputs.monolayer(500, seed=1))
    sizes = inputs.batch_sizes(512)
    assert sizes.min() >= 64 and sizes.max() <= 2048


def test_error_codes_match_header():
    src = open(os.path.join(ROOT, "include", "rpb.h")).read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (RPB_(?:OK|E[A-Z]+)) (\d+)", src)}
    assert set(codes) == {"RPB_OK", "RPB_EINVAL", "RPB_ENOMEM", "RPB_ECUDA", "RPB_ENOCONV", "RPB_ETIMEOUT"}
    for name, value in codes.items():
        assert getattr(rpb, name) == value, name
