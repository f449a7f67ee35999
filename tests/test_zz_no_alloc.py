"""The allocation-free product rpb_mobility_apply_noalloc, called through the C ABI.

Some callers cannot call cudaMalloc (a host that owns all device memory through its own pool, or
code where an allocation's device-wide synchronisation is not allowed), so they cannot create a
context.  This entry point keeps its scratch in a fixed array inside the library instead.  Its
results must agree with the context-based rpb_mobility_apply within the parity tolerances used
elsewhere (1e-10 in float64, 1e-5 in float32), on consecutive calls that reuse the array's stale
contents.  Collected last on purpose; it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

from paper_1612_00474_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.tensor(inputs.to_soa(x), dtype=torch.float64, device="cuda")


def _maxrel(x, ref):
    return float((x - ref).abs().max() / ref.abs().max())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_noalloc_matches_context_product_twice(gpu_lib, precision, tol):
    ctx = gpu_lib.Context(max_N=gpu_lib.NOALLOC_MAX_N, precision=precision, max_iter=8)
    try:
        # call 1: 3000 spheres with forces and torques; call 2: 1000 spheres, forces only, so the
        # second call runs on the array left behind by the first
        for N, seed, with_T in ((3000, 1, True), (1000, 2, False)):
            pos = _dev(inputs.monolayer(N, seed=seed))
            F = _dev(inputs.vectors(N, seed))
            T = _dev(inputs.vectors(N, seed + 50)) if with_T else None
            ref = ctx.mobility_apply(pos, F, T)
            out = torch.full_like(ref, float("nan"))
            got = gpu_lib.mobility_apply_noalloc(pos, F, T, precision=precision, out=out)
            torch.cuda.synchronize()
            assert torch.isfinite(got).all()
            assert _maxrel(got, ref) <= tol
    finally:
        ctx.close()


def test_noalloc_largest_size_and_limit(gpu_lib):
    N = gpu_lib.NOALLOC_MAX_N
    pos = _dev(inputs.monolayer(N, seed=3))
    F = _dev(inputs.vectors(N, 3))
    ctx = gpu_lib.Context(max_N=N, precision="fp32", max_iter=8)
    try:
        ref = ctx.mobility_apply(pos, F, None)
        got = gpu_lib.mobility_apply_noalloc(pos, F, None, precision="fp32")
        assert _maxrel(got, ref) <= 1e-5
    finally:
        ctx.close()
    # one sphere more than the fixed scratch holds is refused with a clear message
    L = gpu_lib.load()
    big = torch.zeros(3 * (N + 1), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(big)
    p = gpu_lib.Params(1.0, 1.0, 1.0, gpu_lib.RPB_FP64)
    rc = L.rpb_mobility_apply_noalloc(N + 1, ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()), None,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.byref(p), None)
    assert rc == gpu_lib.RPB_EINVAL
    assert str(N) in gpu_lib.last_error()
    assert np.isfinite(out.cpu().numpy()).all()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_noalloc_against_oracle_and_null_loads(gpu_lib, precision, tol):
    """Its own error against the FP64 oracle (rather than against another GPU product) at a small N
    that spans tiles and a ragged tail, with forces and torques, torques only, and neither (zeros)."""
    import oracle as O

    N = 300
    pos = inputs.monolayer(N, seed=7)
    F = inputs.vectors(N, 7)
    T = inputs.vectors(N, 57)
    for f, t in ((F, T), (None, T)):
        got = gpu_lib.mobility_apply_noalloc(_dev(pos), None if f is None else _dev(f), _dev(t), precision=precision)
        torch.cuda.synchronize()
        ref = O.mobility_apply(pos, f, t)
        err = float(np.max(np.abs(inputs.from_soa(got.cpu().numpy(), N) - ref)) / np.max(np.abs(ref)))
        assert err <= tol, (precision, f is None, err)
    out = torch.full((3 * N,), float("nan"), dtype=torch.float64, device="cuda")
    gpu_lib.mobility_apply_noalloc(_dev(pos), None, None, precision=precision, out=out)
    torch.cuda.synchronize()
    assert bool((out == 0).all())
