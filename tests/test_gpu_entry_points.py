"""Edge cases of the row-range product, the product hook, the two-right-hand-side product, the batch
tile schedule and the FMA-peak probe, through the C ABI.

  - rpb_mobility_apply_rows: every tile-aligned range of a ragged N (first, middle, last partial
    tile, the whole) equals the same rows of the full product (FP64 1e-12, FP32 1e-5 against the
    oracle); ranges that do not start on a tile or leave [0, N) are refused, and so is
    pseudo-periodic mode.
  - rpb_mobility_apply_part: the shares add up to the product (float32 symmetric shares, torque form,
    pseudo-periodic shares, float64 row shares; more shares than tile units, so that some are empty),
    share 0 of 1 is the product bit for bit, and out-of-range shares are refused.
  - rpb_set_product_hook: an error returned by the hook reaches the caller; the library's own
    products are restored by clearing the hook.
  - rpb_batch_set_tiles / rpb_batch_tune: values outside the documented ranges are refused; a float64
    batch has the one-way kernel as its only candidate.
  - rpb_fma_peak: an unknown kind is refused; the float32 rate exceeds the float64 one.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1612_00474_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.tensor(inputs.to_soa(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_rows_match_full_product(gpu_lib, precision, tol):
    N = 389  # three whole tiles and a ragged tail
    pos = inputs.monolayer(N, seed=9)
    F, T = inputs.vectors(N, 10), inputs.vectors(N, 11)
    ref = O.mobility_apply(pos, F, T)
    ctx = gpu_lib.Context(N, precision=precision, max_iter=8)
    try:
        full = inputs.from_soa(ctx.mobility_apply(dev(pos), dev(F), dev(T)).cpu().numpy(), N)
        for a, b in ((0, 128), (128, 256), (256, 389), (384, 389), (0, 389), (128, 300)):
            rows = ctx.mobility_apply_rows(dev(pos), dev(F), dev(T), a, b).cpu().numpy().reshape(3, b - a).T
            assert np.max(np.abs(rows - ref[a:b])) / np.max(np.abs(ref)) <= tol, (a, b)
            assert np.max(np.abs(rows - full[a:b])) / np.max(np.abs(full)) <= (1e-12 if precision == "fp64" else 2e-5)
        z = ctx.mobility_apply_rows(dev(pos), None, None, 0, 128)
        assert bool((z == 0).all())
        L = gpu_lib.load()
        P, Fd = dev(pos), dev(F)
        out = torch.empty(3 * N, dtype=torch.float64, device="cuda")
        vp = ctypes.c_void_p
        for a, b in ((1, 128), (0, 0), (0, N + 1), (-128, 0), (256, 128)):
            rc = L.rpb_mobility_apply_rows(ctx._h, N, vp(P.data_ptr()), vp(Fd.data_ptr()), None, a, b,
                                           vp(out.data_ptr()))
            assert rc == gpu_lib.RPB_EINVAL, (a, b)
        side = float(np.sqrt(N * np.pi / 0.4))
        ctx.set_periodic(side, side)
        with pytest.raises(gpu_lib.RpbError):
            ctx.mobility_apply_rows(dev(pos), dev(F), None, 0, 128)
    finally:
        ctx.close()


@pytest.mark.parametrize("precision,N,torque,periodic,nparts", [
    ("fp32", 1000, False, False, 2), ("fp32", 1000, False, False, 3), ("fp32", 1000, True, False, 7),
    ("fp32", 600, False, True, 3), ("fp32", 300, False, False, 50), ("fp64", 389, True, False, 3),
    ("fp64", 389, False, True, 2), ("fp32", 200, False, False, 2)])
def test_part_shares_sum_to_product(gpu_lib, precision, N, torque, periodic, nparts):
    pos = inputs.monolayer(N, seed=15)
    F, T = inputs.vectors(N, 16), (inputs.vectors(N, 17) if torque else None)
    side = float(np.sqrt(N * np.pi / 0.4))
    ref = O.mobility_apply(pos, F, T, periodic=(side, side) if periodic else None)
    ctx = gpu_lib.Context(N, precision=precision, max_iter=8)
    try:
        if periodic:
            ctx.set_periodic(side, side)
        P, Fd, Td = dev(pos), dev(F), (dev(T) if torque else None)
        full = ctx.mobility_apply(P, Fd, Td)
        one = ctx.mobility_apply_part(P, Fd, Td, 0, 1)
        assert torch.equal(one, full)
        shares = [ctx.mobility_apply_part(P, Fd, Td, p, nparts) for p in range(nparts)]
        total = torch.stack(shares).sum(0)
        got = inputs.from_soa(total.cpu().numpy(), N)
        full_h = inputs.from_soa(full.cpu().numpy(), N)
        tol = 1e-10 if precision == "fp64" else 1e-5
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= tol
        assert np.max(np.abs(got - full_h)) / np.max(np.abs(full_h)) <= (1e-12 if precision == "fp64" else 2e-6)
        if precision == "fp32" and N >= 256:  # symmetric shares: pairs of their units, both directions
            nb = -(-N // 128)
            units = [(b, t) for b in range(nb) for t in range(b, nb)]
            for p in range(nparts):
                mine = units[len(units) * p // nparts:len(units) * (p + 1) // nparts]
                tiles = {b for b, _ in mine} | {t for _, t in mine}
                want = {i for t in tiles for i in range(128 * t, min(N, 128 * (t + 1)))}
                sp = inputs.from_soa(shares[p].cpu().numpy(), N)
                have = set(np.flatnonzero(np.abs(sp).sum(1)).tolist())
                if p != 0:  # share 0 also holds every sphere's self term
                    assert have == want, (p, len(have), len(want))
        assert bool((ctx.mobility_apply_part(P, None, None, 0, nparts) == 0).all())
        L = gpu_lib.load()
        out = torch.empty(3 * N, dtype=torch.float64, device="cuda")
        vp = ctypes.c_void_p
        for part, np_ in ((-1, 2), (2, 2), (0, 0), (0, 5000)):
            rc = L.rpb_mobility_apply_part(ctx._h, N, vp(P.data_ptr()), vp(Fd.data_ptr()), None, part, np_,
                                           vp(out.data_ptr()))
            assert rc == gpu_lib.RPB_EINVAL, (part, np_)
        # the whole product again after the shares (the shares' schedule is kept apart)
        assert torch.equal(ctx.mobility_apply(P, Fd, Td), full)
    finally:
        ctx.close()


def test_product_hook_error_and_reset(gpu_lib):
    N = 200
    pos = inputs.monolayer(N, seed=12)
    F = inputs.vectors(N, 13)
    ctx = gpu_lib.Context(N, precision="fp64", max_iter=8)
    try:
        calls = []

        def failing(n, p, f, t, u):
            calls.append(n)
            return gpu_lib.RPB_ECUDA

        ctx.set_product_hook(failing)
        with pytest.raises(gpu_lib.RpbError) as e:
            ctx.mobility_apply(dev(pos), dev(F))
        assert e.value.code == gpu_lib.RPB_ECUDA and calls == [N]
        with pytest.raises(gpu_lib.RpbError):  # a step's products go through the hook too
            ctx.ab_step(dev(pos), torch.zeros(3 * N, dtype=torch.float64, device="cuda"), 0, 1)
        with pytest.raises(gpu_lib.RpbError):  # and graph replays are refused with a hook
            ctx.run(dev(pos), torch.zeros(3 * N, dtype=torch.float64, device="cuda"), 0, 1, 2)
        ctx.set_product_hook(None)
        got = inputs.from_soa(ctx.mobility_apply(dev(pos), dev(F)).cpu().numpy(), N)
        ref = O.mobility_apply(pos, F)
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-10
    finally:
        ctx.close()


def test_batch_tiles_validation_and_fp64_tuner(gpu_lib):
    bt = gpu_lib.BatchContext(max_total_N=4000, max_B=8, precision="fp64", max_iter=8)
    try:
        for bad in (dict(seg_tiles=0), dict(seg_tiles=65), dict(ctas_per_sm=3), dict(ctas_per_sm=6)):
            with pytest.raises(gpu_lib.RpbError):
                bt.set_tiles(**bad)
        sizes = [100, 700, 1300]
        poss = [inputs.monolayer(n, seed=30 + k) for k, n in enumerate(sizes)]
        res = bt.tune([dev(p) for p in poss], reps=1)
        assert len(res["candidates"]) == 1 and res["best"]["symmetric"] is False
        Fs = [inputs.vectors(n, 40 + k) for k, n in enumerate(sizes)]
        out = bt.mobility_apply([dev(p) for p in poss], [dev(f) for f in Fs])
        for k, n in enumerate(sizes):
            ref = O.mobility_apply(poss[k], Fs[k])
            got = inputs.from_soa(out[k].cpu().numpy(), n)
            assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-10
    finally:
        bt.close()


def test_fma_peak_kinds(gpu_lib):
    L = gpu_lib.load()
    t, ms = ctypes.c_double(), ctypes.c_double()
    assert L.rpb_fma_peak(7, None, ctypes.byref(t), ctypes.byref(ms)) == gpu_lib.RPB_EINVAL
    f32, _ = gpu_lib.fma_peak("ffma2")
    f64, _ = gpu_lib.fma_peak("dfma")
    assert f32 > 10.0 * f64 > 0.0
