"""GPU parity at the sizes and in the launch configurations the benchmark runs, and the AB step's
increment split into the parts the tolerances of the method's readings apply to.

  - The two-right-hand-side symmetric pass (a step's deterministic velocity M_tt F + M_tr T and its
    first Lanczos product M_tt v_0 from one evaluation of each pair) at N = 65536, on sampled rows
    that the FP64 oracle computes one by one: 1e-5 on both products (FP32 pairs).
  - The FP32-pair Lanczos square root against the FP64 oracle's at N = 4096: the same iteration
    count, eps within tol, and g within 1e-5; also at a forced equal m.
  - One FP64 AB step of the 256-sphere configuration with its increment split: the velocity U^n and
    the Brownian increment g at 1e-10, the drift at its a/delta-amplified bound (reported), and the
    increment without the drift (dt (3/2 U^n - 1/2 U^{n-1}) + sqrt(2 kT dt) g) at 1e-10.
  - The FP32 path's drift (delta = 5e-3 a) against the FP64 oracle's (delta = 1e-6 a), reported.
  - The pair split at N = 65536: four shares of the symmetric pass's triangle add up to the product.
"""
import numpy as np
import pytest

import oracle as O
from paper_1612_00474_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.tensor(inputs.to_soa(x), dtype=torch.float64, device="cuda")


def host(t, N):
    return inputs.from_soa(t.detach().cpu().numpy(), N)


def maxrel(x, ref):
    ref = np.asarray(ref)
    return float(np.max(np.abs(np.asarray(x) - ref)) / np.max(np.abs(ref)))


def test_two_rhs_pass_n65536_sampled_rows(gpu_lib):
    N = 65536
    pos = inputs.monolayer(N, seed=0)
    F = inputs.vectors(N, 9)
    T = np.tile([0.0, 1.0, 0.0], (N, 1))
    W = O.noise(N, 0, 0, 0)
    P = W / np.linalg.norm(W)  # v_0 of the Lanczos iteration
    ctx = gpu_lib.Context(max_N=N, precision="fp32", max_iter=16)
    try:
        U, U2 = ctx.mobility_apply2(dev(pos), dev(F), dev(T), dev(P))
        torch.cuda.synchronize()
        U, U2 = host(U, N), host(U2, N)
    finally:
        ctx.close()
    rows = np.random.default_rng(1).choice(N, 20, replace=False)
    rows = np.concatenate([rows, [0, 127, 128, 255, N - 1]])
    ref = np.concatenate([O.mobility_apply(pos, F, T, rows=(r, r + 1)) for r in rows])
    ref2 = np.concatenate([O.mobility_apply(pos, P, None, rows=(r, r + 1)) for r in rows])
    e1, e2 = maxrel(U[rows], ref), maxrel(U2[rows], ref2)
    assert e1 <= 1e-5 and e2 <= 1e-5, (e1, e2)


def test_two_rhs_entry_point_fallback_fp64(gpu_lib):
    """FP64 contexts take the two products one after the other; the result is the same as two calls."""
    N = 300
    pos = inputs.monolayer(N, seed=4)
    F, T, P = inputs.vectors(N, 1), inputs.vectors(N, 2), inputs.vectors(N, 3)
    ctx = gpu_lib.Context(max_N=N, precision="fp64", max_iter=8)
    try:
        U, U2 = ctx.mobility_apply2(dev(pos), dev(F), dev(T), dev(P))
        assert torch.equal(U, ctx.mobility_apply(dev(pos), dev(F), dev(T)))
        assert torch.equal(U2, ctx.mobility_apply(dev(pos), dev(P)))
        assert maxrel(host(U2, N), O.mobility_apply(pos, P)) <= 1e-10
    finally:
        ctx.close()


def test_lanczos_fp32_against_oracle_n4096(gpu_lib):
    N = 4096
    pos = inputs.monolayer(N, seed=5)
    W = O.noise(N, 3, 0, 0)
    g_ref, m_ref, eps_ref, conv = O.lanczos_sqrt(pos, W, tol=1e-3)
    assert conv
    ctx = gpu_lib.Context(max_N=N, precision="fp32", max_iter=32)
    try:
        g, m, eps, _ = ctx.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-3)
        assert m == m_ref and eps <= 1e-3
        assert O.rel_err(host(g, N), g_ref) <= 1e-5
        # at a forced equal dimension one beyond the stop
        g2, m2, _, _ = ctx.lanczos_sqrt_apply(dev(pos), dev(W), tol=0.0, max_iter=m_ref + 1)
        g2_ref, _, _, _ = O.lanczos_sqrt(pos, W, exact_iters=m_ref + 1)
        assert m2 == m_ref + 1
        assert O.rel_err(host(g2, N), g2_ref) <= 1e-5
    finally:
        ctx.close()


def test_ab_step_increment_parts_n256(gpu_lib):
    N, seed, step, dt, delta = 256, 0, 3, 0.01, 1e-6
    pos0 = inputs.monolayer(N, seed=0)
    Uprev = inputs.vectors(N, 21, scale=0.01)
    new_ref, Un_ref, info = O.ab_step(pos0, Uprev, step, seed=seed, dt=dt, delta=delta, tol=1e-3, detail=True)
    ctx = gpu_lib.Context(max_N=N, precision="fp64", max_iter=64)
    try:
        q, U = dev(pos0), dev(Uprev)
        st = ctx.ab_step(q, U, step, seed, dt=dt, delta=delta, tol=1e-3)
        assert st["m"] == info["m"]
        # the step's own noise and, through the same kernels, its Brownian increment and drift
        W = ctx.philox_normal(N, seed, step, 0)
        Wt = ctx.philox_normal(N, seed, step, 1)
        g, m, _, _ = ctx.lanczos_sqrt_apply(dev(pos0), W, tol=1e-3)
        d = ctx.rfd_drift(dev(pos0), Wt, delta=delta)
        torch.cuda.synchronize()
        q, U, g, d = host(q, N), host(U, N), host(g, N), host(d, N)
    finally:
        ctx.close()
    assert m == info["m"]
    assert maxrel(U, Un_ref) <= 1e-10
    assert maxrel(g, info["g"]) <= 1e-10
    drift_err = maxrel(d, info["drift"])
    assert drift_err <= 1e-4, drift_err  # the product error times a / delta = 1e6
    inc = q - pos0
    inc_ref = new_ref - pos0
    e = maxrel(inc - dt * d, inc_ref - dt * info["drift"])
    assert e <= 1e-10, e
    # and the whole increment, the drift's share included
    assert maxrel(inc, inc_ref) <= 1e-8


def test_fp32_drift_against_fp64_oracle_drift(gpu_lib):
    """The float32 path computes the RFD drift with delta = 5e-3 a (delta ~ eps^(1/3) a for float32
    products, Sec. II.A).  Against the FP64 oracle at the same delta its error is the float32 product
    error amplified by a/delta: bound 1e-3 (max-norm).  Against the oracle at delta = 1e-6 a it also
    carries the finite difference's truncation, which the regularised mobility makes first order
    where it is not smooth -- spheres within delta of the clamp height z = a and pairs within delta of
    contact r = 2a (the oracle alone differs from itself by the same amount between the two deltas);
    that distance is printed and bounded loosely (2-norm 0.05)."""
    N = 4096
    pos = inputs.monolayer(N, seed=31)
    Wt = O.noise(N, 7, 0, 1)
    ref_same = O.rfd_drift(pos, Wt, delta=5e-3)
    ref_fine = O.rfd_drift(pos, Wt, delta=1e-6)
    ctx = gpu_lib.Context(max_N=N, precision="fp32", max_iter=16)
    try:
        got = host(ctx.rfd_drift(dev(pos), dev(Wt), delta=5e-3), N)
    finally:
        ctx.close()
    err = maxrel(got, ref_same)
    fine_max, fine_l2 = maxrel(got, ref_fine), O.rel_err(got, ref_fine)
    oracle_l2 = O.rel_err(ref_same, ref_fine)
    print(f"\nFP32 drift (delta = 5e-3 a), N = {N}: vs the FP64 oracle at the same delta {err:.2e} (max-norm); "
          f"vs the oracle at delta = 1e-6 a {fine_max:.2e} (max-norm), {fine_l2:.2e} (2-norm); the oracle's own "
          f"change between the two deltas {oracle_l2:.2e} (2-norm)")
    assert err <= 1e-3
    assert fine_l2 <= 0.05


def test_pair_shares_n65536(gpu_lib):
    """The pair split at the benchmark's size: four shares of the symmetric pass's triangle
    (rpb_mobility_apply_part) add up to the whole product (float32 partial sums in another order:
    2e-6), and on sampled rows to the FP64 oracle's product (1e-5)."""
    N, W = 65536, 4
    pos = inputs.monolayer(N, seed=0)
    F = inputs.vectors(N, 9)
    ctx = gpu_lib.Context(max_N=N, precision="fp32", max_iter=16)
    try:
        P, Fd = dev(pos), dev(F)
        full = ctx.mobility_apply(P, Fd)
        total = torch.zeros_like(full)
        for p in range(W):
            total += ctx.mobility_apply_part(P, Fd, None, p, W)
        torch.cuda.synchronize()
        full, total = host(full, N), host(total, N)
    finally:
        ctx.close()
    assert maxrel(total, full) <= 2e-6
    rows = np.concatenate([np.random.default_rng(2).choice(N, 16, replace=False), [0, 128, N - 1]])
    ref = np.concatenate([O.mobility_apply(pos, F, None, rows=(r, r + 1)) for r in rows])
    assert maxrel(total[rows], ref) <= 1e-5
