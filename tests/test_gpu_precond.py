"""GPU parity of the optional block-diagonal Lanczos preconditioner (rpb_set_preconditioner; Sec. II.C
reports trying it) against the oracle's lanczos_sqrt / ab_step with precondition=True.

Tolerances as in test_gpu_parity.py: FP64 products 1e-10, g at equal m 1e-10, AB increment 1e-8;
FP32 pairs 1e-5 on products and 2e-5 on the increment."""
import math

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


def with_wall_cases(N, seed):
    """A monolayer with a few spheres overlapping the wall, one on it and one below it."""
    p = inputs.monolayer(N, seed=seed)
    p[1, 2] = 0.55
    p[2, 2] = 0.0
    p[3, 2] = -0.4
    return p


@pytest.fixture()
def ctx64(gpu_lib):
    c = gpu_lib.Context(max_N=2048, precision="fp64", max_iter=64)
    c.set_preconditioner("block-diagonal")
    yield c
    c.close()


@pytest.mark.parametrize("N", [1, 37, 300])
def test_lanczos_preconditioned_equal_m(ctx64, N):
    pos = with_wall_cases(N, 50 + N) if N > 3 else inputs.monolayer(N, seed=1)
    W = O.noise(N, 4, 0, 0)
    g_ref, m_ref, eps_ref, _ = O.lanczos_sqrt(pos, W, tol=1e-3, max_iter=64, precondition=True)
    g, m, eps, conv = ctx64.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-3, max_iter=64)
    assert m == m_ref and conv
    assert maxrel(host(g, N), g_ref) <= 1e-10
    for k in (1, 3):
        g_ref, mk, _, _ = O.lanczos_sqrt(pos, W, exact_iters=k, precondition=True)
        g, m, _, _ = ctx64.lanczos_sqrt_apply(dev(pos), dev(W), tol=0.0, max_iter=k)
        assert m == mk
        assert maxrel(host(g, N), g_ref) <= 1e-10
    if N > 3:  # no noise on the spheres on or below the wall
        gh = host(g, N)
        assert np.all(gh[2] == 0.0) and np.all(gh[3] == 0.0)


def test_preconditioned_step_fp64(ctx64):
    N = 256
    pos0 = with_wall_cases(N, 7)
    Uprev = inputs.vectors(N, 8, scale=0.01)
    new_ref, Un_ref, info = O.ab_step(pos0, Uprev, 2, seed=5, dt=0.01, delta=1e-6, tol=1e-3, precondition=True)
    q, U = dev(pos0), dev(Uprev)
    st = ctx64.ab_step(q, U, 2, seed=5, dt=0.01, delta=1e-6, tol=1e-3)
    assert st["m"] == info["m"]
    assert maxrel(host(U, N), Un_ref) <= 1e-10
    assert maxrel(host(q, N) - pos0, new_ref - pos0) <= 1e-8


def test_preconditioned_step_fp32_two_rhs(gpu_lib):
    """N = 600 in float32: the step's first Lanczos product P M P v_0 shares the pass of the
    deterministic velocity (the two-right-hand-side form)."""
    N = 600
    pos0 = inputs.monolayer(N, seed=19)
    Uprev = inputs.vectors(N, 20, scale=0.01)
    ctx = gpu_lib.Context(max_N=N, precision="fp32", max_iter=64)
    try:
        ctx.set_preconditioner("block-diagonal")
        q, U = dev(pos0), dev(Uprev)
        st = ctx.step(q, U, 3, 9, dt=0.01, delta=5e-3, tol=1e-3)
    finally:
        ctx.close()
    new_ref, Un_ref, info = O.ab_step(pos0, Uprev, 3, seed=9, dt=0.01, delta=5e-3, tol=1e-3, precondition=True)
    assert st["m"] == info["m"]
    assert maxrel(host(U, N), Un_ref) <= 1e-5
    assert maxrel(host(q, N) - pos0, new_ref - pos0) <= 2e-5


def test_switch_off_restores_plain_lanczos(gpu_lib):
    N = 128
    pos = inputs.monolayer(N, seed=3)
    W = O.noise(N, 2, 0, 0)
    a = gpu_lib.Context(max_N=N, precision="fp64", max_iter=32)
    b = gpu_lib.Context(max_N=N, precision="fp64", max_iter=32)
    try:
        a.set_preconditioner("block-diagonal")
        a.set_preconditioner("none")
        ga, ma, _, _ = a.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-3)
        gb, mb, _, _ = b.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-3)
        assert ma == mb and torch.equal(ga, gb)
        with pytest.raises(gpu_lib.RpbError):  # unknown kind, through the C ABI
            gpu_lib._check(gpu_lib.load().rpb_set_preconditioner(a._h, 7))
    finally:
        a.close()
        b.close()


def test_preconditioned_covariance_small(gpu_lib):
    """The map W -> g of the full Krylov space reproduces M as its covariance: with 3N iterations
    g = L W for L = D^{1/2} (P M P)^{1/2}, and L L^T = M (dense, LAPACK)."""
    N = 6
    pos = inputs.monolayer(N, seed=11)
    pos[1, 2] = 0.55  # one overlapping the wall; every sphere above it (D > 0)
    tt, _ = O.dense(pos)
    D = O.self_diagonal(pos).ravel()
    P = 1.0 / np.sqrt(D)
    lam, Q = np.linalg.eigh(P[:, None] * tt * P[None, :])
    L = np.sqrt(D)[:, None] * (Q @ np.diag(np.sqrt(np.clip(lam, 0, None))) @ Q.T)
    ctx = gpu_lib.Context(max_N=N, precision="fp64", max_iter=3 * N)
    try:
        ctx.set_preconditioner("block-diagonal")
        cols = []
        for j in range(3 * N):
            e = np.zeros(3 * N)
            e[j] = 1.0
            g, m, _, _ = ctx.lanczos_sqrt_apply(dev(pos), dev(e.reshape(N, 3)), tol=1e-13, max_iter=3 * N,
                                                raise_on_noconv=False)
            cols.append(host(g, N).ravel())
        Lg = np.stack(cols, axis=1)
    finally:
        ctx.close()
    assert np.allclose(Lg, L, rtol=0, atol=1e-9 * np.abs(L).max())
    assert math.isclose(np.abs(Lg @ Lg.T - tt).max(), 0.0, abs_tol=1e-9 * np.abs(tt).max())


def test_preconditioned_lanczos_periodic(gpu_lib):
    """Pseudo-periodic mode: the block is still each sphere's own self block (its images count as
    other particles); products sum the nine images."""
    L = (20.0, 17.5)
    rng = np.random.default_rng(12)
    N = 60
    pos = np.zeros((N, 3))
    pos[:, 0] = rng.uniform(-0.5 * L[0], 1.5 * L[0], N)
    pos[:, 1] = rng.uniform(-0.5 * L[1], 1.5 * L[1], N)
    pos[:, 2] = rng.uniform(0.8, 3.0, N)
    W = O.noise(N, 6, 0, 0)
    g_ref, m_ref, _, _ = O.lanczos_sqrt(pos, W, tol=1e-3, max_iter=64, periodic=L, precondition=True)
    ctx = gpu_lib.Context(max_N=N, precision="fp64", max_iter=64)
    try:
        ctx.set_periodic(*L)
        ctx.set_preconditioner("block-diagonal")
        g, m, _, conv = ctx.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-3)
    finally:
        ctx.close()
    assert conv and m == m_ref
    assert maxrel(host(g, N), g_ref) <= 1e-10


def test_preconditioned_lanczos_fp32_pairs(gpu_lib):
    """Float32 pairs (the symmetric pass at this size) against the float64 path, both preconditioned."""
    N = 1024
    pos = inputs.monolayer(N, seed=21)
    W = O.noise(N, 7, 0, 0)
    res = {}
    for prec in ("fp64", "fp32"):
        ctx = gpu_lib.Context(max_N=N, precision=prec, max_iter=64)
        try:
            ctx.set_preconditioner("block-diagonal")
            res[prec] = ctx.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-3)
        finally:
            ctx.close()
    g64, m64, _, _ = res["fp64"]
    g32, m32, e32, _ = res["fp32"]
    assert m32 == m64 and e32 <= 1e-3
    assert O.rel_err(host(g32, N), host(g64, N)) <= 1e-5
