"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on seeded inputs.

Tolerances (relative to the largest |oracle| entry of the compared vector unless noted):
  FP64 pair path: 1e-10 for the matvec, Lanczos g (equal m), each RFD matvec, forces 1e-12,
  Philox normals 1e-13 (log / sincospi differ from glibc by a few ulp).
  RFD drift: the matvec error is amplified by a/delta; with delta = 1e-6 the bound is 1e-10 * 1e6
  * (a few) -> 1e-4 is asserted, and the observed value is far below it.
  FP32 pair path: 1e-5 on the matvec.
  AB step: the new positions minus the old ones (the increment) within 1e-8 of the oracle's.
"""
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


def overlapping(N, seed):
    """Monolayer-like configuration with particle overlaps and spheres partly below / at the wall."""
    rng = np.random.default_rng(seed)
    p = np.zeros((N, 3))
    p[:, :2] = rng.uniform(0, 2.2 * math.sqrt(N) + 1, (N, 2))
    p[:, 2] = rng.uniform(-0.3, 3.0, N)
    k = max(1, N // 5)
    p[:k, :2] = p[0, :2] + rng.normal(0, 0.6, (k, 2))
    return p


@pytest.fixture(scope="module")
def ctx64(gpu_lib):
    c = gpu_lib.Context(max_N=70000, precision="fp64", max_iter=64)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx32(gpu_lib):
    c = gpu_lib.Context(max_N=70000, precision="fp32", max_iter=64)
    yield c
    c.close()


# ------------------------------------------------------------------ matvec
@pytest.mark.parametrize("N", [1, 2, 3, 31, 127, 128, 129, 300, 1000])
def test_mobility_fp64(ctx64, N):
    pos = overlapping(N, N)
    F, T = inputs.vectors(N, 1), inputs.vectors(N, 2)
    ref = O.mobility_apply(pos, F, T)
    got = host(ctx64.mobility_apply(dev(pos), dev(F), dev(T)), N)
    assert maxrel(got, ref) <= 1e-10
    assert O.rel_err(got, ref) <= 1e-10


@pytest.mark.parametrize("which", ["F", "T", "none"])
def test_mobility_fp64_partial_loads(ctx64, which):
    N = 200
    pos = overlapping(N, 7)
    F = inputs.vectors(N, 3) if which == "F" else None
    T = inputs.vectors(N, 4) if which == "T" else None
    got = host(ctx64.mobility_apply(dev(pos), None if F is None else dev(F), None if T is None else dev(T)), N)
    if which == "none":
        assert np.all(got == 0.0)
        return
    ref = O.mobility_apply(pos, F, T)
    assert maxrel(got, ref) <= 1e-10


@pytest.mark.parametrize("N", [1, 33, 129, 1000])
def test_mobility_fp32(ctx32, N):
    pos = overlapping(N, 100 + N)
    F, T = inputs.vectors(N, 5), inputs.vectors(N, 6)
    ref = O.mobility_apply(pos, F, T)
    got = host(ctx32.mobility_apply(dev(pos), dev(F), dev(T)), N)
    assert maxrel(got, ref) <= 1e-5


@pytest.mark.parametrize("N", [256, 300, 1000, 4096])
def test_mobility_fp32_translation_only(ctx32, N):
    """F only (the Lanczos and RFD products): the float32 context evaluates each unordered pair once
    and applies it both ways; same tolerance, and deterministic."""
    pos = overlapping(N, 300 + N) if N < 4096 else inputs.monolayer(N, seed=1)
    F = inputs.vectors(N, 7)
    ref = O.mobility_apply(pos, F, None)
    a = ctx32.mobility_apply(dev(pos), dev(F))
    b = ctx32.mobility_apply(dev(pos), dev(F))
    assert torch.equal(a, b)
    assert maxrel(host(a, N), ref) <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mobility_n4096_full(ctx64, ctx32, prec):
    N = 4096
    pos = inputs.monolayer(N, seed=0)
    F, T = inputs.vectors(N, 8), np.tile([0.0, 1.0, 0.0], (N, 1))
    ref = O.mobility_apply(pos, F, T)
    c = ctx64 if prec == "fp64" else ctx32
    got = host(c.mobility_apply(dev(pos), dev(F), dev(T)), N)
    assert maxrel(got, ref) <= (1e-10 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mobility_n65536_sampled_rows(ctx64, ctx32, prec):
    """The 65536-sphere monolayer in the benchmark's launch configuration; the oracle evaluates a
    sample of target rows (all sources) one by one."""
    N = 65536
    pos = inputs.monolayer(N, seed=0)
    F = inputs.vectors(N, 9)
    T = np.tile([0.0, 1.0, 0.0], (N, 1))
    c = ctx64 if prec == "fp64" else ctx32
    got = host(c.mobility_apply(dev(pos), dev(F), dev(T)), N)
    rows = np.random.default_rng(0).choice(N, 24, replace=False)
    rows = np.concatenate([rows, [0, 127, 128, N - 1]])
    ref = np.concatenate([O.mobility_apply(pos, F, T, rows=(r, r + 1)) for r in rows])
    assert maxrel(got[rows], ref) <= (1e-10 if prec == "fp64" else 1e-5)


def test_mobility_deterministic_and_wall_stop(ctx64):
    N = 257
    pos = overlapping(N, 3)
    pos[5, 2] = -0.1   # below the wall: must not move (Appendix A)
    pos[6, 2] = 0.0
    F, T = inputs.vectors(N, 1), inputs.vectors(N, 2)
    a = ctx64.mobility_apply(dev(pos), dev(F), dev(T))
    b = ctx64.mobility_apply(dev(pos), dev(F), dev(T))
    assert torch.equal(a, b)
    U = host(a, N)
    assert np.all(U[5] == 0.0) and np.all(U[6] == 0.0)


# ------------------------------------------------------------------ noise and forces
def test_philox_normals(ctx64):
    N = 1001
    for step, sid in [(0, 0), (0, 1), (17, 0), (2**31 + 5, 1)]:
        got = host(ctx64.philox_normal(N, seed=0x1234_5678_9abc, step=step, stream_id=sid), N)
        ref = O.noise(N, 0x1234_5678_9abc, step, sid)
        assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-13


@pytest.mark.parametrize("N", [1, 2, 300, 1000])
def test_forces(ctx64, N):
    pos = overlapping(N, 40 + N)
    pos[:, 2] = np.abs(pos[:, 2]) + 0.3
    got = host(ctx64.forces(dev(pos), weight=1.0, U0=1.0, b=0.1), N)
    ref = O.forces(pos, 1.0, 1.0, 1.0, 0.1)
    assert maxrel(got, ref) <= 1e-12


# ------------------------------------------------------------------ Lanczos
@pytest.mark.parametrize("N", [1, 16, 256])
def test_lanczos_equal_m(ctx64, N):
    pos = inputs.monolayer(N, seed=N)
    W = O.noise(N, 0, 0, 0)
    g_ref, m_ref, eps_ref, _ = O.lanczos_sqrt(pos, W, tol=1e-3, max_iter=64)
    g, m, eps, conv = ctx64.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-3, max_iter=64)
    assert m == m_ref and conv
    assert maxrel(host(g, N), g_ref) <= 1e-10
    if m >= 2:
        assert abs(eps - eps_ref) <= 1e-8 * max(eps_ref, 1e-12) + 1e-13
    # forced iteration counts (tol <= 0 runs exactly max_iter)
    for k in (1, 2, 5):
        g_ref, mk, _, _ = O.lanczos_sqrt(pos, W, exact_iters=k)
        g, m, _, _ = ctx64.lanczos_sqrt_apply(dev(pos), dev(W), tol=0.0, max_iter=k)
        assert m == mk
        assert maxrel(host(g, N), g_ref) <= 1e-10


def test_lanczos_zero_and_noconv(ctx64, gpu_lib):
    N = 64
    pos = inputs.monolayer(N, seed=2)
    g, m, eps, conv = ctx64.lanczos_sqrt_apply(dev(pos), dev(np.zeros((N, 3))), tol=1e-3)
    assert m == 0 and conv and torch.count_nonzero(g) == 0
    W = O.noise(N, 1, 0, 0)
    g, m, eps, conv = ctx64.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-14, max_iter=2, raise_on_noconv=False)
    assert m == 2 and not conv
    with pytest.raises(gpu_lib.NoConvergence):
        ctx64.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-14, max_iter=2)


def test_lanczos_fp32_pairs(ctx32, ctx64):
    """FP32 pairs with FP64 Lanczos: eps within tol at the FP64 path's iteration count."""
    N = 1024
    pos = inputs.monolayer(N, seed=5)
    W = O.noise(N, 3, 0, 0)
    g64, m64, e64, _ = ctx64.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-3)
    g32, m32, e32, _ = ctx32.lanczos_sqrt_apply(dev(pos), dev(W), tol=1e-3)
    assert m32 == m64 and e32 <= 1e-3
    assert O.rel_err(host(g32, N), host(g64, N)) <= 1e-5


# ------------------------------------------------------------------ RFD
def test_rfd(ctx64):
    N = 256
    pos = inputs.monolayer(N, seed=0)
    Wt = O.noise(N, 0, 0, 1)
    delta = 1e-6
    d_ref, up, um = O.rfd_drift(pos, Wt, delta=delta, parts=True)
    got = host(ctx64.rfd_drift(dev(pos), dev(Wt), delta=delta), N)
    assert maxrel(got, d_ref) <= 1e-4
    # each of its two products at the 1e-10 bar
    for sgn, ref in ((1, up), (-1, um)):
        u = host(ctx64.mobility_apply(dev(pos + sgn * 0.5 * delta * Wt), dev(Wt)), N)
        assert maxrel(u, ref) <= 1e-10


# ------------------------------------------------------------------ AB step
def test_ab_step_n256_two_steps(ctx64):
    """The small FP64 configuration: 256 spheres, dt = 0.01, delta = 1e-6, tol = 1e-3, seed 0."""
    N = 256
    pos0 = inputs.monolayer(N, seed=0)
    q_ref, Up_ref = pos0.copy(), None
    q, Up = dev(pos0), torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    for step in range(2):
        new_ref, Un_ref, info = O.ab_step(q_ref, Up_ref, step, seed=0, dt=0.01, delta=1e-6, tol=1e-3)
        q_before = host(q, N)
        st = ctx64.ab_step(q, Up, step, seed=0, dt=0.01, delta=1e-6, tol=1e-3)
        assert st["m"] == info["m"]
        assert maxrel(host(Up, N), Un_ref) <= 1e-10
        inc = host(q, N) - q_before
        assert maxrel(inc, new_ref - q_ref) <= 1e-8
        q_ref, Up_ref = new_ref, Un_ref
        q = dev(q_ref)   # continue both from the oracle's state


def test_invalid_arguments(ctx64, gpu_lib):
    pos = dev(inputs.monolayer(4, seed=0))
    F = dev(inputs.vectors(4, 1))
    L = gpu_lib.load()
    import ctypes

    out = torch.empty(12, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p
    assert L.rpb_mobility_apply(ctx64._h, 0, p(pos.data_ptr()), p(F.data_ptr()), None, p(out.data_ptr())) == 1
    assert L.rpb_mobility_apply(ctx64._h, 70001, p(pos.data_ptr()), p(F.data_ptr()), None, p(out.data_ptr())) == 1
    assert L.rpb_mobility_apply(ctx64._h, 4, None, p(F.data_ptr()), None, p(out.data_ptr())) == 1
    assert L.rpb_mobility_apply(ctx64._h, 4, p(pos.data_ptr()), p(F.data_ptr()), None, p(pos.data_ptr())) == 1
    assert L.rpb_mobility_apply(ctx64._h, 4, p(pos.data_ptr() + 4), p(F.data_ptr()), None, p(out.data_ptr())) == 1
    assert "aligned" in gpu_lib.last_error()
    with pytest.raises(gpu_lib.RpbError):
        ctx64.lanczos_sqrt_apply(pos, F, max_iter=65)


# ------------------------------------------------------------------ unbounded mode and step variants
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_unbounded_mode(gpu_lib, prec, tol):
    N = 300
    pos = overlapping(N, 501)
    F, T = inputs.vectors(N, 3), inputs.vectors(N, 4)
    ctx = gpu_lib.Context(max_N=N, precision=prec, max_iter=16, wall=False)
    try:
        got = host(ctx.mobility_apply(dev(pos), dev(F), dev(T)), N)
        got_tt = host(ctx.mobility_apply(dev(pos), dev(F)), N)
    finally:
        ctx.close()
    assert maxrel(got, O.mobility_apply(pos, F, T, wall=False)) <= tol
    assert maxrel(got_tt, O.mobility_apply(pos, F, None, wall=False)) <= tol


@pytest.mark.parametrize("scheme,rfd", [("EM", "centred"), ("AB", "one-sided"), ("EM", "one-sided")])
def test_step_variants(ctx64, scheme, rfd):
    N = 64
    pos0 = inputs.monolayer(N, seed=8)
    Uprev = inputs.vectors(N, 9, scale=0.01)
    q, U = dev(pos0), dev(Uprev)
    st = ctx64.step(q, U, 3, 21, scheme=scheme, rfd=rfd, dt=0.01, delta=1e-6, tol=1e-3)
    new_ref, Un_ref, info = O.ab_step(pos0, Uprev, 3, seed=21, dt=0.01, delta=1e-6, tol=1e-3, scheme=scheme,
                                      one_sided=(rfd == "one-sided"))
    assert st["m"] == info["m"]
    assert maxrel(host(q, N) - pos0, new_ref - pos0) <= 1e-8
    assert maxrel(host(U, N), Un_ref) <= 1e-10


def test_checkpoint_resume_bitwise(gpu_lib):
    """State = (positions, U^{n-1}, step index, seed): six steps straight equal three steps, a round
    trip of the state through host memory into a new context, and three more (counter-based noise)."""
    N = 300
    pos0 = inputs.monolayer(N, seed=12)

    def run(q, U, steps, ctx):
        for s in steps:
            ctx.ab_step(q, U, s, 99, dt=0.01, delta=5e-3)

    c1 = gpu_lib.Context(max_N=N, precision="fp32", max_iter=32)
    qa, Ua = dev(pos0), torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    run(qa, Ua, range(6), c1)
    qb, Ub = dev(pos0), torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    run(qb, Ub, range(3), c1)
    saved = (qb.cpu().numpy().copy(), Ub.cpu().numpy().copy())
    c1.close()
    c2 = gpu_lib.Context(max_N=N, precision="fp32", max_iter=32)
    qc = torch.tensor(saved[0], device="cuda")
    Uc = torch.tensor(saved[1], device="cuda")
    run(qc, Uc, range(3, 6), c2)
    c2.close()
    assert torch.equal(qa, qc) and torch.equal(Ua, Uc)


# ------------------------------------------------------------------ pseudo-periodic boundaries (Appendix B)
LXY = (20.0, 17.5)


def periodic_config(N, seed, L=LXY):
    """Spheres scattered over the cell and its neighbours (so the library must fold them), with pairs
    that straddle an edge and a corner of the cell."""
    rng = np.random.default_rng(seed)
    p = np.zeros((N, 3))
    p[:, 0] = rng.uniform(-0.5 * L[0], 1.5 * L[0], N)
    p[:, 1] = rng.uniform(-0.5 * L[1], 1.5 * L[1], N)
    p[:, 2] = rng.uniform(0.8, 3.0, N)
    fixed = [[0.3, 0.5 * L[1], 1.2], [L[0] - 0.6, 0.5 * L[1], 1.3], [0.2, 0.2, 1.1], [L[0] - 0.4, L[1] - 0.3, 1.0]]
    k = min(N, 4)
    p[:k] = np.array(fixed[:k])
    return p


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("N", [1, 4, 129, 300])
def test_periodic_mobility(gpu_lib, prec, tol, N):
    pos = periodic_config(N, 600 + N)
    F, T = inputs.vectors(N, 5), inputs.vectors(N, 6)
    ctx = gpu_lib.Context(max_N=N, precision=prec, max_iter=16)
    try:
        ctx.set_periodic(*LXY)
        got = host(ctx.mobility_apply(dev(pos), dev(F), dev(T)), N)
        got_tt = host(ctx.mobility_apply(dev(pos), dev(F)), N)
        ctx.set_periodic(0.0, 0.0)
        got_open = host(ctx.mobility_apply(dev(pos), dev(F)), N)
    finally:
        ctx.close()
    assert maxrel(got, O.mobility_apply(pos, F, T, periodic=LXY)) <= tol
    assert maxrel(got_tt, O.mobility_apply(pos, F, None, periodic=LXY)) <= tol
    assert maxrel(got_open, O.mobility_apply(pos, F, None)) <= tol


def test_periodic_mobility_fp32_symmetric_size(gpu_lib):
    """N large enough that a float32 context would take the symmetric pass without periodicity."""
    N = 640
    pos = periodic_config(N, 77, L=(40.0, 36.0))
    F = inputs.vectors(N, 7)
    ctx = gpu_lib.Context(max_N=N, precision="fp32", max_iter=16)
    try:
        ctx.set_periodic(40.0, 36.0)
        got = host(ctx.mobility_apply(dev(pos), dev(F)), N)
    finally:
        ctx.close()
    assert maxrel(got, O.mobility_apply(pos, F, None, periodic=(40.0, 36.0))) <= 1e-5


@pytest.mark.parametrize("N", [2, 300])
def test_periodic_forces(gpu_lib, N):
    pos = periodic_config(N, 700 + N)
    ctx = gpu_lib.Context(max_N=N, precision="fp64", max_iter=16)
    try:
        ctx.set_periodic(*LXY)
        got = host(ctx.forces(dev(pos), weight=1.0, U0=1.0, b=0.1), N)
    finally:
        ctx.close()
    ref = O.forces(pos, 1.0, 1.0, 1.0, 0.1, periodic=LXY)
    assert maxrel(got, ref) <= 1e-12


def test_periodic_step(gpu_lib):
    N = 64
    L = (12.0, 11.0)
    pos0 = periodic_config(N, 31, L=L)
    Uprev = inputs.vectors(N, 32, scale=0.01)
    ctx = gpu_lib.Context(max_N=N, precision="fp64", max_iter=64)
    try:
        ctx.set_periodic(*L)
        q, U = dev(pos0), dev(Uprev)
        st = ctx.step(q, U, 2, 5, scheme="AB", dt=0.01, delta=1e-6, tol=1e-3)
    finally:
        ctx.close()
    new_ref, Un_ref, info = O.ab_step(pos0, Uprev, 2, seed=5, dt=0.01, delta=1e-6, tol=1e-3, periodic=L)
    assert st["m"] == info["m"]
    assert maxrel(host(U, N), Un_ref) <= 1e-10
    assert maxrel(host(q, N) - pos0, new_ref - pos0) <= 1e-8


def test_periodic_invalid(gpu_lib):
    ctx = gpu_lib.Context(max_N=8, precision="fp64", max_iter=8)
    try:
        with pytest.raises(gpu_lib.RpbError):
            ctx.set_periodic(3.0, 3.0)      # not above 4a
        with pytest.raises(gpu_lib.RpbError):
            ctx.set_periodic(10.0, 0.0)     # one direction only
        with pytest.raises(gpu_lib.RpbError):
            ctx.set_periodic(float("nan"), 10.0)
    finally:
        ctx.close()


def test_deterministic_step_kT0(gpu_lib):
    """kT = 0: the step is the deterministic Adams-Bashforth step (the oracle computes and multiplies
    the stochastic terms by zero; the library skips them)."""
    N = 200
    pos0 = inputs.monolayer(N, seed=14)
    Uprev = inputs.vectors(N, 15, scale=0.01)
    ctx = gpu_lib.Context(max_N=N, precision="fp64", max_iter=32, kT=0.0)
    try:
        q, U = dev(pos0), dev(Uprev)
        st = ctx.step(q, U, 4, 3, scheme="AB", dt=0.05, delta=1e-6, tol=1e-3, torque=(0.0, 50.0, 0.0))
    finally:
        ctx.close()
    new_ref, Un_ref, _ = O.ab_step(pos0, Uprev, 4, seed=3, dt=0.05, delta=1e-6, tol=1e-3, kT=0.0,
                                   torque=(0.0, 50.0, 0.0))
    assert st["m"] == 0 and st["converged"]
    assert maxrel(host(U, N), Un_ref) <= 1e-10
    assert maxrel(host(q, N) - pos0, new_ref - pos0) <= 1e-10


@pytest.mark.parametrize("with_T", [False, True])
def test_mobility_fp32_far_from_origin(ctx32, with_T):
    """Float32 offsets at large coordinates: a dense patch near (1000a, 4000a) (position ulp 2.4e-4a)
    and spheres spread along a 5000a strip; both forms of the symmetric pass at 1e-5."""
    rng = np.random.default_rng(91)
    N1, N2 = 768, 512
    p1 = np.column_stack([rng.uniform(1000, 1030, N1), rng.uniform(4000, 4030, N1), rng.uniform(0.9, 2.5, N1)])
    p2 = np.column_stack([rng.uniform(0, 60, N2), rng.uniform(0, 5000, N2), rng.uniform(1.0, 3.0, N2)])
    pos = np.vstack([p1, p2])
    N = len(pos)
    F, T = inputs.vectors(N, 92), (inputs.vectors(N, 93) if with_T else None)
    got = host(ctx32.mobility_apply(dev(pos), dev(F), dev(T) if with_T else None), N)
    ref = O.mobility_apply(pos, F, T)
    assert maxrel(got, ref) <= 1e-5


def test_forces_bucket_overflow_fallback(ctx64):
    """600 spheres piled into one 6a x 6a column (one bucket holds more than 512): the cell-list pass
    declines and the all-pairs kernel computes the forces."""
    rng = np.random.default_rng(71)
    N = 600
    pos = np.column_stack([rng.uniform(0, 6, N), rng.uniform(0, 6, N), rng.uniform(0.5, 40.0, N)])
    got = host(ctx64.forces(dev(pos), weight=1.0, U0=1.0, b=0.1), N)
    assert maxrel(got, O.forces(pos, 1.0, 1.0, 1.0, 0.1)) <= 1e-12


def test_forces_hashed_buckets_far_apart(ctx64):
    """Clusters far apart along a 2e5 a strip and on a diagonal, so that distant cells share buckets
    (cells are hashed modulo the bucket grid): the screen must reject the aliased candidates."""
    rng = np.random.default_rng(72)
    parts = []
    for cx in (0.0, 64 * 7.08, 2e5, -3e4):
        for cy in (0.0, 64 * 7.08 * 3, -5e3):
            parts.append(np.column_stack([cx + rng.uniform(0, 8, 40), cy + rng.uniform(0, 8, 40),
                                          rng.uniform(0.8, 3.0, 40)]))
    pos = np.vstack(parts)
    N = len(pos)
    got = host(ctx64.forces(dev(pos), weight=1.0, U0=1.0, b=0.1), N)
    assert maxrel(got, O.forces(pos, 1.0, 1.0, 1.0, 0.1)) <= 1e-12


def test_fp32_step_two_rhs(gpu_lib, monkeypatch):
    """Float32 step at N = 600: the deterministic velocity and the first Lanczos product run as one
    symmetric pass with two right-hand sides; compared with the oracle (same delta) and with the same
    step with that pass switched off (RPB_FP32_SYM_RHS2=0, read when a context is created)."""
    N = 600
    pos0 = inputs.monolayer(N, seed=17)
    Uprev = inputs.vectors(N, 18, scale=0.01)
    res = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("RPB_FP32_SYM_RHS2", flag)
        ctx = gpu_lib.Context(max_N=N, precision="fp32", max_iter=64)
        try:
            q, U = dev(pos0), dev(Uprev)
            st = ctx.step(q, U, 3, 9, dt=0.01, delta=5e-3, tol=1e-3)
            res[flag] = (host(q, N), host(U, N), st)
        finally:
            ctx.close()
    new_ref, Un_ref, info = O.ab_step(pos0, Uprev, 3, seed=9, dt=0.01, delta=5e-3, tol=1e-3)
    for flag in ("1", "0"):
        q, U, st = res[flag]
        assert st["m"] == info["m"]
        assert maxrel(U, Un_ref) <= 1e-5
        assert maxrel(q - pos0, new_ref - pos0) <= 2e-5
    assert maxrel(res["1"][1], res["0"][1]) <= 1e-5
