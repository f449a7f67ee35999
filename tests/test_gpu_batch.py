"""Ragged batches through the C ABI (rpb_batch_*): per-instance parity with the oracle, agreement
with the single-suspension entry points, and an instance's result alone versus inside a batch.

Tolerances as in test_gpu_parity.py: FP64 1e-10 (products, increments relative to their size 1e-8),
FP32 1e-5 on products.  Alone versus mixed: the computation of an instance does not depend on its
companions, so the two agree to 1e-12 relative (bitwise in practice).
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
    return float(np.max(np.abs(np.asarray(x) - ref)) / np.max(np.abs(ref)))


def overlapping(N, seed):
    rng = np.random.default_rng(seed)
    p = np.zeros((N, 3))
    p[:, :2] = rng.uniform(0, 2.2 * math.sqrt(N) + 1, (N, 2))
    p[:, 2] = rng.uniform(-0.3, 3.0, N)
    k = max(1, N // 5)
    p[:k, :2] = p[0, :2] + rng.normal(0, 0.6, (k, 2))
    return p


SIZES = [1, 5, 127, 128, 129, 300, 64]


@pytest.fixture(scope="module")
def batch64(gpu_lib):
    b = gpu_lib.BatchContext(max_total_N=20000, max_B=64, precision="fp64", max_iter=32)
    yield b
    b.close()


@pytest.fixture(scope="module")
def batch32(gpu_lib):
    b = gpu_lib.BatchContext(max_total_N=200000, max_B=600, precision="fp32", max_iter=32)
    yield b
    b.close()


@pytest.mark.parametrize("loads", ["FT", "F", "T"])
def test_batch_mobility_fp64(batch64, loads):
    poss = [overlapping(N, 10 + k) for k, N in enumerate(SIZES)]
    Fs = [inputs.vectors(N, 20 + k) for k, N in enumerate(SIZES)]
    Ts = [inputs.vectors(N, 30 + k) for k, N in enumerate(SIZES)]
    out = batch64.mobility_apply([dev(p) for p in poss], [dev(f) for f in Fs] if "F" in loads else None,
                                 [dev(t) for t in Ts] if "T" in loads else None)
    for k, N in enumerate(SIZES):
        ref = O.mobility_apply(poss[k], Fs[k] if "F" in loads else None, Ts[k] if "T" in loads else None)
        assert maxrel(host(out[k], N), ref) <= 1e-10, (k, N)


def test_batch_mobility_fp32(batch32):
    poss = [overlapping(N, 40 + k) for k, N in enumerate(SIZES)]
    Fs = [inputs.vectors(N, 50 + k) for k, N in enumerate(SIZES)]
    Ts = [inputs.vectors(N, 60 + k) for k, N in enumerate(SIZES)]
    out = batch32.mobility_apply([dev(p) for p in poss], [dev(f) for f in Fs], [dev(t) for t in Ts])
    for k, N in enumerate(SIZES):
        ref = O.mobility_apply(poss[k], Fs[k], Ts[k])
        assert maxrel(host(out[k], N), ref) <= 1e-5, (k, N)


def test_batch_step_matches_single_path_and_oracle(batch64, gpu_lib):
    """Each instance of one batched step equals rpb_ab_step on the same state, seed and step."""
    sizes = [40, 128, 1, 200, 77]
    seeds = [3, 1, 4, 1, 5]
    steps = [0, 2, 0, 7, 1]
    poss = [inputs.monolayer(N, seed=100 + k) for k, N in enumerate(sizes)]
    Ups = [inputs.vectors(N, 70 + k, scale=0.01) for k, N in enumerate(sizes)]
    q = [dev(p) for p in poss]
    U = [dev(u) for u in Ups]
    stats = batch64.ab_step(q, U, steps, seeds, dt=0.01, delta=1e-6, tol=1e-3)
    ctx = gpu_lib.Context(max_N=256, precision="fp64", max_iter=32)
    try:
        for k, N in enumerate(sizes):
            qs, Us = dev(poss[k]), dev(Ups[k])
            st = ctx.ab_step(qs, Us, steps[k], seeds[k], dt=0.01, delta=1e-6, tol=1e-3)
            assert stats[k]["m"] == st["m"]
            inc_b = host(q[k], N) - poss[k]
            inc_s = host(qs, N) - poss[k]
            assert maxrel(inc_b, inc_s) <= 1e-8, k
            assert maxrel(host(U[k], N), host(Us, N)) <= 1e-10, k
    finally:
        ctx.close()
    # and the 40-sphere instance against the oracle
    new_ref, Un_ref, info = O.ab_step(poss[0], None, 0, seed=3, dt=0.01, delta=1e-6, tol=1e-3)
    assert stats[0]["m"] == info["m"]
    assert maxrel(host(q[0], 40) - poss[0], new_ref - poss[0]) <= 1e-8


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_alone_vs_mixed(batch32, batch64, precision):
    bt = batch32 if precision == "fp32" else batch64
    sizes = [300, 64, 129, 1, 250]
    poss = [inputs.monolayer(N, seed=200 + k) for k, N in enumerate(sizes)]
    target = 2
    # alone
    qa, Ua = dev(poss[target]), torch.zeros(3 * sizes[target], dtype=torch.float64, device="cuda")
    sa = bt.ab_step([qa], [Ua], [0], [11], delta=5e-3 if precision == "fp32" else 1e-6)
    sa = bt.ab_step([qa], [Ua], [1], [11], delta=5e-3 if precision == "fp32" else 1e-6)
    # in a mix (other instances at other steps and seeds)
    q = [dev(p) for p in poss]
    U = [torch.zeros(3 * N, dtype=torch.float64, device="cuda") for N in sizes]
    for s in range(2):
        sm = bt.ab_step(q, U, [s, s + 3, s, s + 1, s + 5], [7, 8, 11, 9, 10],
                        delta=5e-3 if precision == "fp32" else 1e-6)
    assert sm[target]["m"] == sa[0]["m"]
    assert maxrel(host(q[target], sizes[target]), host(qa, sizes[target])) <= 1e-12
    assert maxrel(host(U[target], sizes[target]), host(Ua, sizes[target])) <= 1e-12


def test_batch512_like_config_runs(batch32):
    """A slice of the batched workload (log-uniform N in [64, 2048]) steps and converges."""
    sizes = [int(n) for n in inputs.batch_sizes(48, seed=0)]
    q = [dev(inputs.monolayer(N, seed=k)) for k, N in enumerate(sizes)]
    U = [torch.zeros_like(t) for t in q]
    stats = batch32.ab_step(q, U, [0] * len(sizes), list(range(len(sizes))), delta=5e-3)
    assert all(s["converged"] and 2 <= s["m"] <= 20 for s in stats)
    assert all(torch.isfinite(t).all() for t in q)


def test_batch_errors(batch64, gpu_lib):
    q = [dev(inputs.monolayer(10, seed=0))]
    U = [torch.zeros_like(q[0])]
    with pytest.raises(gpu_lib.RpbError):
        batch64.ab_step(q * 65, U * 65, [0] * 65, [0] * 65)     # B > max_B
    big = [dev(inputs.monolayer(20001, seed=0))]
    with pytest.raises(gpu_lib.RpbError):
        batch64.mobility_apply(big, big)                        # total > max_total_N
    assert "max_total_N" in gpu_lib.last_error()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_run_graph_equals_steps(batch32, batch64, precision):
    """rpb_batch_run (the step captured once in a CUDA graph and replayed) gives bitwise the same
    trajectory as the same number of rpb_batch_ab_step calls."""
    bt = batch32 if precision == "fp32" else batch64
    delta = 5e-3 if precision == "fp32" else 1e-6
    sizes = [40, 128, 200, 77, 1]
    seeds = [5, 6, 7, 8, 9]
    steps0 = [0, 2, 0, 5, 0]
    poss = [inputs.monolayer(N, seed=300 + k) for k, N in enumerate(sizes)]
    qa = [dev(p) for p in poss]
    Ua = [torch.zeros(3 * N, dtype=torch.float64, device="cuda") for N in sizes]
    for s in range(4):
        sa = bt.ab_step(qa, Ua, [x + s for x in steps0], seeds, delta=delta)
    qb = [dev(p) for p in poss]
    Ub = [torch.zeros(3 * N, dtype=torch.float64, device="cuda") for N in sizes]
    sb, unconv = bt.run(qb, Ub, steps0, seeds, nsteps=4, lanczos_iters=32, delta=delta)
    assert unconv == 0
    assert [s["m"] for s in sa] == [s["m"] for s in sb]
    for k in range(len(sizes)):
        assert torch.equal(qa[k], qb[k]) and torch.equal(Ua[k], Ub[k]), k


LONG = [2100, 1030, 17, 640]


def test_batch_mobility_fp32_long_rows(batch32):
    """Suspensions of more than eight tiles: rows of the symmetric pass cut into several runs."""
    poss = [overlapping(N, 80 + k) for k, N in enumerate(LONG)]
    Fs = [inputs.vectors(N, 90 + k) for k, N in enumerate(LONG)]
    Ts = [inputs.vectors(N, 95 + k) for k, N in enumerate(LONG)]
    out = batch32.mobility_apply([dev(p) for p in poss], [dev(f) for f in Fs], [dev(t) for t in Ts])
    outF = batch32.mobility_apply([dev(p) for p in poss], [dev(f) for f in Fs], None)
    for k, N in enumerate(LONG):
        assert maxrel(host(out[k], N), O.mobility_apply(poss[k], Fs[k], Ts[k])) <= 1e-5, (k, N)
        assert maxrel(host(outF[k], N), O.mobility_apply(poss[k], Fs[k], None)) <= 1e-5, (k, N)


def test_batch_fp32_symmetric_equals_one_way(batch32, gpu_lib, monkeypatch):
    """The symmetric pass and the one-way kernel (RPB_FP32_BATCH_SYM=0) give the same products up to
    float32 summation order."""
    monkeypatch.setenv("RPB_FP32_BATCH_SYM", "0")
    one = gpu_lib.BatchContext(max_total_N=20000, max_B=8, precision="fp32", max_iter=8)
    try:
        poss = [overlapping(N, 110 + k) for k, N in enumerate(LONG)]
        Fs = [inputs.vectors(N, 120 + k) for k, N in enumerate(LONG)]
        Ts = [inputs.vectors(N, 130 + k) for k, N in enumerate(LONG)]
        a = batch32.mobility_apply([dev(p) for p in poss], [dev(f) for f in Fs], [dev(t) for t in Ts])
        b = one.mobility_apply([dev(p) for p in poss], [dev(f) for f in Fs], [dev(t) for t in Ts])
        for k, N in enumerate(LONG):
            assert maxrel(host(a[k], N), host(b[k], N)) <= 2e-6, (k, N)
    finally:
        one.close()


def test_batch_fp32_alone_vs_mixed_products_bitwise(batch32):
    """A suspension's product does not depend on its companions or its place in the batch."""
    p = overlapping(2100, 140)
    f, t = inputs.vectors(2100, 141), inputs.vectors(2100, 142)
    alone = host(batch32.mobility_apply([dev(p)], [dev(f)], [dev(t)])[0], 2100)
    others = [overlapping(N, 150 + k) for k, N in enumerate([333, 5, 1500])]
    mix = [others[0], others[1], p, others[2]]
    fs = [inputs.vectors(len(x), 160 + k) for k, x in enumerate(mix)]
    ts = [inputs.vectors(len(x), 170 + k) for k, x in enumerate(mix)]
    fs[2], ts[2] = f, t
    mixed = host(batch32.mobility_apply([dev(x) for x in mix], [dev(x) for x in fs], [dev(x) for x in ts])[2], 2100)
    assert np.array_equal(alone, mixed)
