"""The batch context's tile schedules and their autotuner (rpb_batch_set_tiles, rpb_batch_tune).

Under every candidate schedule the tuner may pick -- the symmetric pass with runs of 4, 8, 16 or 32
tiles at 4 or 5 CTAs per SM, and the one-way kernel -- a ragged batch's products match the FP64 oracle
within the FP32 bound (1e-5) and each suspension's result is the same bit for bit alone and inside
the mix (the row cut depends only on its own size).  A step through the graph-replayed run under a
schedule equals the same run under that schedule alone, and the tuner returns one of the candidates
and leaves it in force."""
import numpy as np
import pytest

import oracle as O
from paper_1612_00474_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SIZES = [64, 1000, 129, 3000, 300, 128, 2049]
CANDIDATES = [dict(seg_tiles=s, ctas_per_sm=m, symmetric=True) for s in (4, 8, 16, 32) for m in (4, 5)] + \
             [dict(seg_tiles=8, ctas_per_sm=5, symmetric=False)]


def dev(x):
    return torch.tensor(inputs.to_soa(x), dtype=torch.float64, device="cuda")


def host(t, N):
    return inputs.from_soa(t.detach().cpu().numpy(), N)


@pytest.fixture(scope="module")
def batch(gpu_lib):
    b = gpu_lib.BatchContext(max_total_N=20000, max_B=16, precision="fp32", max_iter=32)
    yield b
    b.close()


@pytest.fixture(scope="module")
def data():
    poss = [inputs.monolayer(N, seed=40 + k) for k, N in enumerate(SIZES)]
    Fs = [inputs.vectors(N, 50 + k) for k, N in enumerate(SIZES)]
    Ts = [inputs.vectors(N, 60 + k) for k, N in enumerate(SIZES)]
    refs = [O.mobility_apply(p, f, t) for p, f, t in zip(poss, Fs, Ts)]
    refs_tt = [O.mobility_apply(p, f) for p, f in zip(poss, Fs)]
    return poss, Fs, Ts, refs, refs_tt


@pytest.mark.parametrize("cand", CANDIDATES, ids=lambda c: f"seg{c['seg_tiles']}_m{c['ctas_per_sm']}_{int(c['symmetric'])}")
def test_every_schedule_parity_and_alone_equals_mixed(batch, data, cand):
    poss, Fs, Ts, refs, refs_tt = data
    batch.set_tiles(**cand)
    assert batch.get_tiles() == cand
    for torque, rr in ((True, refs), (False, refs_tt)):
        mixed = batch.mobility_apply([dev(p) for p in poss], [dev(f) for f in Fs],
                                     [dev(t) for t in Ts] if torque else None)
        for k, N in enumerate(SIZES):
            got = host(mixed[k], N)
            assert np.max(np.abs(got - rr[k])) / np.max(np.abs(rr[k])) <= 1e-5, (cand, k)
            alone = batch.mobility_apply([dev(poss[k])], [dev(Fs[k])], [dev(Ts[k])] if torque else None)[0]
            assert torch.equal(alone, mixed[k]), (cand, k, torque)


def test_run_under_schedule_alone_equals_mixed(batch, data):
    poss = data[0]
    batch.set_tiles(seg_tiles=4, ctas_per_sm=4, symmetric=True)
    seeds = list(range(len(SIZES)))
    q = [dev(p) for p in poss]
    U = [torch.zeros_like(t) for t in q]
    batch.run(q, U, [0] * len(SIZES), seeds, nsteps=2, lanczos_iters=16, delta=5e-3)
    k = 3
    qa, Ua = dev(poss[k]), torch.zeros(3 * SIZES[k], dtype=torch.float64, device="cuda")
    batch.run([qa], [Ua], [0], [seeds[k]], nsteps=2, lanczos_iters=16, delta=5e-3)
    assert torch.equal(qa, q[k]) and torch.equal(Ua, U[k])


def test_tune_picks_a_candidate_and_keeps_it(batch, data):
    poss = data[0]
    res = batch.tune([dev(p) for p in poss], reps=2)
    assert len(res["candidates"]) == len(CANDIDATES)
    assert all(ms > 0 for _, ms in res["candidates"])
    best = res["best"]
    assert best in CANDIDATES
    assert min(res["candidates"], key=lambda c: c[1])[0] == best
    assert batch.get_tiles() == best
