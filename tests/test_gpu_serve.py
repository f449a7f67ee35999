"""The server on the GPU: requests that overlap in time on the device give the same trajectory as
each request served alone (FP32 pairs; same seeds and step counters), and they agree with the
single-suspension path to the FP32 tolerance."""
import numpy as np
import pytest

from paper_1612_00474_gb300 import inputs, serve

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _serve(reqs):
    srv = serve.GpuServer(max_batch=8, max_spheres=4096, precision="fp32", delta=5e-3)
    try:
        sched = serve.Scheduler(budget_bytes=1 << 30, max_batch=8, max_spheres=4096)
        fin, busy, total = serve.run(reqs, sched, srv.step, srv.allocate, srv.finalize, realtime=False)
    finally:
        srv.close()
    return {r.rid: r for r in fin}


def _reqs(arrivals):
    spec = [(300, 5), (1000, 3), (64, 8), (517, 4)]
    return [serve.Request(rid=k, N=N, steps=s, seed=40 + k, arrival=a) for k, ((N, s), a) in enumerate(zip(spec, arrivals))]


def test_alone_equals_mixed(gpu_lib):
    mixed = _serve(_reqs([0.0, 0.0, 0.0, 0.0]))
    for k in range(4):
        alone = _serve([_reqs([0.0] * 4)[k]])[k]
        m = mixed[k]
        assert m.lanczos_m == alone.lanczos_m
        ref = np.abs(alone.result - inputs.monolayer(m.N, seed=m.seed)).max()
        assert np.abs(m.result - alone.result).max() <= 1e-12 * max(ref, 1.0), k


def test_served_equals_single_path(gpu_lib):
    fin = _serve(_reqs([0.0, 0.01, 0.02, 0.03]))
    r = fin[1]
    ctx = gpu_lib.Context(max_N=r.N, precision="fp32", max_iter=64)
    try:
        pos0 = inputs.monolayer(r.N, seed=r.seed)
        q = torch.tensor(inputs.to_soa(pos0), dtype=torch.float64, device="cuda")
        U = torch.zeros_like(q)
        for s in range(r.steps):
            ctx.ab_step(q, U, s, r.seed, delta=5e-3)
        single = inputs.from_soa(q.cpu().numpy(), r.N)
    finally:
        ctx.close()
    disp = np.abs(single - pos0).max()
    assert np.abs(r.result - single).max() <= 1e-5 * disp
