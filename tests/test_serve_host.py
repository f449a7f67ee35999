"""Host logic of the continuous-batching server (no GPU): admission by memory budget and batch
limits in arrival order, retirement, latency accounting, the Poisson request generator."""
import math

import pytest

from paper_1612_00474_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


def _fake_run(requests, budget, max_batch, max_spheres, tick=0.01):
    clk = FakeClock()
    sched = serve.Scheduler(budget, max_batch, max_spheres)
    log = []

    def step(active):
        assert len(active) <= max_batch
        assert sum(r.N for r in active) <= max_spheres
        assert sum(serve.state_bytes(r.N) for r in active) <= budget
        log.append([r.rid for r in active])
        for r in active:
            r.step += 1
        clk.t += tick

    fin, busy, total = serve.run(requests, sched, step, lambda r: ("state", r.rid), lambda r: ("result", r.rid),
                                 clock=clk, sleep=clk.sleep)
    return fin, busy, total, log


def test_all_requests_complete_with_their_step_counts():
    reqs = [serve.Request(rid=k, N=100 * (k + 1), steps=3 + k, seed=k, arrival=0.005 * k) for k in range(6)]
    fin, busy, total, log = _fake_run(reqs, budget=10**9, max_batch=16, max_spheres=10**6)
    assert sorted(r.rid for r in fin) == list(range(6))
    for r in fin:
        assert r.step == r.steps and r.result == ("result", r.rid) and r.state is None
        assert sum(r.rid in ids for ids in log) == r.steps
        assert r.done >= r.arrival + r.steps * 0.01 - 1e-12
    assert busy == pytest.approx(total)


def test_late_arrivals_join_running_batch():
    reqs = [serve.Request(rid=0, N=100, steps=10, seed=0, arrival=0.0),
            serve.Request(rid=1, N=100, steps=2, seed=1, arrival=0.025)]
    fin, _, _, log = _fake_run(reqs, budget=10**9, max_batch=16, max_spheres=10**6)
    joint = [ids for ids in log if ids == [0, 1]]
    assert len(joint) == 2                      # request 1 ran alongside request 0
    assert log.index([0, 1]) == 3               # admitted at the first tick after it arrived


def test_memory_budget_and_fifo():
    b = serve.state_bytes(1000)
    reqs = [serve.Request(rid=k, N=1000, steps=2, seed=k, arrival=0.0) for k in range(5)]
    fin, _, _, log = _fake_run(reqs, budget=2 * b, max_batch=16, max_spheres=10**6)
    assert max(len(ids) for ids in log) == 2
    order = [r.rid for r in sorted(fin, key=lambda r: r.admitted)]
    assert order == [0, 1, 2, 3, 4]
    # a big request at the head blocks later small ones (no overtaking)
    reqs = [serve.Request(rid=0, N=1000, steps=4, seed=0, arrival=0.0),
            serve.Request(rid=1, N=1000, steps=1, seed=1, arrival=0.001),
            serve.Request(rid=2, N=10, steps=1, seed=2, arrival=0.002)]
    fin, _, _, _ = _fake_run(reqs, budget=serve.state_bytes(1500), max_batch=16, max_spheres=10**6)
    adm = {r.rid: r.admitted for r in fin}
    assert adm[2] >= adm[1] > adm[0]


def test_batch_limits_and_rejection():
    reqs = [serve.Request(rid=k, N=50, steps=1, seed=k, arrival=0.0) for k in range(7)]
    _, _, _, log = _fake_run(reqs, budget=10**9, max_batch=3, max_spheres=10**6)
    assert [len(x) for x in log] == [3, 3, 1]
    sched = serve.Scheduler(10**9, 4, 100)
    with pytest.raises(ValueError):
        sched.submit(serve.Request(rid=0, N=101, steps=1, seed=0, arrival=0.0))


def test_poisson_requests_and_percentile():
    reqs = serve.poisson_requests(4000, rate=5.0, seed=3)
    arr = [r.arrival for r in reqs]
    assert arr == sorted(arr) and arr[0] == 0.0
    assert all(128 <= r.N <= 32768 and 10 <= r.steps <= 200 for r in reqs)
    mean_gap = arr[-1] / (len(arr) - 1)
    assert abs(mean_gap - 0.2) < 0.02
    logN = [math.log(r.N) for r in reqs]
    assert abs(sum(logN) / len(logN) - (math.log(128) + math.log(32768)) / 2) < 0.1
    assert serve.percentile([1, 2, 3, 4], 50) == 2.5 and serve.percentile([5], 99) == 5
