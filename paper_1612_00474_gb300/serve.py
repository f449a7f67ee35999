"""Continuous-batching server for Brownian-dynamics trajectory requests.

A request asks for `steps` stochastic Adams-Bashforth steps of one suspension (N spheres, its own
Philox seed).  Requests arrive at any time; the server keeps every admitted request's state (positions
and the previous deterministic velocity U^{n-1}) resident on the device and, at every tick, advances
all admitted requests by one step with a single batched call (rpb_batch_ab_step).  A request that
arrives while others are running is admitted at the next tick if the device-memory budget and the
batch limits allow it, so its work overlaps theirs on the GPU; finished requests leave at the end of
the tick and free their memory.

Each request is advanced with its own seed and step counter and the batched library computes every
instance independently of its companions, so a request's trajectory is the same whether it runs alone
or in a mix (see tests/test_gpu_serve.py).

The scheduling logic (Scheduler) is pure host code: the GPU step and the device buffers are supplied
by the caller, which lets the admission and retirement rules be tested without a GPU.
"""
import collections
import dataclasses
import math
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    N: int
    steps: int
    seed: int
    arrival: float                      # seconds since the start of the run
    pos0: object = None                 # initial positions, host (N, 3) float64
    # filled by the server
    admitted: float = math.nan
    done: float = math.nan
    step: int = 0                       # steps taken so far
    state: object = None                # device state (implementation defined)
    result: object = None               # final positions, host (N, 3)
    lanczos_m: list = dataclasses.field(default_factory=list)

    @property
    def latency(self):
        return self.done - self.arrival


def state_bytes(N):
    """Device bytes a request holds while admitted: positions and U^{n-1}, float64 SoA."""
    return 2 * 3 * 8 * int(N)


class Scheduler:
    """First-come-first-served admission into a continuously batched set of running requests.

    budget_bytes: device memory the admitted requests' state may occupy.
    max_batch / max_spheres: limits of the batch context (instances and total spheres per call).
    A request larger than the limits on its own is rejected at submission (ValueError)."""

    def __init__(self, budget_bytes, max_batch, max_spheres):
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.max_spheres = int(max_spheres)
        self.queue = collections.deque()
        self.active = []
        self.finished = []
        self.used_bytes = 0
        self.used_spheres = 0

    def submit(self, req):
        if req.N > self.max_spheres or state_bytes(req.N) > self.budget:
            raise ValueError(f"request {req.rid} (N={req.N}) can never be admitted")
        self.queue.append(req)

    def admit(self, now, allocate):
        """Move queued requests (in arrival order) into the active set while they fit; allocate(req)
        creates the device state.  Stops at the first request that does not fit (no overtaking)."""
        admitted = []
        while self.queue:
            r = self.queue[0]
            fits = (len(self.active) < self.max_batch and self.used_spheres + r.N <= self.max_spheres
                    and self.used_bytes + state_bytes(r.N) <= self.budget)
            if not fits:
                break
            self.queue.popleft()
            r.state = allocate(r)
            r.admitted = now
            self.active.append(r)
            self.used_bytes += state_bytes(r.N)
            self.used_spheres += r.N
            admitted.append(r)
        return admitted

    def retire(self, now, finalize):
        """Remove requests that have taken all their steps; finalize(req) copies the result out and
        releases the device state."""
        done = [r for r in self.active if r.step >= r.steps]
        for r in done:
            r.result = finalize(r)
            r.state = None
            r.done = now
            self.used_bytes -= state_bytes(r.N)
            self.used_spheres -= r.N
            self.finished.append(r)
        self.active = [r for r in self.active if r.step < r.steps]
        return done

    def idle(self):
        return not self.active and not self.queue


def run(requests, scheduler, step_fn, allocate, finalize, clock=time.perf_counter, sleep=time.sleep,
        realtime=True):
    """Serve `requests` (sorted by arrival) to completion.

    step_fn(active) advances every active request by one step (and increments req.step);
    allocate / finalize as in Scheduler.  With realtime=True arrivals follow the wall clock (the
    server waits for the next arrival when it is idle); otherwise time jumps to the next arrival.
    Returns (finished requests, busy seconds, total seconds)."""
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    t0 = clock()
    busy = 0.0
    offset = 0.0

    def now():
        return clock() - t0 + offset

    while pending or not scheduler.idle():
        t = now()
        while pending and pending[0].arrival <= t:
            scheduler.submit(pending.popleft())
        scheduler.admit(t, allocate)
        if not scheduler.active:
            if pending:
                wait = pending[0].arrival - now()
                if wait > 0:
                    if realtime:
                        sleep(wait)
                    else:
                        offset += wait
            continue
        ts = clock()
        step_fn(scheduler.active)
        busy += clock() - ts
        scheduler.retire(now(), finalize)
    return scheduler.finished, busy, now()


def poisson_requests(n, rate, seed=0, n_lo=128, n_hi=32768, steps_lo=10, steps_hi=200):
    """n requests with exponential inter-arrival times (rate per second), N log-uniform in
    [n_lo, n_hi] and a uniform number of steps in [steps_lo, steps_hi]; seeded."""
    rng = np.random.Generator(np.random.Philox(key=30_000 + seed))
    gaps = rng.exponential(1.0 / rate, n)
    arrivals = np.cumsum(gaps) - gaps[0]
    Ns = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi + 1), n))).astype(int).clip(n_lo, n_hi)
    steps = rng.integers(steps_lo, steps_hi + 1, n)
    return [Request(rid=k, N=int(Ns[k]), steps=int(steps[k]), seed=1000 + k, arrival=float(arrivals[k]))
            for k in range(n)]


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return math.nan
    k = (len(xs) - 1) * q / 100.0
    lo, hi = math.floor(k), math.ceil(k)
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


class GpuServer:
    """The GPU side of the server: a batch context plus per-request device state."""

    def __init__(self, max_batch, max_spheres, precision="fp32", dt=0.01, delta=5e-3, tol=1e-3, max_iter=64,
                 force=dict(weight=1.0, U0=1.0, b=0.1, torque=(0.0, 1.0, 0.0))):
        from . import rpb

        self.bt = rpb.BatchContext(max_total_N=max_spheres, max_B=max_batch, precision=precision, max_iter=max_iter)
        self.kw = dict(dt=dt, delta=delta, tol=tol, max_iter=max_iter, **force)
        self.pairs = 0.0

    def allocate(self, r):
        import torch

        from .inputs import monolayer, to_soa

        pos0 = r.pos0 if r.pos0 is not None else monolayer(r.N, seed=r.seed)
        q = torch.tensor(to_soa(pos0), dtype=torch.float64, device="cuda")
        return (q, torch.zeros_like(q))

    def finalize(self, r):
        from .inputs import from_soa

        return from_soa(r.state[0].cpu().numpy(), r.N)

    def step(self, active):
        stats = self.bt.ab_step([r.state[0] for r in active], [r.state[1] for r in active], [r.step for r in active],
                                [r.seed for r in active], **self.kw)
        for r, s in zip(active, stats):
            r.step += 1
            r.lanczos_m.append(s["m"])
            self.pairs += float(r.N) * r.N * (3 + s["m"])

    def close(self):
        self.bt.close()
