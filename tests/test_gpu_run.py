"""Graph-replayed runs of one suspension (rpb_run) against repeated host-driven steps (rpb_step).

rpb_run captures a step once into a CUDA graph whose Lanczos iterations after the first are
conditional nodes decided on the device, and replays it; the kernels, arguments and order are those
of rpb_step, so K replayed steps must equal K calls of rpb_step bit for bit, Lanczos dimension and
stopping included.  One case also compares the run with the FP64 oracle at the AB-step tolerance.
"""
import numpy as np
import pytest

import oracle as O
from paper_1612_00474_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def dev(x):
    return torch.tensor(inputs.to_soa(x), dtype=torch.float64, device="cuda")


def _pair(gpu_lib, N, precision, kT=1.0, max_iter=32, periodic=None, precondition=False, wall=True):
    cs = []
    for _ in range(2):
        c = gpu_lib.Context(max_N=N, precision=precision, kT=kT, max_iter=max_iter, wall=wall)
        if periodic:
            c.set_periodic(*periodic)
        if precondition:
            c.set_preconditioner("block-diagonal")
        cs.append(c)
    return cs


def _compare(gpu_lib, N, precision, nsteps=3, step0=0, scheme="AB", rfd="centred", kT=1.0, periodic=None,
             precondition=False, delta=None, seed=3):
    delta = delta or (1e-6 if precision == "fp64" else 5e-3)
    c_step, c_run = _pair(gpu_lib, N, precision, kT=kT, periodic=periodic, precondition=precondition)
    try:
        pos0 = inputs.monolayer(N, seed=seed)
        qa, qb = dev(pos0), dev(pos0)
        Ua = torch.zeros_like(qa)
        Ub = torch.zeros_like(qb)
        kw = dict(scheme=scheme, rfd=rfd, dt=0.01, delta=delta, tol=1e-3)
        if step0 > 0:  # a U^{n-1} from an earlier step, the same for both
            c_step.step(qa, Ua, step0 - 1, seed, **kw)
            qb.copy_(qa)
            Ub.copy_(Ua)
        ms = []
        for k in range(nsteps):
            ms.append(c_step.step(qa, Ua, step0 + k, seed, **kw)["m"])
        st, unconv = c_run.run(qb, Ub, step0, seed, nsteps, **kw)
        torch.cuda.synchronize()
        assert unconv == 0
        assert st["m"] == ms[-1]
        assert torch.equal(qa, qb), float((qa - qb).abs().max())
        assert torch.equal(Ua, Ub), float((Ua - Ub).abs().max())
        return ms
    finally:
        c_step.close()
        c_run.close()


@pytest.mark.parametrize("N,precision", [(256, "fp64"), (600, "fp32"), (100, "fp32")])
def test_run_equals_steps(gpu_lib, N, precision):
    ms = _compare(gpu_lib, N, precision)
    assert all(m >= 2 for m in ms)


def test_run_later_steps_and_em_one_sided(gpu_lib):
    _compare(gpu_lib, 300, "fp64", step0=4)
    _compare(gpu_lib, 300, "fp32", scheme="EM", rfd="one-sided")


def test_run_deterministic_preconditioned_periodic(gpu_lib):
    _compare(gpu_lib, 200, "fp64", kT=0.0)
    _compare(gpu_lib, 700, "fp32", precondition=True)
    L = float(np.sqrt(300 * np.pi / 0.4))
    _compare(gpu_lib, 300, "fp32", periodic=(L, L))


def test_run_unconverged_count(gpu_lib):
    N = 128
    c = gpu_lib.Context(max_N=N, precision="fp64", max_iter=8)
    try:
        q = dev(inputs.monolayer(N, seed=1))
        U = torch.zeros_like(q)
        st, unconv = c.run(q, U, 0, 1, 4, tol=1e-14, max_iter=2, raise_on_noconv=False)
        assert unconv == 4 and st["m"] == 2 and not st["converged"]
        with pytest.raises(gpu_lib.NoConvergence):
            c.run(q, U, 4, 1, 1, tol=1e-14, max_iter=2)
    finally:
        c.close()


def test_run_against_oracle_n256(gpu_lib):
    """Two replayed AB steps of the 256-sphere FP64 configuration against two oracle steps (the
    increment within 1e-8, the velocity U^n within 1e-10; equal Lanczos dimension)."""
    N = 256
    pos0 = inputs.monolayer(N, seed=0)
    c = gpu_lib.Context(max_N=N, precision="fp64", max_iter=32)
    try:
        q, U = dev(pos0), torch.zeros(3 * N, dtype=torch.float64, device="cuda")
        st, _ = c.run(q, U, 0, 0, 2, dt=0.01, delta=1e-6, tol=1e-3)
        q1, U1, i1 = O.ab_step(pos0, None, 0, seed=0, dt=0.01, delta=1e-6, tol=1e-3)
        q2, U2, i2 = O.ab_step(q1, U1, 1, seed=0, dt=0.01, delta=1e-6, tol=1e-3)
        assert st["m"] == i2["m"]
        got_q = inputs.from_soa(q.cpu().numpy(), N)
        got_U = inputs.from_soa(U.cpu().numpy(), N)
        assert np.max(np.abs(got_U - U2)) / np.max(np.abs(U2)) <= 1e-10
        assert np.max(np.abs((got_q - pos0) - (q2 - pos0))) / np.max(np.abs(q2 - pos0)) <= 1e-8
    finally:
        c.close()


def test_run_with_falling_lanczos_dimension(gpu_lib):
    """rpb_run runs all its steps from one graph launch (a loop node around the step), and a conditional
    node's condition keeps its value from one pass of the loop to the next, so each step clears the
    Lanczos iterations' conditions first: a step that stops earlier than the one before must not run
    the later iterations again.  A run whose host-driven Lanczos dimension falls from one step to the
    next is compared bit for bit."""
    for seed in range(10):
        ms = _compare(gpu_lib, 64, "fp64", nsteps=10, seed=seed)
        if any(b < a for a, b in zip(ms, ms[1:])):
            return
    pytest.fail("no run with a falling Lanczos dimension among 10 seeds")
