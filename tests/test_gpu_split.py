"""Products shared among processes (split.py over the product hook), on the GPU: by pairs
(rpb_mobility_apply_part, the shares summed by an all-reduce) and by target rows
(rpb_mobility_apply_rows, the rows all-gathered).

Two processes on the same GPU form a gloo group and exchange their shares or row blocks through host
memory (no kernel of one process waits on the other's); every product of their time steps -- the fused
velocity, the Lanczos products and the two RFD products -- is shared out, the rest of the step runs in
both.  Their states must stay equal to each other bit for bit, and match the single-process path and
the FP64 oracle within the parity tolerances (FP64 1e-10 on the products and U^n; the increment
within 1e-8 as the step tests; FP32 pairs 1e-5).  A one-process group takes the same hook path."""
import os
import socket

import numpy as np
import pytest

from paper_1612_00474_gb300 import inputs

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _dev(x):
    return torch.tensor(inputs.to_soa(x), dtype=torch.float64, device="cuda")


def _steps(c, N, precision, nsteps=2):
    pos0 = inputs.monolayer(N, seed=8)
    q = _dev(pos0)
    U = torch.zeros_like(q)
    delta = 1e-6 if precision == "fp64" else 5e-3
    ms = [c.ab_step(q, U, k, 4, dt=0.01, delta=delta, tol=1e-3)["m"] for k in range(nsteps)]
    F = _dev(inputs.vectors(N, 6))
    T = _dev(inputs.vectors(N, 7))
    P = c.mobility_apply(q, F, T)
    torch.cuda.synchronize()
    return q.cpu().numpy(), U.cpu().numpy(), ms, P.cpu().numpy()


def _worker(rank, world, port, N, precision, mode, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1612_00474_gb300.split import SplitContext

        sc = SplitContext(N, host_exchange=True, mode=mode, precision=precision, max_iter=32)
        try:
            out[rank] = _steps(sc, N, precision) + (sc.split(N).mine,)
        finally:
            sc.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["pairs", "rows"])
@pytest.mark.parametrize("N,precision", [(300, "fp64"), (700, "fp32")])
def test_split_two_processes_one_gpu(gpu_lib, N, precision, mode):
    import oracle as O

    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, N, precision, mode, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    q0, U0, m0, P0, rows0 = out[0]
    q1, U1, m1, P1, rows1 = out[1]
    assert rows0 != rows1
    assert np.array_equal(q0, q1) and np.array_equal(U0, U1) and m0 == m1 and np.array_equal(P0, P1)
    # the single-process path
    c = gpu_lib.Context(N, precision=precision, max_iter=32)
    try:
        q, U, m, P = _steps(c, N, precision)
    finally:
        c.close()
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert m == m0
    pos0 = inputs.monolayer(N, seed=8)
    assert np.max(np.abs(U0 - U)) / np.max(np.abs(U)) <= tol
    assert np.max(np.abs(P0 - P)) / np.max(np.abs(P)) <= tol
    inc, inc_ref = q0 - inputs.to_soa(pos0), q - inputs.to_soa(pos0)
    assert np.max(np.abs(inc - inc_ref)) / np.max(np.abs(inc_ref)) <= (1e-8 if precision == "fp64" else 5e-5)
    # the shared product against the oracle at the final positions
    qf = inputs.from_soa(q0, N)
    ref = O.mobility_apply(qf, inputs.vectors(N, 6), inputs.vectors(N, 7))
    assert np.max(np.abs(inputs.from_soa(P0, N) - ref)) / np.max(np.abs(ref)) <= tol


@pytest.mark.parametrize("mode", ["pairs", "rows"])
def test_split_one_process_hook(gpu_lib, mode):
    """Without a process group the hook computes the whole product itself: products equal the oracle's."""
    import oracle as O
    from paper_1612_00474_gb300.split import SplitContext

    N = 257
    pos = inputs.monolayer(N, seed=2)
    F, T = inputs.vectors(N, 3), inputs.vectors(N, 4)
    sc = SplitContext(N, mode=mode, precision="fp64", max_iter=16)
    try:
        got = inputs.from_soa(sc.mobility_apply(_dev(pos), _dev(F), _dev(T)).cpu().numpy(), N)
        with pytest.raises(AttributeError):
            sc.run
    finally:
        sc.close()
    ref = O.mobility_apply(pos, F, T)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-10
