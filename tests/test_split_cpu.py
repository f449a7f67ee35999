"""Sharing one suspension's products by target rows (split.py), on the CPU with the gloo backend.

The row ranges cover every target once on tile boundaries; with two ranks that each compute their
rows of the product with the FP64 oracle and all-gather them, the assembled product and a
5-iteration Lanczos square root built on it equal the one-rank results bit for bit (each row is the
same sum over the same sources whichever rank computes it)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1612_00474_gb300 import inputs  # noqa: E402
from paper_1612_00474_gb300.split import TILE, RowSplit, row_ranges  # noqa: E402


@pytest.mark.parametrize("N,world", [(1, 2), (128, 2), (129, 2), (300, 2), (1000, 3), (65536, 8), (200, 4)])
def test_row_ranges_cover_on_tiles(N, world):
    r = row_ranges(N, world)
    assert len(r) == world
    assert r[0][0] == 0 and r[-1][1] == N
    for (a, b), (c, _) in zip(r, r[1:]):
        assert b == c
    for a, b in r:
        assert a <= b and (a % TILE == 0 or a == b)  # an empty range (more ranks than tiles) may sit anywhere
    sizes = [-(-(b - a) // TILE) for a, b in r]
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rows_soa(pos, v, a, b):
    import oracle as O

    U = O.mobility_apply(pos, None if v is None else v.reshape(-1, 3), None, rows=(a, b))
    return torch.tensor(np.ascontiguousarray(U.T).ravel())


def _worker(rank, world, port, N, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O

        pos = inputs.monolayer(N, seed=11)
        F = inputs.vectors(N, 12)
        sp = RowSplit(N)

        def split_matvec(v):  # particle-major in and out, as the oracle's Lanczos takes it
            U = torch.zeros(3 * N, dtype=torch.float64)
            sp.product(lambda p_, f_, t_, a, b: _rows_soa(pos, v, a, b), None, None, None, U)
            return inputs.from_soa(U.numpy(), N).ravel()

        U = split_matvec(F.ravel())
        W = O.noise(N, 5, 0, 0)
        g, m, eps, _ = O.lanczos_sqrt(pos, W, exact_iters=5, matvec=split_matvec)
        out[rank] = (U, g.ravel(), m, sp.mine)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("N", [300, 513])
def test_split_product_and_lanczos_two_ranks(N):
    import oracle as O

    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, N, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    pos = inputs.monolayer(N, seed=11)
    F = inputs.vectors(N, 12)
    U_ref = O.mobility_apply(pos, F).ravel()
    g_ref, m_ref, _, _ = O.lanczos_sqrt(pos, O.noise(N, 5, 0, 0), exact_iters=5)
    assert out[0][3] != out[1][3]  # the ranks own different rows
    for r in range(world):
        U, g, m, _ = out[r]
        assert np.array_equal(U, U_ref)
        assert m == m_ref == 5
        assert np.array_equal(g, g_ref.ravel())
