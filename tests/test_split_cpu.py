"""Sharing one suspension's products among processes (split.py), on the CPU with the gloo backend.

By target rows: the row ranges cover every target once on tile boundaries; with two ranks that each
compute their rows of the product with the FP64 oracle and all-gather them, the assembled product and a
5-iteration Lanczos square root built on it equal the one-rank results bit for bit (each row is the
same sum over the same sources whichever rank computes it).

By pairs: each rank takes an equal contiguous run of the upper triangle's (target tile, source tile)
units in row-major order -- both directions of each pair it holds, the diagonal units with their self
blocks -- from the oracle's dense mobility, and the all-reduce of the partial products gives every
rank the same vector, equal to the product within rounding; a 5-iteration Lanczos on it matches the
one-rank result."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1612_00474_gb300 import inputs  # noqa: E402
from paper_1612_00474_gb300.split import TILE, PairSplit, RowSplit, row_ranges  # noqa: E402


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


def _share_units(N, part, nparts):
    """The (target tile, source tile >= target tile) units of share `part`: the part-th of nparts equal
    contiguous runs of the triangle in row-major order."""
    nb = -(-N // TILE)
    units = [(b, t) for b in range(nb) for t in range(b, nb)]
    n = len(units)
    return units[n * part // nparts:n * (part + 1) // nparts]


def _share_product(M, v, N, part, nparts):
    """Partial product of share `part` from the dense 3N x 3N (particle-major) mobility M."""
    out = np.zeros(3 * N)
    for b, t in _share_units(N, part, nparts):
        rb = slice(3 * b * TILE, 3 * min(N, (b + 1) * TILE))
        rt = slice(3 * t * TILE, 3 * min(N, (t + 1) * TILE))
        out[rb] += M[rb, rt] @ v[rt]
        if t > b:  # the reversed pairs of the unit: the transposed blocks
            out[rt] += M[rt, rb] @ v[rb]
    return out


def _pair_worker(rank, world, port, N, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O

        pos = inputs.monolayer(N, seed=11)
        F = inputs.vectors(N, 12)
        M, _ = O.dense(pos)
        sp = PairSplit(N)

        def split_matvec(v):
            U = torch.zeros(3 * N, dtype=torch.float64)
            sp.product(lambda p_, f_, t_, r, w, o: o.copy_(torch.from_numpy(_share_product(M, v, N, r, w))), None,
                       None, None, U)
            return U.numpy().copy()

        U = split_matvec(F.ravel())
        W = O.noise(N, 5, 0, 0)
        g, m, eps, _ = O.lanczos_sqrt(pos, W, exact_iters=5, matvec=split_matvec)
        out[rank] = (U, g.ravel(), m, sp.mine)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_share_units_cover_triangle():
    for N, w in ((300, 2), (1000, 3), (129, 7)):
        nb = -(-N // TILE)
        allu = [u for p in range(w) for u in _share_units(N, p, w)]
        assert sorted(allu) == [(b, t) for b in range(nb) for t in range(b, nb)]


@pytest.mark.parametrize("N", [300, 513])
def test_pair_split_product_and_lanczos_two_ranks(N):
    import oracle as O

    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_pair_worker, args=(r, world, port, N, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    pos = inputs.monolayer(N, seed=11)
    F = inputs.vectors(N, 12)
    U_ref = O.mobility_apply(pos, F).ravel()
    g_ref, m_ref, _, _ = O.lanczos_sqrt(pos, O.noise(N, 5, 0, 0), exact_iters=5)
    assert out[0][3] == (0, 2) and out[1][3] == (1, 2)
    U0, g0, m0, _ = out[0]
    U1, g1, m1, _ = out[1]
    assert np.array_equal(U0, U1) and np.array_equal(g0, g1) and m0 == m1 == m_ref == 5  # every rank the same
    assert np.max(np.abs(U0 - U_ref)) <= 1e-13 * np.max(np.abs(U_ref))
    assert np.max(np.abs(g0 - g_ref.ravel())) <= 1e-12 * np.max(np.abs(g_ref))
