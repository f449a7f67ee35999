"""One suspension shared among processes (one per GPU).

The product U = M_tt F + M_tr T is a direct summation over all pairs (Sec. II.B).  Two ways of
sharing it out:

  - by pairs (mode "pairs", PairSplit): the symmetric pass evaluates each unordered pair once, both of
    its directions (M_ji = M_ij^T); process r of a group of W evaluates the r-th of W equal contiguous
    runs of the triangle's (target tile, source tile) units with rpb_mobility_apply_part, which gives
    a partial product over all rows, and an all-reduce sums the W partials.  The W processes share one
    symmetric pass: the pair work per process is 1/W of the single-GPU product's.
  - by target rows (mode "rows", RowSplit): process r owns a contiguous range of target rows (whole
    128-row tiles), computes them with rpb_mobility_apply_rows (one-way kernels: every ordered pair,
    twice the symmetric pass's pair evaluations) and an all-gather assembles the rows.

A SplitContext installs either as the context's product hook (rpb_set_product_hook), so every product
of a time step -- the fused velocity, each Lanczos product of Sec. II.C and the two RFD products of
Sec. II.A -- is shared out, while the rest of the step (forces, noise, the Lanczos recurrence with its
float64 Gram-Schmidt and tridiagonal square root, the drift and the update) runs unchanged in every
process on the identical assembled vectors (an all-reduce and an all-gather give every process the
same values), so every process's state stays bitwise equal.

The exchange uses the group's backend: NCCL on device tensors, or, with host_exchange=True, any
backend (gloo) through host copies.  Only argument marshalling and data movement happen here; the
arithmetic runs in the library's kernels (the all-reduce's sum is the collective's).
"""
import torch
import torch.distributed as dist

from . import rpb

TILE = 128


def row_ranges(N, world, tile=TILE):
    """[(row0, row1)] of each of `world` processes: contiguous, starting on a tile boundary, as equal as
    whole tiles allow (a process may get none when there are fewer tiles than processes)."""
    tiles = -(-int(N) // tile)
    base, extra = divmod(tiles, world)
    out, t = [], 0
    for r in range(world):
        k = base + (1 if r < extra else 0)
        out.append((min(N, t * tile), min(N, (t + k) * tile)))
        t += k
    return out


class RowSplit:
    """The row ranges of a group and the all-gather of row blocks into full SoA vectors."""

    def __init__(self, N, group=None, host_exchange=False):
        self.N = int(N)
        self.group = group
        on = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank(group) if on else 0
        self.world = dist.get_world_size(group) if on else 1
        self.ranges = row_ranges(self.N, self.world)
        self.rows = max(1, max(b - a for a, b in self.ranges))
        self.host_exchange = host_exchange

    @property
    def mine(self):
        return self.ranges[self.rank]

    def gather(self, local, out):
        """local: this process's rows, a (3 nr,) SoA tensor; out: (3N,) SoA, filled with every process's rows."""
        a, b = self.mine
        nr = b - a
        buf = torch.zeros((3, self.rows), dtype=out.dtype, device=out.device)
        if nr > 0:
            buf[:, :nr] = local.view(3, nr)
        if self.world == 1:
            parts = [buf]
        else:
            src = buf.cpu() if self.host_exchange else buf
            parts = [torch.empty_like(src) for _ in range(self.world)]
            dist.all_gather(parts, src, group=self.group)
        full = out.view(3, self.N)
        for r, (ra, rb) in enumerate(self.ranges):
            if rb > ra:
                full[:, ra:rb].copy_(parts[r][:, :rb - ra])
        return out

    def product(self, rows_fn, pos, F, T, out):
        """out = the full product, from rows_fn(pos, F, T, row0, row1) -> this process's rows."""
        a, b = self.mine
        local = rows_fn(pos, F, T, a, b) if b > a else None
        return self.gather(local, out)


class PairSplit:
    """Shares of the triangle's pairs (rpb_mobility_apply_part) and the all-reduce that sums them."""

    def __init__(self, N, group=None, host_exchange=False):
        self.N = int(N)
        self.group = group
        on = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank(group) if on else 0
        self.world = dist.get_world_size(group) if on else 1
        self.host_exchange = host_exchange

    @property
    def mine(self):
        return (self.rank, self.world)

    def reduce(self, share):
        """share: this process's partial product, a (3N,) tensor, replaced in place by the sum over the group."""
        if self.world == 1:
            return share
        if self.host_exchange:
            h = share.cpu()
            dist.all_reduce(h, group=self.group)
            share.copy_(h)
        else:
            dist.all_reduce(share, group=self.group)
        return share

    def product(self, part_fn, pos, F, T, out):
        """out = the full product, from part_fn(pos, F, T, part, nparts, out) -> this process's share in out."""
        part_fn(pos, F, T, self.rank, self.world, out)
        return self.reduce(out)


class _DevPtr:
    """A float64 device vector at a raw address, for torch.as_tensor (no copy)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _wrap(ptr, n):
    return torch.as_tensor(_DevPtr(ptr, n), device="cuda") if ptr else None


class SplitContext:
    """A library context whose products are shared among the processes of a group, by pairs (mode
    "pairs", the default) or by target rows (mode "rows").

    The methods are those of rpb.Context (mobility_apply, lanczos_sqrt_apply, rfd_drift, ab_step, step,
    forces, philox_normal, ...): every process calls them with the same arguments and gets the same
    results.  rpb_run (graph replay) is not available with a shared product."""

    MODES = ("pairs", "rows")

    def __init__(self, max_N, group=None, host_exchange=False, mode="pairs", **ctx_kwargs):
        if mode not in self.MODES:
            raise ValueError(f"mode must be one of {self.MODES}")
        self.ctx = rpb.Context(max_N, **ctx_kwargs)
        self.group = group
        self.host_exchange = host_exchange
        self.mode = mode
        self._split = {}
        self.error = None
        self.ctx.set_product_hook(self._product)

    def split(self, N):
        if N not in self._split:
            cls = PairSplit if self.mode == "pairs" else RowSplit
            self._split[N] = cls(N, self.group, self.host_exchange)
        return self._split[N]

    def _product(self, N, pos_p, F_p, T_p, U_p):
        try:
            n = 3 * N
            sp = self.split(N)
            pos, F, T, U = _wrap(pos_p, n), _wrap(F_p, n), _wrap(T_p, n), _wrap(U_p, n)
            if self.mode == "pairs":
                sp.product(lambda p_, f_, t_, r, w, o: self.ctx.mobility_apply_part(p_, f_, t_, r, w, out=o), pos, F,
                           T, U)
            else:
                sp.product(lambda p_, f_, t_, a, b: self.ctx.mobility_apply_rows(p_, f_, t_, a, b), pos, F, T, U)
            return rpb.RPB_OK
        except Exception as e:  # reported to the library as a failed product
            self.error = e
            return rpb.RPB_ECUDA

    def __getattr__(self, name):
        if name == "run":
            raise AttributeError("graph-replayed runs (rpb_run) are not available with a shared product")
        return getattr(self.ctx, name)

    def close(self):
        self.ctx.set_product_hook(None)
        self.ctx.close()
