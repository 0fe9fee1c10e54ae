"""One split of the norm-1 ADMM sharded over several ranks (Section IV, Table I).

The blocks of an M x N split are spread over a grid of Rr x Rc ranks: rank
(a, b) holds the row blocks of row group a and the column blocks of column
group b, as one library handle of that sub-matrix (``admm_shard_*`` in
include/admm.h).  Per iteration two sums cross ranks:

* the estimated data of Eq. (g_columns) / (g_rows_columns): per row, the sum
  over all column blocks of ghat_iq, reduced over the ranks holding the same
  rows (the row communicator) -- column splits only;
* the consensus average of Eq. (v_variable) / (v_variable_rows_columns): per
  column, the sum over all replicas of u^i + s^i, reduced over the ranks
  holding the same columns (the column communicator) -- row splits only.

Consensus (M, 1) therefore shards rows (Rr = ranks, one all-reduce of n
values), sectioning (1, N) shards columns (Rc = ranks, one all-reduce of m
values), and consensus-and-sectioning uses both sub-communicators, the
exchanges Table I counts.  The residual partials of every rank are summed
over all ranks.

A communicator has three collectives on lists of the local ranks' tensors
(sum in place): ``rows``, ``cols``, ``world``.  ``TorchComm`` runs one rank per
process over torch.distributed; ``LocalComm`` runs every rank in one process
(each rank's engine a handle of its own) and sums directly.  The per-rank
work is the engine's: ``CudaShardEngine`` calls the library.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import _binding as B


def balanced(total: int, parts: int) -> list[tuple[int, int]]:
    """Contiguous [start, stop) ranges, sizes differing by at most one, larger first."""
    base, extra = divmod(total, parts)
    out, start = [], 0
    for p in range(parts):
        size = base + (1 if p < extra else 0)
        out.append((start, start + size))
        start += size
    return out


def default_grid(M: int, N: int, world: int, m: int, n: int) -> tuple[int, int]:
    """Rr x Rc = world ranks for an M x N split of an m x n problem: all ranks
    on the row blocks for consensus, on the column blocks for sectioning; for
    both, the factorisation with Rr <= M and Rc <= N whose ranks exchange the
    fewest elements per iteration, counted as in Table I: m / Rr estimated data
    when Rc > 1, and 2 n / Rc (replica out, consensus back) when Rr > 1."""
    if N == 1:
        if world > M:
            raise ValueError("more ranks than row blocks")
        return world, 1
    if M == 1:
        if world > N:
            raise ValueError("more ranks than column blocks")
        return 1, world
    best = None
    for Rr in range(1, world + 1):
        if world % Rr:
            continue
        Rc = world // Rr
        if Rr > M or Rc > N:
            continue
        cost = (m / Rr if Rc > 1 else 0.0) + (2.0 * n / Rc if Rr > 1 else 0.0)
        if best is None or cost < best[0]:
            best = (cost, Rr, Rc)
    if best is None:
        raise ValueError("no rank grid fits the split")
    return best[1], best[2]


@dataclass
class ShardLayout:
    """The blocks of rank `rank` in an Rr x Rc grid over the M x N split of an m x n problem."""

    m: int
    n: int
    M: int
    N: int
    Rr: int
    Rc: int
    rank: int

    def __post_init__(self):
        if self.Rr * self.Rc < 1 or not 0 <= self.rank < self.Rr * self.Rc:
            raise ValueError("bad rank grid")
        self.row_group, self.col_group = divmod(self.rank, self.Rc)
        self.blocks_i = balanced(self.M, self.Rr)[self.row_group]
        self.blocks_j = balanced(self.N, self.Rc)[self.col_group]
        ro = [0] + [b for _, b in balanced(self.m, self.M)]
        co = [0] + [b for _, b in balanced(self.n, self.N)]
        self.rows = (ro[self.blocks_i[0]], ro[self.blocks_i[1]])
        self.cols = (co[self.blocks_j[0]], co[self.blocks_j[1]])
        self.M_loc = self.blocks_i[1] - self.blocks_i[0]
        self.N_loc = self.blocks_j[1] - self.blocks_j[0]

    @property
    def world(self) -> int:
        return self.Rr * self.Rc

    def row_peers(self) -> list[int]:
        """Ranks holding the same rows (the estimated-data exchange)."""
        return [self.row_group * self.Rc + b for b in range(self.Rc)]

    def col_peers(self) -> list[int]:
        """Ranks holding the same columns (the consensus average)."""
        return [a * self.Rc + self.col_group for a in range(self.Rr)]


class TorchComm:
    """One rank per process over torch.distributed (NCCL with device tensors,
    gloo through host copies).  Creates every row and column sub-group (each
    rank must construct it, in the same order)."""

    def __init__(self, layout: ShardLayout):
        import torch.distributed as dist
        self.dist = dist
        self.layout = layout
        self.rows_group = self.cols_group = None
        for a in range(layout.Rr):
            g = dist.new_group([a * layout.Rc + b for b in range(layout.Rc)])
            if a == layout.row_group:
                self.rows_group = g
        for b in range(layout.Rc):
            g = dist.new_group([a * layout.Rc + b for a in range(layout.Rr)])
            if b == layout.col_group:
                self.cols_group = g
        self.host = dist.get_backend() != "nccl"

    def _reduce(self, tensors, group):
        import torch
        for t in tensors:
            on_device = not self.host   # NCCL reduces device tensors, gloo host tensors
            x = t if t.is_cuda == on_device else (t.cuda() if on_device else t.cpu())
            r = torch.view_as_real(x) if x.is_complex() else x
            self.dist.all_reduce(r, op=self.dist.ReduceOp.SUM, group=group)
            if x is not t:
                t.copy_(x)

    def rows(self, tensors):
        self._reduce(tensors, self.rows_group)

    def cols(self, tensors):
        self._reduce(tensors, self.cols_group)

    def world(self, tensors):
        self._reduce(tensors, None)


class LocalComm:
    """Every rank of the grid in this process: the list holds one tensor per
    rank, in rank order, and each collective sums over the peers directly."""

    def __init__(self, layouts: list[ShardLayout]):
        self.layouts = layouts

    def _reduce(self, tensors, peers_of):
        sums = {}
        for lay, t in zip(self.layouts, tensors):
            key = tuple(peers_of(lay))
            sums[key] = t.clone() if key not in sums else sums[key] + t
        for lay, t in zip(self.layouts, tensors):
            t.copy_(sums[tuple(peers_of(lay))])

    def rows(self, tensors):
        self._reduce(tensors, ShardLayout.row_peers)

    def cols(self, tensors):
        self._reduce(tensors, ShardLayout.col_peers)

    def world(self, tensors):
        self._reduce(tensors, lambda lay: list(range(lay.world)))


class CudaShardEngine:
    """The blocks of one rank on its GPU: a library handle of the rank's
    sub-matrix (its row blocks and column blocks) in sharded mode."""

    def __init__(self, H, g, layout: ShardLayout, lam: float, rho: float, stream=None):
        import torch
        from .solver import Solver
        self._torch = torch
        r0, r1 = layout.rows
        c0, c1 = layout.cols
        if isinstance(H, np.ndarray):
            H, g = torch.from_numpy(np.ascontiguousarray(H)), torch.from_numpy(np.ascontiguousarray(g))
        Hl = H[r0:r1, c0:c1].contiguous()
        gl = g[r0:r1].contiguous()
        self.layout = layout
        self.stream = stream
        self.solver = Solver(Hl, gl, layout.M_loc, layout.N_loc, lam, rho, stream=stream)
        B.admm_shard_enable(self.solver.h, layout.M, stream)
        self.m, self.n = r1 - r0, c1 - c0
        dev = Hl.device if Hl.is_cuda else "cuda"
        self.t = torch.empty(self.m, dtype=torch.complex64, device=dev)
        self.S = torch.empty(self.n, dtype=torch.complex64, device=dev)

    def ghat_sum(self):
        B.admm_shard_ghat_sum(self.solver.h, self.t, self.stream)
        self._sync()
        return self.t

    def set_exchange(self, t) -> None:
        B.admm_shard_set_exchange(self.solver.h, t, self.stream)

    def ustep(self):
        B.admm_shard_ustep(self.solver.h, self.S, self.stream)
        self._sync()
        return self.S

    def vstep(self, S) -> np.ndarray:
        return B.admm_shard_vstep(self.solver.h, S, self.stream)

    def _sync(self):
        st = self.stream
        if st is not None and isinstance(st, self._torch.cuda.Stream):
            st.synchronize()
        else:
            self._torch.cuda.synchronize()

    def v(self):
        return self.solver.v()

    def state(self):
        return self.solver.state()

    def close(self) -> None:
        self.solver.close()


class ShardedSolver:
    """Runs the sharded iteration over the local ranks `parts` = [(layout,
    engine), ...] (one per process with TorchComm; all of them with
    LocalComm).  ``hist`` holds the whole problem's residual records, (||r_p||^2,
    ||r_d||^2, ||u||^2, ||v||^2, ||s||^2) stacked as in the unsharded split."""

    def __init__(self, parts, comm, rho: float):
        self.parts = list(parts)
        self.comm = comm
        self.rho = float(rho)
        lay = self.parts[0][0]
        self.M, self.N = lay.M, lay.N
        self.hist = []

    def iterate(self, iters: int = 1) -> "ShardedSolver":
        import torch
        for _ in range(int(iters)):
            if self.N > 1:
                ts = [e.ghat_sum() for _, e in self.parts]
                self.comm.rows(ts)
                for (_, e), t in zip(self.parts, ts):
                    e.set_exchange(t)
            Ss = [e.ustep() for _, e in self.parts]
            self.comm.cols(Ss)
            recs = []
            for (lay, e), S in zip(self.parts, Ss):
                r = e.vstep(S)
                if lay.row_group != 0:   # v is held by every row group: count it once
                    r[1] = r[3] = 0.0
                recs.append(torch.from_numpy(r))
            self.comm.world(recs)
            r = recs[0].numpy()
            self.hist.append((r[0], self.rho * self.rho * self.M * r[1], r[2], self.M * r[3], r[4]))
        return self

    def residuals(self) -> np.ndarray:
        return np.array(self.hist, dtype=np.float64).reshape(-1, 5)
