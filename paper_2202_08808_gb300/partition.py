"""Row-sharded dynamic SpGEMM over several ranks (host-side plan and exchange).

The paper distributes A, B and C over a 2D process grid and moves only the
hypersparse update matrices between processes (Section 5.1: the update
matrices are broadcast, never B' or A).  On GPUs the natural split is 1D:

* rows of A and of C are cut into contiguous blocks, one per rank, balanced
  by the number of entries of A;
* B is replicated on every rank (when C = A A, each rank holds all of A as
  its B and its own block of rows as its A);
* the one exchange per batch is an allgather of the batch itself: each rank
  passes the slice of the batch it received, the slices are concatenated in
  rank order (which keeps the batch's arrival order when the caller cut it
  into consecutive pieces), and every rank then applies the whole batch to
  its copy of B and the entries of its own rows to its block of A.

A rank's block is then an ordinary instance C_r = A_r B with a separate B:
its affected rows are rows(A_r*) u {i : A_r(i,k) != 0, k in rows(B*)}, which
are exactly the rows of the full R that the rank owns, and its recompute and
splice touch only its own rows.  The per-rank step is one call of the
library (``DynamicSpGEMM(A_r, B).apply_batch(local, full)``); this module
plans the blocks, routes and exchanges the batches, and has no arithmetic
of the method itself.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .dspg import CsrArrays as CSR


@dataclass
class Batch:
    """An update list in arrival order (row/col int32, val, op uint8), as
    apply_batch takes it."""

    row: np.ndarray
    col: np.ndarray
    val: np.ndarray
    op: np.ndarray

    def __len__(self) -> int:
        return int(self.row.shape[0])


class RowPartition:
    """Contiguous row blocks [lo_r, hi_r) of an n-row matrix for `world`
    ranks, balanced by the given per-row weights (entries of A; equal rows
    when weights is None)."""

    def __init__(self, nrows: int, world: int, weights: np.ndarray | None = None):
        if world < 1:
            raise ValueError("world must be >= 1")
        self.nrows, self.world = int(nrows), int(world)
        if weights is None or nrows == 0:
            cuts = [(self.nrows * r) // world for r in range(world + 1)]
        else:
            w = np.asarray(weights, dtype=np.float64) + 1.0  # an empty row still costs its header
            pre = np.concatenate([[0.0], np.cumsum(w)])
            targets = pre[-1] * np.arange(world + 1) / world
            cuts = np.searchsorted(pre, targets, side="left").tolist()
            cuts[0], cuts[-1] = 0, self.nrows
            for r in range(1, world + 1):  # monotone
                cuts[r] = max(cuts[r], cuts[r - 1])
        self.bounds = np.array(cuts, dtype=np.int64)

    def block(self, rank: int) -> tuple[int, int]:
        return int(self.bounds[rank]), int(self.bounds[rank + 1])

    def owner(self, rows) -> np.ndarray:
        """Rank owning each row index."""
        return np.searchsorted(self.bounds, np.asarray(rows, dtype=np.int64), side="right") - 1


def shard_rows(M, lo: int, hi: int) -> CSR:
    """Rows [lo, hi) of M as an (hi - lo)-row CSR with M's column indices."""
    a, b = int(M.rowptr[lo]), int(M.rowptr[hi])
    return CSR(hi - lo, M.ncols, (np.asarray(M.rowptr[lo:hi + 1]) - a).astype(np.int64),
               np.asarray(M.col[a:b]), np.asarray(M.val[a:b]))


def split_in_order(batch, world: int) -> list[Batch]:
    """The batch cut into `world` consecutive pieces (arrival order kept):
    what each rank receives before the exchange."""
    cuts = [(len(batch) * r) // world for r in range(world + 1)]
    return [Batch(batch.row[a:b], batch.col[a:b], batch.val[a:b], batch.op[a:b]) for a, b in zip(cuts, cuts[1:])]


def local_entries(batch, part: RowPartition, rank: int) -> Batch:
    """The entries of `batch` in rank's rows, arrival order kept, with rows
    renumbered from the block's first row (the rank's A block is local)."""
    lo, hi = part.block(rank)
    m = (batch.row >= lo) & (batch.row < hi)
    return Batch((batch.row[m] - lo).astype(np.int32), batch.col[m], batch.val[m], batch.op[m])


def allgather_batch(piece, group=None) -> Batch:
    """Every rank's piece, concatenated in rank order (torch.distributed
    all_gather of the piece's sizes, then of its padded arrays).  With the
    pieces from split_in_order this is the whole batch in arrival order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([len(piece)], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(max(sizes), 1)

    def gather(a: np.ndarray) -> np.ndarray:
        t = torch.zeros(cap, dtype=torch.from_numpy(a[:0].copy()).dtype)
        t[:len(a)] = torch.from_numpy(np.ascontiguousarray(a))
        out = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(out, t, group=group)
        return np.concatenate([o[:k].numpy() for o, k in zip(out, sizes)])

    return Batch(gather(piece.row), gather(piece.col), gather(piece.val), gather(piece.op))


class ShardPlan:
    """What rank `rank` holds and receives: its block of A's rows (an
    ordinary left operand), the replicated B (all of A when B is A), and per
    batch the local entries of the A batch and the whole batch for B."""

    def __init__(self, A, B, world: int, rank: int, balance: bool = True):
        self.b_is_a = B is None
        weights = np.diff(np.asarray(A.rowptr)) if balance else None
        self.part = RowPartition(A.nrows, world, weights)
        self.rank = rank
        self.lo, self.hi = self.part.block(rank)
        self.A_local = shard_rows(A, self.lo, self.hi)
        self.B = A if B is None else B

    def batches(self, piece_a, piece_b=None, group=None):
        """Exchange this rank's pieces; returns (local A batch, whole B batch).
        When B is A the B batch is the whole A batch (every rank's copy of B
        takes every update)."""
        full_a = allgather_batch(piece_a, group)
        local_a = local_entries(full_a, self.part, self.rank)
        if self.b_is_a:
            return local_a, full_a
        full_b = allgather_batch(piece_b, group) if piece_b is not None else None
        return local_a, full_b

    def global_rows(self, local_rows) -> np.ndarray:
        return np.asarray(local_rows, dtype=np.int64) + self.lo
