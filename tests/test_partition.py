"""The row-sharded plan (paper_2202_08808_gb300/partition.py) on CPU ranks.

Two gloo ranks each hold a block of A's rows and the whole B (all of A when
C = A A).  Each receives a consecutive piece of the batch, the pieces are
allgathered, and each rank applies its local A entries and the whole batch
to its instance C_r = A_r B -- here with the CPU oracle standing in for the
library call the GPU path makes.  The union of the ranks' affected rows and
of their rows of C' must equal the single-process oracle's R and C'.  No
GPU is used; nothing of this runs on more than one GPU in this build.
"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from oracle import OMat
from paper_2202_08808_gb300.partition import RowPartition, ShardPlan, local_entries, split_in_order
from workloads import MIN_PLUS_I32, PLUS_TIMES_F64, random_batch, random_csr


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _csr_rows(M, rows):
    return {int(i): (M.col[M.rowptr[i]:M.rowptr[i + 1]].tolist(), M.val[M.rowptr[i]:M.rowptr[i + 1]].tolist())
            for i in rows}


def _rank(rank, world, port, case, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sr, separate_b, seed = case
        A = random_csr(240, 180 if separate_b else 240, 7, seed, sr, empty_frac=0.1)
        B = random_csr(180, 260, 6, seed + 1, sr, empty_frac=0.1) if separate_b else None
        plan = ShardPlan(A, B, world, rank)
        Ao = OMat.from_csr(plan.A_local)
        Bo = OMat.from_csr(plan.B)
        Co = Ao.multiply(Bo)
        results = []
        for t in range(3):
            ba = random_batch(A.nrows, A.ncols, 300, seed + 10 + t, sr, A=A)
            bb = random_batch(B.nrows, B.ncols, 200, seed + 20 + t, sr, A=B) if separate_b else None
            piece_a = split_in_order(ba, world)[rank]
            piece_b = split_in_order(bb, world)[rank] if separate_b else None
            local_a, full_b = plan.batches(piece_a, piece_b)
            if not separate_b:
                # the exchange restores the whole batch in arrival order
                assert np.array_equal(full_b.row, ba.row) and np.array_equal(full_b.op, ba.op)
            R = oracle.row_dynamic(Ao, Co, local_a, Bo, full_b)
            C = Co.to_csr()
            results.append((plan.global_rows(R).tolist(), _csr_rows(C, range(C.nrows)), plan.lo))
        out[rank] = results
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", [(PLUS_TIMES_F64, False, 3), (MIN_PLUS_I32, False, 5), (PLUS_TIMES_F64, True, 7),
                                  (MIN_PLUS_I32, True, 9)])
def test_two_ranks_equal_one_process(case):
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), case, out), nprocs=world, join=True)
        res = dict(out)
    sr, separate_b, seed = case
    # the single-process oracle on the same inputs
    A = random_csr(240, 180 if separate_b else 240, 7, seed, sr, empty_frac=0.1)
    B = random_csr(180, 260, 6, seed + 1, sr, empty_frac=0.1) if separate_b else None
    Ao = OMat.from_csr(A)
    Bo = OMat.from_csr(B) if separate_b else None
    Co = Ao.multiply(Bo if separate_b else Ao)
    for t in range(3):
        ba = random_batch(A.nrows, A.ncols, 300, seed + 10 + t, sr, A=A)
        bb = random_batch(B.nrows, B.ncols, 200, seed + 20 + t, sr, A=B) if separate_b else None
        R = oracle.row_dynamic(Ao, Co, ba, Bo, bb) if separate_b else oracle.row_dynamic(Ao, Co, ba)
        got_R = sorted(res[0][t][0] + res[1][t][0])
        assert got_R == R.tolist(), f"batch {t}: union of the ranks' R"
        C = Co.to_csr()
        for r in range(world):
            lo = res[r][t][2]
            for i, row in res[r][t][1].items():
                g = lo + i
                assert row[0] == C.col[C.rowptr[g]:C.rowptr[g + 1]].tolist(), f"batch {t} row {g}: columns"
                assert row[1] == C.val[C.rowptr[g]:C.rowptr[g + 1]].tolist(), f"batch {t} row {g}: values"
        assert sum(len(res[r][t][1]) for r in range(world)) == C.nrows


def test_partition_blocks_and_routing():
    w = np.array([5, 0, 0, 9, 1, 1, 1, 20, 0, 3], np.int64)
    p = RowPartition(10, 3, w)
    b = p.bounds
    assert b[0] == 0 and b[-1] == 10 and np.all(np.diff(b) >= 0)
    assert [p.owner([i])[0] for i in range(10)] == [int(np.searchsorted(b, i, side="right") - 1) for i in range(10)]
    q = RowPartition(10, 4)
    assert q.bounds.tolist() == [0, 2, 5, 7, 10]
    from paper_2202_08808_gb300.partition import Batch
    bt = Batch(np.array([0, 9, 3, 5, 2], np.int32), np.array([1, 2, 3, 4, 5], np.int32), np.arange(5.0),
               np.zeros(5, np.uint8))
    loc = local_entries(bt, q, 1)  # rows 2..4
    assert loc.row.tolist() == [1, 0] and loc.col.tolist() == [3, 5]
    pieces = split_in_order(bt, 2)
    assert [len(x) for x in pieces] == [2, 3] and pieces[1].row.tolist() == [3, 5, 2]


@pytest.mark.gpu
@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_shard_handles_on_one_gpu(dspg, sr):
    """The per-rank step through the library: three shards of an R-MAT
    A A, each an ordinary handle on (its rows of A, all of A as B), run one
    after the other on one GPU (no kernel waits on another; the exchange is
    the host concatenation that the allgather performs across ranks).  The
    union of the shards' R and rows of C' equals the oracle's."""
    from paper_2202_08808_gb300.partition import local_entries
    from workloads import rmat_edge_batch, rmat_symmetric
    A, held = rmat_symmetric(11, 8, (0.57, 0.19, 0.19, 0.05), seed=71, kind=sr, holdout=3000)
    world = 3
    plans = [ShardPlan(A, None, world, r) for r in range(world)]
    hs = [dspg.DynamicSpGEMM(p.A_local, p.B) for p in plans]
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    for t in range(3):
        b = rmat_edge_batch(Ao.to_csr(), held, 400, seed=72 + t)
        R = oracle.row_dynamic(Ao, Co, b)
        got = []
        for p, h in zip(plans, hs):
            h.apply_batch(local_entries(b, p.part, p.rank), b)
            got.extend(p.global_rows(h.last_affected()).tolist())
        assert sorted(got) == R.tolist(), f"batch {t}: union of R"
        C = Co.to_csr()
        for p, h in zip(plans, hs):
            Cg = h.read_C()
            a, z = int(C.rowptr[p.lo]), int(C.rowptr[p.hi])
            assert np.array_equal(Cg.rowptr, C.rowptr[p.lo:p.hi + 1] - a), f"batch {t} rank {p.rank}: rows"
            assert np.array_equal(Cg.col, C.col[a:z])
            if sr == MIN_PLUS_I32:
                assert np.array_equal(Cg.val, C.val[a:z])
            else:
                S = Ao.multiply(Ao, absval=True).to_csr()
                assert np.all(np.abs(Cg.val - C.val[a:z]) <= 1e-12 * S.val[a:z])
    for h in hs:
        h.close()
