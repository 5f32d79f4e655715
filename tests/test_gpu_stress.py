"""Longer sequences on skewed graphs, against the oracle (GPU).

- A consecutive run of 10^4-edge batches on an R-MAT graph with hubs, C = A A
  in (+,.): the shape (hub rows whose A' and B' rows the batch has just
  rewritten, and whose product bounds cross the hash-table sizes) where the
  sizing pass must read the rows the commit has just written.  After every
  batch R must equal the oracle's, and a sample of rows of R and of all of C
  must match the oracle's A' A'.  Tables are sized by the product bound, so a
  table smaller than its row's products can only come from a stale bound; the
  library reports that as DSPG_ERR_TIMEOUT (apply_batch raises), and the
  learned-overflow count stays 0.
- A group of 64 uneven instances (the batched configuration's mix of
  semirings and sizes, at smaller scales) over an eager apply, the capturing
  apply and replays: every member against the oracle.
"""

import numpy as np
import pytest

import oracle
from oracle import OMat
from parity import assert_matches, assert_rows_match, oracle_product
from workloads import MIN_PLUS_I32, PLUS_TIMES_F64, rmat_edge_batch, rmat_symmetric

pytestmark = pytest.mark.gpu

SKEWED = (0.45, 0.15, 0.15, 0.25)
G500 = (0.57, 0.19, 0.19, 0.05)


def _rows_against_oracle(g, Ao, rows, what):
    rp, col, val = g.read_rows_C(rows)
    orp, ocol, oval = Ao.multiply_rows(Ao, rows)
    _, _, sabs = Ao.multiply_rows(Ao, rows, absval=True)
    assert_rows_match(rp, col, val, orp, ocol, oval, sabs, what=what)
    # relative to the entry itself where the entry does not cancel much (|C| >= S / 100)
    keep = np.abs(oval) * 100 >= sabs
    assert (np.abs(val - oval)[keep] / np.abs(oval[keep])).max(initial=0.0) <= 1e-12, what


def test_rmat18_consecutive_1e4_edge_batches(dspg):
    A, held = rmat_symmetric(18, 8, SKEWED, seed=81, kind=PLUS_TIMES_F64, holdout=1 << 17)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    rng = np.random.default_rng(82)
    for k in range(8):
        b = rmat_edge_batch(Ao.to_csr(), held, 10000, seed=83 + k)
        st = g.apply_batch(b)
        pre = Ao.presence(b)
        Ao.apply(b)
        post = Ao.presence(b)
        R = oracle.affected_rows(Ao, b, pre, post, b_nrows=A.nrows, b_is_a=True)
        assert np.array_equal(g.last_affected(), R), f"batch {k}: R"
        assert st["affected_rows"] == R.shape[0]
        assert st["est_overflows"] == 0
        pick = np.sort(rng.choice(R, size=min(5000, R.shape[0]), replace=False)).astype(np.int32)
        _rows_against_oracle(g, Ao, pick, f"batch {k}: rows of R")
        other = np.sort(rng.choice(A.nrows, size=5000, replace=False)).astype(np.int32)
        _rows_against_oracle(g, Ao, other, f"batch {k}: sample of C")
    # the hub rows themselves (the longest A' rows) after the whole sequence
    lens = np.diff(Ao.to_csr().rowptr)
    hubs = np.sort(np.argsort(lens)[-64:]).astype(np.int32)
    _rows_against_oracle(g, Ao, hubs, "hub rows")


def test_group_of_64_uneven_instances(dspg):
    rng = np.random.default_rng(91)
    insts = []
    for t in range(64):
        sr = PLUS_TIMES_F64 if t % 2 == 0 else MIN_PLUS_I32
        scale = int(rng.integers(7, 12))
        A, held = rmat_symmetric(scale, 8, G500, seed=9100 + t, kind=sr, holdout=200)
        size = int(10 ** rng.uniform(1, 3))
        insts.append((A, held, size))
    gs = [dspg.DynamicSpGEMM(A) for A, _, _ in insts]
    Aos = [OMat.from_csr(A) for A, _, _ in insts]
    Cos = [Ao.multiply(Ao) for Ao in Aos]
    grp = dspg.Group(gs)
    for rep in range(4):  # eager, capture, replay, replay
        bs = [rmat_edge_batch(Aos[t].to_csr(), held, size, seed=5000 * rep + t)
              for t, (A, held, size) in enumerate(insts)]
        stats, status = grp.apply(bs)
        assert status == [0] * len(gs)
        for t, (g, Ao, Co) in enumerate(zip(gs, Aos, Cos)):
            R = oracle.row_dynamic(Ao, Co, bs[t])
            assert stats[t]["affected_rows"] == R.shape[0], f"rep {rep} member {t}"
            assert np.array_equal(g.last_affected(), R), f"rep {rep} member {t}: R"
            C_o, S_o = oracle_product(Ao, Ao)
            assert_matches(g.read_C(), C_o, S_o, what=f"rep {rep} member {t}")
    grp.close()
