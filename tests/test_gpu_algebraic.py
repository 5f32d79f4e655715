"""The delta path of Eq. 1 (dspg_apply_batch_algebraic) against the oracle.

Section 5, algebraic updates: for a batch that only inserts, C' = C (+) C*
with C* = A* B' (+) A B*.  The library forms C* entry by entry and folds it
into C; C' must equal the oracle's static A' B' (patterns exact; (min,+)
values bit-exact; (+,.) values within 1e-12 sum|ab|, and bit-exact on
integer-valued data, where every summation order is exact).  The rows that
took a contribution must be exactly Eq. 1's: rows of A* whose B' row is not
empty, and rows i with A(i,k) != 0 before the batch for a row k of B*.
A batch with a write to a present entry or a delete takes the row path
(stats["algebraic"] == 0) with the same result.
"""

import numpy as np
import pytest

from oracle import OMat
from parity import assert_matches, oracle_product
from workloads import (CSR, MIN_PLUS_I32, OP_DELETE, OP_INSERT, PLUS_TIMES_F64, Batch, concat_batches, er_matrix,
                       random_batch, random_csr, rmat_symmetric, stencil7)

pytestmark = pytest.mark.gpu


def _integer_valued(M: CSR, seed: int) -> CSR:
    rng = np.random.default_rng(seed)
    if M.val.dtype == np.float64:
        v = rng.integers(1, 10, M.col.shape[0]).astype(np.float64)
    else:
        v = rng.integers(1, 101, M.col.shape[0]).astype(np.int32)
    return CSR(M.nrows, M.ncols, M.rowptr, M.col, v)


def _inserts(M: CSR, n: int, seed: int, integer: bool = True, dup: int = 0, rows=None) -> Batch:
    """n insertions at distinct positions absent from M (uniform, or in the
    given rows only), then `dup` of them written again with another value
    (the last write wins)."""
    rng = np.random.default_rng(seed)
    present = set((M.row_ids().astype(np.int64) * M.ncols + M.col).tolist())
    keys = set()
    while len(keys) < n:
        if rows is None:
            k = int(rng.integers(0, M.nrows * M.ncols))
        else:
            k = int(rng.choice(rows)) * M.ncols + int(rng.integers(0, M.ncols))
        if k not in present:
            keys.add(k)
    keys = np.array(sorted(keys), np.int64)
    rng.shuffle(keys)
    r, c = (keys // M.ncols).astype(np.int32), (keys % M.ncols).astype(np.int32)
    if M.val.dtype == np.float64:
        v = rng.integers(1, 10, n).astype(np.float64) if integer else rng.random(n)
    else:
        v = rng.integers(1, 101, n).astype(np.int32)
    b = Batch(r, c, v, np.full(n, OP_INSERT, np.uint8))
    if dup:
        pick = rng.choice(n, dup, replace=False)
        v2 = (v[pick] + 1).astype(v.dtype)
        b = concat_batches(b, Batch(r[pick], c[pick], v2, np.full(dup, OP_INSERT, np.uint8)))
    return b


def _touched_rows(A_old: CSR, B_new: CSR, star_a: Batch, star_b: Batch) -> np.ndarray:
    """Rows of C that Eq. 1's C* reaches: X = A* B' reaches row i of an A*
    entry (i,k) when B'(k,:) is not empty; Y = A B* reaches every row i with
    A(i,k) != 0 (before the batch) for a row k of B*."""
    blen = np.diff(B_new.rowptr)
    rows = {int(i) for i, k in zip(star_a.row, star_a.col) if blen[k] > 0}
    kset = set(star_b.row.tolist())
    ar = A_old.row_ids()
    for i, k in zip(ar.tolist(), A_old.col.tolist()):
        if k in kset:
            rows.add(i)
    return np.array(sorted(rows), np.int32)


def _check_C(g, Ao, Bo, what, rel=False):
    C_o, S_o = oracle_product(Ao, Bo)
    assert_matches(g.read_C(), C_o, S_o, what=what, rel_check=rel)


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_insert_only_er_bitwise(dspg, sr):
    """ER n=4096, 8 per row (integer-valued): two batches of 1024 and 3000
    insertions (the second with repeated keys); C' bit-exact."""
    A = _integer_valued(er_matrix(4096, 8, seed=1, kind=sr), 3)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    for t, (n, dup) in enumerate([(1024, 0), (3000, 200)]):
        A_old = Ao.to_csr()
        b = _inserts(A_old, n, 10 + t, dup=dup)
        st = g.apply_batch(b, algebraic=True)
        assert st["algebraic"] == 1 and st["n_insert"] == n and st["n_update"] == 0
        Ao.apply(b)
        want = _touched_rows(A_old, Ao.to_csr(), b, b)
        assert np.array_equal(g.last_affected(), want), f"batch {t}: touched rows"
        C_o = Ao.multiply(Ao).to_csr()
        Cg = g.read_C()
        assert np.array_equal(Cg.rowptr, C_o.rowptr) and np.array_equal(Cg.col, C_o.col), f"batch {t}: pattern"
        assert np.array_equal(Cg.val, C_o.val), f"batch {t}: values"
        Ag = g.read_A()
        assert np.array_equal(Ag.col, Ao.to_csr().col) and np.array_equal(Ag.val, Ao.to_csr().val)


def test_insert_only_stencil_real_values(dspg):
    """32^3 stencil, real values: three consecutive insert-only batches, each
    4000 uniform insertions plus 40 into each of 30 rows (those rows of C
    outgrow their capacity and move, and later grow past the length that is
    searched, so the row path recomputes them); C' within 1e-12 sum|ab|."""
    A = stencil7(32, 32, 32, seed=4)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    relocations = 0
    hot = np.random.default_rng(19).choice(A.nrows, 30, replace=False)
    for t in range(3):
        A_old = Ao.to_csr()
        b1 = _inserts(A_old, 4000, 20 + t, integer=False)
        b2 = _inserts(A_old, 1200, 30 + t, integer=False, rows=hot)
        keep = ~np.isin(b2.row.astype(np.int64) * A.ncols + b2.col, b1.row.astype(np.int64) * A.ncols + b1.col)
        b = concat_batches(b1, Batch(b2.row[keep], b2.col[keep], b2.val[keep], b2.op[keep]))
        b = Batch(b.row, b.col, np.abs(b.val) + 0.5, b.op)
        st = g.apply_batch(b, algebraic=True)
        assert st["algebraic"] == 1
        relocations += st["relocations"]
        Ao.apply(b)
        assert np.array_equal(g.last_affected(), _touched_rows(A_old, Ao.to_csr(), b, b))
    assert relocations > 0, "no row of C moved: the append path is untested"
    C_o, S_o = oracle_product(Ao, Ao)
    assert_matches(g.read_C(), C_o, S_o, what="stencil delta path")


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_general_batch_takes_the_row_path(dspg, sr):
    """A batch with deletes and value changes is applied by the row path:
    stats say so, and C' equals the oracle's."""
    A = _integer_valued(random_csr(800, 800, 10, 31, sr), 32)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    b = random_batch(800, 800, 500, 33, sr, A=A)
    assert np.any(b.op != OP_INSERT)
    st = g.apply_batch(b, algebraic=True)
    assert st["algebraic"] == 0
    Ao.apply(b)
    _check_C(g, Ao, Ao, "row path fallback")
    # then an insert-only batch on the same handle takes the delta path
    A_old = Ao.to_csr()
    b2 = _inserts(A_old, 600, 34)
    st = g.apply_batch(b2, algebraic=True)
    assert st["algebraic"] == 1
    Ao.apply(b2)
    _check_C(g, Ao, Ao, "delta path after the row path")


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_insert_only_separate_b(dspg, sr):
    """C = A B with insertions into both A and B in one call: X = A* B' and
    Y = A B* with A's pattern before the batch."""
    A = _integer_valued(random_csr(700, 500, 8, 41, sr, empty_frac=0.1), 42)
    B = _integer_valued(random_csr(500, 900, 8, 43, sr, empty_frac=0.1), 44)
    g = dspg.DynamicSpGEMM(A, B)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    for t in range(2):
        A_old, B_old = Ao.to_csr(), Bo.to_csr()
        ba, bb = _inserts(A_old, 400, 45 + t), _inserts(B_old, 300, 47 + t)
        st = g.apply_batch(ba, bb, algebraic=True)
        assert st["algebraic"] == 1
        Ao.apply(ba)
        Bo.apply(bb)
        assert np.array_equal(g.last_affected(), _touched_rows(A_old, Bo.to_csr(), ba, bb))
        C_o = Ao.multiply(Bo).to_csr()
        Cg = g.read_C()
        assert np.array_equal(Cg.rowptr, C_o.rowptr) and np.array_equal(Cg.col, C_o.col)
        assert np.array_equal(Cg.val, C_o.val)


def test_long_rows_recomputed(dspg):
    """R-MAT scale 11 (hub rows of C with thousands of entries): contributions
    to rows longer than 256 entries are not searched; those rows are
    recomputed by the row path, and C' still equals the oracle's."""
    A, _ = rmat_symmetric(11, 8, (0.57, 0.19, 0.19, 0.05), seed=51, kind=PLUS_TIMES_F64)
    A = _integer_valued(A, 52)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    assert np.diff(Ao.multiply(Ao).to_csr().rowptr).max() > 256
    A_old = Ao.to_csr()
    b = _inserts(A_old, 1500, 53)
    st = g.apply_batch(b, algebraic=True)
    assert st["algebraic"] == 1
    Ao.apply(b)
    assert np.array_equal(g.last_affected(), _touched_rows(A_old, Ao.to_csr(), b, b))
    C_o = Ao.multiply(Ao).to_csr()
    Cg = g.read_C()
    assert np.array_equal(Cg.rowptr, C_o.rowptr) and np.array_equal(Cg.col, C_o.col)
    assert np.array_equal(Cg.val, C_o.val)


def test_empty_and_noop_batches(dspg):
    """An empty batch, and a batch of deletes of absent entries only, change
    nothing (the delta path with no contribution)."""
    A = _integer_valued(random_csr(300, 300, 6, 61, PLUS_TIMES_F64), 62)
    g = dspg.DynamicSpGEMM(A)
    before = g.read_C()
    z = np.zeros(0, np.int32)
    st = g.apply_batch(Batch(z, z, np.zeros(0), np.zeros(0, np.uint8)), algebraic=True)
    assert st["affected_rows"] == 0
    b = _inserts(A, 50, 63)
    nb = Batch(b.row, b.col, b.val, np.full(50, OP_DELETE, np.uint8))  # absent: no-ops
    st = g.apply_batch(nb, algebraic=True)
    assert st["algebraic"] == 1 and st["n_noop"] == 50 and st["affected_rows"] == 0
    after = g.read_C()
    assert np.array_equal(after.rowptr, before.rowptr) and np.array_equal(after.col, before.col)
    assert np.array_equal(after.val, before.val)
