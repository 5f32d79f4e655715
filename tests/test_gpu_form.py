"""The product form of Section 3 against the oracle: C = alpha op(A) op(B)
(+) beta X with transposed operands (Section 5.3), through dspg_build_form.

The oracle side transposes the caller's matrices on the CPU (a stable sort
of the entries by column), multiplies with the oracle, and forms alpha P
(+) beta X entry by entry from its definition; batches are applied to the
caller's A and B, so a transposed operand's update (i, j) must land at
(j, i) inside the library.  Patterns and (min,+) values must match exactly,
(+,.) values within 1e-12 (|alpha| sum|ab| + |beta x|).
"""

import numpy as np
import pytest

from oracle import OMat
from workloads import CSR, MIN_PLUS_I32, PLUS_TIMES_F64, random_batch, random_csr

pytestmark = pytest.mark.gpu


def _transpose(M: CSR) -> CSR:
    r = M.row_ids()
    order = np.lexsort((r, M.col))  # by column, then row
    rowptr = np.zeros(M.ncols + 1, np.int64)
    np.cumsum(np.bincount(M.col.astype(np.int64), minlength=M.ncols), out=rowptr[1:])
    return CSR(M.ncols, M.nrows, rowptr, r[order].astype(np.int32), M.val[order])


def _dense(M: CSR):
    P = np.zeros((M.nrows, M.ncols), bool)
    V = np.zeros((M.nrows, M.ncols), np.float64 if M.val.dtype == np.float64 else np.int64)
    r = M.row_ids()
    P[r, M.col] = True
    V[r, M.col] = M.val
    return P, V


def _expected(Ao, Bo, ta, tb, sr, alpha, beta, X):
    """(presence, values, bound) of alpha op(A) op(B) (+) beta X."""
    A = Ao.to_csr()
    B = Bo.to_csr() if Bo is not None else A
    opA = _transpose(A) if ta else A
    opB = _transpose(B) if tb else B
    a, b = OMat.from_csr(opA), OMat.from_csr(opB)
    PP, PV = _dense(a.multiply(b).to_csr())
    if X is None:
        PX = np.zeros_like(PP)
        XV = np.zeros_like(PV)
    else:
        PX, XV = _dense(X)
    pres = PP | PX
    if sr == PLUS_TIMES_F64:
        _, SA = _dense(a.multiply(b, absval=True).to_csr())
        val = np.where(PP, alpha * PV, 0.0) + np.where(PX, beta * XV, 0.0)
        bound = abs(alpha) * SA + abs(beta) * np.abs(XV)
    else:
        big = np.iinfo(np.int64).max
        val = np.minimum(np.where(PP, alpha + PV, big), np.where(PX, beta + XV, big))
        bound = None
    return pres, val, bound


def _check(g, Ao, Bo, ta, tb, sr, alpha, beta, X, what):
    pres, val, bound = _expected(Ao, Bo, ta, tb, sr, alpha, beta, X)
    Cg = g.read_C()
    P, V = _dense(Cg)
    assert np.array_equal(P, pres), f"{what}: pattern"
    if sr == PLUS_TIMES_F64:
        assert np.all(np.abs(V - val)[pres] <= 1e-12 * bound[pres]), f"{what}: values"
    else:
        assert np.array_equal(V[pres], val[pres]), f"{what}: values"
    # a few rows through dspg_read_rows_C
    rows = np.array([0, Cg.nrows - 1, Cg.nrows // 2, 0], np.int32)
    rp, col, v = g.read_rows_C(rows)
    for t, i in enumerate(rows):
        js = col[rp[t]:rp[t + 1]]
        assert np.array_equal(js, np.nonzero(pres[i])[0]), f"{what}: row {i} read alone"


CASES = [
    # (trans_a, trans_b, separate B)
    (1, 0, True), (0, 1, True), (1, 1, True), (1, 0, False), (0, 1, False), (1, 1, False),
]


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
@pytest.mark.parametrize("ta,tb,sep", CASES)
def test_transposed_operands_dynamic(dspg, sr, ta, tb, sep):
    """C = op(A) op(B) (B separate, or B is A: A^T A, A A^T, A^T A^T) over
    three batches given in the caller's coordinates."""
    rng = np.random.default_rng(ta * 4 + tb * 2 + sep)
    if sep:
        A = random_csr(150, 120, 6, 11, sr, empty_frac=0.1)
        # op(A) op(B) needs op(A).ncols == op(B).nrows
        ka = A.nrows if ta else A.ncols
        B = random_csr(ka, 170, 6, 12, sr, empty_frac=0.1) if not tb else random_csr(170, ka, 6, 12, sr, empty_frac=0.1)
    else:
        A = random_csr(140, 140 if ta == tb else 110, 6, 13, sr, empty_frac=0.1)
        B = None
    g = dspg.DynamicSpGEMM(A, B, trans_a=bool(ta), trans_b=bool(tb))
    Ao = OMat.from_csr(A)
    Bo = OMat.from_csr(B) if B is not None else None
    one = 1 if sr == PLUS_TIMES_F64 else 0  # the neutral scalar: times 1, plus 0
    _check(g, Ao, Bo, ta, tb, sr, one, one, None, "build")
    for t in range(3):
        ba = random_batch(A.nrows, A.ncols, 120, 20 + t, sr, A=Ao.to_csr())
        bb = random_batch(B.nrows, B.ncols, 90, 30 + t, sr, A=Bo.to_csr()) if B is not None else None
        g.apply_batch(ba, bb)
        Ao.apply(ba)
        if bb is not None:
            Bo.apply(bb)
        _check(g, Ao, Bo, ta, tb, sr, one, one, None, f"batch {t}")
        Ag = g.read_A()
        Aw = Ao.to_csr()
        assert np.array_equal(Ag.rowptr, Aw.rowptr) and np.array_equal(Ag.col, Aw.col), "A in the caller's coordinates"
        assert np.array_equal(Ag.val, Aw.val)
    g.close()


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_alpha_beta_x(dspg, sr):
    """C = alpha A B (+) beta X with a fixed X (some entries where A B has
    none), static and after batches; the affected rows are those of A B."""
    A = random_csr(200, 160, 6, 41, sr, empty_frac=0.1)
    B = random_csr(160, 180, 5, 42, sr, empty_frac=0.1)
    X = random_csr(200, 180, 4, 43, sr, empty_frac=0.2)
    alpha, beta = (2.5, -0.75) if sr == PLUS_TIMES_F64 else (3, 5)
    g = dspg.DynamicSpGEMM(A, B, alpha=alpha, beta=beta, X=X)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    _check(g, Ao, Bo, 0, 0, sr, alpha, beta, X, "build")
    assert g.info()["nnz_c"] == int(_expected(Ao, Bo, 0, 0, sr, alpha, beta, X)[0].sum())
    for t in range(2):
        ba = random_batch(A.nrows, A.ncols, 150, 44 + t, sr, A=Ao.to_csr())
        g.apply_batch(ba)
        Ao.apply(ba)
        _check(g, Ao, Bo, 0, 0, sr, alpha, beta, X, f"batch {t}")
    g.close()


def test_transposed_gram_with_form(dspg):
    """A^T A with alpha and an X, (+,.): all three parts of the form at once."""
    sr = PLUS_TIMES_F64
    A = random_csr(120, 90, 7, 51, sr, empty_frac=0.05)
    X = random_csr(90, 90, 3, 52, sr)
    g = dspg.DynamicSpGEMM(A, None, trans_a=True, alpha=0.5, beta=2.0, X=X)
    Ao = OMat.from_csr(A)
    _check(g, Ao, None, 1, 0, sr, 0.5, 2.0, X, "build")
    b = random_batch(A.nrows, A.ncols, 200, 53, sr, A=A)
    g.apply_batch(b)
    Ao.apply(b)
    _check(g, Ao, None, 1, 0, sr, 0.5, 2.0, X, "after a batch")


def test_form_rejects_bad_shapes(dspg):
    A = random_csr(30, 20, 3, 61, PLUS_TIMES_F64)
    B = random_csr(25, 40, 3, 62, PLUS_TIMES_F64)
    with pytest.raises(dspg.DspgError) as e:  # A B: 20 != 25
        dspg.DynamicSpGEMM(A, B, alpha=1.0)
    assert e.value.status == 1
    B2 = random_csr(20, 40, 3, 63, PLUS_TIMES_F64)
    X = random_csr(30, 39, 3, 64, PLUS_TIMES_F64)
    with pytest.raises(dspg.DspgError) as e:
        dspg.DynamicSpGEMM(A, B2, X=X)
    assert e.value.status == 1
    with pytest.raises(dspg.DspgError):  # A^T B2: 30 != 20
        dspg.DynamicSpGEMM(A, B2, trans_a=True)
