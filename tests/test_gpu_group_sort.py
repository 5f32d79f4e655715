"""The group-sort recompute kernels (rows of at most 64, 128 or 256
products, sorted by column in registers by 8, 16 or 32 lanes), against the
oracle.

The rows are built so that each path of the kernels is taken:
- every product of a row lands on one column, so one run of equal columns
  spans every lane of the group and the cross-lane fold carries it through;
- every product has its own column, at product counts on both sides of each
  group size (64/65, 128/129, 256/257: the rows above a size go to the next
  group, or to the hash kernels);
- overlapping B rows give runs of two and three equal columns at arbitrary
  places, split between lanes or not.
Patterns and (min,+) values are bit-exact; (+,.) values within 1e-12 of the
oracle's (all values positive, so componentwise is relative).
"""

import numpy as np
import pytest

from oracle import OMat
from parity import assert_matches, oracle_product
from workloads import CSR, MIN_PLUS_I32, PLUS_TIMES_F64, random_batch

pytestmark = pytest.mark.gpu

NB = 300  # B rows of each kind


def _csr(nrows, ncols, rows, sr, rng):
    rp = np.zeros(nrows + 1, np.int64)
    for i, cs in rows.items():
        rp[i + 1] = len(cs)
    rp = np.cumsum(rp)
    col = np.zeros(rp[-1], np.int32)
    for i, cs in rows.items():
        col[rp[i]:rp[i + 1]] = np.sort(np.asarray(cs, np.int32))
    n = col.shape[0]
    val = rng.random(n) + 0.5 if sr == PLUS_TIMES_F64 else rng.integers(1, 101, n).astype(np.int32)
    return CSR(nrows, ncols, rp, col, val)


def _operands(sr, seed=5):
    rng = np.random.default_rng(seed)
    # B: rows [0, NB) hold column 5 only; rows [NB, 2 NB) column k - NB + 7
    # (all distinct); rows [2 NB, 3 NB) columns j, j + 1, j + 2
    brows = {}
    for k in range(NB):
        brows[k] = [5]
        brows[NB + k] = [k + 7]
        brows[2 * NB + k] = [k, k + 1, k + 2]
    B = _csr(3 * NB, NB + 16, brows, sr, rng)
    arows = {}
    i = 0
    for L in (1, 8, 9, 63, 64, 65, 127, 128, 129, 200, 255, 256, 257):
        arows[i] = list(range(L))                        # one column, L products
        arows[i + 1] = list(range(NB, NB + L))           # L distinct columns
        i += 2
    for L in (5, 21, 22, 42, 43, 60, 85, 86):            # 3 L products in runs of up to three
        arows[i] = sorted(rng.choice(np.arange(2 * NB, 3 * NB), size=L, replace=False).tolist())
        i += 1
    for _ in range(40):                                   # mixed rows
        k = int(rng.integers(1, 40))
        arows[i] = sorted(rng.choice(3 * NB, size=k, replace=False).tolist())
        i += 1
    A = _csr(i + 10, 3 * NB, arows, sr, rng)              # and ten empty rows
    return A, B


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
@pytest.mark.parametrize("sort_max", [64, 128, 256])
def test_group_sort_rows_against_the_oracle(dspg, sr, sort_max):
    A, B = _operands(sr)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    g = dspg.DynamicSpGEMM(A, B)
    g.set_tuning(dict(dspg.tuning_candidates()[0], sort_max=sort_max))
    g.recompute_all()
    C_o, S_o = oracle_product(Ao, Bo)
    assert_matches(g.read_C(), C_o, S_o, what=f"static sort_max={sort_max}", rel_check=True)
    # batches on A: rows keep their kind but change length and values
    for k in range(3):
        b = random_batch(A.nrows, A.ncols, 150, 60 + k, sr, A=Ao.to_csr())
        g.apply_batch(b)
        Ao.apply(b)
        C_o, S_o = oracle_product(Ao, Bo)
        assert_matches(g.read_C(), C_o, S_o, what=f"batch {k} sort_max={sort_max}", rel_check=True)
    g.close()


def test_group_sort_one_column_row_sums(dspg):
    """A row of L products on one column is the plain sum of its products,
    for every L up to a group's size; checked against numpy as well."""
    A, B = _operands(PLUS_TIMES_F64)
    g = dspg.DynamicSpGEMM(A, B)
    g.set_tuning(dict(dspg.tuning_candidates()[0], sort_max=256))
    g.recompute_all()
    C = g.read_C()
    for i in range(0, 26, 2):
        a = A.val[A.rowptr[i]:A.rowptr[i + 1]]
        b = B.val[B.rowptr[A.col[A.rowptr[i]:A.rowptr[i + 1]]]]
        lo, hi = C.rowptr[i], C.rowptr[i + 1]
        assert hi - lo == 1 and C.col[lo] == 5
        want = float(np.sum(a * b))
        assert abs(C.val[lo] - want) <= 1e-12 * want
    g.close()
