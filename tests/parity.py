"""Comparison helpers for the CUDA path against the oracle (test code only).

Tolerance for (+,.) on double (the stated bar is 1e-12 relative): every
summation order of n products has error at most gamma_n * sum_k |a_ik b_kj|
with gamma_n = n u / (1 - n u), u = 2^-53, so two implementations differ by
at most 2 gamma_n sum|ab| <= 1e-12 * sum|ab| while n <= 4500 terms per entry.
The check is therefore componentwise against S = |A'| |B'| (the oracle's
product of absolute values): |g - o| <= 1e-12 * S.  Patterns must be equal,
and (min,+) values bit-for-bit.
"""

import numpy as np

from oracle import OMat

RTOL = 1e-12


def assert_same_pattern(g, o, what="C"):
    assert g.nrows == o.nrows, f"{what}: nrows {g.nrows} != {o.nrows}"
    assert np.array_equal(np.asarray(g.rowptr), np.asarray(o.rowptr)), f"{what}: row lengths differ"
    assert np.array_equal(np.asarray(g.col), np.asarray(o.col)), f"{what}: column indices differ"


def assert_values(g, o, o_abs=None, what="C", rel_check=False):
    gv, ov = np.asarray(g.val), np.asarray(o.val)
    if ov.dtype != np.float64:
        bad = np.nonzero(gv != ov)[0]
        assert bad.shape[0] == 0, f"{what}: {bad.shape[0]} (min,+) values differ, first at {bad[:5]}"
        return
    assert o_abs is not None
    bound = RTOL * np.asarray(o_abs.val)
    err = np.abs(gv - ov)
    bad = np.nonzero(err > bound)[0]
    assert bad.shape[0] == 0, f"{what}: {bad.shape[0]} values outside 1e-12*sum|ab|, e.g. {err[bad[:3]]} vs {bound[bad[:3]]}"
    if rel_check:
        nz = ov != 0
        rel = err[nz] / np.abs(ov[nz])
        assert rel.size == 0 or rel.max() <= RTOL, f"{what}: max relative error {rel.max()}"


def oracle_product(A_or: OMat, B_or: OMat):
    C = A_or.multiply(B_or).to_csr()
    S = A_or.multiply(B_or, absval=True).to_csr() if A_or.sr == 0 else None
    return C, S


def assert_matches(g, o, o_abs=None, what="C", rel_check=False):
    assert_same_pattern(g, o, what)
    assert_values(g, o, o_abs, what, rel_check)


def assert_rows_match(g_rp, g_col, g_val, o_rp, o_col, o_val, o_abs_val=None, what="rows"):
    assert np.array_equal(g_rp, o_rp), f"{what}: row lengths differ"
    assert np.array_equal(g_col, o_col), f"{what}: columns differ"
    if o_val.dtype != np.float64:
        assert np.array_equal(g_val, o_val), f"{what}: (min,+) values differ"
    else:
        assert np.all(np.abs(g_val - o_val) <= RTOL * o_abs_val), f"{what}: values outside tolerance"
