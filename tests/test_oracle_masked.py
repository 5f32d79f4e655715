"""Pins of the oracle's Bloom filter (Section 5.2) and of its route through
Algorithm 2 (oracle/masked.py), no GPU needed.

* F by brute force: a dense triple loop over (i, k, j) on tiny inputs;
* the l = 64 fold: columns k and k + 64 of A share a bit;
* the hand-worked fixture tests/golden/masked_3x3_hand.json (C*, F*, R,
  A^R, the product count, C' and F' after two batches);
* Algorithm 2 against the definition: after sequences of mixed batches the
  route's C' equals the oracle's plain product of A', B' and its F' the
  oracle's Bloom filter, in both semirings, with B = A and B separate;
* the mask: entries outside C* keep their values, and every entry of C
  that changes is an entry of C*.
"""

import json
import os

import numpy as np
import pytest

from oracle import OMat
from oracle import masked as om
from workloads import CSR, Batch, MIN_PLUS_I32, PLUS_TIMES_F64, random_batch, random_csr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr_from_rows(rows, ncols, sr):
    rp = np.zeros(len(rows) + 1, np.int64)
    for i, r in enumerate(rows):
        rp[i + 1] = rp[i] + len(r)
    col = np.array([j for r in rows for j in sorted(r)], np.int32)
    val = np.array([r[j] for r in rows for j in sorted(r)], np.float64 if sr == PLUS_TIMES_F64 else np.int32)
    return CSR(len(rows), ncols, rp, col, val)


def test_bloom_by_brute_force():
    rng = np.random.default_rng(1)
    for seed in range(4):
        A = random_csr(9, 130, 12, 10 + seed)
        B = random_csr(130, 11, 6, 20 + seed)
        PA = np.zeros((9, 130), bool)
        PB = np.zeros((130, 11), bool)
        PA[A.row_ids(), A.col] = True
        PB[B.row_ids(), B.col] = True
        want = np.zeros((9, 11), np.uint64)
        for i in range(9):
            for k in range(130):
                for j in range(11):
                    if PA[i, k] and PB[k, j]:
                        want[i, j] |= np.uint64(1) << np.uint64(k % 64)
        rp, col, words = OMat.from_csr(A).bloom(OMat.from_csr(B))
        got = np.zeros((9, 11), np.uint64)
        pat = np.zeros((9, 11), bool)
        for i in range(9):
            got[i, col[rp[i]:rp[i + 1]]] = words[rp[i]:rp[i + 1]]
            pat[i, col[rp[i]:rp[i + 1]]] = True
        assert np.array_equal(pat, (PA.astype(int) @ PB.astype(int)) > 0)
        assert np.array_equal(got, want)
    del rng


def test_bloom_bits_fold_modulo_64():
    """A(0,3) and A(0,67) both reach column 5: one bit (3); A(0,64) alone
    reaches column 6: bit 0."""
    A = _csr_from_rows([{3: 1.0, 67: 2.0, 64: 1.0}], 70, PLUS_TIMES_F64)
    brows = [dict() for _ in range(70)]
    brows[3] = {5: 1.0}
    brows[67] = {5: 1.0}
    brows[64] = {6: 1.0}
    B = _csr_from_rows(brows, 8, PLUS_TIMES_F64)
    rp, col, words = OMat.from_csr(A).bloom(OMat.from_csr(B))
    assert list(col) == [5, 6]
    assert list(words) == [1 << 3, 1]


def test_golden_masked_hand_worked():
    with open(os.path.join(GOLDEN, "masked_3x3_hand.json")) as f:
        g = json.load(f)
    a = g["A"]
    A = CSR(a["nrows"], a["ncols"], np.array(a["rowptr"], np.int64), np.array(a["col"], np.int32),
            np.array(a["val"], np.float64))
    rows = om.rows_of(A)
    C0 = om.product(rows, rows, 0)
    F0 = om.bloom(rows, rows)
    rp, col, val = om.to_csr_arrays(C0, 3, np.float64)
    assert rp.tolist() == g["C"]["rowptr"] and col.tolist() == g["C"]["col"] and val.tolist() == g["C"]["val"]
    rp, col, w = om.to_csr_arrays(F0, 3, np.uint64)
    assert col.tolist() == g["F"]["col"] and w.tolist() == g["F"]["words"]
    for k, step in enumerate(g["batches"]):
        b = step["batch"]
        batch = Batch(np.array(b["row"], np.int32), np.array(b["col"], np.int32), np.array(b["val"], np.float64),
                      np.array(b["op"], np.uint8))
        r = om.masked_update(rows, None, batch, b_is_a=True, sr=0)
        cs = step["C_star"]
        assert r["C_star"] == {(i, j): f for i, j, f in zip(cs["row"], cs["col"], cs["fstar"])}, f"batch {k} C*"
        assert r["R"] == dict(zip(step["R"]["row"], step["R"]["bits"])), f"batch {k} R"
        assert r["kept"] == step["kept"] and r["products"] == step["products"], f"batch {k} A^R"
        rp, col, val = om.to_csr_arrays(r["C"], 3, np.float64)
        assert rp.tolist() == step["C_after"]["rowptr"] and col.tolist() == step["C_after"]["col"]
        assert val.tolist() == step["C_after"]["val"], f"batch {k} C'"
        rp, col, w = om.to_csr_arrays(r["F"], 3, np.uint64)
        assert col.tolist() == step["F_after"]["col"] and w.tolist() == step["F_after"]["words"], f"batch {k} F'"
        # and the oracle's plain product and Bloom filter of A' agree
        An = _csr_from_rows(r["A"], 3, PLUS_TIMES_F64)
        Ao = OMat.from_csr(An)
        Cd = Ao.multiply(Ao).to_csr()
        assert np.array_equal(Cd.col, col) and np.array_equal(Cd.val, val)
        _, _, wd = Ao.bloom(Ao)
        assert np.array_equal(wd, w)
        rows = r["A"]


def _check_against_definition(r, sr, nrows, b_is_a):
    An = _csr_from_rows(r["A"], len(r["B"]), sr)
    Bn = An if b_is_a else _csr_from_rows(r["B"], r["ncols"], sr)
    Ao, Bo = OMat.from_csr(An), OMat.from_csr(Bn)
    Cd = Ao.multiply(Bo).to_csr()
    rp, col, val = om.to_csr_arrays(r["C"], nrows, np.float64 if sr == PLUS_TIMES_F64 else np.int32)
    assert np.array_equal(rp, Cd.rowptr) and np.array_equal(col, Cd.col), "C' pattern"
    if sr == PLUS_TIMES_F64:
        S = Ao.multiply(Bo, absval=True).to_csr()
        assert np.all(np.abs(val - Cd.val) <= 1e-12 * S.val), "C' values"
    else:
        assert np.array_equal(val, Cd.val), "C' values"
    brp, bcol, bw = Ao.bloom(Bo)
    frp, fcol, fw = om.to_csr_arrays(r["F"], nrows, np.uint64)
    assert np.array_equal(frp, brp) and np.array_equal(fcol, bcol) and np.array_equal(fw, bw), "F'"


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
@pytest.mark.parametrize("b_is_a", [True, False])
def test_masked_route_equals_the_definition(sr, b_is_a):
    n, k, m = 60, (60 if b_is_a else 150), (60 if b_is_a else 40)
    A = random_csr(n, k, 9, 3, sr, empty_frac=0.1)
    B = A if b_is_a else random_csr(k, m, 7, 4, sr, empty_frac=0.1)
    A_rows, B_rows = om.rows_of(A), om.rows_of(B)
    for step in range(4):
        Acsr = _csr_from_rows(A_rows, k, sr)
        ba = random_batch(n, k, 40, 50 + step, sr, A=Acsr, dup_frac=0.2)
        bb = None
        if not b_is_a:
            bb = random_batch(k, m, 30, 70 + step, sr, A=_csr_from_rows(B_rows, m, sr), dup_frac=0.2)
        r = om.masked_update(A_rows, B_rows, ba, bb, b_is_a=b_is_a, sr=sr)
        r["ncols"] = m
        _check_against_definition(r, sr, n, b_is_a)
        # the mask: outside C* nothing changes, and every change is in C*
        for key, v in r["C_old"].items():
            if key not in r["C_star"]:
                assert r["C"].get(key) == v
        for key in set(r["C_old"]) | set(r["C"]):
            if r["C_old"].get(key) != r["C"].get(key):
                assert key in r["C_star"], f"change outside C* at {key}"
        A_rows = r["A"]
        B_rows = r["A"] if b_is_a else r["B"]


def test_absent_delete_changes_nothing():
    """A delete of an absent entry is no change: C* is empty, nothing is
    kept or multiplied, C and F stay.  A set that writes a present entry's
    own value counts as a change (the reading of A*)."""
    A = _csr_from_rows([{0: 1.0, 1: 2.0}, {1: 3.0}], 2, PLUS_TIMES_F64)
    rows = om.rows_of(A)
    r = om.masked_update(rows, None, Batch(np.array([1], np.int32), np.array([0], np.int32),
                                           np.array([0.0]), np.array([om.OP_DELETE], np.uint8)), b_is_a=True, sr=0)
    assert r["C_star"] == {} and r["kept"] == 0 and r["products"] == 0
    assert r["C"] == r["C_old"] and r["F"] == r["F_old"]
    r = om.masked_update(rows, None, Batch(np.array([1], np.int32), np.array([1], np.int32),
                                           np.array([3.0]), np.array([om.OP_SET], np.uint8)), b_is_a=True, sr=0)
    # (1,1) changed: A* B' gives (1,1) bit 1; A B*: rows with A(i,1): 0, 1 -> (0,1), (1,1) bit 1
    assert r["C_star"] == {(1, 1): 2, (0, 1): 2}
    assert r["C"] == r["C_old"]
