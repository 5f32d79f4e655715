"""The entry-level masked recompute (Section 5.2, Algorithm 2) and the
Bloom filter F it keeps, through the C ABI, against the oracle.

- F of the static product equals the oracle's Bloom filter of A B, word
  for word (rows short enough for the warp kernel and rows over 512
  entries for the CTA kernel);
- after each batch of general updates C' equals the oracle's product of
  A', B' (patterns and (min,+) values bit-exact, (+,.) within 1e-12 of
  sum|ab|), F' equals the oracle's Bloom filter of A', B', and the counts
  of the algorithm's steps equal those of the oracle's route through
  Algorithm 2 (oracle/masked.py): |C*|, the rows of C*, |A^R| and the
  products of the masked multiplication;
- entries of C outside C* keep their values bit for bit;
- a tight arena (rows that outgrow their room move, the arena regrows)
  gives the same results;
- the calls that would take the row path on such a handle are refused.
"""

import numpy as np
import pytest

from oracle import OMat
from oracle import masked as om
from parity import assert_matches, oracle_product
from workloads import (MIN_PLUS_I32, PLUS_TIMES_F64, Batch, random_batch, random_csr, rmat_edge_batch,
                       rmat_symmetric)

pytestmark = pytest.mark.gpu

G500 = (0.57, 0.19, 0.19, 0.05)


def _bloom_matches(g, Ao, Bo, what):
    F = g.read_bloom()
    rp, col, words = Ao.bloom(Bo)
    assert np.array_equal(F.rowptr, rp), f"{what}: F row lengths"
    assert np.array_equal(F.col, col), f"{what}: F columns"
    bad = np.nonzero(F.val != words)[0]
    assert bad.size == 0, f"{what}: {bad.size} Bloom words differ, first at {bad[:5]}"


def _csr_from_rows(rows, ncols, sr):
    from workloads import CSR
    rp = np.zeros(len(rows) + 1, np.int64)
    for i, r in enumerate(rows):
        rp[i + 1] = rp[i] + len(r)
    col = np.array([j for r in rows for j in sorted(r)], np.int32)
    val = np.array([r[j] for r in rows for j in sorted(r)], np.float64 if sr == PLUS_TIMES_F64 else np.int32)
    return CSR(len(rows), ncols, rp, col, val)


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_bloom_of_the_static_product(dspg, sr):
    # B rows of up to 40 entries under A rows of up to 40: rows of C beyond
    # 512 entries go to the CTA kernel
    A = random_csr(400, 300, 40, 1, sr, empty_frac=0.1)
    B = random_csr(300, 2000, 40, 2, sr, empty_frac=0.1)
    g = dspg.DynamicSpGEMM(A, B, bloom=True)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    lens = np.diff(Ao.multiply(Bo).to_csr().rowptr)
    assert lens.max() > 512 and (lens <= 512).sum() > 100
    _bloom_matches(g, Ao, Bo, "static")
    C_o, S_o = oracle_product(Ao, Bo)
    assert_matches(g.read_C(), C_o, S_o, what="static C")
    g.recompute_all()  # a second static product rebuilds F
    _bloom_matches(g, Ao, Bo, "recompute_all")
    g.close()


def _run_sequence(dspg, g, A_rows, B_rows, batches_a, batches_b, sr, b_is_a, nrows, ncols_b):
    for k, ba in enumerate(batches_a):
        bb = batches_b[k] if batches_b is not None else None
        r = om.masked_update(A_rows, B_rows, ba, bb, b_is_a=b_is_a, sr=sr)
        C_before = g.read_C()
        st = g.apply_batch(ba, bb)
        Ao = OMat.from_csr(_csr_from_rows(r["A"], len(r["B"]) if b_is_a else len(B_rows), sr))
        Bo = Ao if b_is_a else OMat.from_csr(_csr_from_rows(r["B"], ncols_b, sr))
        C_o, S_o = oracle_product(Ao, Bo)
        assert_matches(g.read_C(), C_o, S_o, what=f"batch {k} C", rel_check=(sr == PLUS_TIMES_F64))
        _bloom_matches(g, Ao, Bo, f"batch {k}")
        assert st["masked_entries"] == len(r["C_star"]), f"batch {k}: |C*|"
        assert np.array_equal(g.last_affected(), r["rows"]), f"batch {k}: rows of C*"
        assert st["affected_rows"] == r["rows"].shape[0]
        assert st["a_entries"] == r["kept"], f"batch {k}: |A^R|"
        assert st["products"] == r["products"], f"batch {k}: products"
        # entries outside C* keep their values bit for bit
        C_after = g.read_C()
        before = {(i, int(j)): v for i in range(nrows)
                  for j, v in zip(C_before.col[C_before.rowptr[i]:C_before.rowptr[i + 1]],
                                  C_before.val[C_before.rowptr[i]:C_before.rowptr[i + 1]])}
        after = {(i, int(j)): v for i in range(nrows)
                 for j, v in zip(C_after.col[C_after.rowptr[i]:C_after.rowptr[i + 1]],
                                 C_after.val[C_after.rowptr[i]:C_after.rowptr[i + 1]])}
        for key, v in before.items():
            if key not in r["C_star"]:
                assert key in after and after[key].tobytes() == v.tobytes(), f"batch {k}: {key} outside C* changed"
        A_rows = r["A"]
        B_rows = r["A"] if b_is_a else r["B"]
    return A_rows, B_rows


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_masked_batches_b_is_a(dspg, sr):
    A = random_csr(500, 500, 12, 3, sr, empty_frac=0.1)
    g = dspg.DynamicSpGEMM(A, bloom=True)
    rows = om.rows_of(A)
    batches = []
    cur = rows
    for k in range(4):
        b = random_batch(500, 500, 150 + 50 * k, 30 + k, sr, A=_csr_from_rows(cur, 500, sr), dup_frac=0.2)
        batches.append(b)
        cur, _ = om.apply_updates(cur, b)
    _run_sequence(dspg, g, rows, rows, batches, None, sr, True, 500, 500)
    g.close()


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_masked_batches_separate_b(dspg, sr):
    A = random_csr(300, 200, 10, 5, sr, empty_frac=0.1)
    B = random_csr(200, 350, 9, 6, sr, empty_frac=0.1)
    g = dspg.DynamicSpGEMM(A, B, bloom=True)
    a_rows, b_rows = om.rows_of(A), om.rows_of(B)
    ba_list, bb_list = [], []
    ca, cb = a_rows, b_rows
    for k in range(3):
        ba = random_batch(300, 200, 120, 40 + k, sr, A=_csr_from_rows(ca, 200, sr))
        bb = random_batch(200, 350, 90, 50 + k, sr, A=_csr_from_rows(cb, 350, sr))
        ba_list.append(ba)
        bb_list.append(bb)
        ca, _ = om.apply_updates(ca, ba)
        cb, _ = om.apply_updates(cb, bb)
    # a batch on A only at the end
    ba_list.append(random_batch(300, 200, 60, 77, sr, A=_csr_from_rows(ca, 200, sr)))
    bb_list.append(None)
    _run_sequence(dspg, g, a_rows, b_rows, ba_list, bb_list, sr, False, 300, 350)
    g.close()


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_masked_rmat_hubs(dspg, sr):
    """R-MAT scale 10, Graph500 parameters: hub rows of C with hundreds of
    entries, where a batch masks a few of them."""
    A, held = rmat_symmetric(10, 8, G500, seed=7, kind=sr, holdout=800)
    g = dspg.DynamicSpGEMM(A, bloom=True)
    rows = om.rows_of(A)
    cur = _csr_from_rows(rows, A.ncols, sr)
    batches = []
    crow = rows
    for k in range(3):
        b = rmat_edge_batch(cur, held, 60, seed=80 + k)
        batches.append(b)
        crow, _ = om.apply_updates(crow, b)
        cur = _csr_from_rows(crow, A.ncols, sr)
    _run_sequence(dspg, g, rows, rows, batches, None, sr, True, A.nrows, A.ncols)
    g.close()


def test_masked_tight_arena_and_empty_batches(dspg):
    sr = PLUS_TIMES_F64
    A = random_csr(300, 300, 8, 9, sr, empty_frac=0.0)
    g = dspg.DynamicSpGEMM(A, bloom=True, arena_headroom=1.0, slack_min=0, slack_div=1 << 20)
    rows = om.rows_of(A)
    # inserts only: rows of C grow past their room
    cur = rows
    batches = []
    for k in range(3):
        rng = np.random.default_rng(90 + k)
        n = 400
        b = Batch(rng.integers(0, 300, n).astype(np.int32), rng.integers(0, 300, n).astype(np.int32),
                  rng.random(n), np.zeros(n, np.uint8))
        batches.append(b)
        cur, _ = om.apply_updates(cur, b)
    empty = Batch(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), np.zeros(0, np.uint8))
    absent = Batch(np.array([0], np.int32), np.array([299], np.int32), np.zeros(1), np.array([1], np.uint8))
    if 299 in cur[0]:
        absent = empty
    batches += [empty, absent]
    _run_sequence(dspg, g, rows, rows, batches, None, sr, True, 300, 300)
    st = g.apply_batch(empty)
    assert st["masked_entries"] == 0 and st["affected_rows"] == 0
    g.close()


def test_masked_handle_refuses_the_row_path_calls(dspg):
    A = random_csr(50, 50, 5, 11, PLUS_TIMES_F64)
    g = dspg.DynamicSpGEMM(A, bloom=True)
    b = random_batch(50, 50, 10, 12, PLUS_TIMES_F64)
    with pytest.raises(dspg.DspgError) as e:
        g.apply_batch(b, algebraic=True)
    assert e.value.status == 5
    with pytest.raises(dspg.DspgError) as e:
        g.apply_batch_async(b)
    assert e.value.status == 5
    with pytest.raises(dspg.DspgError) as e:
        g.autotune([b])
    assert e.value.status == 5
    with pytest.raises(dspg.DspgError) as e:
        dspg.Group([g])
    assert e.value.status == 5
    plain = dspg.DynamicSpGEMM(A)
    with pytest.raises(dspg.DspgError) as e:
        plain.read_bloom()
    assert e.value.status == 5
    # the handle still works after the refusals
    Ao = OMat.from_csr(A)
    g.apply_batch(b)
    Ao.apply(b)
    C_o, S_o = oracle_product(Ao, Ao)
    assert_matches(g.read_C(), C_o, S_o, what="after refusals")
    _bloom_matches(g, Ao, Ao, "after refusals")
    g.close()
    plain.close()


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_masked_staging_growth(dspg, sr):
    """A batch whose rebuilt rows of A need more staging than a batch of its
    size starts with (100 rows of 1,500 entries each): the merge is redone
    with grown staging, and the result matches as before."""
    rng = np.random.default_rng(61)
    from workloads import CSR
    rows = []
    for i in range(200):
        k = 1500 if i < 100 else 5
        rows.append({int(c): (float(rng.random()) if sr == PLUS_TIMES_F64 else int(rng.integers(1, 101)))
                     for c in rng.choice(3000, size=k, replace=False)})
    A = _csr_from_rows(rows, 3000, sr)
    B = random_csr(3000, 50, 3, 62, sr, empty_frac=0.0)
    g = dspg.DynamicSpGEMM(A, B, bloom=True)
    n = 300
    ops = rng.integers(0, 3, n).astype(np.uint8)
    vals = rng.random(n) if sr == PLUS_TIMES_F64 else rng.integers(1, 101, n).astype(np.int32)
    b = Batch(rng.integers(0, 100, n).astype(np.int32), rng.integers(0, 3000, n).astype(np.int32), vals, ops)
    _run_sequence(dspg, g, om.rows_of(A), om.rows_of(B), [b], [None], sr, False, 200, 50)
    g.close()
