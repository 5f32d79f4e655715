"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every test builds a handle on the GPU, applies batches with the library, and
compares C', A' and the affected row set R element by element with the
oracle's results on the same seeded inputs: patterns and (min,+) values
bit-exact, (+,.) values within 1e-12 * sum|ab| (see parity.py).
"""

import numpy as np
import pytest

import oracle
from oracle import OMat
from parity import assert_matches, assert_same_pattern, oracle_product
from workloads import (CSR, MIN_PLUS_I32, OP_DELETE, OP_SET, PLUS_TIMES_F64, Batch, bernoulli_sparse, er_batch,
                       er_matrix, random_batch, random_csr, rmat_edge_batch, rmat_symmetric, stencil7,
                       stencil_batch)

pytestmark = pytest.mark.gpu


def _check_state(g, A_or, B_or, what, rel=False):
    """C', A' (and R if given) of handle g against the oracle's A', B'."""
    C_o, S_o = oracle_product(A_or, B_or if B_or is not None else A_or)
    assert_matches(g.read_C(), C_o, S_o, what=f"{what} C", rel_check=rel)
    Ag = g.read_A()
    Ao = A_or.to_csr()
    assert_same_pattern(Ag, Ao, what=f"{what} A")
    assert np.array_equal(Ag.val, Ao.val), f"{what} A values"


def _apply_both(g, A_or, C_or, b, B_or=None, bb=None):
    st = g.apply_batch(b, bb)
    R = oracle.row_dynamic(A_or, C_or, b, B_or, bb)
    assert np.array_equal(g.last_affected(), R), "affected rows differ"
    assert st["affected_rows"] == R.shape[0]
    return st


# ------------------------------------------------------------------ static


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_static_build_er_config1(dspg, sr):
    A = er_matrix(4096, 8, seed=1, kind=sr)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    _check_state(g, Ao, None, "build", rel=(sr == PLUS_TIMES_F64))


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_static_build_skewed_all_bins(dspg, sr):
    """R-MAT rows give product bounds from 0 to tens of thousands, so every
    hash / dense bin of the recompute runs (the square has hubs)."""
    A, _ = rmat_symmetric(12, 16, (0.57, 0.19, 0.19, 0.05), seed=5, kind=sr)
    g = dspg.DynamicSpGEMM(A)
    _check_state(g, OMat.from_csr(A), None, "rmat12")


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_static_build_small_m_dense(dspg, sr):
    """C with 256 columns: the dense shared-memory accumulators (warp and CTA)."""
    A, _ = rmat_symmetric(12, 16, (0.57, 0.19, 0.19, 0.05), seed=6, kind=sr)
    B = bernoulli_sparse(A.ncols, 256, 0.08, seed=7, kind=sr)
    g = dspg.DynamicSpGEMM(A, B)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    C_o, S_o = oracle_product(Ao, Bo)
    assert_matches(g.read_C(), C_o, S_o, what="dense C")


def test_static_empty_and_ragged(dspg):
    for seed in range(4):
        A = random_csr(37, 53, 9, seed, PLUS_TIMES_F64, empty_frac=0.4)
        B = random_csr(53, 29, 7, seed + 1, PLUS_TIMES_F64, empty_frac=0.4)
        g = dspg.DynamicSpGEMM(A, B)
        C_o, S_o = oracle_product(OMat.from_csr(A), OMat.from_csr(B))
        assert_matches(g.read_C(), C_o, S_o, what=f"ragged {seed}")


def test_build_rejects_noncanonical_input(dspg):
    A = random_csr(10, 10, 4, 0, PLUS_TIMES_F64)
    i = int(np.argmax(np.diff(A.rowptr) >= 2))
    bad = A.col.copy()
    s = A.rowptr[i]
    bad[s], bad[s + 1] = bad[s + 1], bad[s]
    from workloads import CSR
    with pytest.raises(dspg.DspgError) as e:
        dspg.DynamicSpGEMM(CSR(10, 10, A.rowptr, bad, A.val))
    assert e.value.status == 1


# ------------------------------------------------------------------ dynamic


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_config1_batch(dspg, sr):
    """ER n=4096, 8 per row; one batch of 512 inserts, 256 deletes, 256 value
    changes; C' against the oracle's A' A' and R against the oracle's R."""
    A = er_matrix(4096, 8, seed=1, kind=sr)
    b = er_batch(A, seed=2)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    st = _apply_both(g, Ao, Co, b)
    assert st["n_insert"] == 512 and st["n_delete"] == 256 and st["n_update"] == 256 and st["n_noop"] == 0
    _check_state(g, Ao, None, "config1", rel=(sr == PLUS_TIMES_F64))


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
@pytest.mark.parametrize("seed", range(6))
def test_random_batches_sequence(dspg, sr, seed):
    """Uneven rows, empty rows, duplicate keys in a batch, deletes of absent
    entries, several batches in a row (state carries over)."""
    n = 300
    A = random_csr(n, n, 12, seed, sr, empty_frac=0.2)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    for k in range(4):
        b = random_batch(n, n, [1, 17, 300, 2500][k], seed * 10 + k, sr, A=Ao.to_csr(), dup_frac=0.3)
        _apply_both(g, Ao, Co, b)
        _check_state(g, Ao, None, f"seed{seed} batch{k}")


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_separate_b_with_both_batches(dspg, sr):
    A = random_csr(200, 150, 10, 3, sr)
    B = random_csr(150, 180, 10, 4, sr)
    g = dspg.DynamicSpGEMM(A, B)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    Co = Ao.multiply(Bo)
    for k in range(3):
        ba = random_batch(200, 150, 120, 40 + k, sr, A=Ao.to_csr())
        bb = random_batch(150, 180, 90, 50 + k, sr, A=Bo.to_csr())
        _apply_both(g, Ao, Co, ba, Bo, bb)
        C_o, S_o = oracle_product(Ao, Bo)
        assert_matches(g.read_C(), C_o, S_o, what=f"AB batch {k}")
    # a batch on A only, after the transposed pattern exists
    ba = random_batch(200, 150, 60, 77, sr, A=Ao.to_csr())
    _apply_both(g, Ao, Co, ba, Bo, None)
    C_o, S_o = oracle_product(Ao, Bo)
    assert_matches(g.read_C(), C_o, S_o, what="A-only batch")


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_short_rows_with_more_products_than_columns(dspg, sr):
    """C with 20 columns, A rows of at most 8 entries reading B rows of up to
    18: a row's product bound (up to 144) exceeds both the column count and
    the thread-merge staging size, so the merge bins must be chosen by the
    uncapped bound, every tuning candidate alike."""
    A = random_csr(300, 30, 8, 5, sr, empty_frac=0.05)
    B = random_csr(30, 20, 18, 6, sr, empty_frac=0.0)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    for cand in dspg.tuning_candidates():
        g = dspg.DynamicSpGEMM(A, B)
        g.set_tuning(cand)
        Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
        Co = Ao.multiply(Bo)
        C_o, S_o = oracle_product(Ao, Bo)
        assert_matches(g.read_C(), C_o, S_o, what=f"static {cand}")
        ba = random_batch(300, 30, 200, 7, sr, A=A)
        _apply_both(g, Ao, Co, ba, Bo, None)
        C_o, S_o = oracle_product(Ao, Bo)
        assert_matches(g.read_C(), C_o, S_o, what=f"batch {cand}")
        g.close()


def test_locality_rows_outside_R_unchanged_bitwise(dspg):
    A = er_matrix(2048, 8, seed=11)
    g = dspg.DynamicSpGEMM(A)
    before = g.read_C()
    b = er_batch(A, seed=12, n_insert=20, n_delete=10, n_set=10)
    g.apply_batch(b)
    R = g.last_affected()
    after = g.read_C()
    keep = np.setdiff1d(np.arange(A.nrows), R)
    for i in keep[:: max(1, keep.shape[0] // 500)]:
        s0, s1 = before.rowptr[i], before.rowptr[i + 1]
        t0, t1 = after.rowptr[i], after.rowptr[i + 1]
        assert np.array_equal(before.col[s0:s1], after.col[t0:t1])
        assert np.array_equal(before.val[s0:s1].view(np.int64), after.val[t0:t1].view(np.int64))


def test_edge_batches(dspg):
    sr = PLUS_TIMES_F64
    A = random_csr(120, 120, 8, 9, sr)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    # empty batch
    empty = Batch(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), np.zeros(0, np.uint8))
    st = _apply_both(g, Ao, Co, empty)
    assert st["affected_rows"] == 0
    # only deletes of absent entries: nothing changes, R empty
    present = set(zip(A.row_ids().tolist(), A.col.tolist()))
    absent = [(i, j) for i in range(5) for j in range(120) if (i, j) not in present][:10]
    b = Batch(np.array([p[0] for p in absent], np.int32), np.array([p[1] for p in absent], np.int32),
              np.zeros(len(absent)), np.full(len(absent), OP_DELETE, np.uint8))
    st = _apply_both(g, Ao, Co, b)
    assert st["affected_rows"] == 0 and st["n_noop"] == len(absent)
    # delete every entry of the longest row, and write the last row
    r = int(np.argmax(np.diff(A.rowptr)))
    cols = A.col[A.rowptr[r]:A.rowptr[r + 1]]
    b = Batch(np.concatenate([np.full(cols.shape[0], r, np.int32), np.full(3, 119, np.int32)]),
              np.concatenate([cols, np.array([0, 60, 119], np.int32)]),
              np.concatenate([np.zeros(cols.shape[0]), np.array([1.5, -2.0, 0.0])]),
              np.concatenate([np.full(cols.shape[0], OP_DELETE, np.uint8), np.full(3, OP_SET, np.uint8)]))
    _apply_both(g, Ao, Co, b)
    _check_state(g, Ao, None, "edge")


def test_invalid_batch_leaves_state(dspg):
    sr = MIN_PLUS_I32
    A = random_csr(80, 80, 6, 21, sr)
    g = dspg.DynamicSpGEMM(A)
    C0, A0 = g.read_C(), g.read_A()
    for bad in ("row", "op", "value"):
        b = random_batch(80, 80, 40, 22, sr, A=A)
        if bad == "row":
            b.row[7] = 80
        elif bad == "op":
            b.op[3] = 9
        else:
            b.op[5] = OP_SET
            b.val[5] = np.iinfo(np.int32).max
        with pytest.raises(dspg.DspgError) as e:
            g.apply_batch(b)
        assert e.value.status == 1
        C1, A1 = g.read_C(), g.read_A()
        assert np.array_equal(C1.col, C0.col) and np.array_equal(C1.val, C0.val)
        assert np.array_equal(A1.col, A0.col) and np.array_equal(A1.val, A0.val)


def test_growth_paths_tight_arena(dspg):
    """No slack and no arena headroom: every insert relocates its row, the
    tails run out and the arenas are rebuilt mid-batch; results unchanged."""
    sr = PLUS_TIMES_F64
    A = random_csr(400, 400, 10, 31, sr)
    g = dspg.DynamicSpGEMM(A, slack_min=0, slack_div=1 << 20, arena_headroom=1.0)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    total = 0
    for k in range(3):
        b = random_batch(400, 400, 3000, 60 + k, sr, A=Ao.to_csr(), hit_frac=0.1)
        st = _apply_both(g, Ao, Co, b)
        total += st["compactions"]
        _check_state(g, Ao, None, f"tight {k}")
    assert total > 0


@pytest.mark.parametrize("nupd,sr", [(1023, PLUS_TIMES_F64), (1024, PLUS_TIMES_F64), (1025, PLUS_TIMES_F64),
                                     (2049, PLUS_TIMES_F64), (6000, PLUS_TIMES_F64), (8192, PLUS_TIMES_F64),
                                     (8193, PLUS_TIMES_F64), (10000, PLUS_TIMES_F64), (10000, MIN_PLUS_I32),
                                     (15000, MIN_PLUS_I32), (16384, PLUS_TIMES_F64), (16385, PLUS_TIMES_F64)])
def test_batch_sizes_at_the_sort_tile_bounds(dspg, nupd, sr):
    """Batch sizes around the sort's tiles (1024 words per CTA, up to 16 CTAs
    in one cluster where the device allows it, else 2048 words in up to 8;
    above 8192 entries the cluster's radix sort where clusters of 16 are
    allowed; 16385 takes the multi-pass radix path), half of the entries
    repeating keys, so that a key's last write and its dead copies sit in
    different tiles."""
    A = er_matrix(3000, 6, seed=43, kind=sr)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    b = random_batch(3000, 3000, nupd, 44 + nupd, sr, A=A, dup_frac=0.5)
    st = _apply_both(g, Ao, Co, b)
    assert st["n_unique"] < nupd
    _check_state(g, Ao, None, f"batch of {nupd}")


def test_large_batch_multi_cta_sort(dspg):
    """Batches above the single-CTA sort size take the multi-pass radix sort."""
    sr = MIN_PLUS_I32
    A = er_matrix(20000, 6, seed=41, kind=sr)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    b = random_batch(20000, 20000, 30000, 42, sr, A=A, dup_frac=0.3)
    _apply_both(g, Ao, Co, b)
    _check_state(g, Ao, None, "big batch")


# ------------------------------------------------------------ full configs


def _sampled_rows(g, A_or, B_or, rows, what):
    rp, col, val = g.read_rows_C(rows)
    orp, ocol, oval = A_or.multiply_rows(B_or, rows)
    assert np.array_equal(rp, orp), f"{what}: row lengths"
    assert np.array_equal(col, ocol), f"{what}: columns"
    if oval.dtype == np.float64:
        _, _, sabs = A_or.multiply_rows(B_or, rows, absval=True)
        assert np.all(np.abs(val - oval) <= 1e-12 * sabs), f"{what}: values"
    else:
        assert np.array_equal(val, oval), f"{what}: values"


def test_config2_stencil_full_size(dspg):
    """128^3 7-point stencil, C = A A (51,742,208 non-zeros), batches of
    10^3 and 10^4 mixed updates within two grid hops: full C' compared."""
    A = stencil7(128, 128, 128, seed=1)
    g = dspg.DynamicSpGEMM(A)
    assert g.info()["nnz_c"] == 51742208
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    for k, nb in enumerate([1000, 10000]):
        b = stencil_batch(128, 128, 128, nb, seed=10 + k)
        _apply_both(g, Ao, Co, b)
    C_o = Co.to_csr()
    Cg = g.read_C()
    assert_same_pattern(Cg, C_o, "stencil C")
    S_o = Ao.multiply(Ao, absval=True).to_csr()
    err = np.abs(Cg.val - C_o.val)
    assert np.all(err <= 1e-12 * S_o.val)
    # and relative to the entry itself (no entry of this C cancels: S / |C| <= 3.4 here)
    nz = C_o.val != 0
    assert (err[nz] / np.abs(C_o.val[nz])).max() <= 1e-12


def test_config3_rmat_minplus_full_size(dspg):
    """R-MAT scale 20, edge factor 16, min-plus A B with B n x 256 at 1%;
    edge batches of 10^2 and 10^4 (inserts of held-out edges, deletes of
    present ones); C' bit-exact on all affected rows and a row sample."""
    A, held = rmat_symmetric(20, 16, (0.57, 0.19, 0.19, 0.05), seed=3, kind=MIN_PLUS_I32, holdout=1 << 16)
    B = bernoulli_sparse(A.ncols, 256, 0.01, seed=4, kind=MIN_PLUS_I32)
    g = dspg.DynamicSpGEMM(A, B)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    rng = np.random.default_rng(0)
    _sampled_rows(g, Ao, Bo, np.sort(rng.choice(A.nrows, 4000, replace=False)), "rmat build")
    for k, ne in enumerate([100, 10000]):
        b = rmat_edge_batch(Ao.to_csr() if k else A, held, ne, seed=30 + k)
        g.apply_batch(b)
        pre = None
        Ao.apply(b)
        R = g.last_affected()
        assert np.array_equal(R, np.unique(b.row)), "R = rows of the A batch when B does not change"
        _sampled_rows(g, Ao, Bo, R, f"rmat batch {k} R")
        _sampled_rows(g, Ao, Bo, np.sort(rng.choice(A.nrows, 2000, replace=False)), f"rmat batch {k} sample")


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_repeated_shape_captured_pipeline(dspg, sr):
    """Equal-size batches: the first runs eagerly, the second is captured as a
    CUDA graph, later ones replay it; every result must match the oracle."""
    n = 2000
    A = random_csr(n, n, 10, 77, sr)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    for k in range(5):
        b = random_batch(n, n, 700, 500 + k, sr, A=Ao.to_csr(), dup_frac=0.2)
        _apply_both(g, Ao, Co, b)
        _check_state(g, Ao, None, f"replay {k}")


def test_graph_and_eager_agree_minplus(dspg):
    """Same batches through captured graphs and through the eager path
    (profiling on) give bit-identical (min,+) results."""
    n = 1500
    A = random_csr(n, n, 9, 88, MIN_PLUS_I32)
    g1 = dspg.DynamicSpGEMM(A)
    g2 = dspg.DynamicSpGEMM(A)
    g2.set_profiling(True)
    for k in range(4):
        b = random_batch(n, n, 400, 900 + k, MIN_PLUS_I32, A=A)
        g1.apply_batch(b)
        g2.apply_batch(b)
        assert g2.stage_times()["numeric"] >= 0.0
    c1, c2 = g1.read_C(), g2.read_C()
    assert np.array_equal(c1.rowptr, c2.rowptr) and np.array_equal(c1.col, c2.col)
    assert np.array_equal(c1.val, c2.val)


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_exact_two_pass_static_layout(dspg, sr):
    """The static product laid out from exact row counts (count pass, then
    write pass) gives the same C, and later batches still match."""
    A, _ = rmat_symmetric(11, 8, (0.57, 0.19, 0.19, 0.05), seed=9, kind=sr)
    g = dspg.DynamicSpGEMM(A, exact_static=1)
    Ao = OMat.from_csr(A)
    _check_state(g, Ao, None, "exact static")
    Co = Ao.multiply(Ao)
    b = random_batch(A.nrows, A.ncols, 500, 19, sr, A=A)
    _apply_both(g, Ao, Co, b)
    _check_state(g, Ao, None, "exact static + batch")
    g.recompute_all()
    _check_state(g, Ao, None, "exact static recompute")


def _with_hubs(n, k, hub_rows, hub_len, sr, seed, short_max=12):
    """n x k matrix: rows of 0..short_max random columns, and the rows in
    hub_rows with hub_len columns each (the hubs of skewed graphs)."""
    from workloads import CSR
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        L = hub_len if i in hub_rows else int(rng.integers(0, short_max + 1))
        c = rng.choice(k, size=min(L, k), replace=False)
        rows.append(np.full(c.shape[0], i, np.int64))
        cols.append(c.astype(np.int64))
    r, c = np.concatenate(rows), np.concatenate(cols)
    order = np.argsort(r * k + c, kind="stable")
    r, c = r[order], c[order]
    v = rng.random(r.shape[0]) if sr == PLUS_TIMES_F64 else rng.integers(1, 101, r.shape[0]).astype(np.int32)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rowptr[1:])
    return CSR(n, k, rowptr, c.astype(np.int32), v)


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_hub_rows_split_across_ctas_small_m(dspg, sr):
    """C with 256 columns (dense accumulators): rows of A with 3000-5000
    entries over B rows of ~25 entries have over 16384 products each, so the
    split kernel recomputes them with every CTA (a chunk of the A row each);
    their A rows are also longer than a warp sizes (a CTA sizes them).  Static
    build and batches that touch the hubs, against the oracle."""
    hubs = {3, 700, 701, 1999}
    A = _with_hubs(2000, 6000, hubs, 4000, sr, 151)
    B = bernoulli_sparse(6000, 256, 0.1, seed=152, kind=sr)
    g = dspg.DynamicSpGEMM(A, B)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    _check_state(g, Ao, Bo, "hub build")
    Co = Ao.multiply(Bo)
    for k in range(3):
        b = random_batch(A.nrows, A.ncols, 400, 153 + k, sr, A=A)
        # a few more updates on the hub rows themselves
        extra = random_batch(A.nrows, A.ncols, 60, 160 + k, sr, A=A)
        extra.row[:] = np.array(sorted(hubs), np.int32)[np.arange(60) % len(hubs)]
        from workloads import concat_batches
        bb = concat_batches(b, extra)
        st = g.apply_batch(bb)
        R = oracle.row_dynamic(Ao, Co, bb, Bo)
        assert np.array_equal(g.last_affected(), R)
        _check_state(g, Ao, Bo, f"hub batch {k}")
    g.recompute_all()
    _check_state(g, Ao, Bo, "hub recompute")


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_long_rows_sized_by_a_cta_wide_m(dspg, sr):
    """C with 5000 columns (hash and global dense bins): A rows longer than
    512 entries are sized by a CTA each; static build and batches against
    the oracle."""
    hubs = {0, 10, 11, 1499}
    A = _with_hubs(1500, 5000, hubs, 3000, sr, 171)
    B = random_csr(5000, 5000, 6, 172, sr)
    g = dspg.DynamicSpGEMM(A, B)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    _check_state(g, Ao, Bo, "long-row build")
    Co = Ao.multiply(Bo)
    for k in range(2):
        b = random_batch(A.nrows, A.ncols, 300, 173 + k, sr, A=A)
        b.row[:40] = np.array(sorted(hubs), np.int32)[np.arange(40) % len(hubs)]
        g.apply_batch(b)
        R = oracle.row_dynamic(Ao, Co, b, Bo)
        assert np.array_equal(g.last_affected(), R)
        _check_state(g, Ao, Bo, f"long-row batch {k}")


@pytest.mark.parametrize("cta_max", [8192, 16384])
def test_rows_longer_than_the_tables_are_read_in_order(dspg, cta_max):
    """Rows of C with 9,000 to 30,000 entries (hub rows of A over 60,000
    columns): beyond the shared-memory tables they go to the global dense
    kernel (or, with cta_max 16384, partly to the 16384-slot CTA table), and
    every read returns them in column order, equal to the oracle's."""
    sr = PLUS_TIMES_F64
    hubs = {2, 300, 599}
    A = _with_hubs(600, 3000, hubs, 2900, sr, 201)
    B = random_csr(3000, 60000, 20, 202, sr)
    g = dspg.DynamicSpGEMM(A, B)
    g.set_tuning(dict(dspg.tuning_candidates()[0], cta_max=cta_max))
    g.recompute_all()
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    _check_state(g, Ao, Bo, f"long rows (cta_max {cta_max})")
    Co = Ao.multiply(Bo)
    lens = np.diff(Co.to_csr().rowptr)
    assert lens.max() > 16384, "no row beyond the largest table"
    b = random_batch(A.nrows, A.ncols, 200, 203, sr, A=A)
    b.row[:30] = np.array(sorted(hubs), np.int32)[np.arange(30) % len(hubs)]
    g.apply_batch(b)
    R = oracle.row_dynamic(Ao, Co, b, Bo)
    assert np.array_equal(g.last_affected(), R)
    _check_state(g, Ao, Bo, f"long rows after a batch (cta_max {cta_max})")
    rows = np.array(sorted(hubs) + [0, 1], np.int32)
    rp, col, val = g.read_rows_C(rows)
    o_rp, o_col, o_val = Ao.multiply_rows(Bo, rows)
    assert np.array_equal(rp, o_rp) and np.array_equal(col, o_col)


def _hub_lengths(n, k, hub_lens, sr, seed, short_max=6):
    """n x k matrix whose rows 0..len(hub_lens)-1 have the given lengths and
    the others 0..short_max random columns."""
    from workloads import CSR
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        L = hub_lens[i] if i < len(hub_lens) else int(rng.integers(0, short_max + 1))
        c = np.sort(rng.choice(k, size=min(L, k), replace=False))
        rows.append(np.full(c.shape[0], i, np.int64))
        cols.append(c.astype(np.int64))
    r, c = np.concatenate(rows), np.concatenate(cols)
    v = rng.random(r.shape[0]) if sr == PLUS_TIMES_F64 else rng.integers(1, 101, r.shape[0]).astype(np.int32)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rowptr[1:])
    return CSR(n, k, rowptr, c.astype(np.int32), v)


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_rows_in_cluster_tables_and_beyond(dspg, sr):
    """Rows of C with about 20,000, 45,000, 100,000 and 150,000 products
    over 400,000 columns (nearly all distinct): they go to the tables that
    span 4 and 8 CTAs of a cluster (distributed shared memory), to the one of
    8 CTAs x 16384 slots, and past it to the global dense kernel; C' equals
    the oracle's, statically, after a batch on the hub rows, and in every
    read (rows longer than a CTA can sort are sorted together)."""
    A = _hub_lengths(64, 20000, [2000, 4500, 10000, 15000], sr, 211)
    B = random_csr(20000, 400000, 20, 212, sr, empty_frac=0.0)
    g = dspg.DynamicSpGEMM(A, B)
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    Co = Ao.multiply(Bo)
    blen = np.diff(B.rowptr)
    prods = [int(blen[A.col[A.rowptr[i]:A.rowptr[i + 1]]].sum()) for i in range(4)]
    assert 2 * 8192 < prods[0] <= 4 * 8192 < prods[1] <= 8 * 8192 < prods[2] <= 8 * 16384 < prods[3], prods
    assert np.diff(Co.to_csr().rowptr)[:4].min() > 16384
    _check_state(g, Ao, Bo, "cluster tables, static")
    b = random_batch(A.nrows, A.ncols, 400, 213, sr, A=A)
    b.row[:40] = np.arange(40, dtype=np.int32) % 4
    _apply_both(g, Ao, Co, b, Bo, None)
    _check_state(g, Ao, Bo, "cluster tables, after a batch")
    rows = np.array([3, 0, 2, 1, 17], np.int32)
    rp, col, val = g.read_rows_C(rows)
    o_rp, o_col, o_val = Ao.multiply_rows(Bo, rows)
    assert np.array_equal(rp, o_rp) and np.array_equal(col, o_col)


def test_row_reads_between_batches(dspg):
    """A two-call read of C's rows (count, then fill) reuses the count's row
    pointers only for the same rows of the same C: the affected rows read
    twice, another list of the same length, a read of all of C in between,
    and the next batches each give the oracle's rows."""
    sr = PLUS_TIMES_F64
    n = 4000
    A = er_matrix(n, 6, seed=71, kind=sr)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    rng = np.random.default_rng(72)
    for t in range(3):
        _apply_both(g, Ao, Co, random_batch(n, n, 400, 73 + t, sr, A=A))
        R = g.last_affected()
        assert R.size > 0
        _sampled_rows(g, Ao, Ao, R, f"batch {t}: R")
        _sampled_rows(g, Ao, Ao, R, f"batch {t}: R again")
        other = np.sort(rng.choice(n, size=R.size, replace=False)).astype(np.int32)
        _sampled_rows(g, Ao, Ao, other, f"batch {t}: other rows")
        g.read_C()
        _sampled_rows(g, Ao, Ao, R, f"batch {t}: R after a read of C")


@pytest.mark.parametrize("bloom", [False, True])
@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_read_affected_in_one_call(dspg, sr, bloom):
    """dspg_read_affected_C returns R ascending and its rows of C' in one
    call: the same as dspg_last_affected and a read of those rows, against
    the oracle (row path, masked path, the delta path's batches, an empty
    batch, and buffers that start too small)."""
    n = 3000
    A = er_matrix(n, 6, seed=81, kind=sr)
    g = dspg.DynamicSpGEMM(A, bloom=bloom)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    g._aff_cap = (4, 4)  # too small: the binding grows them and calls again
    empty = Batch(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, A.val.dtype), np.zeros(0, np.uint8))
    batches = [random_batch(n, n, 300 + 200 * t, 82 + t, sr, A=A) for t in range(3)] + [empty]
    for t, b in enumerate(batches):
        if bloom:
            g.apply_batch(b)
            Ao.apply(b)
        else:
            _apply_both(g, Ao, Co, b)
        rows, rp, col, val = g.read_affected()
        R = g.last_affected()
        assert np.array_equal(rows, R), f"batch {t}: rows"
        assert np.all(np.diff(rows) > 0)
        orp, ocol, oval = Ao.multiply_rows(Ao, rows)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol), f"batch {t}: pattern"
        if sr == MIN_PLUS_I32:
            assert np.array_equal(val, oval)
        else:
            _, _, sabs = Ao.multiply_rows(Ao, rows, absval=True)
            assert np.all(np.abs(val - oval) <= 1e-12 * sabs), f"batch {t}: values"
    if not bloom:
        # an insert-only batch through the delta path, then the read
        Ag = g.read_A()
        rng = np.random.default_rng(90)
        present = set(zip(np.repeat(np.arange(n), np.diff(Ag.rowptr)).tolist(), Ag.col.tolist()))
        ins = [(int(i), int(j)) for i, j in zip(rng.integers(0, n, 400), rng.integers(0, n, 400)) if (i, j) not in present]
        ins = list(dict.fromkeys(ins))
        vals = rng.random(len(ins)) if sr == PLUS_TIMES_F64 else rng.integers(1, 101, len(ins)).astype(np.int32)
        b = Batch(np.array([i for i, _ in ins], np.int32), np.array([j for _, j in ins], np.int32), vals,
                  np.zeros(len(ins), np.uint8))
        g.apply_batch(b, algebraic=True)
        Ao.apply(b)
        rows, rp, col, val = g.read_affected()
        assert np.array_equal(rows, g.last_affected())
        orp, ocol, _ = Ao.multiply_rows(Ao, rows)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    g.close()


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_captured_pipeline_serves_uneven_sizes(dspg, sr, monkeypatch):
    """Batches of different sizes within one launch size (a multiple of 1024
    up to 16384, powers of two beyond): after the first two, every batch
    replays the same captured pipeline (no new kernels are captured), which
    reads each batch's own length on the device; every result matches the
    oracle.  Sizes cross the cluster sort's limit too (LSD path).  Every
    recompute bin is launched here (a batch whose rows first reach a bin
    that is off is captured anew: test_bins_off_go_to_global_dense)."""
    n = 3000
    A = random_csr(n, n, 10, 311, sr)
    # room in the arenas, so that no buffer moves (which would retire the
    # captured pipeline) during the sequence
    monkeypatch.setenv("DSPG_ALL_BINS", "1")
    g = dspg.DynamicSpGEMM(A, arena_headroom=4.0)
    monkeypatch.delenv("DSPG_ALL_BINS")
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    for sizes in ([700, 900, 1000, 13, 333, 1024, 1], [20000, 17000, 30000, 16385]):
        r0 = g.run_counts()
        for k, m in enumerate(sizes):
            b = random_batch(n, n, m, 312 + 17 * k + m, sr, A=Ao.to_csr(), dup_frac=0.2)
            _apply_both(g, Ao, Co, b)
            _check_state(g, Ao, None, f"size {m}")
        r1 = g.run_counts()
        # one launch size: run eagerly once, captured once, then replayed
        # (a buffer that still has to grow once costs one more of each)
        assert r1["eager"] - r0["eager"] <= 2 and r1["captured"] - r0["captured"] <= 2, (r0, r1)
        assert r1["replayed"] - r0["replayed"] >= len(sizes) - 4, (r0, r1)


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_bins_off_go_to_global_dense(dspg, sr, monkeypatch):
    """After its first batch a handle launches only the recompute bins that
    batch used (plus the global dense bin).  A first batch confined to a
    low-degree corner of an R-MAT square leaves most bins off; the next,
    spread over the hubs, sends the rows of the bins that are off to the
    global dense bin (seen in its larger tables against a handle that
    launches every bin), and turns those bins on.  C' and R match the oracle
    after every batch on both handles."""
    A, _ = rmat_symmetric(12, 16, (0.57, 0.19, 0.19, 0.05), seed=9, kind=sr)
    g = dspg.DynamicSpGEMM(A)
    monkeypatch.setenv("DSPG_ALL_BINS", "1")
    g_all = dspg.DynamicSpGEMM(A)
    monkeypatch.delenv("DSPG_ALL_BINS")
    Ao = OMat.from_csr(A)
    deg = np.diff(A.rowptr)
    # an entry (i, j) with both ends of degree 1 or 2: few affected rows, few products
    rows = np.repeat(np.arange(A.nrows), deg)
    pick = np.flatnonzero((deg[rows] <= 2) & (deg[A.col] <= 2))
    assert pick.size > 0
    p = pick[0]
    val = A.val[p:p + 1].copy()
    first = Batch(np.array([rows[p]], np.int32), np.array([A.col[p]], np.int32), val + 1,
                  np.array([OP_SET], np.uint8))
    batches = [first] + [random_batch(A.nrows, A.ncols, 600, 40 + k, sr, A=None, dup_frac=0.2) for k in range(3)]
    slots = []
    for k, b in enumerate(batches):
        Co = Ao.multiply(Ao)
        st = _apply_both(g, Ao, Co, b)
        st_all = g_all.apply_batch(b)
        assert st_all["affected_rows"] == st["affected_rows"]
        Ao.apply(b)
        _check_state(g, Ao, None, f"gated batch {k}")
        _check_state(g_all, Ao, None, f"all-bins batch {k}")
        slots.append((st["table_slots"], st_all["table_slots"]))
    # the second batch's hub rows went to the global dense bin (m slots each)
    assert slots[1][0] > slots[1][1], slots
    # once the bins the batches need are on, batches of one launch size replay
    r0 = g.run_counts()
    for k in range(4):
        b = random_batch(A.nrows, A.ncols, 600, 60 + k, sr, A=None, dup_frac=0.2)
        Co = Ao.multiply(Ao)
        _apply_both(g, Ao, Co, b)
        Ao.apply(b)
    _check_state(g, Ao, None, "gated, bins learned")
    r1 = g.run_counts()
    assert r1["replayed"] - r0["replayed"] >= 2, (r0, r1)


def _csr_of_rows(cols_per_row, ncols, sr, rng):
    rp = np.zeros(len(cols_per_row) + 1, np.int64)
    rp[1:] = np.cumsum([len(c) for c in cols_per_row])
    col = np.concatenate([np.sort(np.asarray(c, np.int64)) for c in cols_per_row]).astype(np.int32)
    nnz = col.shape[0]
    val = rng.random(nnz) + 0.5 if sr == PLUS_TIMES_F64 else rng.integers(1, 101, nnz).astype(np.int32)
    return CSR(len(cols_per_row), ncols, rp, col, val)


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_read_affected_rows_of_every_length(dspg, sr, monkeypatch):
    """The one-call read writes the rows of C' straight into page-locked host
    arrays: rows of up to 64 entries put in column order in registers (the
    group sort's rows arrive in order; rows of colliding products from the
    hash tables do not), longer ones in shared memory, and rows of more than
    16384 entries out of order (hub rows of A over B rows of ~20 entries,
    from the cluster tables) by the radix sort.  R and every row equal the
    oracle's, and the read that stages the rows on the device first; so do
    those of apply_read_affected into page-locked arrays (the read enqueued
    behind the batch)."""
    import torch
    rng = np.random.default_rng(93)
    n, k, m = 1200, 4000, 400000
    bcols = [rng.choice(m, size=int(rng.integers(0, 41)), replace=False) for _ in range(k)]
    shared = rng.choice(m, size=30, replace=False)
    for q in range(10):  # B rows 0..9 share their 30 columns: rows of A over them collide
        bcols[q] = shared
    B = _csr_of_rows(bcols, m, sr, rng)
    acols = [rng.choice(np.arange(10, k), size=int(rng.choice([0, 1, 2, 3, 6, 12])), replace=False) for _ in range(n)]
    for i in range(100, 120):
        acols[i] = np.arange(10)
    for i in (5, 600, 1111):
        acols[i] = rng.choice(np.arange(10, k), size=1000, replace=False)  # hubs
    A = _csr_of_rows(acols, k, sr, rng)
    g = dspg.DynamicSpGEMM(A, B)
    monkeypatch.setenv("DSPG_NO_DIRECT_READ", "1")
    g_staged = dspg.DynamicSpGEMM(A, B)
    monkeypatch.delenv("DSPG_NO_DIRECT_READ")
    g_one = dspg.DynamicSpGEMM(A, B)
    vt = torch.float64 if sr == PLUS_TIMES_F64 else torch.int32
    out = tuple(torch.empty(q, dtype=dt, pin_memory=True).numpy()
                for q, dt in ((n, torch.int32), (n + 1, torch.int64), (2000000, torch.int32), (2000000, vt)))
    Ao, Bo = OMat.from_csr(A), OMat.from_csr(B)
    for t in range(2):
        b = random_batch(n, k, 600, 95 + t, sr, A=Ao.to_csr(), dup_frac=0.1)
        b.row[:23] = np.array([5, 600, 1111] + list(range(100, 120)), np.int32)  # hubs and colliding rows in R
        b.col[:23] = np.array([10 + t] * 3 + [0] * 20, np.int32)
        b.op[:23] = OP_SET
        b.val[:23] = b.val[:23] * 0 + 2
        g.apply_batch(b)
        g_staged.apply_batch(b)
        _, (rows_1, rp_1, col_1, val_1) = g_one.apply_read_affected(b, out=out)
        Ao.apply(b)
        rows, rp_g, col, val = g.read_affected()
        rows_s, rp_s, col_s, val_s = g_staged.read_affected()
        assert np.shares_memory(col_1, out[2]), "out arrays not used"
        assert np.array_equal(rows_1, rows) and np.array_equal(rp_1, rp_g) and np.array_equal(col_1, col)
        assert np.array_equal(rows, g.last_affected()) and np.array_equal(rows, rows_s)
        lens_c = np.diff(rp_g)
        assert lens_c.max() > 16384 and ((lens_c > 64) & (lens_c <= 16384)).any() and (lens_c <= 64).any()
        orp, ocol, oval = Ao.multiply_rows(Bo, rows)
        assert np.array_equal(rp_g, orp) and np.array_equal(col, ocol), f"batch {t}: pattern"
        assert np.array_equal(rp_s, rp_g) and np.array_equal(col_s, col)
        if sr == MIN_PLUS_I32:
            # (min,+) is order-free; (+,.) sums of the hash bins depend on the
            # order of their shared-memory atomics, so the two handles' values
            # are each checked against the oracle below instead
            assert np.array_equal(val_s, val) and np.array_equal(val_1, val)
            assert np.array_equal(val, oval)
        else:
            _, _, sabs = Ao.multiply_rows(Bo, rows, absval=True)
            assert np.all(np.abs(val - oval) <= 1e-12 * sabs), f"batch {t}: values"
            assert np.all(np.abs(val_s - oval) <= 1e-12 * sabs), f"batch {t}: staged values"
            assert np.all(np.abs(val_1 - oval) <= 1e-12 * sabs), f"batch {t}: one-call values"


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_read_affected_into_caller_arrays(dspg, sr):
    """read_affected(out=...) fills caller-owned arrays: page-locked ones
    (written from the device directly), pageable ones (staged and copied),
    and arrays too small for the result (the binding then returns arrays of
    its own); every result equals the default read and the oracle's rows."""
    import torch
    n = 3000
    A = er_matrix(n, 6, seed=97, kind=sr)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    vt = torch.float64 if sr == PLUS_TIMES_F64 else torch.int32
    vn = np.float64 if sr == PLUS_TIMES_F64 else np.int32
    pinned = tuple(torch.empty(m, dtype=dt, pin_memory=True).numpy()
                   for m, dt in ((n, torch.int32), (n + 1, torch.int64), (200000, torch.int32), (200000, vt)))
    pageable = (np.empty(n, np.int32), np.empty(n + 1, np.int64), np.empty(200000, np.int32), np.empty(200000, vn))
    small = (np.empty(4, np.int32), np.empty(5, np.int64), np.empty(4, np.int32), np.empty(4, vn))
    for t, out in enumerate((pinned, pageable, small, pinned)):
        b = random_batch(n, n, 400, 98 + t, sr, A=Ao.to_csr())
        g.apply_batch(b)
        Ao.apply(b)
        rows, rp, col, val = g.read_affected(out=out)
        if out is not small:
            assert rows.base is not None and np.shares_memory(rows, out[0]), "out arrays not used"
        r2, rp2, c2, v2 = g.read_affected()
        assert np.array_equal(rows, r2) and np.array_equal(rp, rp2) and np.array_equal(col, c2)
        assert np.array_equal(val, v2)
        orp, ocol, oval = Ao.multiply_rows(Ao, rows)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol), f"read {t}: pattern"
        if sr == MIN_PLUS_I32:
            assert np.array_equal(val, oval)
        else:
            _, _, sabs = Ao.multiply_rows(Ao, rows, absval=True)
            assert np.all(np.abs(val - oval) <= 1e-12 * sabs), f"read {t}: values"


def _check_rows_of_c(Ao, rows, rp, col, val, sr, what):
    orp, ocol, oval = Ao.multiply_rows(Ao, rows)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol), f"{what}: pattern"
    if sr == MIN_PLUS_I32:
        assert np.array_equal(val, oval), f"{what}: values"
    else:
        _, _, sabs = Ao.multiply_rows(Ao, rows, absval=True)
        assert np.all(np.abs(val - oval) <= 1e-12 * sabs), f"{what}: values"


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_apply_read_affected_one_call(dspg, sr):
    """apply_read_affected: a batch and the read of its affected rows in one
    call.  With page-locked arrays the read is enqueued behind the batch and
    takes R's size from the device (one synchronisation); pageable arrays,
    arrays too small for the result and batches that need a second pass (a
    tight arena rebuilt mid-batch) take the read on its own after the batch.
    Every result is the oracle's R and rows of C', and A' the oracle's."""
    import torch
    vt = torch.float64 if sr == PLUS_TIMES_F64 else torch.int32
    vn = np.float64 if sr == PLUS_TIMES_F64 else np.int32

    def page_locked(nr, ne):
        return tuple(torch.empty(m, dtype=dt, pin_memory=True).numpy()
                     for m, dt in ((nr, torch.int32), (nr + 1, torch.int64), (ne, torch.int32), (ne, vt)))

    n = 3000
    A = er_matrix(n, 6, seed=111, kind=sr)
    g = dspg.DynamicSpGEMM(A)
    Ao = OMat.from_csr(A)
    Co = Ao.multiply(Ao)
    pinned = page_locked(n, 200000)
    pageable = (np.empty(n, np.int32), np.empty(n + 1, np.int64), np.empty(200000, np.int32), np.empty(200000, vn))
    small = page_locked(4, 4)
    for t, out in enumerate((pinned, pinned, pageable, small, pinned)):
        b = random_batch(n, n, 400 + 300 * t, 112 + t, sr, A=Ao.to_csr())
        st, (rows, rp, col, val) = g.apply_read_affected(b, out=out)
        R = oracle.row_dynamic(Ao, Co, b, None, None)  # A' and C' of the oracle, and its R
        if out is not small:
            assert np.shares_memory(rows, out[0]) and np.shares_memory(col, out[2]), "out arrays not used"
        assert st["affected_rows"] == rows.shape[0]
        assert np.array_equal(rows, R), f"batch {t}: affected rows"
        _check_rows_of_c(Ao, rows, rp, col, val, sr, f"batch {t}")
        _check_state(g, Ao, None, f"batch {t}")
    # arenas without room: every batch is applied in two passes, and the read
    # enqueued behind the first is replaced by one after the second
    A2 = random_csr(400, 400, 10, 31, sr)
    g2 = dspg.DynamicSpGEMM(A2, slack_min=0, slack_div=1 << 20, arena_headroom=1.0)
    Ao2 = OMat.from_csr(A2)
    Co2 = Ao2.multiply(Ao2)
    out2 = page_locked(400, 160000)
    grown = 0
    for k in range(3):
        b = random_batch(400, 400, 3000, 60 + k, sr, A=Ao2.to_csr(), hit_frac=0.1)
        st, (rows, rp, col, val) = g2.apply_read_affected(b, out=out2)
        R = oracle.row_dynamic(Ao2, Co2, b, None, None)
        grown += st["compactions"]
        assert np.array_equal(rows, R), f"tight {k}: affected rows"
        _check_rows_of_c(Ao2, rows, rp, col, val, sr, f"tight {k}")
        _check_state(g2, Ao2, None, f"tight {k}")
    assert grown > 0


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_host_batches_page_locked_pageable_and_device(dspg, sr):
    """The same batches given as page-locked host arrays, pageable host
    arrays (both copied to the device first) and device arrays (read where
    they are) leave the same A' and C' as the oracle's, in sizes on both
    sides of the cluster sort's limits (one CTA, radix cluster, multi-pass)."""
    import torch
    n = 3000
    A = er_matrix(n, 6, seed=103, kind=sr)
    handles = [dspg.DynamicSpGEMM(A) for _ in range(3)]
    Ao = OMat.from_csr(A)
    for t, m in enumerate((500, 9000, 20000)):
        b = random_batch(n, n, m, 104 + t, sr, A=Ao.to_csr(), dup_frac=0.2)
        pinned = Batch(*(torch.from_numpy(x).pin_memory().numpy() for x in (b.row, b.col, b.val, b.op)))
        dev = Batch(*(torch.from_numpy(x).cuda() for x in (b.row, b.col, b.val, b.op)))
        for g, bb in zip(handles, (pinned, b, dev)):
            g.apply_batch(bb)
        Ao.apply(b)
        for g, what in zip(handles, ("page-locked", "pageable", "device")):
            _check_state(g, Ao, None, f"batch {t} {what}")
