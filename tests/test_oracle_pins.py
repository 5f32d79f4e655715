"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test ties the oracle to a fact the paper or mathematics fixes:

* dense brute force over the semiring on tiny non-square inputs;
* numpy's dense matmul (plus-times) and boolean pattern products;
* Floyd-Warshall and Dijkstra from scipy (min-plus, shortest paths with
  multiple sources, the application named in Section 1);
* a Python dictionary model of sequential updates (Section 4.1);
* Eq. 1 (algebraic updates: C' = C + A*B' + AB*) on integer-valued data,
  where every summation order is exact;
* the locality of general updates (Section 5: C' differs from C only in the
  rows of C*), checked against a full static recompute;
* a closed form for the 7-point stencil square (path counts on the grid);
* hand-worked fixtures in tests/golden/.
"""

import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import OMat, OracleError
from workloads import (CSR, Batch, MIN_PLUS_I32, OP_DELETE, OP_INSERT, OP_SET, PLUS_TIMES_F64,
                       er_batch, er_matrix, random_batch, random_csr, stencil7)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = np.iinfo(np.int64).max


def dense_parts(m: CSR):
    """(presence bool matrix, value matrix) of a CSR; absent values are 0."""
    P = np.zeros((m.nrows, m.ncols), dtype=bool)
    V = np.zeros((m.nrows, m.ncols), dtype=np.float64 if m.val.dtype == np.float64 else np.int64)
    r = m.row_ids()
    P[r, m.col] = True
    V[r, m.col] = m.val
    return P, V


def brute_force_product(A: CSR, B: CSR):
    """Triple loop over the semiring on dense arrays: (i,j) present iff some k
    has A(i,k) and B(k,j) present; value = fold of (a (x) b) over those k."""
    PA, VA = dense_parts(A)
    PB, VB = dense_parts(B)
    n, kk, m = A.nrows, A.ncols, B.ncols
    P = np.zeros((n, m), dtype=bool)
    V = np.zeros((n, m), dtype=VA.dtype)
    for i in range(n):
        for j in range(m):
            acc = None
            for k in range(kk):
                if PA[i, k] and PB[k, j]:
                    if A.semiring == PLUS_TIMES_F64:
                        t = VA[i, k] * VB[k, j]
                        acc = t if acc is None else acc + t
                    else:
                        t = int(VA[i, k]) + int(VB[k, j])
                        acc = t if acc is None else min(acc, t)
            if acc is not None:
                P[i, j] = True
                V[i, j] = acc
    return P, V


def to_dense(m: CSR):
    return dense_parts(m)


def csr_from_coords(nrows, ncols, r, c, v) -> CSR:
    """CSR from coordinates given in row-major order without duplicates."""
    rowptr = np.zeros(nrows + 1, np.int64)
    np.cumsum(np.bincount(np.asarray(r, np.int64), minlength=nrows), out=rowptr[1:])
    return CSR(nrows, ncols, rowptr, np.asarray(c, np.int32), np.asarray(v))


def integer_valued(m: CSR, seed: int, lo=-5, hi=6) -> CSR:
    rng = np.random.default_rng(seed)
    return CSR(m.nrows, m.ncols, m.rowptr, m.col, rng.integers(lo, hi, size=m.nnz).astype(np.float64))


# ----------------------------------------------------------------- static


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
@pytest.mark.parametrize("seed", range(6))
def test_static_product_matches_brute_force(sr, seed):
    n, k, m = 13 + seed, 9 + 2 * seed, 17 - seed  # non-square: a transposed operand fails
    A = random_csr(n, k, 5, seed, sr)
    B = random_csr(k, m, 6, 100 + seed, sr)
    if sr == PLUS_TIMES_F64:  # integer-valued data: every summation order is exact
        A, B = integer_valued(A, seed), integer_valued(B, seed + 50)
    C = OMat.from_csr(A).multiply(OMat.from_csr(B)).to_csr()
    P, V = brute_force_product(A, B)
    PC, VC = to_dense(C)
    assert np.array_equal(PC, P)
    assert np.array_equal(VC[P], V[P])


def test_structural_zero_is_kept():
    """Section 3: a product that sums to the number 0 is still a non-zero."""
    A = CSR(1, 2, np.array([0, 2]), np.array([0, 1], np.int32), np.array([1.0, -1.0]))
    B = CSR(2, 1, np.array([0, 1, 2]), np.array([0, 0], np.int32), np.array([2.0, 2.0]))
    C = OMat.from_csr(A).multiply(OMat.from_csr(B)).to_csr()
    assert C.nnz == 1 and C.col[0] == 0 and C.val[0] == 0.0


@pytest.mark.parametrize("seed", range(3))
def test_plus_times_matches_numpy_matmul(seed):
    A = random_csr(60, 45, 12, seed, PLUS_TIMES_F64)
    B = random_csr(45, 70, 12, seed + 9, PLUS_TIMES_F64)
    C = OMat.from_csr(A).multiply(OMat.from_csr(B)).to_csr()
    PA, VA = to_dense(A)
    PB, VB = to_dense(B)
    pattern = (PA.astype(np.int64) @ PB.astype(np.int64)) > 0
    PC, VC = to_dense(C)
    assert np.array_equal(PC, pattern)
    ref = VA @ VB
    assert np.allclose(VC[pattern], ref[pattern], rtol=1e-13, atol=1e-13)
    assert np.all(ref[~pattern] == 0)


def minplus_closure_oracle(W: CSR) -> CSR:
    """(W (+) I0) squared ceil(log2 n) times with the oracle: I0 (diagonal 0)
    is written with SET updates, then X <- X X in (min,+)."""
    n = W.nrows
    X = OMat.from_csr(W)
    diag = np.arange(n, dtype=np.int32)
    X.apply(Batch(diag, diag, np.zeros(n, np.int32), np.full(n, OP_SET, np.uint8)))
    for _ in range(int(np.ceil(np.log2(max(n, 2))))):
        X = X.multiply(X)
    return X.to_csr()


@pytest.mark.parametrize("seed", range(4))
def test_minplus_squaring_equals_floyd_warshall(seed):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import floyd_warshall
    n = 40
    W = random_csr(n, n, 3, seed, MIN_PLUS_I32, empty_frac=0.2)
    D = floyd_warshall(csr_matrix((W.val.astype(np.float64), W.col, W.rowptr), shape=(n, n)), directed=True)
    X = minplus_closure_oracle(W)
    PX, VX = to_dense(X)
    assert np.array_equal(PX, np.isfinite(D))
    assert np.array_equal(VX[PX], D[PX].astype(np.int64))


@pytest.mark.parametrize("seed", range(3))
def test_minplus_relaxation_fixed_point_equals_dijkstra(seed):
    """Multi-source shortest distances: iterate X <- (W (+) I0) X from X0 = B
    with the oracle's row-dynamic route (each step applies the changed entries
    of X as a batch to the right operand) until nothing changes; compare with
    Dijkstra from a super-source per column of B on the reversed graph."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import dijkstra
    n, s = 30, 4
    W = random_csr(n, n, 3, seed, MIN_PLUS_I32, empty_frac=0.3)
    B0 = random_csr(n, s, 2, seed + 7, MIN_PLUS_I32, empty_frac=0.6)
    A = OMat.from_csr(W)
    diag = np.arange(n, dtype=np.int32)
    A.apply(Batch(diag, diag, np.zeros(n, np.int32), np.full(n, OP_SET, np.uint8)))
    Bm = OMat.from_csr(B0)
    C = A.multiply(Bm)
    for _ in range(n + 1):
        cur, nxt = Bm.to_csr(), C.to_csr()
        Pc, Vc = to_dense(cur)
        Pn, Vn = to_dense(nxt)
        changed = np.argwhere(Pn & (~Pc | (Vn != Vc)))
        if changed.shape[0] == 0:
            break
        upd = Batch(changed[:, 0].astype(np.int32), changed[:, 1].astype(np.int32),
                    Vn[changed[:, 0], changed[:, 1]].astype(np.int32),
                    np.full(changed.shape[0], OP_SET, np.uint8))
        oracle.row_dynamic(A, C, Batch(np.zeros(0, np.int32), np.zeros(0, np.int32),
                                       np.zeros(0, np.int32), np.zeros(0, np.uint8)), Bm, upd)
        assert np.array_equal(to_dense(C.to_csr())[0], to_dense(A.multiply(Bm).to_csr())[0])
    X = Bm.to_csr()
    PX, VX = to_dense(X)
    # Dijkstra: node n+j is the super-source of column j; reversed edges of W
    for j in range(s):
        r = W.row_ids()
        rows = list(W.col.astype(np.int64))
        cols = list(r)
        vals = list(W.val.astype(np.float64))
        P0, V0 = to_dense(B0)
        for k in np.nonzero(P0[:, j])[0]:
            rows.append(n)
            cols.append(int(k))
            vals.append(float(V0[k, j]))
        G = coo_matrix((vals, (rows, cols)), shape=(n + 1, n + 1)).tocsr()
        d = dijkstra(G, directed=True, indices=n)[:n]
        assert np.array_equal(PX[:, j], np.isfinite(d))
        assert np.array_equal(VX[PX[:, j], j], d[PX[:, j]].astype(np.int64))


def test_stencil_square_closed_form():
    """7-point stencil with diagonal 6 and off-diagonals exactly -1: (A^2)(i,j)
    is 36 + deg(i) on the diagonal, -12 for grid neighbours (the grid is
    bipartite, so adjacent points share no neighbour), and the number of
    common neighbours (1 along an axis, 2 across a face diagonal) for points
    two hops apart; every other entry is absent."""
    nx, ny, nz = 5, 4, 3
    A = stencil7(nx, ny, nz, seed=0)
    A = CSR(A.nrows, A.ncols, A.rowptr, A.col, np.where(A.col == A.row_ids(), 6.0, -1.0))
    C = OMat.from_csr(A).multiply(OMat.from_csr(A)).to_csr()
    got = {(int(i), int(j)): float(v) for i, j, v in zip(C.row_ids(), C.col, C.val)}
    want = {}
    pts = list(itertools.product(range(nx), range(ny), range(nz)))
    idx = {p: p[0] + nx * (p[1] + ny * p[2]) for p in pts}

    def nbrs(p):
        for d in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
            q = (p[0] + d[0], p[1] + d[1], p[2] + d[2])
            if q in idx:
                yield q

    for p in pts:
        want[(idx[p], idx[p])] = 36.0 + len(list(nbrs(p)))
        for q in nbrs(p):
            want[(idx[p], idx[q])] = -12.0
        two = {}
        for q in nbrs(p):
            for r in nbrs(q):
                if r != p and sum(abs(a - b) for a, b in zip(p, r)) == 2:
                    two[r] = two.get(r, 0) + 1
        for r, c in two.items():
            want[(idx[p], idx[r])] = float(c)
    assert got == want


# ----------------------------------------------------------------- updates


def dict_model(A: CSR, batch: Batch) -> dict:
    d = {(int(i), int(j)): v for i, j, v in zip(A.row_ids(), A.col, A.val)}
    for i, j, v, op in zip(batch.row, batch.col, batch.val, batch.op):
        if op == OP_DELETE:
            d.pop((int(i), int(j)), None)
        else:
            d[(int(i), int(j))] = v
    return d


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
@pytest.mark.parametrize("seed", range(5))
def test_apply_matches_dictionary_model(sr, seed):
    A = random_csr(50, 40, 8, seed, sr)
    b = random_batch(50, 40, 300, seed + 11, sr, A=A, dup_frac=0.4)
    M = OMat.from_csr(A)
    M.apply(b)
    out = M.to_csr()
    got = {(int(i), int(j)): v for i, j, v in zip(out.row_ids(), out.col, out.val)}
    assert got == dict_model(A, b)
    assert np.all(np.diff(out.col)[np.diff(out.row_ids()) == 0] > 0)  # rows stay sorted


@pytest.mark.parametrize("bad", ["row", "col", "op", "nan", "inf_minplus"])
def test_invalid_batch_changes_nothing(bad):
    sr = MIN_PLUS_I32 if bad == "inf_minplus" else PLUS_TIMES_F64
    A = random_csr(20, 20, 5, 3, sr)
    b = random_batch(20, 20, 50, 4, sr, A=A)
    if bad == "row":
        b.row[17] = 20
    elif bad == "col":
        b.col[3] = -1
    elif bad == "op":
        b.op[9] = 7
    elif bad == "nan":
        b.op[5] = OP_INSERT
        b.val[5] = np.nan
    else:
        b.op[5] = OP_SET
        b.val[5] = np.iinfo(np.int32).max
    M = OMat.from_csr(A)
    with pytest.raises(OracleError):
        M.apply(b)
    out = M.to_csr()
    assert np.array_equal(out.rowptr, A.rowptr) and np.array_equal(out.col, A.col)
    assert np.array_equal(out.val, A.val)


# ------------------------------------------------------------- dynamic


def csr_equal(x: CSR, y: CSR) -> bool:
    return (np.array_equal(x.rowptr, y.rowptr) and np.array_equal(x.col, y.col)
            and np.array_equal(x.val, y.val))


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
@pytest.mark.parametrize("seed", range(6))
def test_row_dynamic_equals_static_and_is_local(sr, seed):
    """Section 5: C' = A'A' whichever route computes it, and C' differs from
    C only in R; every row outside R of the static A'A' equals the old row."""
    n = 80
    A = random_csr(n, n, 6, seed, sr)
    b = random_batch(n, n, 40, seed + 1, sr, A=A)
    Am = OMat.from_csr(A)
    C0 = Am.multiply(Am).to_csr()
    Cm = OMat.from_csr(C0)
    R = oracle.row_dynamic(Am, Cm, b)
    dyn = Cm.to_csr()
    A2 = OMat.from_csr(A)
    A2.apply(b)
    static = A2.multiply(A2).to_csr()
    assert csr_equal(dyn, static)
    outside = np.setdiff1d(np.arange(n), R)
    for i in outside:
        s0, s1 = C0.rowptr[i], C0.rowptr[i + 1]
        t0, t1 = static.rowptr[i], static.rowptr[i + 1]
        assert np.array_equal(C0.col[s0:s1], static.col[t0:t1])
        assert np.array_equal(C0.val[s0:s1], static.val[t0:t1])


@pytest.mark.parametrize("seed", range(4))
def test_row_dynamic_separate_b(seed):
    sr = MIN_PLUS_I32 if seed % 2 else PLUS_TIMES_F64
    A = random_csr(60, 30, 5, seed, sr)
    B = random_csr(30, 45, 5, seed + 3, sr)
    ba = random_batch(60, 30, 25, seed + 5, sr, A=A)
    bb = random_batch(30, 45, 15, seed + 6, sr, A=B)
    Am, Bm = OMat.from_csr(A), OMat.from_csr(B)
    Cm = Am.multiply(Bm)
    oracle.row_dynamic(Am, Cm, ba, Bm, bb)
    A2, B2 = OMat.from_csr(A), OMat.from_csr(B)
    A2.apply(ba)
    B2.apply(bb)
    assert csr_equal(Cm.to_csr(), A2.multiply(B2).to_csr())


def test_affected_rows_same_with_old_or_new_pattern():
    """R computed with A' (as stated) equals R computed with A's pattern
    before the batch: a pattern difference at (i,k) puts i in rows(A*)."""
    for seed in range(8):
        n = 70
        A = random_csr(n, n, 5, seed, PLUS_TIMES_F64)
        b = random_batch(n, n, 30, seed + 2, PLUS_TIMES_F64, A=A)
        M = OMat.from_csr(A)
        pre = M.presence(b)
        M.apply(b)
        post = M.presence(b)
        R = oracle.affected_rows(M, b, pre, post, b_nrows=n, b_is_a=True)
        changed = (pre | post).astype(bool)
        star_rows = set(b.row[changed].tolist())
        PA, _ = to_dense(A)
        R_old = set(star_rows)
        for i in range(n):
            if any(PA[i, k] for k in star_rows):
                R_old.add(i)
        assert sorted(R_old) == R.tolist()


@pytest.mark.parametrize("seed", range(4))
def test_algebraic_identity_eq1(seed):
    """Eq. 1: for A' = A + A*, B' = B + B* (here B = A, so B* = A*),
    C' = C + A* B' + A B*, on integer-valued data (exact in any order)."""
    n = 50
    A = integer_valued(random_csr(n, n, 5, seed, PLUS_TIMES_F64), seed)
    rng = np.random.default_rng(seed + 40)
    PA, VA = to_dense(A)
    # A*: some new positions and some additive changes of existing ones
    pos = np.sort(rng.choice(n * n, size=60, replace=False))
    Astar = csr_from_coords(n, n, pos // n, pos % n, rng.integers(1, 4, size=60).astype(np.float64))
    PS, VS = to_dense(Astar)
    upd_r, upd_c = np.nonzero(PS)
    b = Batch(upd_r.astype(np.int32), upd_c.astype(np.int32),
              (VA + VS)[upd_r, upd_c], np.full(upd_r.shape[0], OP_SET, np.uint8))
    Am = OMat.from_csr(A)
    C = Am.multiply(Am).to_csr()
    A1 = OMat.from_csr(A)
    A1.apply(b)  # A' = A + A*
    Cnew = A1.multiply(A1).to_csr()
    Sm = OMat.from_csr(Astar)
    X = Sm.multiply(A1).to_csr()          # A* B'
    Y = Am.multiply(Sm).to_csr()          # A B*
    PC, VC = to_dense(C)
    PX, VX = to_dense(X)
    PY, VY = to_dense(Y)
    Pn, Vn = to_dense(Cnew)
    assert np.array_equal(Pn, PC | PX | PY)
    assert np.array_equal(Vn, VC + VX + VY)
    # the equivalent form of the footnote: C' = C + A* B + A' B*
    X2 = Sm.multiply(Am).to_csr()
    Y2 = A1.multiply(Sm).to_csr()
    P2, V2 = to_dense(X2)
    P3, V3 = to_dense(Y2)
    assert np.array_equal(Vn, VC + V2 + V3)


def test_er_batch_recipe_and_dynamic_config1_small():
    A = er_matrix(512, 8, seed=1)
    b = er_batch(A, seed=2, n_insert=64, n_delete=32, n_set=32)
    assert len(b) == 128 and len(set(zip(b.row.tolist(), b.col.tolist()))) == 128
    M = OMat.from_csr(A)
    pre = M.presence(b)
    assert np.all(pre[b.op == OP_INSERT] == 0) and np.all(pre[b.op != OP_INSERT] == 1)
    C = M.multiply(M)
    R = oracle.row_dynamic(M, C, b)
    A2 = OMat.from_csr(A)
    A2.apply(b)
    assert csr_equal(C.to_csr(), A2.multiply(A2).to_csr())
    assert R.shape[0] > 0


# ------------------------------------------------------------- golden


def _golden_cases():
    # the product-and-batch fixtures (masked_*.json, Algorithm 2's steps, are
    # read by test_oracle_masked.py)
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".json") and not f.startswith("masked_"))


@pytest.mark.parametrize("name", _golden_cases())
def test_golden_hand_worked(name):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    sr = PLUS_TIMES_F64 if g["semiring"] == "plus_times" else MIN_PLUS_I32
    dt = np.float64 if sr == PLUS_TIMES_F64 else np.int32

    def csr(d):
        return CSR(d["nrows"], d["ncols"], np.array(d["rowptr"], np.int64),
                   np.array(d["col"], np.int32), np.array(d["val"], dt))

    A = csr(g["A"])
    Am = OMat.from_csr(A)
    C = Am.multiply(Am)
    assert csr_equal(C.to_csr(), csr(g["C"]))
    bt = g["batch"]
    b = Batch(np.array(bt["row"], np.int32), np.array(bt["col"], np.int32),
              np.array(bt["val"], dt), np.array(bt["op"], np.uint8))
    R = oracle.row_dynamic(Am, C, b)
    assert R.tolist() == g["R"]
    assert csr_equal(Am.to_csr(), csr(g["A_after"]))
    assert csr_equal(C.to_csr(), csr(g["C_after"]))


# ------------------------------------------- the bound and the B != A rows


@pytest.mark.parametrize("seed", range(4))
def test_absval_product_is_abs_matmul(seed):
    """The (+,.) tolerance bound S = |A| |B| (Section 3's product on the
    entrywise magnitudes): on integer-valued data of both signs every sum is
    exact, so the oracle's absval product equals numpy's |A| @ |B| bit for
    bit on the product's pattern, and that pattern is the plain product's.
    An inflated bound (|a| + |b|, or a fold into a stale accumulator) fails."""
    A = integer_valued(random_csr(40, 30, 5, seed, PLUS_TIMES_F64), seed, lo=-7, hi=8)
    B = integer_valued(random_csr(30, 50, 4, seed + 11, PLUS_TIMES_F64), seed + 1, lo=-7, hi=8)
    Am, Bm = OMat.from_csr(A), OMat.from_csr(B)
    S = Am.multiply(Bm, absval=True).to_csr()
    C = Am.multiply(Bm).to_csr()
    PA, VA = to_dense(A)
    PB, VB = to_dense(B)
    want_p = (PA.astype(np.int64) @ PB.astype(np.int64)) > 0
    want_v = np.abs(VA) @ np.abs(VB)
    PS, VS = to_dense(S)
    PC, _ = to_dense(C)
    assert np.array_equal(PS, want_p) and np.array_equal(PC, want_p)
    assert np.array_equal(VS[PS], want_v[PS])
    # the rows-only route of the oracle gives the same bound
    rows = np.array([0, 7, 13, 39], np.int32)
    rp, col, val = Am.multiply_rows(Bm, rows, absval=True)
    for t, i in enumerate(rows):
        js = col[rp[t]:rp[t + 1]]
        assert np.array_equal(js, np.nonzero(want_p[i])[0])
        assert np.array_equal(val[rp[t]:rp[t + 1]], want_v[i, js])


def _presence_model(M: CSR, batch: Batch):
    """Presence of each batch key before and after applying the batch in
    array order, from a set of (row, col) pairs (Section 4.1 semantics:
    INSERT and SET store, DELETE removes)."""
    present = set(zip(M.row_ids().tolist(), M.col.tolist()))
    pre = np.array([(int(r), int(c)) in present for r, c in zip(batch.row, batch.col)], np.uint8)
    for r, c, o in zip(batch.row.tolist(), batch.col.tolist(), batch.op.tolist()):
        if o == OP_DELETE:
            present.discard((r, c))
        else:
            present.add((r, c))
    post = np.array([(int(r), int(c)) in present for r, c in zip(batch.row, batch.col)], np.uint8)
    return pre, post, present


@pytest.mark.parametrize("seed", range(6))
def test_affected_rows_separate_b_brute_force(seed):
    """R for C = A B with separate batches of A and B, against Eq. 1's row
    set written out on dense patterns: R = rows(A*) u {i : A'(i,k) != 0,
    k in rows(B*)}, where A* (B*) holds the batch keys present before or
    after the batch.  R must also contain every row whose product changed
    (the rows of C' - C), and nothing else may enter it: a B batch made
    partly of deletes of absent entries (no change) and of rows whose column
    in A' is empty checks that R is not over-inclusive."""
    rng = np.random.default_rng(seed + 70)
    n, k, m = 50, 40, 45
    A = random_csr(n, k, 3, seed, PLUS_TIMES_F64)
    B = random_csr(k, m, 3, seed + 20, PLUS_TIMES_F64)
    ba = random_batch(n, k, 12, seed + 5, PLUS_TIMES_F64, A=A)
    bb = random_batch(k, m, 10, seed + 6, PLUS_TIMES_F64, A=B)
    # no-op deletes in B rows that A' reads: they change nothing
    PB, _ = to_dense(B)
    absent = np.argwhere(~PB)
    pick = absent[rng.choice(absent.shape[0], size=6, replace=False)]
    bb = Batch(np.concatenate([bb.row, pick[:, 0].astype(np.int32)]),
               np.concatenate([bb.col, pick[:, 1].astype(np.int32)]),
               np.concatenate([bb.val, np.zeros(6)]),
               np.concatenate([bb.op, np.full(6, OP_DELETE, np.uint8)]))
    pre_a, post_a, a_after = _presence_model(A, ba)
    pre_b, post_b, _ = _presence_model(B, bb)
    star_a = {int(r) for r, p, q in zip(ba.row, pre_a, post_a) if p or q}
    star_b = {int(r) for r, p, q in zip(bb.row, pre_b, post_b) if p or q}
    want = set(star_a)
    for (i, kk) in a_after:
        if kk in star_b:
            want.add(i)
    Am, Bm = OMat.from_csr(A), OMat.from_csr(B)
    # the oracle's own presence agrees with the set model
    assert np.array_equal(Am.presence(ba), pre_a) and np.array_equal(Bm.presence(bb), pre_b)
    Cm = Am.multiply(Bm)
    C0 = Cm.to_csr()
    R = oracle.row_dynamic(Am, Cm, ba, Bm, bb)
    assert R.tolist() == sorted(want)
    P0, V0 = to_dense(C0)
    P1, V1 = to_dense(Cm.to_csr())
    changed = set(np.nonzero((P0 != P1).any(axis=1) | (V0 != V1).any(axis=1))[0].tolist())
    assert changed <= set(R.tolist())


def test_affected_rows_separate_b_worked_example():
    """A 3 x 3 example by hand.  A has (0,1), (1,2), (2,0); B has (0,0),
    (1,1), (2,2).  The A batch sets (2,0) (an existing entry: A* = {(2,0)});
    the B batch inserts (1,0) and deletes the absent (0,2).  B* = {(1,0)},
    rows(B*) = {1}, and the only row of A' with column 1 is row 0, so
    R = {2} u {0} = {0, 2}: row 1, whose A row reads B row 2, is untouched,
    and the no-op delete in B row 0 adds nothing (row 2 reads B row 0 but is
    already in R for its own change)."""
    A = CSR(3, 3, np.array([0, 1, 2, 3], np.int64), np.array([1, 2, 0], np.int32), np.array([1.0, 2.0, 3.0]))
    B = CSR(3, 3, np.array([0, 1, 2, 3], np.int64), np.array([0, 1, 2], np.int32), np.array([4.0, 5.0, 6.0]))
    ba = Batch(np.array([2], np.int32), np.array([0], np.int32), np.array([7.0]), np.array([OP_SET], np.uint8))
    bb = Batch(np.array([1, 0], np.int32), np.array([0, 2], np.int32), np.array([8.0, 0.0]),
               np.array([OP_INSERT, OP_DELETE], np.uint8))
    Am, Bm = OMat.from_csr(A), OMat.from_csr(B)
    Cm = Am.multiply(Bm)
    R = oracle.row_dynamic(Am, Cm, ba, Bm, bb)
    assert R.tolist() == [0, 2]
    # C' by hand: row 0 = 1 * B'(1,:) = {0: 8, 1: 5}; row 1 = 2 * B(2,:) = {2: 12};
    # row 2 = 7 * B(0,:) = {0: 28}
    Cn = Cm.to_csr()
    assert Cn.rowptr.tolist() == [0, 2, 3, 4]
    assert Cn.col.tolist() == [0, 1, 2, 0]
    assert Cn.val.tolist() == [8.0, 5.0, 12.0, 28.0]


@pytest.mark.parametrize("sr", [PLUS_TIMES_F64, MIN_PLUS_I32])
def test_all_cores_route_is_identical(sr):
    """The all-cores timing of the oracle (its row loops over threads) gives
    bit for bit the single-threaded result: R, C' and A'."""
    A = random_csr(3000, 3000, 9, 91, sr)
    b = random_batch(3000, 3000, 2500, 92, sr, A=A)
    out = []
    for threads in (1, 4):
        oracle.set_threads(threads)
        try:
            M = OMat.from_csr(A)
            C = M.multiply(M)
            R = oracle.row_dynamic(M, C, b)
            out.append((R, C.to_csr(), M.to_csr()))
        finally:
            oracle.set_threads(1)
    (R1, C1, A1), (R4, C4, A4) = out
    assert np.array_equal(R1, R4) and csr_equal(C1, C4) and csr_equal(A1, A4)
    assert np.array_equal(C1.val, C4.val)
