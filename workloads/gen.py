"""Seeded synthetic matrices and update batches.

Every function takes an explicit integer seed and draws from
``numpy.random.default_rng(seed)``. Nothing here multiplies, merges or
detects anything: the functions only build random inputs in canonical CSR
(rows ascending, columns strictly ascending within a row) and random update
lists.

Value types follow the two semirings of the library:

* plus-times: float64 values (``PLUS_TIMES_F64``);
* min-plus: int32 values (``MIN_PLUS_I32``), weights in [1, 100].

Update operations (Section 4.1 "Dynamic Updates": insertion of a new
non-zero, deletion of an existing non-zero, change of a value):

* ``OP_INSERT`` (0) and ``OP_SET`` (2) both write the value at (i, j);
* ``OP_DELETE`` (1) removes (i, j) if it is present.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

PLUS_TIMES_F64 = 0
MIN_PLUS_I32 = 1

OP_INSERT = 0
OP_DELETE = 1
OP_SET = 2


@dataclass
class CSR:
    """Canonical CSR: ``rowptr`` int64[nrows+1], ``col`` int32, ``val`` f64 or i32."""

    nrows: int
    ncols: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def semiring(self) -> int:
        return PLUS_TIMES_F64 if self.val.dtype == np.float64 else MIN_PLUS_I32

    def row_ids(self) -> np.ndarray:
        return np.repeat(np.arange(self.nrows, dtype=np.int64), np.diff(self.rowptr))


@dataclass
class Batch:
    """Update list in arrival order: row/col int32, val f64 or i32, op uint8."""

    row: np.ndarray
    col: np.ndarray
    val: np.ndarray
    op: np.ndarray

    def __len__(self) -> int:
        return int(self.row.shape[0])


def _values(rng: np.random.Generator, n: int, kind: int) -> np.ndarray:
    if kind == PLUS_TIMES_F64:
        return rng.random(n)
    return rng.integers(1, 101, size=n, dtype=np.int32)


def _csr_from_unique_coo(nrows, ncols, r, c, v) -> CSR:
    """Canonical CSR from coordinates that are already free of duplicates."""
    r = np.asarray(r, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    order = np.argsort(r * max(int(ncols), 1) + c, kind="stable")  # row-major order
    r, c, v = r[order], c[order], np.asarray(v)[order]
    counts = np.bincount(r, minlength=nrows).astype(np.int64)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(nrows, ncols, rowptr, c.astype(np.int32), v)


def er_matrix(n: int, per_row: int, seed: int, kind: int = PLUS_TIMES_F64) -> CSR:
    """Erdos-Renyi style n x n matrix: each row has ``per_row`` distinct columns
    drawn uniformly without replacement; values U(0,1) (f64) or U[1,100] (i32)."""
    rng = np.random.default_rng(seed)
    cols = np.empty((n, per_row), dtype=np.int64)
    for i in range(n):
        cols[i] = rng.choice(n, size=per_row, replace=False)
    r = np.repeat(np.arange(n, dtype=np.int64), per_row)
    v = _values(rng, n * per_row, kind)
    return _csr_from_unique_coo(n, n, r, cols.reshape(-1), v)


def random_csr(nrows: int, ncols: int, nnz_per_row_max: int, seed: int,
               kind: int = PLUS_TIMES_F64, empty_frac: float = 0.1) -> CSR:
    """Small random matrix with uneven rows (some empty): row lengths uniform in
    [0, nnz_per_row_max], columns distinct, for property tests."""
    rng = np.random.default_rng(seed)
    rr, cc = [], []
    for i in range(nrows):
        if rng.random() < empty_frac:
            continue
        k = int(rng.integers(0, min(nnz_per_row_max, ncols) + 1))
        cs = rng.choice(ncols, size=k, replace=False)
        rr.append(np.full(k, i, dtype=np.int64))
        cc.append(cs.astype(np.int64))
    r = np.concatenate(rr) if rr else np.zeros(0, np.int64)
    c = np.concatenate(cc) if cc else np.zeros(0, np.int64)
    v = _values(rng, r.shape[0], kind)
    return _csr_from_unique_coo(nrows, ncols, r, c, v)


def _stencil_index(x, y, z, nx, ny):
    return x + nx * (y + ny * z)


def stencil7(nx: int, ny: int, nz: int, seed: int) -> CSR:
    """7-point stencil pattern on an nx*ny*nz grid, row i = x + nx*(y + ny*z).
    Diagonal 6.0; each off-diagonal -1 + U(-0.1, 0.1)."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    rs, cs, ds = [], [], []
    for dx, dy, dz in [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]:
        ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny) & (z + dz >= 0) & (z + dz < nz)
        rs.append(idx[ok])
        cs.append(_stencil_index(x[ok] + dx, y[ok] + dy, z[ok] + dz, nx, ny))
        ds.append(np.full(int(ok.sum()), (dx, dy, dz) == (0, 0, 0)))
    r = np.concatenate(rs)
    c = np.concatenate(cs)
    diag = np.concatenate(ds)
    v = -1.0 + rng.uniform(-0.1, 0.1, size=r.shape[0])
    v[diag] = 6.0
    return _csr_from_unique_coo(n, n, r, c, v)


def _rmat_directed(scale: int, nedges: int, abcd, rng) -> tuple[np.ndarray, np.ndarray]:
    a, b, c, _ = abcd
    u = np.zeros(nedges, dtype=np.int64)
    v = np.zeros(nedges, dtype=np.int64)
    for level in range(scale):
        r = rng.random(nedges)
        row_bit = r >= (a + b)
        col_bit = ((r >= a) & (r < a + b)) | (r >= a + b + c)
        u |= row_bit.astype(np.int64) << level
        v |= col_bit.astype(np.int64) << level
    return u, v


def rmat_symmetric(scale: int, edge_factor: int, abcd, seed: int, kind: int,
                   holdout: int = 0):
    """Symmetrised R-MAT adjacency matrix (Graph500-style recursive quadrant
    sampling of ``edge_factor * 2**scale`` directed edges). Self-loops are
    dropped, undirected duplicates merged, one weight per undirected edge,
    and both (u,v) and (v,u) stored.

    ``holdout`` undirected edges are removed uniformly at random and returned
    as the insertion pool (u, v, w) for held-out-edge insertion batches
    (the protocol of Section 7.2 "Insertions": insert from the held-back part).
    Returns (A, (hu, hv, hw))."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    u, v = _rmat_directed(scale, edge_factor * n, abcd, rng)
    keep = u != v
    lo = np.minimum(u[keep], v[keep])
    hi = np.maximum(u[keep], v[keep])
    key = np.sort(lo * n + hi)
    key = key[np.concatenate([[True], key[1:] != key[:-1]])] if key.shape[0] else key
    lo, hi = key // n, key % n
    w = _values(rng, key.shape[0], kind)
    if holdout > 0:
        pick = rng.choice(key.shape[0], size=min(holdout, key.shape[0]), replace=False)
        mask = np.zeros(key.shape[0], dtype=bool)
        mask[pick] = True
        held = (lo[mask].astype(np.int32), hi[mask].astype(np.int32), w[mask])
        lo, hi, w = lo[~mask], hi[~mask], w[~mask]
    else:
        held = (np.zeros(0, np.int32), np.zeros(0, np.int32), w[:0])
    r = np.concatenate([lo, hi])
    c = np.concatenate([hi, lo])
    vv = np.concatenate([w, w])
    return _csr_from_unique_coo(n, n, r, c, vv), held


def bernoulli_sparse(nrows: int, ncols: int, p: float, seed: int, kind: int) -> CSR:
    """Each (i, j) present independently with probability p (positions drawn as
    a Bernoulli process over the row-major index space via geometric gaps)."""
    rng = np.random.default_rng(seed)
    total = nrows * ncols
    expect = int(total * p)
    chunks = []
    pos = -1
    while True:
        gaps = rng.geometric(p, size=max(1024, expect // 4 + 1024))
        steps = pos + np.cumsum(gaps)
        inside = steps[steps < total]
        chunks.append(inside)
        if inside.shape[0] < steps.shape[0]:
            break
        pos = int(steps[-1])
    flat = np.concatenate(chunks)
    r = flat // ncols
    c = flat % ncols
    v = _values(rng, flat.shape[0], kind)
    return _csr_from_unique_coo(nrows, ncols, r, c, v)


def _present_keys(A: CSR) -> np.ndarray:
    return A.row_ids() * A.ncols + A.col.astype(np.int64)


def er_batch(A: CSR, seed: int, n_insert: int = 512, n_delete: int = 256,
             n_set: int = 256) -> Batch:
    """Distinct positions: ``n_insert`` INSERTs at absent (i,j) drawn uniformly,
    ``n_delete`` DELETEs and ``n_set`` SETs of distinct present entries; values
    like the matrix's. The list is shuffled."""
    rng = np.random.default_rng(seed)
    kind = A.semiring
    present = _present_keys(A)
    pset = set(present.tolist())
    ins = []
    seen = set()
    while len(ins) < n_insert:
        i = int(rng.integers(0, A.nrows))
        j = int(rng.integers(0, A.ncols))
        k = i * A.ncols + j
        if k in pset or k in seen:
            continue
        seen.add(k)
        ins.append(k)
    pick = rng.choice(present.shape[0], size=n_delete + n_set, replace=False)
    dels = present[pick[:n_delete]]
    sets = present[pick[n_delete:]]
    keys = np.concatenate([np.array(ins, dtype=np.int64), dels, sets])
    op = np.concatenate([np.full(n_insert, OP_INSERT), np.full(n_delete, OP_DELETE),
                         np.full(n_set, OP_SET)]).astype(np.uint8)
    val = _values(rng, keys.shape[0], kind)
    if kind == PLUS_TIMES_F64:
        val[op == OP_DELETE] = 0.0
    else:
        val[op == OP_DELETE] = 0
    perm = rng.permutation(keys.shape[0])
    keys, op, val = keys[perm], op[perm], val[perm]
    return Batch((keys // A.ncols).astype(np.int32), (keys % A.ncols).astype(np.int32), val, op)


_HOP2 = [(dx, dy, dz) for dx in range(-2, 3) for dy in range(-2, 3) for dz in range(-2, 3)
         if abs(dx) + abs(dy) + abs(dz) <= 2]


def stencil_batch(nx: int, ny: int, nz: int, nupd: int, seed: int) -> Batch:
    """Mixed updates (one third each INSERT / DELETE / SET, in random order) at
    (i, j) with j within L1 distance 2 of i on the grid (25 offsets including
    the diagonal), i uniform; values -1 + U(-0.1, 0.1). Positions may repeat and
    may or may not be present, so upserts and no-op deletes both occur."""
    rng = np.random.default_rng(seed)
    offs = np.array(_HOP2, dtype=np.int64)
    rows = np.empty(0, np.int64)
    cols = np.empty(0, np.int64)
    while rows.shape[0] < nupd:
        m = (nupd - rows.shape[0]) * 2 + 16
        i = rng.integers(0, nx * ny * nz, size=m)
        o = offs[rng.integers(0, offs.shape[0], size=m)]
        x = i % nx + o[:, 0]
        y = (i // nx) % ny + o[:, 1]
        z = i // (nx * ny) + o[:, 2]
        ok = (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
        rows = np.concatenate([rows, i[ok]])
        cols = np.concatenate([cols, _stencil_index(x[ok], y[ok], z[ok], nx, ny)])
    rows, cols = rows[:nupd], cols[:nupd]
    op = rng.permutation(np.arange(nupd) % 3).astype(np.uint8)
    val = -1.0 + rng.uniform(-0.1, 0.1, size=nupd)
    val[op == OP_DELETE] = 0.0
    return Batch(rows.astype(np.int32), cols.astype(np.int32), val, op)


_HOP2_ONLY = [o for o in _HOP2 if abs(o[0]) + abs(o[1]) + abs(o[2]) == 2]


def stencil_insert_batch(nx: int, ny: int, nz: int, nupd: int, seed: int, taken: set,
                         present: np.ndarray | None = None) -> Batch:
    """Insertions only, for the algebraic (Eq. 1) comparison: nupd distinct
    positions (i, j) with j at L1 distance exactly 2 of i on the grid (18
    offsets; absent from the 7-point pattern), i uniform, none of them in
    ``taken`` (positions inserted before, which the call adds to) nor in
    ``present`` (sorted keys i * n + j of a matrix's entries); values
    -1 + U(-0.1, 0.1)."""
    rng = np.random.default_rng(seed)
    offs = np.array(_HOP2_ONLY, dtype=np.int64)
    n = nx * ny * nz
    keys = []
    fresh = set()
    while len(keys) < nupd:
        m = (nupd - len(keys)) * 2 + 16
        i = rng.integers(0, n, size=m)
        o = offs[rng.integers(0, offs.shape[0], size=m)]
        x = i % nx + o[:, 0]
        y = (i // nx) % ny + o[:, 1]
        z = i // (nx * ny) + o[:, 2]
        ok = (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz)
        kk = i[ok] * n + _stencil_index(x[ok], y[ok], z[ok], nx, ny)
        if present is not None and present.shape[0] > 0:
            p = np.minimum(np.searchsorted(present, kk), present.shape[0] - 1)
            kk = kk[present[p] != kk]
        for k in kk.tolist():
            if k not in taken and k not in fresh:
                fresh.add(k)
                keys.append(k)
                if len(keys) == nupd:
                    break
    taken |= fresh
    keys = np.array(keys, np.int64)
    val = -1.0 + rng.uniform(-0.1, 0.1, size=nupd)
    return Batch((keys // n).astype(np.int32), (keys % n).astype(np.int32), val,
                 np.full(nupd, OP_INSERT, np.uint8))


def rmat_edge_batch(A: CSR, held, n_edges: int, seed: int) -> Batch:
    """Undirected-edge batch for a symmetric A: half INSERTs of edges drawn
    without replacement from the held-out pool ``held`` = (u, v, w), half
    DELETEs of present undirected edges drawn uniformly. Each edge update is
    emitted as (u,v) and (v,u) with the same value, so the list has
    2 * n_edges entries.  A pool (or edge set) smaller than its half of the
    batch is drawn with replacement: repeated edges within the batch are
    then written twice and the last write wins."""
    rng = np.random.default_rng(seed)
    kind = A.semiring
    n_ins = n_edges // 2
    n_del = n_edges - n_ins
    hu, hv, hw = held
    if n_ins > 0 and hu.shape[0] == 0:
        raise ValueError("empty held-out pool")
    pi = rng.choice(hu.shape[0], size=n_ins, replace=n_ins > hu.shape[0])
    iu, iv, iw = hu[pi].astype(np.int64), hv[pi].astype(np.int64), hw[pi]
    r = A.row_ids()
    c = A.col.astype(np.int64)
    upper = np.nonzero(r < c)[0]
    pd = rng.choice(upper.shape[0], size=n_del, replace=n_del > upper.shape[0])
    du, dv = r[upper[pd]], c[upper[pd]]
    dw = np.zeros(n_del, dtype=hw.dtype)
    u = np.concatenate([iu, du])
    v = np.concatenate([iv, dv])
    w = np.concatenate([iw, dw])
    op = np.concatenate([np.full(n_ins, OP_INSERT), np.full(n_del, OP_DELETE)]).astype(np.uint8)
    perm = rng.permutation(u.shape[0])
    u, v, w, op = u[perm], v[perm], w[perm], op[perm]
    rows = np.stack([u, v], axis=1).reshape(-1)
    cols = np.stack([v, u], axis=1).reshape(-1)
    vals = np.repeat(w, 2)
    ops = np.repeat(op, 2)
    return Batch(rows.astype(np.int32), cols.astype(np.int32), vals, ops)


def mlp_init_params(seed: int, n_in: int = 4, n_hid: int = 64) -> np.ndarray:
    """Seeded initial parameters of the row-size estimator's network
    (x -> n_hid -> n_hid -> 1), flat in the order W1, b1, W2, b2, W3, b3:
    He-uniform weights (bound sqrt(6 / fan_in)), zero biases, float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((n_hid, n_in), (n_hid, n_hid), (1, n_hid)):
        bound = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-bound, bound, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


class EdgeStream:
    """A stream of undirected-edge batches for a symmetric A, as
    ``rmat_edge_batch`` draws them (half INSERTs from the held-out pool,
    half DELETEs of edges of A, both directions emitted), but with the edge
    lists prepared once so that each batch costs O(its size)."""

    def __init__(self, A: CSR, held, seed: int):
        self.rng = np.random.default_rng(seed)
        r = A.row_ids()
        c = A.col.astype(np.int64)
        upper = r < c
        self.du, self.dv = r[upper], c[upper]
        self.hu, self.hv, self.hw = (np.asarray(x) for x in held)
        self.kind = A.semiring

    def batch(self, n_edges: int) -> Batch:
        rng = self.rng
        n_ins = n_edges // 2
        n_del = n_edges - n_ins
        pi = rng.integers(0, self.hu.shape[0], size=n_ins)
        pd = rng.integers(0, self.du.shape[0], size=n_del)
        u = np.concatenate([self.hu[pi].astype(np.int64), self.du[pd]])
        v = np.concatenate([self.hv[pi].astype(np.int64), self.dv[pd]])
        w = np.concatenate([self.hw[pi], np.zeros(n_del, dtype=self.hw.dtype)])
        op = np.concatenate([np.full(n_ins, OP_INSERT), np.full(n_del, OP_DELETE)]).astype(np.uint8)
        perm = rng.permutation(u.shape[0])
        u, v, w, op = u[perm], v[perm], w[perm], op[perm]
        rows = np.stack([u, v], axis=1).reshape(-1)
        cols = np.stack([v, u], axis=1).reshape(-1)
        return Batch(rows.astype(np.int32), cols.astype(np.int32), np.repeat(w, 2), np.repeat(op, 2))


def random_batch(nrows: int, ncols: int, nupd: int, seed: int, kind: int,
                 A: CSR | None = None, hit_frac: float = 0.5,
                 dup_frac: float = 0.2) -> Batch:
    """Adversarial mixed batch for property tests: ops uniform over
    INSERT/DELETE/SET; a ``hit_frac`` share of positions is drawn from A's
    present entries (when A is given), the rest uniformly; a ``dup_frac`` share
    repeats earlier positions so that one key is written several times."""
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, nrows, size=nupd).astype(np.int64)
    cols = rng.integers(0, ncols, size=nupd).astype(np.int64)
    if A is not None and A.nnz > 0 and nupd > 0:
        hit = rng.random(nupd) < hit_frac
        pk = _present_keys(A)
        pick = pk[rng.integers(0, pk.shape[0], size=int(hit.sum()))]
        rows[hit] = pick // A.ncols
        cols[hit] = pick % A.ncols
    if nupd > 1:
        dup = rng.random(nupd) < dup_frac
        dup[0] = False
        src = (rng.random(nupd) * np.arange(nupd)).astype(np.int64)
        rows[dup] = rows[src[dup]]
        cols[dup] = cols[src[dup]]
    op = rng.integers(0, 3, size=nupd).astype(np.uint8)
    val = _values(rng, nupd, kind)
    return Batch(rows.astype(np.int32), cols.astype(np.int32), val, op)


def concat_batches(*batches: Batch) -> Batch:
    return Batch(np.concatenate([b.row for b in batches]),
                 np.concatenate([b.col for b in batches]),
                 np.concatenate([b.val for b in batches]),
                 np.concatenate([b.op for b in batches]))
