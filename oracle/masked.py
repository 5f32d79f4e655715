"""Algorithm 2 (Section 5.2), general updates by the entry-level masked
recompute, as plain Python over dictionaries -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module.  It takes the algorithm's steps in
the paper's order, on small inputs:

1. A' and B' from A and B by the batches, applied one update at a time in
   array order (insert and set write the entry, delete removes it).
2. A* (B*): the keys whose entry a batch changes.  Reading: a delete of a
   present entry, and every write (insert or set, present or absent, equal
   value or not), count as changes; a delete of an absent entry does not.
   When B is A the A batch is also the B batch.
3. computePattern: C* = A* B' + A B* (Eq. 1) as a pattern with F*, where
   bit (k mod l) of F*(i,j) is set when (i,k) in A* and B'(k,j) != 0, or
   A(i,k) != 0 and (k,j) in B*.
4. E = F | F* at the entries of C* (F(i,j) = 0 where C has no entry), and
   R_i = OR of E over row i.
5. A^R: the entries (i,k) of A' with bit (k mod l) set in R_i.
6. Z, H = A^R B' masked at C*: the terms a b of the kept entries whose
   column is an entry of C*, folded per entry in ascending k, with bit
   (k mod l) of H set for each.
7. C' and F': at each entry of C*, Z and H where Z has the entry, no entry
   where it has none; elsewhere C and F unchanged.

C and F before the batch are the plain product and Bloom filter of A and B
(Gustavson over dictionaries; F(i,j) has bit (k mod l) for every k with
A(i,k) and B(k,j) non-zero), so that a test can check the route's C', F'
against the oracle's plain product and Bloom filter of A', B'.
"""

from __future__ import annotations

import numpy as np

ELL = 64
OP_INSERT, OP_DELETE, OP_SET = 0, 1, 2


def rows_of(csr) -> list[dict]:
    """Row dictionaries {col: value} of a CSR."""
    rp, col, val = np.asarray(csr.rowptr), np.asarray(csr.col), np.asarray(csr.val)
    return [{int(col[p]): val[p].item() for p in range(rp[i], rp[i + 1])} for i in range(csr.nrows)]


def apply_updates(rows: list[dict], batch) -> tuple[list[dict], set]:
    """The rows after the batch, and the keys it changes (step 2's reading)."""
    new = [dict(r) for r in rows]
    last = {}
    for t in range(len(batch.row)):
        key = (int(batch.row[t]), int(batch.col[t]))
        op = int(batch.op[t])
        i, j = key
        if op == OP_DELETE:
            new[i].pop(j, None)
        else:
            new[i][j] = batch.val[t].item()
        last[key] = op
    changed = set()
    for (i, j), op in last.items():
        if op != OP_DELETE or j in rows[i]:
            changed.add((i, j))
    return new, changed


def _mul(a, b, sr):
    return a * b if sr == 0 else a + b


def _add(a, b, sr):
    return a + b if sr == 0 else min(a, b)


def product(A: list[dict], B: list[dict], sr: int) -> dict:
    """Gustavson over dictionaries: {(i,j): value} of A B."""
    C = {}
    for i, row in enumerate(A):
        for k in sorted(row):
            for j in sorted(B[k]):
                t = _mul(row[k], B[k][j], sr)
                C[(i, j)] = t if (i, j) not in C else _add(C[(i, j)], t, sr)
    return C


def bloom(A: list[dict], B: list[dict]) -> dict:
    """{(i,j): word} with bit (k mod l) set for every term A(i,k) B(k,j)."""
    F = {}
    for i, row in enumerate(A):
        for k in row:
            for j in B[k]:
                F[(i, j)] = F.get((i, j), 0) | (1 << (k % ELL))
    return F


def masked_update(A_rows, B_rows, batch_a, batch_b=None, b_is_a=True, sr=0):
    """One batch by Algorithm 2.  Returns a dict with the new operand rows
    (A, B), C and F before and after, C* with F*, R per row, |A^R| and the
    number of products of the masked multiplication."""
    C_old = product(A_rows, B_rows if not b_is_a else A_rows, sr)
    F_old = bloom(A_rows, B_rows if not b_is_a else A_rows)
    A_new, A_star = apply_updates(A_rows, batch_a)
    if b_is_a:
        B_old_rows, B_new, B_star = A_rows, A_new, A_star
    elif batch_b is not None and len(batch_b.row) > 0:
        B_old_rows = B_rows
        B_new, B_star = apply_updates(B_rows, batch_b)
    else:
        B_old_rows, B_new, B_star = B_rows, [dict(r) for r in B_rows], set()
    # step 3: computePattern (A before the batch for the second term)
    a_cols = {}
    for i, row in enumerate(A_rows):
        for k in row:
            a_cols.setdefault(k, []).append(i)
    C_star = {}
    for (i, k) in A_star:
        for j in B_new[k]:
            C_star[(i, j)] = C_star.get((i, j), 0) | (1 << (k % ELL))
    for (k, j) in B_star:
        for i in a_cols.get(k, []):
            C_star[(i, j)] = C_star.get((i, j), 0) | (1 << (k % ELL))
    # step 4: E and R
    R = {}
    for (i, j), fs in C_star.items():
        R[i] = R.get(i, 0) | F_old.get((i, j), 0) | fs
    # step 5: A^R
    kept = [(i, k) for i in sorted(R) for k in sorted(A_new[i]) if (R[i] >> (k % ELL)) & 1]
    # step 6: the masked product
    Z, H = {}, {}
    products = 0
    for (i, k) in kept:
        a = A_new[i][k]
        products += len(B_new[k])
        for j in sorted(B_new[k]):
            if (i, j) in C_star:
                t = _mul(a, B_new[k][j], sr)
                Z[(i, j)] = t if (i, j) not in Z else _add(Z[(i, j)], t, sr)
                H[(i, j)] = H.get((i, j), 0) | (1 << (k % ELL))
    # step 7: the merge at C*
    C_new, F_new = dict(C_old), dict(F_old)
    for key in C_star:
        if key in Z:
            C_new[key] = Z[key]
            F_new[key] = H[key]
        else:
            C_new.pop(key, None)
            F_new.pop(key, None)
    return {
        "A": A_new, "B": B_new, "C_old": C_old, "F_old": F_old, "C": C_new, "F": F_new,
        "C_star": C_star, "R": R, "rows": np.array(sorted(R), dtype=np.int32), "kept": len(kept),
        "products": products, "B_old": B_old_rows,
    }


def to_csr_arrays(d: dict, nrows: int, dtype):
    """(rowptr, col, val) of a {(i,j): value} dictionary, rows ascending."""
    keys = sorted(d)
    rp = np.zeros(nrows + 1, np.int64)
    for (i, _) in keys:
        rp[i + 1] += 1
    rp = np.cumsum(rp)
    col = np.array([j for (_, j) in keys], dtype=np.int32)
    val = np.array([d[k] for k in keys], dtype=dtype)
    return rp, col, val
