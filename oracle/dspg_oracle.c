/*
 * dspg_oracle.c -- CPU oracle for batch-dynamic SpGEMM.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, single-threaded
 * restatement of what the library computes. Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it. It shares no code,
 * header, table or helper with the CUDA library, and nothing here is tuned.
 *
 * What it follows (van der Grinten et al., "Fast Dynamic Updates and Dynamic
 * SpGEMM on MPI-Distributed Graphs"):
 *
 *  - Section 3 (Preliminaries): matrices over a semiring (+,.) or (min,+);
 *    an entry is a non-zero iff it is stored ("structural" non-zero), even
 *    when its value is the number 0; absent entries equal the semiring's
 *    additive neutral element (infinity for (min,+)).
 *  - Section 4.1 (Dynamic Updates): an update inserts a new non-zero, deletes
 *    an existing one, or changes a value.  Insert and value change are the
 *    paper's merge(A, A*) (overwrite or add the entry); delete is
 *    mask(A, A*) (remove the entry if present).  Updates are applied here one
 *    by one in array order, so a later update of the same (i,j) wins.
 *  - Section 5, problem statement: given C = A B and the updated A', B',
 *    compute C' = A' B'.  For general updates C' can only differ from C where
 *    C* = A* B' + A B* (Eq. 1) has a non-zero; the row set of C* is the set
 *    of rows this oracle recomputes in its row-dynamic route.
 *  - Section 5.2: the Bloom filter F of C (orc_bloom), by its definition.
 *  - Section 6.1: the local product is Gustavson's row-wise algorithm with a
 *    sparse accumulator.  Here the accumulator is a dense value array plus a
 *    presence flag per column and a list of touched columns, the plainest
 *    form of that algorithm; the touched list is sorted before output.
 *
 * Value types: (+,.) on double; (min,+) on int32 with plain int32 addition.
 * The (min,+) inputs must satisfy |v| < 2^30 so that a product a+b never
 * overflows; the value INT32_MAX (the library's infinity) is rejected.
 *
 * Every function taking an update list validates it completely before any
 * mutation; an invalid list returns ORC_ERR_INVALID and changes nothing.
 *
 * Threads: single-threaded unless orc_set_threads(n > 1) is called (the CPU
 * baseline's all-cores timing only).  Then the two row loops of the
 * row-dynamic route -- the scan of A' for the affected rows and the
 * recompute of those rows -- are split over n OpenMP threads.  Each row is
 * still computed by one thread in the same order with its own accumulator,
 * so every result is identical to the single-threaded one.  Updates are
 * always applied one by one in array order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_OOM 2

#define ORC_PLUS_TIMES 0
#define ORC_MIN_PLUS 1

#define ORC_OP_INSERT 0
#define ORC_OP_DELETE 1
#define ORC_OP_SET 2

#define ORC_MINPLUS_LIMIT (1 << 30)

/* threads of the row loops (see the header comment); 1 = single-threaded */
static int g_threads = 1;
void orc_set_threads(int n) { g_threads = n > 1 ? n : 1; }
int orc_threads(void) { return g_threads; }

typedef struct {
    int32_t len, cap;
    int32_t *col;   /* strictly ascending */
    double *fv;     /* (+,.) values, or NULL */
    int32_t *iv;    /* (min,+) values, or NULL */
} orc_row;

typedef struct {
    int64_t nrows, ncols;
    int sr;
    orc_row *rows;
} orc_mat;

/* ------------------------------------------------------------------ basics */

orc_mat *orc_new(int64_t nrows, int64_t ncols, int sr) {
    orc_mat *m = (orc_mat *)calloc(1, sizeof(orc_mat));
    if (!m) return NULL;
    m->nrows = nrows;
    m->ncols = ncols;
    m->sr = sr;
    m->rows = (orc_row *)calloc((size_t)(nrows > 0 ? nrows : 1), sizeof(orc_row));
    if (!m->rows) { free(m); return NULL; }
    return m;
}

void orc_free(orc_mat *m) {
    if (!m) return;
    for (int64_t i = 0; i < m->nrows; i++) {
        free(m->rows[i].col);
        free(m->rows[i].fv);
        free(m->rows[i].iv);
    }
    free(m->rows);
    free(m);
}

static int row_reserve(orc_row *r, int sr, int32_t need) {
    if (need <= r->cap) return ORC_OK;
    int32_t cap = r->cap ? r->cap : 4;
    while (cap < need) cap *= 2;
    int32_t *c = (int32_t *)realloc(r->col, sizeof(int32_t) * (size_t)cap);
    if (!c) return ORC_ERR_OOM;
    r->col = c;
    if (sr == ORC_PLUS_TIMES) {
        double *v = (double *)realloc(r->fv, sizeof(double) * (size_t)cap);
        if (!v) return ORC_ERR_OOM;
        r->fv = v;
    } else {
        int32_t *v = (int32_t *)realloc(r->iv, sizeof(int32_t) * (size_t)cap);
        if (!v) return ORC_ERR_OOM;
        r->iv = v;
    }
    r->cap = cap;
    return ORC_OK;
}

/* Position of column c in row r: index if present, else -(insertion point)-1. */
static int64_t row_find(const orc_row *r, int32_t c) {
    int64_t lo = 0, hi = r->len;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (r->col[mid] < c) lo = mid + 1; else hi = mid;
    }
    if (lo < r->len && r->col[lo] == c) return lo;
    return -lo - 1;
}

static int valid_value(int sr, const void *val, int64_t t) {
    if (sr == ORC_PLUS_TIMES) {
        double v = ((const double *)val)[t];
        return !isnan(v) && !isinf(v);
    }
    int32_t v = ((const int32_t *)val)[t];
    return v > -ORC_MINPLUS_LIMIT && v < ORC_MINPLUS_LIMIT;
}

int64_t orc_nnz(const orc_mat *m) {
    int64_t s = 0;
    for (int64_t i = 0; i < m->nrows; i++) s += m->rows[i].len;
    return s;
}

/* Import a canonical CSR (columns strictly ascending in each row). */
int orc_from_csr(orc_mat **out, int64_t nrows, int64_t ncols, int sr,
                 const int64_t *rowptr, const int32_t *col, const void *val) {
    *out = NULL;
    if (nrows < 0 || ncols < 0 || (sr != ORC_PLUS_TIMES && sr != ORC_MIN_PLUS)) return ORC_ERR_INVALID;
    if (rowptr[0] != 0) return ORC_ERR_INVALID;
    for (int64_t i = 0; i < nrows; i++) {
        if (rowptr[i + 1] < rowptr[i]) return ORC_ERR_INVALID;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
            if (col[p] < 0 || col[p] >= ncols) return ORC_ERR_INVALID;
            if (p > rowptr[i] && col[p] <= col[p - 1]) return ORC_ERR_INVALID;
            if (!valid_value(sr, val, p)) return ORC_ERR_INVALID;
        }
    }
    orc_mat *m = orc_new(nrows, ncols, sr);
    if (!m) return ORC_ERR_OOM;
    for (int64_t i = 0; i < nrows; i++) {
        int32_t len = (int32_t)(rowptr[i + 1] - rowptr[i]);
        orc_row *r = &m->rows[i];
        if (row_reserve(r, sr, len) != ORC_OK) { orc_free(m); return ORC_ERR_OOM; }
        memcpy(r->col, col + rowptr[i], sizeof(int32_t) * (size_t)len);
        if (sr == ORC_PLUS_TIMES)
            memcpy(r->fv, (const double *)val + rowptr[i], sizeof(double) * (size_t)len);
        else
            memcpy(r->iv, (const int32_t *)val + rowptr[i], sizeof(int32_t) * (size_t)len);
        r->len = len;
    }
    *out = m;
    return ORC_OK;
}

/* Export to canonical CSR; rowptr has nrows+1 entries, col/val nnz entries. */
void orc_to_csr(const orc_mat *m, int64_t *rowptr, int32_t *col, void *val) {
    int64_t p = 0;
    rowptr[0] = 0;
    for (int64_t i = 0; i < m->nrows; i++) {
        const orc_row *r = &m->rows[i];
        if (col) memcpy(col + p, r->col, sizeof(int32_t) * (size_t)r->len);
        if (val) {
            if (m->sr == ORC_PLUS_TIMES)
                memcpy((double *)val + p, r->fv, sizeof(double) * (size_t)r->len);
            else
                memcpy((int32_t *)val + p, r->iv, sizeof(int32_t) * (size_t)r->len);
        }
        p += r->len;
        rowptr[i + 1] = p;
    }
}

orc_mat *orc_copy(const orc_mat *m) {
    orc_mat *c = orc_new(m->nrows, m->ncols, m->sr);
    if (!c) return NULL;
    for (int64_t i = 0; i < m->nrows; i++) {
        const orc_row *s = &m->rows[i];
        orc_row *d = &c->rows[i];
        if (row_reserve(d, m->sr, s->len) != ORC_OK) { orc_free(c); return NULL; }
        memcpy(d->col, s->col, sizeof(int32_t) * (size_t)s->len);
        if (m->sr == ORC_PLUS_TIMES) memcpy(d->fv, s->fv, sizeof(double) * (size_t)s->len);
        else memcpy(d->iv, s->iv, sizeof(int32_t) * (size_t)s->len);
        d->len = s->len;
    }
    return c;
}

/* ------------------------------------------------------- dynamic updates */

/* Section 4.1: apply an update list one entry at a time in array order.
 * INSERT and SET write the value (merge: overwrite, or add the entry when
 * absent); DELETE removes the entry when present (mask) and is a no-op
 * otherwise. */
int orc_apply(orc_mat *m, int64_t n, const int32_t *row, const int32_t *col,
              const void *val, const uint8_t *op) {
    for (int64_t t = 0; t < n; t++) {
        if (row[t] < 0 || row[t] >= m->nrows || col[t] < 0 || col[t] >= m->ncols) return ORC_ERR_INVALID;
        if (op[t] != ORC_OP_INSERT && op[t] != ORC_OP_DELETE && op[t] != ORC_OP_SET) return ORC_ERR_INVALID;
        if (op[t] != ORC_OP_DELETE && !valid_value(m->sr, val, t)) return ORC_ERR_INVALID;
    }
    for (int64_t t = 0; t < n; t++) {
        orc_row *r = &m->rows[row[t]];
        int64_t at = row_find(r, col[t]);
        if (op[t] == ORC_OP_DELETE) {
            if (at < 0) continue;
            memmove(r->col + at, r->col + at + 1, sizeof(int32_t) * (size_t)(r->len - at - 1));
            if (m->sr == ORC_PLUS_TIMES)
                memmove(r->fv + at, r->fv + at + 1, sizeof(double) * (size_t)(r->len - at - 1));
            else
                memmove(r->iv + at, r->iv + at + 1, sizeof(int32_t) * (size_t)(r->len - at - 1));
            r->len--;
            continue;
        }
        if (at < 0) {
            at = -at - 1;
            if (row_reserve(r, m->sr, r->len + 1) != ORC_OK) return ORC_ERR_OOM;
            memmove(r->col + at + 1, r->col + at, sizeof(int32_t) * (size_t)(r->len - at));
            if (m->sr == ORC_PLUS_TIMES)
                memmove(r->fv + at + 1, r->fv + at, sizeof(double) * (size_t)(r->len - at));
            else
                memmove(r->iv + at + 1, r->iv + at, sizeof(int32_t) * (size_t)(r->len - at));
            r->col[at] = col[t];
            r->len++;
        }
        if (m->sr == ORC_PLUS_TIMES) r->fv[at] = ((const double *)val)[t];
        else r->iv[at] = ((const int32_t *)val)[t];
    }
    return ORC_OK;
}

/* present[t] = 1 iff (row[t], col[t]) is a non-zero of m (indices must be
 * in range; out-of-range entries report 0). */
void orc_presence(const orc_mat *m, int64_t n, const int32_t *row, const int32_t *col,
                  uint8_t *present) {
    for (int64_t t = 0; t < n; t++) {
        if (row[t] < 0 || row[t] >= m->nrows || col[t] < 0 || col[t] >= m->ncols) { present[t] = 0; continue; }
        present[t] = row_find(&m->rows[row[t]], col[t]) >= 0;
    }
}

/* ------------------------------------------------------------- Gustavson */

typedef struct {
    int64_t m;
    uint8_t *present;
    double *facc;
    int32_t *iacc;
    int32_t *touched;
} orc_spa;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int spa_init(orc_spa *s, int64_t m) {
    s->m = m;
    s->present = (uint8_t *)calloc((size_t)(m > 0 ? m : 1), 1);
    s->facc = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    s->iacc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    s->touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    return (s->present && s->facc && s->iacc && s->touched) ? ORC_OK : ORC_ERR_OOM;
}

static void spa_free(orc_spa *s) {
    free(s->present); free(s->facc); free(s->iacc); free(s->touched);
}

/* Row i of C = A B (Section 6.1): for each A(i,k) in ascending k and each
 * B(k,j) in ascending j, form t = a (x) b and fold it into the accumulator
 * of column j with (+); the first contribution to a column initialises it.
 * A column is a non-zero of the output row iff some product reaches it
 * (structural semantics, Section 3: a value 0 stays a non-zero).
 * With absval set, the (+,.) products use |a| |b| (used for error bounds). */
static int gustavson_row(const orc_mat *A, const orc_mat *B, int64_t i, orc_spa *s,
                         orc_row *out, int absval) {
    const orc_row *ar = &A->rows[i];
    int32_t nt = 0;
    for (int32_t p = 0; p < ar->len; p++) {
        int32_t k = ar->col[p];
        const orc_row *br = &B->rows[k];
        for (int32_t q = 0; q < br->len; q++) {
            int32_t j = br->col[q];
            if (A->sr == ORC_PLUS_TIMES) {
                double a = ar->fv[p], b = br->fv[q];
                double t = absval ? fabs(a) * fabs(b) : a * b;
                if (!s->present[j]) { s->present[j] = 1; s->facc[j] = t; s->touched[nt++] = j; }
                else s->facc[j] = s->facc[j] + t;
            } else {
                int32_t t = ar->iv[p] + br->iv[q];
                if (!s->present[j]) { s->present[j] = 1; s->iacc[j] = t; s->touched[nt++] = j; }
                else if (t < s->iacc[j]) s->iacc[j] = t;
            }
        }
    }
    qsort(s->touched, (size_t)nt, sizeof(int32_t), cmp_i32);
    out->len = 0;
    if (row_reserve(out, A->sr, nt) != ORC_OK) return ORC_ERR_OOM;
    for (int32_t t = 0; t < nt; t++) {
        int32_t j = s->touched[t];
        out->col[t] = j;
        if (A->sr == ORC_PLUS_TIMES) out->fv[t] = s->facc[j];
        else out->iv[t] = s->iacc[j];
        s->present[j] = 0;
    }
    out->len = nt;
    return ORC_OK;
}

/* C = A B over all rows (the static product). */
orc_mat *orc_multiply(const orc_mat *A, const orc_mat *B, int absval) {
    if (A->ncols != B->nrows || A->sr != B->sr) return NULL;
    orc_mat *C = orc_new(A->nrows, B->ncols, A->sr);
    if (!C) return NULL;
    orc_spa s;
    if (spa_init(&s, B->ncols) != ORC_OK) { spa_free(&s); orc_free(C); return NULL; }
    for (int64_t i = 0; i < A->nrows; i++) {
        if (gustavson_row(A, B, i, &s, &C->rows[i], absval) != ORC_OK) {
            spa_free(&s); orc_free(C); return NULL;
        }
    }
    spa_free(&s);
    return C;
}

/* Rows `rows[0..nr)` of A B as a CSR; two calls: with col == NULL only
 * rowptr (nr+1 entries) is filled. */
int orc_multiply_rows(const orc_mat *A, const orc_mat *B, const int32_t *rows, int64_t nr,
                      int absval, int64_t *rowptr, int32_t *col, void *val) {
    if (A->ncols != B->nrows || A->sr != B->sr) return ORC_ERR_INVALID;
    orc_spa s;
    if (spa_init(&s, B->ncols) != ORC_OK) { spa_free(&s); return ORC_ERR_OOM; }
    orc_row tmp = {0, 0, NULL, NULL, NULL};
    rowptr[0] = 0;
    for (int64_t t = 0; t < nr; t++) {
        if (rows[t] < 0 || rows[t] >= A->nrows) { spa_free(&s); return ORC_ERR_INVALID; }
        if (gustavson_row(A, B, rows[t], &s, &tmp, absval) != ORC_OK) { spa_free(&s); return ORC_ERR_OOM; }
        int64_t p = rowptr[t];
        if (col) {
            memcpy(col + p, tmp.col, sizeof(int32_t) * (size_t)tmp.len);
            if (A->sr == ORC_PLUS_TIMES) memcpy((double *)val + p, tmp.fv, sizeof(double) * (size_t)tmp.len);
            else memcpy((int32_t *)val + p, tmp.iv, sizeof(int32_t) * (size_t)tmp.len);
        }
        rowptr[t + 1] = p + tmp.len;
    }
    free(tmp.col); free(tmp.fv); free(tmp.iv);
    spa_free(&s);
    return ORC_OK;
}

/* ---------------------------------------------------- the Bloom filter F */

/* Section 5.2: the Bloom filter of C = A B is a matrix F with C's pattern
 * whose entry F(i,j) is an l-bit field (l = 64 here, as in the paper) with
 * bit (k mod l) set iff the term A(i,k) B(k,j) contributes to C(i,j), i.e.
 * iff both A(i,k) and B(k,j) are non-zeros.  Computed by definition, row by
 * row like the product: for each A(i,k), each B(k,j), OR the bit into the
 * word of column j.  Two calls: with col == NULL only rowptr (nrows+1
 * entries) is filled. */
int orc_bloom(const orc_mat *A, const orc_mat *B, int64_t *rowptr, int32_t *col, uint64_t *words) {
    if (A->ncols != B->nrows) return ORC_ERR_INVALID;
    int64_t m = B->ncols;
    uint8_t *present = (uint8_t *)calloc((size_t)(m > 0 ? m : 1), 1);
    uint64_t *acc = (uint64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(uint64_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!present || !acc || !touched) { free(present); free(acc); free(touched); return ORC_ERR_OOM; }
    rowptr[0] = 0;
    for (int64_t i = 0; i < A->nrows; i++) {
        const orc_row *ar = &A->rows[i];
        int32_t nt = 0;
        for (int32_t p = 0; p < ar->len; p++) {
            int32_t k = ar->col[p];
            uint64_t bit = (uint64_t)1 << (k % 64);
            const orc_row *br = &B->rows[k];
            for (int32_t q = 0; q < br->len; q++) {
                int32_t j = br->col[q];
                if (!present[j]) { present[j] = 1; acc[j] = 0; touched[nt++] = j; }
                acc[j] |= bit;
            }
        }
        qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
        int64_t o = rowptr[i];
        for (int32_t t = 0; t < nt; t++) {
            int32_t j = touched[t];
            if (col) { col[o + t] = j; words[o + t] = acc[j]; }
            present[j] = 0;
        }
        rowptr[i + 1] = o + nt;
    }
    free(present); free(acc); free(touched);
    return ORC_OK;
}

/* ---------------------------------------------------- affected rows (R) */

/* The rows of C that a batch may change (Section 5, general updates: C'
 * differs from C only at non-zeros of C* = A* B' + A B*, Eq. 1).
 *
 * A* holds the entries of a batch that really change A: a batch key (i,j)
 * belongs to A* iff it is a non-zero of A or of A' (a delete of an absent
 * entry changes nothing; every write counts as a change).  The caller passes
 * the presence of each batch entry before (pre) and after (post) the batch.
 * B* likewise for the B batch.  At row granularity
 *
 *     R = rows(A*)  u  { i : A'(i,k) != 0 for some k in rows(B*) }.
 *
 * When B is A (C = A A) the single batch is both A* and B*.
 * `a_new` is A'.  Writes R ascending into `out` (room for nrows) and
 * returns |R|. */
int64_t orc_affected_rows(const orc_mat *a_new,
                          int64_t na, const int32_t *arow, const uint8_t *apre, const uint8_t *apost,
                          int64_t nb, const int32_t *brow, const uint8_t *bpre, const uint8_t *bpost,
                          int64_t b_nrows, int b_is_a, int32_t *out) {
    uint8_t *in_r = (uint8_t *)calloc((size_t)(a_new->nrows > 0 ? a_new->nrows : 1), 1);
    uint8_t *brows = (uint8_t *)calloc((size_t)(b_nrows > 0 ? b_nrows : 1), 1);
    if (!in_r || !brows) { free(in_r); free(brows); return -1; }
    for (int64_t t = 0; t < na; t++)
        if (apre[t] || apost[t]) in_r[arow[t]] = 1;
    if (b_is_a) {
        for (int64_t t = 0; t < na; t++)
            if (apre[t] || apost[t]) brows[arow[t]] = 1;
    } else {
        for (int64_t t = 0; t < nb; t++)
            if (bpre[t] || bpost[t]) brows[brow[t]] = 1;
    }
#pragma omp parallel for num_threads(g_threads) schedule(static, 4096) if (g_threads > 1)
    for (int64_t i = 0; i < a_new->nrows; i++) {
        const orc_row *r = &a_new->rows[i];
        for (int32_t p = 0; p < r->len && !in_r[i]; p++)
            if (brows[r->col[p]]) in_r[i] = 1;
    }
    int64_t cnt = 0;
    for (int64_t i = 0; i < a_new->nrows; i++)
        if (in_r[i]) out[cnt++] = (int32_t)i;
    free(in_r);
    free(brows);
    return cnt;
}

/* Replace rows `rows[0..nr)` of C by the rows of A B, in place; every other
 * row of C is left as it is (the row-dynamic route). */
int orc_replace_rows(orc_mat *C, const orc_mat *A, const orc_mat *B, const int32_t *rows, int64_t nr) {
    if (A->ncols != B->nrows || A->sr != B->sr || C->nrows != A->nrows || C->ncols != B->ncols) return ORC_ERR_INVALID;
    for (int64_t t = 0; t < nr; t++)
        if (rows[t] < 0 || rows[t] >= A->nrows) return ORC_ERR_INVALID;
    int err = ORC_OK;
#pragma omp parallel num_threads(g_threads) if (g_threads > 1)
    {
        orc_spa s;  /* one accumulator per thread */
        int mine = spa_init(&s, B->ncols);
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < nr; t++)
            if (mine == ORC_OK) mine = gustavson_row(A, B, rows[t], &s, &C->rows[rows[t]], 0);
        spa_free(&s);
        if (mine != ORC_OK) {
#pragma omp critical
            err = mine;
        }
    }
    return err;
}

/* Row accessors for sampled comparisons. */
int32_t orc_row_len(const orc_mat *m, int64_t i) { return m->rows[i].len; }

void orc_get_row(const orc_mat *m, int64_t i, int32_t *col, void *val) {
    const orc_row *r = &m->rows[i];
    memcpy(col, r->col, sizeof(int32_t) * (size_t)r->len);
    if (m->sr == ORC_PLUS_TIMES) memcpy(val, r->fv, sizeof(double) * (size_t)r->len);
    else memcpy(val, r->iv, sizeof(int32_t) * (size_t)r->len);
}
