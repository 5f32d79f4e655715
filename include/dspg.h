/*
 * dspg.h -- C ABI of the batch-dynamic SpGEMM library for one GB300 GPU.
 *
 * The problem (van der Grinten et al., "Fast Dynamic Updates and Dynamic
 * SpGEMM on MPI-Distributed Graphs", Section 5): A is n x k, B is k x m,
 * C = A B over a semiring.  A batch of updates turns A, B into A', B'; the
 * library then produces C' = A' B' by recomputing only the rows of C that
 * the batch can change (general updates, Section 5: C' differs from C only
 * where C* = A* B' + A B* (Eq. 1) has a non-zero), instead of the whole
 * product.
 *
 * Semirings (Section 3): (+,.) on double, and (min,+) on int32 (the
 * shortest-path semiring).  An entry is a non-zero iff it is stored
 * ("structural" non-zero, Section 3), even when its value is 0; absent
 * entries are the additive neutral element (infinity for (min,+)).
 * (min,+) values must satisfy |v| < 2^30; sums use plain int32 addition.
 *
 * Updates (Section 4.1): INSERT and SET write a value at (i,j) (the paper's
 * merge: overwrite, or add the entry when absent); DELETE removes (i,j)
 * when present (the paper's mask) and is a no-op otherwise.  Within one
 * batch, updates of the same (i,j) take effect in array order: the last
 * one wins.
 *
 * Conventions for every call:
 *  - Indices are int32 (rows, columns), offsets int64.
 *  - Pointers marked "host or device" are device pointers when the
 *    accompanying on_device flag is 1 and host pointers otherwise; they are
 *    only read during the call (borrowed) and copied into library memory.
 *  - The handle owns A', B', C' and all working memory on the device; no
 *    pointer into library memory is ever returned.
 *  - All work is enqueued on the given stream (0 = legacy default stream);
 *    calls that return a status or sizes synchronise that stream.
 *  - Errors are reported as dspg_status codes only; dspg_last_error gives a
 *    message.  An invalid input returns DSPG_ERR_INVALID and leaves the
 *    handle exactly as it was (validation precedes mutation).
 *  - A handle is not thread-safe: one call at a time per handle.
 */
#ifndef DSPG_H
#define DSPG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DSPG_PLUS_TIMES_F64 = 0, /* (+,.) with double values */
    DSPG_MIN_PLUS_I32 = 1    /* (min,+) with int32 values, |v| < 2^30 */
} dspg_semiring;

typedef enum {
    DSPG_OK = 0,
    DSPG_ERR_INVALID = 1, /* bad argument or batch; the handle is unchanged */
    DSPG_ERR_OOM = 2,     /* device memory exhausted; the handle is unchanged */
    DSPG_ERR_CUDA = 3,    /* a CUDA runtime error; the handle should be destroyed */
    DSPG_ERR_TIMEOUT = 4, /* a bounded device-side loop gave up */
    DSPG_ERR_STATE = 5    /* call not valid in the handle's current state */
} dspg_status;

typedef enum { DSPG_OP_INSERT = 0, DSPG_OP_DELETE = 1, DSPG_OP_SET = 2 } dspg_op;

/* A canonical CSR matrix: rowptr[nrows+1] (rowptr[0] = 0, non-decreasing),
 * col[nnz] strictly ascending within each row and in [0, ncols), val[nnz]
 * of the semiring's value type.  Host or device memory per on_device. */
typedef struct {
    int64_t nrows, ncols, nnz;
    const int64_t *rowptr;
    const int32_t *col;
    const void *val;
    int on_device;
} dspg_csr;

/* An update batch in arrival order (Section 4.1): n entries of
 * (row, col, val, op); val is ignored for DELETE.  Host or device memory
 * per on_device. */
typedef struct {
    int64_t n;
    const int32_t *row;
    const int32_t *col;
    const void *val;
    const uint8_t *op;
    int on_device;
} dspg_updates;

/* Tuning knobs; pass NULL for the defaults given here. */
typedef struct {
    int32_t slack_min;      /* free slots reserved per row: max(slack_min, len/slack_div); default 4 */
    int32_t slack_div;      /* default 4 */
    double arena_headroom;  /* arena capacity / total row capacity at build; default 1.5 */
    int32_t keep_transpose; /* 1: maintain A's transposed pattern (needed when B is A or B changes); -1: auto */
    int32_t exact_static;   /* static product: 1 = count rows exactly before laying C out (two passes);
                               0 = auto (exact only when the bound-sized layout would take over a quarter
                               of the free device memory) */
    int32_t bloom;          /* 1: keep the Bloom filter F of C (Section 5.2: a 64-bit word per entry of C,
                               bit (k mod 64) set when A(i,k) B(k,j) contributes to C(i,j)) and apply every
                               batch by the entry-level masked recompute of Algorithm 2 (general updates);
                               0 (default): the row path.  See dspg_apply_batch. */
} dspg_options;

/* What one apply_batch did.  Counts of the unique, last-writer-wins batch
 * entries of A and B together. */
typedef struct {
    int64_t n_updates;      /* entries received (A and B batches) */
    int64_t n_unique;       /* distinct (matrix, row, col) keys */
    int64_t n_insert;       /* writes of absent entries */
    int64_t n_update;       /* writes of present entries */
    int64_t n_delete;       /* deletes of present entries */
    int64_t n_noop;         /* deletes of absent entries */
    int64_t touched_rows;   /* rows of A and B rewritten by the merge */
    int64_t affected_rows;  /* |R|: rows of C recomputed */
    int64_t products;       /* semiring products formed in the recompute */
    int64_t nnz_written;    /* entries of C written by the recompute */
    int64_t relocations;    /* rows moved to the arena tail (A, B, transpose, C) */
    int64_t compactions;    /* arena rebuilds (growth) during this batch */
    int64_t a_entries;      /* entries of A' rows read by the recompute */
    int64_t est_rows;       /* rows sized by the learned estimator */
    int64_t est_overflows;  /* of those, rows whose table was too small (counted exactly, recomputed) */
    int64_t algebraic;      /* 1: the batch took the delta path of Eq. 1 (dspg_apply_batch_algebraic) */
    int64_t table_slots;    /* accumulator slots of the recompute's rows (hash-table or dense-row size per
                               row, summed; what the sizing decides, the learned estimator's gain) */
    int64_t masked_entries; /* handles with the Bloom filter: entries of C* (Algorithm 2's mask), the
                               entries of C the batch may change; affected_rows then counts C*'s rows,
                               a_entries the entries of A' the filter kept (A^R) and products the
                               products of the masked multiplication */
} dspg_batch_stats;

/* Stages of apply_batch, in pipeline order, for dspg_stage_times. */
enum {
    DSPG_STAGE_SORT = 0,      /* radix sort + last-writer de-duplication (Section 4.2 grouping) */
    DSPG_STAGE_CLASSIFY = 1,  /* row segments, insert/update/delete classification */
    DSPG_STAGE_DETECT = 2,    /* affected rows R (Section 5, rows of C*) */
    DSPG_STAGE_MERGE = 3,     /* rebuild changed rows of A (and B) in staging */
    DSPG_STAGE_COMMIT = 4,    /* write them into the slack-CSR (Section 4.1 merge/mask) */
    DSPG_STAGE_TRANSPOSE = 5, /* keep A's transposed pattern in step */
    DSPG_STAGE_SIZE = 6,      /* product bounds and bins of the rows of R */
    DSPG_STAGE_NUMERIC = 7,   /* Gustavson recompute of the rows of R (Section 6.1), written into C */
    DSPG_NSTAGES = 8
};

typedef struct dspg_handle dspg_handle;

/* Build a handle holding A, B and C = A B (Section 5's starting point; the
 * product itself is Gustavson's row-wise algorithm, Section 6.1).
 * B == NULL means B is A (C = A A): one batch then updates both operands.
 * A->ncols must equal B->nrows.  On success *out receives the handle.
 * Returns DSPG_ERR_INVALID for a non-canonical or out-of-range input. */
dspg_status dspg_build(dspg_handle **out, const dspg_csr *A, const dspg_csr *B, dspg_semiring sr,
                       const dspg_options *opt, void *stream);

/* The general product form of Section 3: C = alpha op(A) op(B) (+) beta X,
 * where op is the identity or the transpose (Section 5.3, handling
 * transposition).  In (+,.): alpha (x) p = alpha p and (+) = +; in (min,+):
 * alpha (x) p = alpha + p and (+) = min.
 *   trans_a, trans_b: 1 = the product uses A^T (B^T).  The operand is stored
 *     transposed (built on the device); batches of A and B and dspg_read_A
 *     stay in the caller's coordinates (an update (i, j) of A is applied as
 *     (j, i) to A^T).  With B == NULL (B is A) and trans_a != trans_b (for
 *     instance A^T A), the library keeps A and A^T and every batch of A
 *     updates both.
 *   alpha, beta (+,.) or alpha_i, beta_i ((min,+), |.| < 2^29): the scalars.
 *   X: NULL, or a canonical CSR with the shape of op(A) op(B); borrowed for
 *     the call (copied), fixed afterwards.
 * The handle keeps P = op(A) op(B) up to date; alpha, beta and X are applied
 * when rows are read (dspg_read_C, dspg_read_rows_C): the rows of C a batch
 * can change are the rows of P it recomputes (dspg_last_affected).  A form
 * with alpha = 1 (alpha_i = 0) and no X reads P itself.  dspg_footprint
 * rejects handles with a transposed operand.  Returns DSPG_ERR_INVALID for
 * mismatched shapes, an X of the wrong shape, or out-of-range scalars. */
typedef struct {
    int32_t trans_a, trans_b;
    double alpha, beta;
    int32_t alpha_i, beta_i;
    const dspg_csr *X;
} dspg_form;
dspg_status dspg_build_form(dspg_handle **out, const dspg_csr *A, const dspg_csr *B, dspg_semiring sr,
                            const dspg_form *form, const dspg_options *opt, void *stream);

/* Apply one batch to A (dA) and to B (dB; must be NULL or empty when B is
 * A) and bring C up to date: C' = A' B' (Section 5, general updates).
 * Rows of C outside the affected set R = rows(A*) u {i : A(i,k) != 0,
 * k in rows(B*)} are left bit-for-bit as they were.  stats may be NULL.
 * Synchronises the stream once to return the status.
 *
 * A handle built with options.bloom = 1 applies the batch entry by entry
 * instead (Section 5.2, Algorithm 2): the pattern of C* = A* B' + A B*
 * with its Bloom words F*, E = F | F* at C*'s entries and its OR per row
 * R_i, the entries of A' that R_i's bits keep (A^R), their products masked
 * at C*, and the merge of the results into C and F.  Entries of C outside
 * C* are left bit-for-bit as they were, the rows of C* are what
 * dspg_last_affected lists, and masked_entries in stats counts C*.  It
 * runs eagerly with several stream synchronisations (no graph); such a
 * handle rejects dspg_apply_batch_algebraic, dspg_apply_batch_async,
 * dspg_autotune and groups (DSPG_ERR_STATE). */
dspg_status dspg_apply_batch(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB,
                             dspg_batch_stats *stats, void *stream);

/* dspg_apply_batch in two halves, so that other work can run while the batch
 * is on the GPU.  dspg_apply_batch_async checks the batch, uploads it and
 * enqueues the whole pipeline on `stream`, then returns; the batch arrays
 * (host or device) must stay unchanged until dspg_apply_batch_wait returns.
 * dspg_apply_batch_wait waits for it, grows buffers and re-runs failed
 * stages as dspg_apply_batch would, fills stats, and returns the status.
 * In between, the handle takes no other call but dspg_read_C and
 * dspg_read_rows_C (others return DSPG_ERR_STATE); those reads are
 * consistent only for rows the batch cannot change (outside its
 * footprint, dspg_footprint), which a serving loop uses to read one wave's
 * rows while the next wave runs.  The reads may use another stream. */
dspg_status dspg_apply_batch_async(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB, void *stream);
dspg_status dspg_apply_batch_wait(dspg_handle *h, dspg_batch_stats *stats, void *stream);

/* Apply one batch as dspg_apply_batch does, by the delta path of Section 5's
 * algebraic updates when the batch qualifies: C' = C (+) C* with
 * C* = A* B' (+) A B* (Eq. 1; Section 5.1's local step), formed entry by
 * entry from the update matrices instead of recomputing rows.  A batch
 * qualifies when every entry that changes A or B writes an absent entry
 * (an insertion: A' = A (+) A* with the semiring's addition; deletes of
 * absent entries are ignored).  Any write to a present entry or delete of
 * one makes the call apply the batch by the row path instead (general
 * updates), with the same result as dspg_apply_batch; stats->algebraic says
 * which path ran.  Each contribution a (x) b is folded into C'(i,j) where
 * row i of C holds column j (an atomic (+) on the value, so in (+,.) the
 * summation order varies, within the library's tolerance), and otherwise
 * appended to row i (rows of C carry no column order); rows of C longer
 * than 256 entries are recomputed by the row path instead of searched.
 * After the call, C' = A' B' as after dspg_apply_batch; affected_rows and
 * dspg_last_affected give the rows of C that took a contribution (a subset
 * of the row path's R), products the contributions formed.  Runs eagerly
 * (no captured graph) and synchronises the stream several times.  Errors
 * as dspg_apply_batch. */
dspg_status dspg_apply_batch_algebraic(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB,
                                       dspg_batch_stats *stats, void *stream);

/* Read C (with dspg_build_form: alpha op(A) op(B) (+) beta X) in canonical
 * CSR (rows in order, columns ascending) into caller
 * buffers: rowptr[nrows+1], col[nnz], val[nnz], host or device per
 * on_device (host buffers may be pageable or page-locked; page-locked ones
 * are copied to at full speed).  Two-call convention: with rowptr == NULL
 * only *nnz_out is written.  The handle keeps the read's device scratch
 * (up to 256 MiB per buffer) for later reads; a larger read allocates and
 * frees its scratch within the call. */
dspg_status dspg_read_C(dspg_handle *h, int64_t *nnz_out, int64_t *rowptr, int32_t *col, void *val,
                        int on_device, void *stream);

/* The Bloom filter F of C (handles with options.bloom = 1; Section 5.2):
 * the same two-call protocol and canonical order as dspg_read_C, with the
 * 64-bit word of each entry in words (bit (k mod 64) set when A(i,k) B(k,j)
 * contributes to C(i,j)).  DSPG_ERR_STATE for a handle without F. */
dspg_status dspg_read_bloom(dspg_handle *h, int64_t *nnz_out, int64_t *rowptr, int32_t *col, uint64_t *words,
                            int on_device, void *stream);

/* Read A' (the updated left operand) in canonical CSR; same convention.
 * A' is in the caller's coordinates: rowptr has A->nrows + 1 entries of the
 * A given to dspg_build (dspg_build_form turns a stored transpose back). */
dspg_status dspg_read_A(dspg_handle *h, int64_t *nnz_out, int64_t *rowptr, int32_t *col, void *val,
                        int on_device, void *stream);

/* Read selected rows of C: rows[nrows] (host or device per on_device);
 * rowptr[nrows+1], col, val as in dspg_read_C, in the order given.  The
 * fill call reuses the row pointers its count call computed when the host
 * row list is the same (by content) and C has not changed in between. */
dspg_status dspg_read_rows_C(dspg_handle *h, const int32_t *rows, int64_t nrows, int64_t *nnz_out,
                             int64_t *rowptr, int32_t *col, void *val, int on_device, void *stream);

/* Host-side fault injection, a testing aid with no counterpart in the
 * paper.  spec: NULL or "" (off), or "site@N" items separated by commas:
 * alloc@N fails the N-th device allocation from now on (DSPG_ERR_OOM),
 * validate@N fails the N-th batch check (DSPG_ERR_INVALID).  Counted per
 * process; each fires once.  The environment variable DSPG_FAULT sets the
 * same at the first use of the library.  A batch that fails in its checks
 * or while its buffers grow (before A, B or C change) leaves the handle as
 * it was; a failure after that (an exhausted arena that cannot grow, a
 * probe limit, a CUDA error) leaves the handle's matrices undefined, and
 * every later call on it returns DSPG_ERR_STATE.  Returns
 * DSPG_ERR_INVALID for a malformed spec. */
dspg_status dspg_fault_inject(const char *spec);

/* 1 for the debug build (compiled with DSPG_DEBUG=1: kernels check indices
 * and room before their accesses, and a failed check fails the batch with
 * DSPG_ERR_CUDA naming the check), else 0. */
int dspg_debug_build(void);

/* The rows of C the last batch affected (the set dspg_last_affected lists)
 * and their entries, in one call: R ascending into rows, and the rows of C'
 * in canonical CSR (rowptr n+1 entries, columns ascending per row) into
 * rowptr, col and val, host or device memory per on_device.  *nrows_out and
 * *nnz_out receive the sizes; with rows == NULL nothing else is written.
 * Buffers smaller than rows_cap < n or nnz_cap < nnz: DSPG_ERR_INVALID with
 * the sizes written (the caller grows and calls again).  Synchronises the
 * stream once when col and val are page-locked host memory, twice
 * otherwise.  Not for handles with alpha, beta or X (DSPG_ERR_STATE).
 * Not part of the paper: the read a server makes after each batch. */
dspg_status dspg_read_affected_C(dspg_handle *h, int64_t rows_cap, int64_t nnz_cap, int64_t *nrows_out,
                                 int64_t *nnz_out, int32_t *rows, int64_t *rowptr, int32_t *col, void *val,
                                 int on_device, void *stream);

/* dspg_apply_batch followed by dspg_read_affected_C (host memory,
 * on_device = 0), with the same arguments and results, in one call.  When
 * rows, rowptr, col and val are all page-locked host memory (cudaHostAlloc,
 * cudaHostRegister), rows_cap >= 0 and the handle keeps no Bloom filter, the
 * read is enqueued behind the batch and the stream is synchronised once:
 * the read's kernels take R's size from the device, check it against
 * rows_cap, and write R, its row pointers and its rows of C' into the
 * caller's arrays.  When the batch needed a second pass (a buffer grew, a
 * learned table overflowed) or the arrays are too small, the enqueued read
 * is discarded and the read runs again on its own after the batch
 * (DSPG_ERR_INVALID with the sizes written, as dspg_read_affected_C, for
 * arrays that are too small).  Any other host memory: the two calls one
 * after the other.  A batch that fails returns its error with nothing read.
 * Not part of the paper: the step of a server that returns every batch's
 * affected rows. */
dspg_status dspg_apply_read_affected(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB,
                                     int64_t rows_cap, int64_t nnz_cap, int64_t *nrows_out, int64_t *nnz_out,
                                     int32_t *rows, int64_t *rowptr, int32_t *col, void *val,
                                     dspg_batch_stats *stats, void *stream);

/* The affected row set R of the last apply_batch, ascending, into rows
 * (room for *count rows; with rows == NULL only *count is written). */
dspg_status dspg_last_affected(dspg_handle *h, int64_t *count, int32_t *rows, int on_device, void *stream);

/* Recompute every row of C from the current A', B' (the static product, used
 * as the comparison point for the dynamic path). */
dspg_status dspg_recompute_all(dspg_handle *h, void *stream);

/* Shapes and sizes: nrows(A), ncols(A) = nrows(B), ncols(B), nnz(A'), nnz(C'). */
dspg_status dspg_info(dspg_handle *h, int64_t *n, int64_t *k, int64_t *m, int64_t *nnz_a, int64_t *nnz_c);

/* Turn per-stage timing on (1) or off (0).  When on, apply_batch records a
 * CUDA event between its stages on the caller's stream; dspg_stage_times
 * then returns the device time of each stage of the last apply_batch in
 * milliseconds (ms[DSPG_NSTAGES]; n = room in ms).  Re-runs after a buffer
 * grew are not included. */
dspg_status dspg_set_profiling(dspg_handle *h, int on);
dspg_status dspg_stage_times(dspg_handle *h, float *ms, int n);

/* Number of CUDA kernels this library has launched in this process (all
 * handles), for auditing how many launches a call makes. */
unsigned long long dspg_kernel_launches(void);

/* How the handle's batches have run so far (the row path, alone or in a
 * group): replaying a captured pipeline, capturing one, or eagerly.  A
 * captured pipeline serves every later batch of the same launch sizes (the
 * batch length rounded up to a multiple of 1024 up to 16384, to a power of
 * two beyond) while no buffer moves.  Not part of the paper. */
dspg_status dspg_run_counts(const dspg_handle *h, int64_t *replayed, int64_t *captured, int64_t *eager);

/* Reserve launch sizes for batches of up to nA (and nB) entries when the
 * handle runs inside a group (dspg_group_apply): the member then launches
 * its pipeline at those sizes whatever its batch's length (a shorter batch
 * runs as a zero-padded one, an empty batch as a zero-length one), so one
 * captured group pipeline serves every combination of the members' batch
 * sizes up to their reservations; a larger batch raises the member's
 * reservation.  Buffers are grown now.  Not part of the paper. */
dspg_status dspg_reserve(dspg_handle *h, int64_t nA, int64_t nB, void *stream);

/* Row bins of the recompute.  Section 6.1 fixes only that each row is formed
 * in a sparse accumulator; which accumulator serves which row is this
 * library's choice.  A row of R is binned by its product bound ub (the sum of
 * the lengths of the B rows it reads, capped at the column count):
 *  - group sort: rows with an uncapped bound ub <= sort_max (0..256; 0 turns
 *    it off), whose products a group of 8, 16 or 32 lanes (for ub up to 64,
 *    128, 256) holds in registers, sorts by column and folds;
 *  - thread merge (the rows the group sort leaves): A rows with at most merge_k entries (0..8; 0 turns the
 *    merge off) and an uncapped bound ub <= 64, in two kernels: ub <=
 *    merge_ub (0..64) in one whose threads stage merge_ub entries in shared
 *    memory, so that a lower bound lets more threads run at once (at 49,
 *    three 128-thread blocks per SM for double, at the cost of L1 cache),
 *    the rest in one staging 64;
 *  - hash tables in shared memory of at least ub << table_shift slots
 *    (table_shift 0 or 1), served by 8, 16 or 32 lanes per row while the
 *    table has at most 32, 64 or warp_max slots (lanes_min = 8, 16 or 32:
 *    the fewest lanes a row may get; warp_max in 0..1024), then by a whole
 *    CTA while it has at most cta_max slots (0..16384);
 *  - longer rows: a CTA with a dense accumulator in global memory.
 * Every setting gives the same C: a table never has fewer slots than the
 * row's bound, which no row's distinct columns can exceed.  Only the speed
 * changes.  C with at most 1024 columns uses dense shared-memory
 * accumulators for all rows outside the thread-merge bin instead. */
typedef struct {
    int32_t merge_k, merge_ub;
    int32_t lanes_min;
    int32_t table_shift;
    int32_t warp_max;
    int32_t cta_max;
    int32_t sort_max;
} dspg_tuning;

/* Set (t == NULL: restore the defaults {8, 64, 8, 0, 1024, 16384, 64}) or read
 * the tuning of h.  Out-of-range fields return DSPG_ERR_INVALID. */
dspg_status dspg_set_tuning(dspg_handle *h, const dspg_tuning *t);
dspg_status dspg_get_tuning(dspg_handle *h, dspg_tuning *t);

/* Choose the tuning of h by measurement.  Each of the nbatches batches
 * (updates of A; of B too when dB != NULL, as arrays of nbatches) is applied
 * in full, in order, as by dspg_apply_batch: they are real updates.  After
 * each, the recompute of its affected rows (sizing and numeric stages) is
 * replayed once under every candidate of a built-in list of tunings, in a
 * rotating order, and timed on the device; replaying rewrites the same rows
 * of C from the same A', B'.  The candidate with the least total time is set
 * on h and written to *best (may be NULL); ms[k] (room for n_ms entries, may
 * be NULL) receives candidate k's total and *n_cand the list's length. */
dspg_status dspg_autotune(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB, int64_t nbatches,
                          dspg_tuning *best, float *ms, int n_ms, int *n_cand, void *stream);

/* The k-th built-in candidate tuning (k < *n_cand of dspg_autotune). */
dspg_status dspg_tuning_candidate(int k, dspg_tuning *t);

/* A group of independent handles whose batches are applied together: every
 * handle's whole pipeline is enqueued as one branch of a single CUDA graph,
 * so one graph launch runs all of them and their kernels overlap on the
 * device.  The paper distributes one product over many processes; a group
 * instead packs many small, unrelated products onto one GPU (no counterpart
 * in the paper).  handles[n]: distinct handles on the current device; they
 * must outlive the group, and a handle may belong to several groups.  The
 * group keeps its graphs keyed by every member's batch sizes and buffers: the
 * first apply of a key runs eagerly (branches on the members' own streams),
 * the second captures the graph, later ones replay it. */
typedef struct dspg_group dspg_group;
dspg_status dspg_group_create(dspg_group **out, dspg_handle *const *handles, int64_t n);

/* Apply dA[t] (and dB[t] when dB != NULL) to member t, for every t, as
 * dspg_apply_batch would one by one; a NULL or empty batch leaves its member
 * as it is.  stats and status may be NULL, else arrays of n: per-member
 * statistics and status.  Members whose run needs more memory are grown and
 * re-run eagerly after the graph.  Returns DSPG_OK when every member
 * succeeded, else the first failing member's status (its message is in
 * dspg_last_error of the group and of the member); the others are applied.
 * Synchronises the stream. */
dspg_status dspg_group_apply(dspg_group *g, const dspg_updates *dA, const dspg_updates *dB,
                             dspg_batch_stats *stats, dspg_status *status, void *stream);

/* ---------------------------------------------------------------------------
 * Sizing of the recompute's hash tables, and the learned row-size estimator.
 *
 * Each affected row is recomputed in a hash table in shared memory
 * (Section 6.1's sparse accumulator) whose size the library must choose
 * before the row is formed.  Three ways (the paper prescribes none):
 *  DSPG_SIZE_BOUND    the product bound ub_i (never too small; default);
 *  DSPG_SIZE_EXACT    a symbolic pass first counts nnz(C'_i) exactly, then
 *                     the numeric pass uses tables of that size;
 *  DSPG_SIZE_LEARNED  a small network (the estimator) predicts nnz(C'_i) from
 *                     len(A_i) and the sum, maximum and mean of the lengths
 *                     of the B rows it reads, for rows whose bound exceeds
 *                     est_min; the table is the prediction times (1 + margin),
 *                     clamped to [max_k len(B_k), ub_i].  A row whose table
 *                     overflows is counted exactly and recomputed afterwards.
 * The three give the same C (tables never decide the result); only the time
 * differs.  The estimator has no counterpart in the paper. */
enum { DSPG_SIZE_BOUND = 0, DSPG_SIZE_EXACT = 1, DSPG_SIZE_LEARNED = 2 };

/* The estimator's network: x -> 64 ReLU -> 64 ReLU -> 1 with
 * x = log2(1 + [len(A_i), sum_k len(B_k), max_k len(B_k), mean_k len(B_k)])
 * and output o = log2(1 + nnz(C_i)).  Parameters: one float32 vector of
 * DSPG_EST_PARAMS numbers, W1 (64 x 4, row-major), b1 (64), W2 (64 x 64,
 * row-major), b2 (64), W3 (64), b3 (1).  Every forward pass uses the weights
 * rounded to bfloat16 (nearest, ties to even) and accumulates in float32;
 * training keeps a float32 master copy. */
#define DSPG_EST_PARAMS 4545
typedef struct dspg_estimator dspg_estimator;

/* New estimator with the given initial parameters (host, float32). */
dspg_status dspg_estimator_create(dspg_estimator **out, const float *params);

/* Its float32 parameters into params (host, DSPG_EST_PARAMS). */
dspg_status dspg_estimator_params(dspg_estimator *e, float *params, void *stream);

/* Mean squared error L = mean_r (o_r - y_r)^2 over the n rows X (device,
 * n x 4 float32, row-major) with targets y (device, n), and dL/dw at the
 * bfloat16 weights into grad (host, DSPG_EST_PARAMS; may be NULL) and L into
 * *loss (may be NULL).  The parameters do not change. */
dspg_status dspg_estimator_grad(dspg_estimator *e, const float *X, const float *y, int64_t n, float *grad,
                                double *loss, void *stream);

/* `steps` SGD steps (w <- w - lr dL/dw) over consecutive mini-batches of
 * `batch` rows of X, y (device; wrapping around); *loss (may be NULL)
 * receives the loss over all n rows afterwards. */
dspg_status dspg_estimator_train(dspg_estimator *e, const float *X, const float *y, int64_t n, int64_t batch,
                                 int64_t steps, float lr, double *loss, void *stream);

/* Outputs o for n rows X (device) into out (device, n float32). */
dspg_status dspg_estimator_predict(dspg_estimator *e, const float *X, int64_t n, float *out, void *stream);

const char *dspg_estimator_last_error(const dspg_estimator *e);
void dspg_estimator_destroy(dspg_estimator *e);

/* Training data from a handle: the features of rows rows[n] of C (device;
 * rows == NULL: all rows, n = nrows(C)) into X (device, n x 4 float32) and,
 * when y != NULL, log2(1 + nnz(C_i)) into y (device, n).  C's rows are exact
 * after every build and batch, so these are exact symbolic counts. */
dspg_status dspg_row_features(dspg_handle *h, const int32_t *rows, int64_t n, float *X, float *y, void *stream);

/* Choose the sizing of h's dynamic recompute (the static product always uses
 * the bound).  For DSPG_SIZE_LEARNED, e's current bfloat16 weights are
 * copied into h (e may be destroyed afterwards), with est_min >= 0 and
 * margin >= 0. */
dspg_status dspg_set_sizing(dspg_handle *h, int mode, const dspg_estimator *e, int32_t est_min, float margin);

/* ---------------------------------------------------------------------------
 * Serving support: merging queued batches without changing any result.
 * (No counterpart in the paper, which applies one batch at a time.)
 *
 * A server that receives many small batches for the same handle can apply
 * several in one call, concatenated in arrival order, when no one of them
 * can change a row of C that another reports: the result of each is then
 * the same as if it had been applied alone, in order.  The footprint of a
 * batch dA is the set of rows of C it can touch, plus the rows its entries
 * could connect: its rows, and, when B is A, its columns and every row i
 * with A(i,k) != 0 for a row k of the batch (the rows of C* = A* B' + A B*,
 * Eq. 1, on the current pattern).  Two batches whose footprints are
 * disjoint can share a call.  (With B distinct from A the footprint is the
 * batch's rows; batches of B are not covered.) */

/* Write the footprint of dA into f (device, ceil(nrows/32) words, bit i of
 * word i/32 for row i; f is cleared first) and its number of rows into *rows
 * (may be NULL).  When u != NULL (device, same size, the rows a wave already
 * holds): if f and u share no bit, u |= f and *admitted = 1; otherwise
 * *admitted = 0, and u |= f only when or_anyway != 0 (a server marks a
 * request it passes over, so that no later request that conflicts with it
 * overtakes it).  Working memory is the handle's (kept between calls); one
 * synchronisation.  DSPG_ERR_INVALID for an entry out of range. */
dspg_status dspg_footprint(dspg_handle *h, const dspg_updates *dA, uint32_t *f, uint32_t *u, int or_anyway,
                           int *admitted, int64_t *rows, void *stream);

/* Footprints of k batches and their admission in one call (one
 * synchronisation), as k calls of dspg_footprint in a row would give:
 * f[j * words .. ) receives batch j's footprint (words = (rows of C + 31)
 * / 32, device), and the footprints are tested against u and added to it in
 * order.  admitted[j] = 1 when batch j met no footprint before it: with
 * or_anyway = 0 the first batch that meets one ends the run (it and every
 * later batch are not admitted, and u takes only the admitted footprints);
 * with or_anyway = 1 a batch that meets one is passed over but its
 * footprint still joins u (so a later batch overtakes only batches it
 * commutes with).  rows (may be NULL): rows set in each footprint.
 * Borrowed batches are read during the call.  DSPG_ERR_INVALID for an entry
 * out of range, DSPG_ERR_STATE while an asynchronous batch is in flight.
 * Not part of the paper; the serving loop's admission. */
dspg_status dspg_footprint_batch(dspg_handle *h, const dspg_updates *batches, int64_t k, uint32_t *f, uint32_t *u,
                                 int or_anyway, int *admitted, int64_t *rows, void *stream);

/* Free the group (not its handles). */
void dspg_group_destroy(dspg_group *g);
const char *dspg_group_last_error(const dspg_group *g);

/* Rows of C = A B for callers that cannot let a library allocate device
 * memory: their memory belongs to another allocator (a framework's caching
 * pool, an arena fixed at start-up), or their latency budget cannot absorb
 * cudaMalloc/cudaFree, which synchronise the device.  The paper has no
 * counterpart of this call; it is a service of this library.
 *
 * A and B: canonical CSR in device memory (on_device = 1), A->ncols ==
 * B->nrows, and B->ncols <= 65536 (larger B is rejected with
 * DSPG_ERR_INVALID: the working memory is a fixed array).  rows[nrows]:
 * device array of row indices of A (any order, repeats allowed).
 * Outputs (device, caller-owned): rowptr[nrows+1], then col and val with
 * room for `capacity` entries; row t of the result is row rows[t] of C with
 * columns ascending.  Two-call convention: with col == NULL only rowptr and
 * *nnz_out are written; a result larger than capacity returns
 * DSPG_ERR_INVALID with *nnz_out set to the size needed.
 *
 * Allocation: none.  The working memory is a fixed array of about 4.1 MiB
 * (4,260,096 bytes) of device memory in this library image, held by every
 * GPU that loads the library until the process exits.  The first call on
 * each device looks up that array's device address (with the device
 * current); make that first call before any stream capture begins.  The
 * stream must belong to the current device (another device's stream is
 * rejected with DSPG_ERR_INVALID).  All calls share the array: calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race and give wrong results.  Each call synchronises the stream before it
 * returns (twice when it writes the rows).
 *
 * Errors: a row index outside [0, A->nrows), or a column index of A or B
 * outside its matrix, makes the call return DSPG_ERR_INVALID ("row or
 * column index out of range") without writing col/val (the kernel skips
 * the bad index instead of reading through it). */
dspg_status dspg_multiply_rows_noalloc(const dspg_csr *A, const dspg_csr *B, dspg_semiring sr, const int32_t *rows,
                                       int64_t nrows, int64_t *rowptr, int32_t *col, void *val, int64_t capacity,
                                       int64_t *nnz_out, void *stream);

/* Free the handle and all its device memory (synchronises the device). */
void dspg_destroy(dspg_handle *h);

/* Message of the last error on h, or of the calling thread's last failed
 * dspg_build when h == NULL.  Valid until the next call on h / the thread. */
const char *dspg_last_error(const dspg_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* DSPG_H */
