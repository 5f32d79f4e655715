// internal.h -- job descriptors passed by value to the kernels, and the host
// entry points of each translation unit.
#pragma once

#include <string>

#include "common.cuh"

namespace dspg {

// One sorted batch being applied to one slack-CSR (A, B, or A's transposed
// pattern).  Per sorted entry arrays have n entries; per merge item arrays
// have n entries too (at most one item per entry).
struct UpdJob {
    int which;  // index into Ctl::u
    int64_t n;  // launch size: at least the sorted entries (batch_bucket)
    const int64_t *n_dev;  // the sorted entries (the argument block's n, on the device)
    // sorted batch (output of sort_updates)
    int32_t *row, *col;
    void *val;  // nullptr for a pattern
    uint8_t *op;
    // classification
    uint8_t *kind;
    int32_t *pos, *insx, *delx;
    // merge items: rows with an effective change; their updates are the
    // sorted entries [m_lo, m_hi)
    int32_t *m_row, *m_lo, *m_hi, *m_len, *m_nins, *m_ndel;
    int64_t *m_soff;
    // commit plan per item
    int64_t *m_dest;
    int32_t *m_cap;
    // copy work items (item, part)
    int32_t *ch_item, *ch_part;
    int64_t ch_cap;
    int32_t *cc_item, *cc_part;
    int64_t cc_cap;
    // staging for rebuilt rows
    int32_t *st_col;
    void *st_val;
    int64_t st_cap;
};

// Staged rows -> slack-CSR.
struct CommitJob {
    const int32_t *rows;      // matrix row of each item
    const int32_t *lens;      // new length of each item
    const int64_t *soff;      // staging offset of each item
    const long long *count;   // number of items (device)
    const int32_t *st_col;
    const void *st_val;
    int64_t *dest;
    int32_t *ncap;
    int32_t *cc_item, *cc_part;
    long long *cc_count;
    int64_t cc_cap;
    long long *reloc;
    unsigned arena_bit, stage_bit;
};

struct DetectBufs {
    uint32_t *bmR;   // bitmap over rows of A (rows of C)
    uint32_t *bmK;   // bitmap over rows of B
    int32_t *R;      // affected rows (unordered)
    int32_t *K;      // rows of B*
    long long *nK;
};

// The recompute of rows of C (static build: all rows).
struct CJob {
    const int32_t *R;         // rows to recompute
    int32_t *bins;            // NBINS lists of rows of C, bin_cap each
    int64_t bin_cap;
    void *gd_acc;             // per-CTA dense accumulators (global), gd_w entries each
    uint32_t *gd_mask;        // per-CTA presence bits, gd_w / 32 words each
    uint32_t *gd_sum;         // per-CTA summary: bit w set when mask word w is touched, gd_w / 1024 words each
    int64_t gd_w;
    int gd_ctas;
    int64_t m;                // columns of C
    int dense_mode;           // 1: all rows use the dense small-m kernels
    int static_mode;          // 1: C is laid out afresh by the sizing pass
    int slack_min, slack_div;
    int count_only;           // 1: only count each row's entries into C.len (exact sizing pass)
    int64_t rows_hint;        // upper bound on the rows to recompute (caps the grids)
    // row-bin thresholds (dspg_tuning): thread-merge limits, smallest hash
    // executor, table oversizing, warp/CTA and CTA/global crossovers
    int tm_k, tm_ub, lanes_min, table_shift, warp_max, cta_max;
    int sort_max;             // rows of at most this many products: group sort
    // bins (bit b) whose kernels the recompute launches; a row whose bin is
    // off goes to the global dense bin (any row fits it), and the bin is
    // recorded in Ctl::bins_wanted.  All bits set in dense mode.
    unsigned long long bin_on;
    // sizing of the hash tables: SIZE_BOUND by the product bound; SIZE_COUNT
    // by C.len (an exact count written by a count_only pass); SIZE_LEARNED by
    // the estimator for rows with bound above est_min (tables may then
    // overflow: the row goes to the overflow list instead of C)
    int sizing;
    int est_min;
    float est_margin;
    const uint16_t *est_w;    // estimator weights, bfloat16 bits (EST_PARAMS)
    int4 *est;                // rows waiting for an estimate: {i, len(A_i), max len(B_k), bound}
    int32_t *ovf;             // rows (of C) whose learned table overflowed
    // split rows (dense mode): rows with many A entries or products are cut
    // into chunks recomputed by different CTAs and combined in global
    // accumulators (sp_rows rows at a time)
    int64_t sp_rows;
    void *sp_acc;             // sp_rows x mp accumulators
    uint32_t *sp_mask;        // sp_rows x mp/32 presence bits
    int *sp_done;             // sp_rows counters of folded chunks
    int64_t *sp_pre;          // sp_rows + 1: prefix of the split rows' chunk counts
};
enum { SIZE_BOUND = 0, SIZE_COUNT = 1, SIZE_LEARNED = 2 };

// The masked path (masked.cu): the contributions to the pattern of C*.
struct PatJob {
    const int32_t *xr, *xc;  // the sorted A batch and its kinds
    const uint8_t *xk;
    int64_t xn;
    const int32_t *yr, *yc;  // the sorted B batch (the A batch when B is A)
    const uint8_t *yk;
    int64_t yn;
    uint64_t *key;           // (i << cb | j) of each contribution
    uint64_t *bits;          // its bit (k mod 64)
    int64_t cap;
    int cb;
};

// C* as sorted entries (row, column, F*) in runs of one row each, and the
// masked product's working arrays, one entry per entry of C*.
struct MaskJob {
    int32_t *urow, *ucol;
    unsigned long long *ufs;  // F*
    const int64_t *nu_dev;    // |C*| (device)
    int64_t *run_start;       // runs + 1
    int32_t *run_row;
    const int64_t *nruns_dev; // runs (device)
    int64_t max_runs;         // a bound on the runs (grid sizes)
    int32_t *upos;            // place of the entry in its row of C, -1 if C has none
    unsigned long long *ue;   // F there (0 if none)
    unsigned long long *rbits;  // R_i per run
    int32_t *kept_run;        // A^R: run and A' entry of each kept entry
    int64_t *kept_a;
    int64_t kcap;
    const long long *nkept_dev;  // entries kept (device; beyond kcap the list overflowed)
    void *z;                  // Z: the masked product's values
    unsigned long long *h;    // H: its Bloom words
    uint8_t *hit;             // 1 where some product reached the entry
    int64_t *dest;            // per run: the row's new place (-1: in place)
    int32_t *dcap;
};

void bloom_rows(const MatView &A, const MatView &B, const MatView &C, unsigned long long *F, int32_t *rows_long,
                long long *n_long, long long cap_long, cudaStream_t s, int num_sms);
void bloom_long_rows(const MatView &A, const MatView &B, const MatView &C, unsigned long long *F,
                     const int32_t *rows_long, const long long *n_long, long long cap_long, int32_t *posmap,
                     int ctas, cudaStream_t s);
void pat_contrib(const PatJob &J, const MatView &B, const MatView &AT, Ctl *ctl, unsigned mask, cudaStream_t s,
                 int num_sms);
void iota_u32(uint32_t *v, int64_t n, cudaStream_t s, int num_sms);
void pat_heads(const uint64_t *K, int64_t n, int32_t *flag, cudaStream_t s, int num_sms);
void pat_unique(const uint64_t *K, const uint32_t *I, const uint64_t *bits, int64_t n, const int64_t *ex, int cb,
                const MaskJob &M, int32_t *rflag, cudaStream_t s, int num_sms);
void pat_runs(const MaskJob &M, const int32_t *rflag, const int64_t *rex, int64_t max_u, uint32_t *bm, cudaStream_t s,
              int num_sms);
void mask_scan(const MaskJob &M, const MatView &C, const unsigned long long *F, cudaStream_t s, int num_sms);
void mask_keep(const MaskJob &M, const MatView &A, Ctl *ctl, cudaStream_t s, int num_sms);
void mask_init_acc(int sr, const MaskJob &M, int64_t nu, cudaStream_t s, int num_sms);
void mask_product(int sr, const MaskJob &M, const MatView &A, const MatView &B, Ctl *ctl, unsigned mask,
                  cudaStream_t s, int num_sms);
void mask_plan(const MaskJob &M, const MatView &C, Ctl *ctl, unsigned mask, int slack_min, int slack_div,
               cudaStream_t s, int num_sms);
void mask_splice(int sr, const MaskJob &M, const MatView &C, unsigned long long *F, Ctl *ctl, unsigned mask,
                 cudaStream_t s, int num_sms);

// update.cu
void run_classify(const UpdJob &J, const MatView &M, int vsize, Ctl *ctl, unsigned mask, unsigned stage_bit,
                  const DetectBufs &D, bool mark_rows, bool mark_cols, cudaStream_t s, int num_sms);
void run_merge_copy(const UpdJob &J, const MatView &M, int vsize, Ctl *ctl, unsigned mask, cudaStream_t s,
                    int num_sms);
void run_commit(const CommitJob &J, const MatView &M, int vsize, int64_t max_items, Ctl *ctl, unsigned plan_mask,
                unsigned copy_mask, int slack_min, int slack_div, cudaStream_t s, int num_sms);
void run_detect_cols(const MatView &AT, const DetectBufs &D, Ctl *ctl, unsigned mask, cudaStream_t s, int num_sms);
void run_collect_rows(uint32_t *bm, int64_t words, int32_t *R, long long *chunk, Ctl *ctl, unsigned mask,
                      cudaStream_t s, int num_sms);
void run_detect_merge_plan(const MatView &AT, const DetectBufs &D, const UpdJob &J, const MatView &M,
                           const CommitJob &CJ, int vsize, Ctl *ctl, unsigned mask, int slack_min, int slack_div,
                           int64_t max_items, cudaStream_t s, int num_sms);
void run_collect_copy(uint32_t *bm, int64_t words, int32_t *R, long long *chunk, const CommitJob &CJ, const MatView &M,
                      int vsize, Ctl *ctl, unsigned collect_mask, unsigned copy_mask, cudaStream_t s, int num_sms);
void run_detect_merge(const MatView &AT, const DetectBufs &D, const UpdJob &J, const MatView &M, int vsize, Ctl *ctl,
                      unsigned mask, cudaStream_t s, int num_sms);
void run_transpose_feed(const UpdJob &J, int32_t pad_row, int32_t *trow, int32_t *tcol, uint8_t *top, Ctl *ctl,
                        unsigned mask, cudaStream_t s);
void run_footprint(const int32_t *row, const int32_t *col, int64_t n, int64_t nrows, int64_t ncols, bool b_is_a,
                   const MatView &AT, uint32_t *bm, unsigned *bad, cudaStream_t s, int num_sms);
void run_bitmap_overlap(const uint32_t *f, const uint32_t *u, int64_t words, unsigned long long *cnt, cudaStream_t s,
                        int num_sms);
void run_bitmap_or(const uint32_t *f, uint32_t *u, int64_t words, const unsigned long long *cnt, int or_anyway,
                   cudaStream_t s, int num_sms, unsigned *stopped = nullptr);

// algebraic.cu: the delta path of Eq. 1 (batches that only insert)
constexpr int ALG_SCAN = 256;  // rows of C up to this length take contributions in place
struct AlgJob {
    // X = A* B': the sorted A batch (entries of kind K_INS are A*)
    const int32_t *xr, *xc;
    const void *xv;
    const uint8_t *xk;
    int64_t xn;
    // Y = A B*: the sorted B batch (the A batch when B is A)
    const int32_t *yr, *yc;
    const void *yv;
    const uint8_t *yk;
    int64_t yn;
    // new entries of C (columns not yet in their row): room for ncap
    int32_t *nr, *nc;
    void *nv;
    uint8_t *nop;
    int64_t ncap;
    uint32_t *bm_touch;  // rows of C that take a contribution
    uint32_t *bm_long;   // rows longer than ALG_SCAN: recomputed by the row path
};
// The sorted new entries of C (equal keys adjacent) and their rows' plan.
struct AlgNew {
    const int32_t *row, *col;
    const void *val;
    int64_t n;
    int64_t *dest;  // per row-run head: where the row goes
    int32_t *cap;   // per row-run head: its capacity there
};
void run_alg_contrib(int sr, const AlgJob &J, const MatView &A, const MatView &B, const MatView &AT, const MatView &C,
                     Ctl *ctl, unsigned mask, cudaStream_t s, int num_sms);
void run_alg_append(int sr, const AlgNew &N, const MatView &C, Ctl *ctl, unsigned plan_mask, unsigned copy_mask,
                    int slack_min, int slack_div, bool plan, cudaStream_t s, int num_sms);

// form.cu: C = alpha op(A) op(B) (+) beta X (Section 3), transposed operands
struct FormScalars {
    double alpha, beta;       // (+,.)
    int32_t alpha_i, beta_i;  // (min,+): added to the products / to X
};
void permute_entries(const uint32_t *idx, const uint32_t *row_of, const void *val, int64_t nnz, int32_t *out_col,
                     void *out_val, int vsize, cudaStream_t s, int num_sms);
void form_count(const int32_t *rows, int64_t n, const MatView &P, const int64_t *xrp, const int32_t *xcol,
                int64_t *cnt, cudaStream_t s, int num_sms);
void form_merge(int sr, const int32_t *rows, int64_t n, const int64_t *prp, const int32_t *pcol, const void *pval,
                const int64_t *xrp, const int32_t *xcol, const void *xval, const int64_t *orp, int32_t *ocol,
                void *oval, const FormScalars &f, cudaStream_t s, int num_sms);

// spgemm.cu
constexpr int64_t DENSE_M_MAX = 1024;  // C columns up to this use dense accumulators
void run_size_bins(const MatView &A, const MatView &B, const MatView &C, const CJob &J, int64_t max_rows, Ctl *ctl,
                   unsigned mask, cudaStream_t s, int num_sms);
void run_numeric(int sr, const MatView &A, const MatView &B, const MatView &C, const CJob &J, Ctl *ctl, unsigned mask,
                 const cudaStream_t *ss, int ns, int num_sms);
// The bins a handle launches after a batch whose control block is c, given
// the bins it launched (on) and whether it has narrowed them before: the
// first time, the bins that got rows; then those plus every bin a row was
// redirected from.  The global dense bin is always on.
unsigned long long next_bin_mask(const Ctl &c, unsigned long long on, bool narrowed);
void init_dense_scratch(int sr, void *acc, uint32_t *mask, int64_t entries, int64_t words, cudaStream_t s);
// Accumulator slots a row of bin `bin` gets (hash table or dense row of m
// columns; 0 for the thread-merge bins, which keep no table).
int64_t bin_table_slots(int bin, int64_t m);

// Message for dspg_last_error(NULL) on the calling thread (handle.cu).
void set_thread_error(const char *msg);

// estimator.cu: features of rows of C for the estimator
void row_features(const MatView &A, const MatView &B, const MatView &C, const int32_t *rows, int64_t n, float *X,
                  float *y, unsigned *bad, cudaStream_t s);

// layout.cu: building and reading slack-CSRs
void fill_iota(int32_t *a, int64_t n, cudaStream_t s);
void begin_batch(const InArgs *host_args, InArgs *dev_args, Ctl *ctl, cudaStream_t s);
void end_batch(const Ctl *ctl, Ctl *host_ctl, cudaStream_t s);
void caps_from_lens(const int32_t *len, int32_t *cap, int64_t n, int slack_min, int slack_div, cudaStream_t s);
void lens_from_rowptr(const int64_t *rowptr, int32_t *len, int64_t n, cudaStream_t s);
// Copy rows: dst row i gets src[src_off[i] .. +len[i]) at dst_off[i] (per index i < n, with an
// optional row map rows[i]).
void copy_rows(const int32_t *rows, int64_t n, const int64_t *src_off, const int32_t *len, const int32_t *src_col,
               const void *src_val, const int64_t *dst_off, int32_t *dst_col, void *dst_val, int vsize,
               cudaStream_t s, int num_sms);
void gather_rows_out(const int32_t *rows, int64_t n, const MatView &M, const int64_t *out_rowptr, int32_t *out_col,
                     void *out_val, int vsize, cudaStream_t s, int num_sms);
// Sort each row of a gathered CSR (rowptr over n rows) by column, in place;
// rows longer than 16384 entries that are out of order are counted in
// *n_listed and their indices written to listed[0, list_cap) instead, for
// sort_listed_rows.
void sort_rows(const int64_t *rowptr, int64_t n, int32_t *col, void *val, int vsize, unsigned *n_listed,
               int64_t *listed, int64_t list_cap, cudaStream_t s, int num_sms);
struct SortScratch {  // for `total` entries: keys, indices (two each), radix counts, scans, gather space
    uint64_t *k0, *k1;
    uint32_t *i0, *i1, *counts;
    int64_t *scan_tmp, *scan_out;
    int32_t *tcol;
    void *tval;
};
// Sorts the listed rows (nl of them, `total` entries, pre[k] = entries before
// listed row k, pre[nl] = total; all on the device) by column, in place.
void sort_listed_rows(const int64_t *rowptr, const int64_t *listed, const int64_t *pre, int nl, int64_t total,
                      int cb, int32_t *col, void *val, int vsize, const SortScratch &w, cudaStream_t s, int num_sms);
void lens_of_rows(const int32_t *rows, int64_t n, const int32_t *len, int32_t *out, cudaStream_t s);
// A read of rows of C straight into page-locked host buffers (layout.cu):
// what it found, for the one host synchronisation after it.
struct ReadOut {
    long long nnz;   // entries of the rows (rp[n])
    unsigned n_long; // rows of more than 64 entries (listed)
    unsigned n_huge; // of those, rows over 16384 entries that are out of order (left in the scratch)
    unsigned flags;  // READ_TOO_SMALL, READ_UNORDERED: nothing was written
    unsigned pad;
    long long nr;    // the rows of R (n, as read on the device)
};
enum : unsigned { READ_TOO_SMALL = 1u, READ_UNORDERED = 2u };
// rows[0..n) (ascending, R from its collection when r_total is given: its
// chunk total must equal n), their row pointers rp (device, rp[n] = entries)
// -> out_col/out_val (device addresses of page-locked host memory, at least
// nnz_cap entries; out_val may be null).  Scratch: nnz_cap entries; lists:
// n entries each; res zeroed by the caller.
// n_dev (or null): n read on the device, n then bounding it (grid sizes).
void read_rows_direct(const int32_t *rows, int64_t n, const long long *n_dev, const MatView &M, int vsize,
                      const int64_t *rp, const int64_t *r_total, int64_t nnz_cap, int32_t *out_col, void *out_val,
                      int32_t *scr_col, void *scr_val, int64_t *long_list, int64_t *huge_list, ReadOut *res,
                      cudaStream_t s, int num_sms);
// R (n rows, as collected: ascending within each 8192-row chunk, chunk c's
// rows at chunk[2c] with chunk[2c+1] of them) into out in row order; cnt and
// ex (nch + 1) and tmp (scan_tmp_entries(nch) + 1) are scratch, and ex[nch]
// is the number of rows placed (n when R came from one collection).
void rows_in_order(const int32_t *R, const long long *chunk, int64_t nch, int64_t n, int64_t *cnt, int64_t *ex,
                   int64_t *tmp, int32_t *out, cudaStream_t s);
// The same in two launches, with R's row pointers: out (n) gets R in row
// order, lens (n) its rows' lengths in C (len), S (nch) the lengths summed per
// chunk, rp (n + 1) the row pointers, *r_total the rows placed; h_rows and
// h_rp (device addresses of page-locked host arrays of at least n and n + 1
// entries, or null) get copies of out and rp, and res (or null) is zeroed
// with its nr set.  For nch <= read_nch_max(); nothing but *r_total is
// written when it is not n.  With n_dev, n is read on the device (behind a
// batch still on the stream): rows_cap bounds it (the arrays are sized for
// rows_cap), and a nonzero *status (a failed batch) or a larger n makes
// *r_total -1, so that nothing is read.
int64_t read_nch_max();
void read_order_rowptr(const int32_t *R, const long long *chunk, int64_t nch, int64_t n, const long long *n_dev,
                       int64_t rows_cap, const unsigned *status, const int32_t *len, int32_t *out, int32_t *lens,
                       int64_t *S, int64_t *r_total, int64_t *rp, int32_t *h_rows, int64_t *h_rp, ReadOut *res,
                       cudaStream_t s, int num_sms);
void validate_rowptr(int64_t nrows, int64_t nnz, const int64_t *rowptr, unsigned *bad, cudaStream_t s);
void validate_csr_entries(int64_t nrows, int64_t ncols, const int64_t *rowptr, const int32_t *col, const void *val,
                          int sr, unsigned *bad, cudaStream_t s);
void hist_cols(const int32_t *col, int64_t nnz, int32_t *counts, cudaStream_t s);
void rows_of_entries(const int64_t *rowptr, int64_t nrows, uint32_t *rows_out, cudaStream_t s, int num_sms);
void keys_from_cols(const int32_t *col, int64_t nnz, uint64_t *keys, cudaStream_t s);
void sort_i32_values(int32_t *a, int64_t n, int bits, uint64_t *k0, uint64_t *k1, uint32_t *i0, uint32_t *i1,
                     uint32_t *counts, int64_t *scan_tmp, int64_t *scan_out, cudaStream_t s);

}  // namespace dspg

// The learned row-size estimator (estimator.cu): float32 master weights, their
// bfloat16 copy used by every forward pass, and training buffers.
struct dspg_estimator {
    float *master = nullptr;   // float32 parameters (device)
    float *grad = nullptr;     // last gradient (device)
    uint16_t *w = nullptr;     // bfloat16 bits of master (device)
    float *H1 = nullptr, *H2 = nullptr, *D = nullptr, *DZ1 = nullptr, *DZ2 = nullptr, *O = nullptr;
    int64_t cap = 0;           // rows the activation buffers hold
    double *loss_d = nullptr;  // device accumulator
    std::string err;
};
