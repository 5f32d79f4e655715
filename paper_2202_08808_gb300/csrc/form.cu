// form.cu -- the general product form of Section 3: C = alpha op(A) op(B) (+) beta X.
//
// Section 3 states SpGEMM as C = alpha A B + beta X with A and B optionally
// transposed; Section 5.3 extends the dynamic algorithms to transposed
// operands by reading A* and B* with their indices swapped.  On one GPU:
//
//  * a transposed operand is stored transposed (op(A) as a slack-CSR, built
//    by k_permute_entries after a stable radix sort of the entries by
//    column), and an update (i, j) of A is applied as (j, i) to it, so the
//    row path below is the plain one;
//  * the handle keeps P = op(A) op(B) up to date, and alpha, beta and X are
//    applied when rows of C are read: k_form_count sizes each output row as
//    |P_i u X_i| (P's rows carry no column order, so each entry is searched
//    in the sorted X row), and k_form_merge merges the sorted rows of P with
//    those of X, giving alpha (x) p (+) beta (x) x, alpha (x) p alone, or
//    beta (x) x alone.  X does not change, so the rows of C a batch can
//    change are still the rows of P it recomputes.
#include "internal.h"

namespace dspg {

namespace {

// out[t] = (row of entry idx[t], its value): the entries of a CSR sorted
// by column (idx from a stable sort) become the rows of its transpose.
__global__ void k_permute_entries(const uint32_t *idx, const uint32_t *row_of, const char *val, int64_t nnz,
                                  int32_t *out_col, char *out_val, int vsize) {
    pdl_begin();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = idx[t];
        out_col[t] = (int32_t)row_of[e];
        if (vsize == 8) ((double *)out_val)[t] = ((const double *)val)[e];
        else if (vsize == 4) ((int32_t *)out_val)[t] = ((const int32_t *)val)[e];
    }
}

// A warp per output row: |P_i u X_i| = len(P_i) + len(X_i) - |P_i n X_i|.
__global__ void k_form_count(const int32_t *rows, int64_t n, MatView P, const int64_t *xrp, const int32_t *xcol,
                             int64_t *cnt) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n; t += nw) {
        const int32_t i = rows ? rows[t] : (int32_t)t;
        const int64_t po = P.off[i];
        const int pl = P.len[i];
        const int64_t x0 = xrp[i], x1 = xrp[i + 1];
        int both = 0;
        for (int p = lane; p < pl; p += 32) {
            const int32_t j = P.col[po + p];
            const int64_t q = lower_bound_dev<int32_t>(xcol, x0, x1, j);
            both += q < x1 && xcol[q] == j;
        }
        both = warp_sum<int>(both);
        if (lane == 0) cnt[t] = (int64_t)pl + (x1 - x0) - both;
    }
}

template <int SR>
struct FormSr;
template <>
struct FormSr<SR_PT> {
    using T = double;
    __device__ static T scale(T s, T v) { return __dmul_rn(s, v); }
    __device__ static T add(T a, T b) { return __dadd_rn(a, b); }
};
template <>
struct FormSr<SR_MP> {
    using T = int32_t;
    __device__ static T scale(T s, T v) { return s + v; }
    __device__ static T add(T a, T b) { return a < b ? a : b; }
};

// A thread per output row: merge the sorted row t of P (prp/pcol/pval, as
// read) with the sorted row rows[t] of X into the output at orp[t].
template <int SR>
__global__ void k_form_merge(const int32_t *rows, int64_t n, const int64_t *prp, const int32_t *pcol, const void *pval,
                             const int64_t *xrp, const int32_t *xcol, const void *xval, const int64_t *orp,
                             int32_t *ocol, void *oval, FormScalars f) {
    pdl_begin();
    using T = typename FormSr<SR>::T;
    const T a = SR == SR_PT ? (T)f.alpha : (T)f.alpha_i;
    const T b = SR == SR_PT ? (T)f.beta : (T)f.beta_i;
    const T *pv = (const T *)pval;
    const T *xv = (const T *)xval;
    T *ov = (T *)oval;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = rows ? rows[t] : (int32_t)t;
        int64_t p = prp[t];
        const int64_t p1 = prp[t + 1];
        int64_t x = xrp[i];
        const int64_t x1 = xrp[i + 1];
        int64_t o = orp[t];
        while (p < p1 || x < x1) {
            const int32_t jp = p < p1 ? pcol[p] : 0x7fffffff;
            const int32_t jx = x < x1 ? xcol[x] : 0x7fffffff;
            if (jp == jx) {
                ocol[o] = jp;
                ov[o] = FormSr<SR>::add(FormSr<SR>::scale(a, pv[p]), FormSr<SR>::scale(b, xv[x]));
                p++;
                x++;
            } else if (jp < jx) {
                ocol[o] = jp;
                ov[o] = FormSr<SR>::scale(a, pv[p]);
                p++;
            } else {
                ocol[o] = jx;
                ov[o] = FormSr<SR>::scale(b, xv[x]);
                x++;
            }
            o++;
        }
    }
}

unsigned grid_of(int64_t items, int per_block, int num_sms) {
    int64_t g = (items + per_block - 1) / per_block;
    if (g > (int64_t)num_sms * 16) g = (int64_t)num_sms * 16;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

void permute_entries(const uint32_t *idx, const uint32_t *row_of, const void *val, int64_t nnz, int32_t *out_col,
                     void *out_val, int vsize, cudaStream_t s, int num_sms) {
    if (nnz <= 0) return;
    launch_k(k_permute_entries, grid_of(nnz, 256, num_sms), 256, 0, s, idx, row_of, (const char *)val, nnz, out_col,
             (char *)out_val, vsize);
}

void form_count(const int32_t *rows, int64_t n, const MatView &P, const int64_t *xrp, const int32_t *xcol,
                int64_t *cnt, cudaStream_t s, int num_sms) {
    if (n <= 0) return;
    launch_k(k_form_count, grid_of(n * 32, 256, num_sms), 256, 0, s, rows, n, P, xrp, xcol, cnt);
}

void form_merge(int sr, const int32_t *rows, int64_t n, const int64_t *prp, const int32_t *pcol, const void *pval,
                const int64_t *xrp, const int32_t *xcol, const void *xval, const int64_t *orp, int32_t *ocol,
                void *oval, const FormScalars &f, cudaStream_t s, int num_sms) {
    if (n <= 0) return;
    if (sr == SR_PT)
        launch_k(k_form_merge<SR_PT>, grid_of(n, 128, num_sms), 128, 0, s, rows, n, prp, pcol, pval, xrp, xcol, xval,
                 orp, ocol, oval, f);
    else
        launch_k(k_form_merge<SR_MP>, grid_of(n, 128, num_sms), 128, 0, s, rows, n, prp, pcol, pval, xrp, xcol, xval,
                 orp, ocol, oval, f);
}

}  // namespace dspg
