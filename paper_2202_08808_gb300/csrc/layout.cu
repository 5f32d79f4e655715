// layout.cu -- building slack-CSRs from row-wise sources and reading them back.
//
// These kernels move whole rows between a CSR-like source (row start + row
// length) and a destination layout, one warp per row, and sort read rows by
// column; they carry no semiring arithmetic.
#include <algorithm>

#include "internal.h"

namespace dspg {

static unsigned blocks_for(int64_t n, int nt, int64_t cap = 1 << 20) {
    int64_t g = (n + nt - 1) / nt;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

__global__ void k_iota(int32_t *a, int64_t n) {
    pdl_begin();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        a[x] = (int32_t)x;
}
// First and last steps of a batch.  The host keeps the batch pointers and
// receives the control block in pinned, mapped memory; these two small
// kernels move them (the pointers read uncached, as the host rewrites them
// between batches), which costs less on the stream than a memset and two
// copy-engine transfers.
static_assert(sizeof(Ctl) % sizeof(unsigned long long) == 0, "control block in 8-byte words");
constexpr int CTL_WORDS = (int)(sizeof(Ctl) / sizeof(unsigned long long));
constexpr int ARG_WORDS = (int)(3 * sizeof(InArgs) / sizeof(unsigned long long));

__global__ void k_begin_batch(const InArgs *host_args, InArgs *dev_args, Ctl *ctl) {
    pdl_begin();
    unsigned long long *c = (unsigned long long *)ctl;
    for (int k = threadIdx.x; k < CTL_WORDS; k += blockDim.x) c[k] = 0ull;
    if (threadIdx.x < ARG_WORDS)
        ((unsigned long long *)dev_args)[threadIdx.x] = __ldcv((const unsigned long long *)host_args + threadIdx.x);
}

__global__ void k_end_batch(const Ctl *ctl, Ctl *host_ctl) {
    pdl_begin();
    const unsigned long long *c = (const unsigned long long *)ctl;
    for (int k = threadIdx.x; k < CTL_WORDS; k += blockDim.x) ((unsigned long long *)host_ctl)[k] = c[k];
    __threadfence_system();
}

void begin_batch(const InArgs *host_args, InArgs *dev_args, Ctl *ctl, cudaStream_t s) {
    launch_k(k_begin_batch, 1, 128, 0, s, host_args, dev_args, ctl);
}

void end_batch(const Ctl *ctl, Ctl *host_ctl, cudaStream_t s) { launch_k(k_end_batch, 1, 128, 0, s, ctl, host_ctl); }

void fill_iota(int32_t *a, int64_t n, cudaStream_t s) {
    if (n > 0) launch_k(k_iota, blocks_for(n, 256, 8192), 256, 0, s, a, n);
}

__global__ void k_caps(const int32_t *len, int32_t *cap, int64_t n, int smin, int sdiv) {
    pdl_begin();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        cap[x] = slack_cap(len[x], smin, sdiv);
}
void caps_from_lens(const int32_t *len, int32_t *cap, int64_t n, int smin, int sdiv, cudaStream_t s) {
    if (n > 0) launch_k(k_caps, blocks_for(n, 256, 8192), 256, 0, s, len, cap, n, smin, sdiv);
}

__global__ void k_lens_rowptr(const int64_t *rowptr, int32_t *len, int64_t n) {
    pdl_begin();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        len[x] = (int32_t)(rowptr[x + 1] - rowptr[x]);
}
void lens_from_rowptr(const int64_t *rowptr, int32_t *len, int64_t n, cudaStream_t s) {
    if (n > 0) launch_k(k_lens_rowptr, blocks_for(n, 256, 8192), 256, 0, s, rowptr, len, n);
}

__global__ void k_lens_of_rows(const int32_t *rows, int64_t n, const int32_t *len, int32_t *out) {
    pdl_begin();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        out[x] = len[rows[x]];
}
void lens_of_rows(const int32_t *rows, int64_t n, const int32_t *len, int32_t *out, cudaStream_t s) {
    if (n > 0) launch_k(k_lens_of_rows, blocks_for(n, 256, 8192), 256, 0, s, rows, n, len, out);
}

// R in row order from its collection: each chunk of 8192 rows wrote its
// (ascending) rows at chunk[2c] in R, chunk[2c+1] of them, so laying the
// chunks end to end in chunk order sorts R.  k_chunk_counts lists the
// counts for a scan, k_chunk_copy moves each chunk (a block per chunk).
__global__ void k_chunk_counts(const long long *chunk, int64_t nch, int64_t *cnt) {
    pdl_begin();
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nch; c += (int64_t)gridDim.x * blockDim.x)
        cnt[c] = chunk[2 * c + 1];
}

__global__ void k_chunk_copy(const int32_t *R, const long long *chunk, int64_t nch, const int64_t *ex, int64_t n,
                             int32_t *out) {
    pdl_begin();
    for (int64_t c = blockIdx.x; c < nch; c += gridDim.x) {
        const long long b = chunk[2 * c], k = chunk[2 * c + 1];
        const int64_t o = ex[c];
        if (k <= 0 || b < 0 || b + k > n || o + k > n) continue;  // not one collection: the caller checks ex[nch]
        for (long long t = threadIdx.x; t < k; t += blockDim.x) out[o + t] = R[b + t];
    }
}

void rows_in_order(const int32_t *R, const long long *chunk, int64_t nch, int64_t n, int64_t *cnt, int64_t *ex,
                   int64_t *tmp, int32_t *out, cudaStream_t s) {
    if (nch <= 0) return;
    launch_k(k_chunk_counts, blocks_for(nch, 256, 1024), 256, 0, s, chunk, nch, cnt);
    scan_i64(cnt, ex, nch, tmp, s);
    launch_k(k_chunk_copy, (unsigned)std::min<int64_t>(nch, 8192), 256, 0, s, R, chunk, nch, ex, n, out);
}

// R in row order and its row pointers for a read, in two launches while
// the chunk table is small enough for one block to scan (READ_NCH_MAX
// chunks): every block scans the chunk counts itself, so no scan launches
// come between.  k_read_order lays each chunk's rows at the scan of the
// counts, looks up their lengths in C and sums them per chunk;
// k_read_rowptr scans the sums and each chunk's lengths into the rows' first
// entries.  Both also write the caller's page-locked arrays when given
// (h_rows, h_rp: device addresses), and both leave everything untouched when
// the counts do not add up to n (R was not collected in one pass; the caller
// sees *r_total != n).
constexpr int RD_NT = 1024;
constexpr int RD_IPT = 2;

int64_t read_nch_max() { return (int64_t)RD_NT * RD_IPT; }

// Exclusive scan of the m <= RD_NT * RD_IPT values load(0..m) into s_ex;
// returns their total.  Every thread of the block calls it.
template <class F>
__device__ __forceinline__ int64_t rd_scan_table(F load, int m, int64_t *s_ex, int64_t *s_w) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int64_t v[RD_IPT];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < RD_IPT; j++) {
        const int c = tid * RD_IPT + j;
        v[j] = c < m ? load(c) : 0;
        sum += v[j];
    }
    const int64_t incl = warp_incl_scan<int64_t>(sum);
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int64_t t = s_w[lane];
        const int64_t ti = warp_incl_scan<int64_t>(t);
        s_w[lane] = ti - t;
        if (lane == 31) s_w[32] = ti;
    }
    __syncthreads();
    int64_t e = s_w[w] + incl - sum;
#pragma unroll
    for (int j = 0; j < RD_IPT; j++) {
        const int c = tid * RD_IPT + j;
        if (c < m) s_ex[c] = e;
        e += v[j];
    }
    const int64_t total = s_w[32];
    __syncthreads();
    return total;
}

// Exclusive scan of one value per thread; *total gets the block's sum.
__device__ __forceinline__ int64_t rd_block_scan(int64_t v, int64_t *s_w, int64_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t incl = warp_incl_scan<int64_t>(v);
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int64_t t = s_w[lane];
        const int64_t ti = warp_incl_scan<int64_t>(t);
        s_w[lane] = ti - t;
        if (lane == 31) s_w[32] = ti;
    }
    __syncthreads();
    const int64_t r = s_w[w] + incl - v;
    *total = s_w[32];
    __syncthreads();
    return r;
}

// chunk c of R holds k = chunk[2c+1] rows at chunk[2c]; they go to o = ex[c]
__device__ __forceinline__ bool rd_chunk_ok(long long b, long long k, int64_t o, int64_t n) {
    return k > 0 && b >= 0 && b + k <= n && o + k <= n;
}

__global__ void __launch_bounds__(RD_NT)
k_read_order(const int32_t *R, const long long *chunk, int nch, int64_t n_arg, const long long *n_dev, int64_t rows_cap,
             const unsigned *status, const int32_t *len, int32_t *out, int32_t *lens, int64_t *S, int64_t *r_total,
             int32_t *h_rows, ReadOut *res) {
    pdl_begin();
    __shared__ int64_t s_ex[RD_NT * RD_IPT];
    __shared__ int64_t s_w[33];
    const int64_t n = n_dev ? (int64_t)*n_dev : n_arg;
    // enqueued behind an apply (n on the device): nothing is read after a
    // failed batch or when R would not fit the buffers sized for it
    const bool skip = (status && *status) || n < 0 || n > rows_cap;
    const int64_t tot = rd_scan_table([&](int c) { return (int64_t)chunk[2 * c + 1]; }, nch, s_ex, s_w);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *r_total = skip ? -1 : tot;
        if (res) {
            ReadOut z{};
            z.nr = n;
            *res = z;
        }
    }
    if (skip || tot != n) return;
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const long long b = chunk[2 * c], k = chunk[2 * c + 1];
        const int64_t o = s_ex[c];
        int64_t sum = 0;
        if (rd_chunk_ok(b, k, o, n))
            for (long long t = threadIdx.x; t < k; t += RD_NT) {
                const int32_t r = R[b + t];
                out[o + t] = r;
                if (h_rows) h_rows[o + t] = r;
                const int32_t L = len[r];
                lens[o + t] = L;
                sum += L;
            }
        sum = warp_sum<int64_t>(sum);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x < 32) {
            int64_t t = s_w[threadIdx.x];
            t = warp_sum<int64_t>(t);
            if (threadIdx.x == 0) S[c] = t;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(RD_NT)
k_read_rowptr(const long long *chunk, int nch, int64_t n_arg, const long long *n_dev, const int32_t *lens,
              const int64_t *S, const int64_t *r_total, int64_t *rp, int64_t *h_rp) {
    pdl_begin();
    __shared__ int64_t s_ex[RD_NT * RD_IPT];
    __shared__ int64_t s_base[RD_NT * RD_IPT];
    __shared__ int64_t s_w[33];
    const int64_t n = n_dev ? (int64_t)*n_dev : n_arg;
    if (*r_total != n) return;
    rd_scan_table([&](int c) { return (int64_t)chunk[2 * c + 1]; }, nch, s_ex, s_w);
    const int64_t nnz = rd_scan_table([&](int c) { return S[c]; }, nch, s_base, s_w);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        rp[n] = nnz;
        if (h_rp) h_rp[n] = nnz;
    }
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const long long b = chunk[2 * c], k = chunk[2 * c + 1];
        const int64_t o = s_ex[c];
        if (!rd_chunk_ok(b, k, o, n)) continue;  // the same for the whole block
        int64_t carry = s_base[c];
        for (long long t0 = 0; t0 < k; t0 += RD_NT) {
            const long long t = t0 + threadIdx.x;
            const int64_t L = t < k ? lens[o + t] : 0;
            int64_t round = 0;
            const int64_t e = rd_block_scan(L, s_w, &round);
            if (t < k) {
                rp[o + t] = carry + e;
                if (h_rp) h_rp[o + t] = carry + e;
            }
            carry += round;
        }
    }
}

void read_order_rowptr(const int32_t *R, const long long *chunk, int64_t nch, int64_t n, const long long *n_dev,
                       int64_t rows_cap, const unsigned *status, const int32_t *len, int32_t *out, int32_t *lens,
                       int64_t *S, int64_t *r_total, int64_t *rp, int32_t *h_rows, int64_t *h_rp, ReadOut *res,
                       cudaStream_t s, int num_sms) {
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nch, (int64_t)num_sms * 2));
    launch_k(k_read_order, g, RD_NT, 0, s, R, chunk, (int)nch, n, n_dev, rows_cap, status, len, out, lens, S, r_total,
             h_rows, res);
    launch_k(k_read_rowptr, g, RD_NT, 0, s, chunk, (int)nch, n, n_dev, (const int32_t *)lens, (const int64_t *)S,
             (const int64_t *)r_total, rp, h_rp);
}

template <typename T>
__global__ void k_copy_rows(const int32_t *rows, int64_t n, const int64_t *src_off, const int32_t *len,
                            const int32_t *src_col, const T *src_val, const int64_t *dst_off, int32_t *dst_col,
                            T *dst_val) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
        const int64_t r = rows ? rows[x] : x;
        const int64_t so = src_off[r], d = dst_off[r];
        const int L = len[r];
        for (int e = lane; e < L; e += 32) {
            dst_col[d + e] = src_col[so + e];
            if (dst_val) dst_val[d + e] = src_val[so + e];
        }
    }
}

void copy_rows(const int32_t *rows, int64_t n, const int64_t *src_off, const int32_t *len, const int32_t *src_col,
               const void *src_val, const int64_t *dst_off, int32_t *dst_col, void *dst_val, int vsize,
               cudaStream_t s, int num_sms) {
    if (n <= 0) return;
    unsigned g = blocks_for(n * 32, 256, (int64_t)num_sms * 16);
    if (vsize == 8)
        launch_k(k_copy_rows<double>, g, 256, 0, s, rows, n, src_off, len, src_col, (const double *)src_val, dst_off,
                                              dst_col, (double *)dst_val);
    else
        launch_k(k_copy_rows<int32_t>, g, 256, 0, s, rows, n, src_off, len, src_col, (const int32_t *)src_val, dst_off,
                                               dst_col, (int32_t *)dst_val);
}

template <typename T>
__global__ void k_gather_out(const int32_t *rows, int64_t n, MatView M, const int64_t *out_rowptr, int32_t *out_col,
                             T *out_val) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const T *mv = (const T *)M.val;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
        const int64_t r = rows ? rows[x] : x;
        const int64_t so = M.off[r], d = out_rowptr[x];
        const int L = M.len[r];
        for (int e = lane; e < L; e += 32) {
            out_col[d + e] = M.col[so + e];
            if (out_val) out_val[d + e] = mv[so + e];
        }
    }
}

void gather_rows_out(const int32_t *rows, int64_t n, const MatView &M, const int64_t *out_rowptr, int32_t *out_col,
                     void *out_val, int vsize, cudaStream_t s, int num_sms) {
    if (n <= 0) return;
    unsigned g = blocks_for(n * 32, 256, (int64_t)num_sms * 16);
    if (vsize == 8) launch_k(k_gather_out<double>, g, 256, 0, s, rows, n, M, out_rowptr, out_col, (double *)out_val);
    else launch_k(k_gather_out<int32_t>, g, 256, 0, s, rows, n, M, out_rowptr, out_col, (int32_t *)out_val);
}

// ------------------------------------------------------- row sorting

// C's rows are stored in any column order (the hash bins write long rows in
// table order); every read returns canonical rows, so the gathered rows are
// sorted by column here.  Rows already in order are left as they are.
constexpr int SORT_SHORT = 64;     // rows up to this length: a warp each
constexpr int SORT_MAX = 16384;    // longer rows are listed and sorted together (sort_listed_rows)

template <typename T>
__global__ void k_sort_short_rows(const int64_t *rowptr, int64_t n, int32_t *col, T *val) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
        const int64_t lo = rowptr[x];
        const int len = (int)(rowptr[x + 1] - lo);
        if (len < 2 || len > SORT_SHORT) continue;
        const int32_t k0 = lane < len ? col[lo + lane] : INT32_MAX;
        const int32_t k1 = lane + 32 < len ? col[lo + lane + 32] : INT32_MAX;
        T v0 = T(0), v1 = T(0);
        if (val) {
            if (lane < len) v0 = val[lo + lane];
            if (lane + 32 < len) v1 = val[lo + lane + 32];
        }
        // rank of each key among the row's (distinct) columns
        int r0 = 0, r1 = 0;
        for (int j = 0; j < 32; j++) {
            const int32_t a = __shfl_sync(0xffffffffu, k0, j), b = __shfl_sync(0xffffffffu, k1, j);
            r0 += (a < k0) + (b < k0);
            r1 += (a < k1) + (b < k1);
        }
        __syncwarp();
        if (lane < len) {
            col[lo + r0] = k0;
            if (val) val[lo + r0] = v0;
        }
        if (lane + 32 < len) {
            col[lo + r1] = k1;
            if (val) val[lo + r1] = v1;
        }
    }
}

// Bitonic sort by column of the N (a power of two) keys in sk, with their
// values in sv when hv, in the block's shared memory (padding keys INT32_MAX).
template <typename T>
__device__ __forceinline__ void block_sort_row(int32_t *sk, T *sv, int N, bool hv) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int q = tid; q < N / 2; q += nt) {
                const int a = 2 * q - (q & (stride - 1)), b = a + stride;
                const bool up = (a & size) == 0;
                const int32_t ka = sk[a], kb = sk[b];
                if ((ka > kb) == up) {
                    sk[a] = kb;
                    sk[b] = ka;
                    if (hv) {
                        const T t = sv[a];
                        sv[a] = sv[b];
                        sv[b] = t;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(512) k_sort_long_rows(const int64_t *rowptr, int64_t n, int32_t *col, T *val,
                                                        unsigned *n_listed, int64_t *listed, int64_t list_cap) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem[];
    T *sv = (T *)smem;
    int32_t *sk = (int32_t *)(sv + SORT_MAX);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int64_t x = blockIdx.x; x < n; x += gridDim.x) {
        const int64_t lo = rowptr[x];
        const int64_t len = rowptr[x + 1] - lo;
        if (len <= SORT_SHORT) continue;
        int unsorted = 0;
        for (int64_t e = tid; e + 1 < len; e += nt) unsorted |= col[lo + e] > col[lo + e + 1];
        if (!__syncthreads_or(unsorted)) continue;
        if (len > SORT_MAX) {  // too long for shared memory: listed for sort_listed_rows
            if (tid == 0) {
                const unsigned k = atomicAdd(n_listed, 1u);
                if (k < list_cap) listed[k] = x;
            }
            continue;
        }
        int N = 128;
        while (N < len) N <<= 1;
        for (int e = tid; e < N; e += nt) {
            sk[e] = e < len ? col[lo + e] : INT32_MAX;
            if (val && e < len) sv[e] = val[lo + e];
        }
        __syncthreads();
        block_sort_row<T>(sk, sv, N, val != nullptr);
        for (int e = tid; e < len; e += nt) {
            col[lo + e] = sk[e];
            if (val) val[lo + e] = sv[e];
        }
        __syncthreads();
    }
}

// ------------------------------------------- direct read into host memory
//
// Rows of C read straight into the caller's page-locked host buffers, which
// the GPU reaches over the C2C link (out_col, out_val: their device
// addresses), with one host synchronisation for the whole read.  Each warp
// takes a row: a row of up to SORT_SHORT entries is put in column order in
// registers (ranked by shuffles unless it is in order already) and written
// out; a longer row is copied to device scratch at its place and listed for
// k_long_rows_out.  Nothing is written when R is not the ordered list of its
// collection (r_total != n) or the entries do not fit the caller's buffers;
// the flags say which, and the caller takes the general path.
template <typename T>
__global__ void k_gather_sort_out(const int32_t *rows, int64_t n_arg, const long long *n_dev, MatView M,
                                  const int64_t *rp, const int64_t *r_total, int64_t nnz_cap, int32_t *out_col,
                                  T *out_val, int32_t *scr_col, T *scr_val, int64_t *long_list, ReadOut *res) {
    pdl_begin();
    const int64_t n = n_dev ? (int64_t)*n_dev : n_arg;
    // rp[n] exists only when R was placed (r_total == n)
    const bool unordered = r_total && *r_total != n;
    const int64_t nnz = unordered ? 0 : rp[n];
    const unsigned bad = (unordered ? READ_UNORDERED : 0u) | (nnz > nnz_cap ? READ_TOO_SMALL : 0u);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        res->nnz = nnz;
        if (bad) atomicOr(&res->flags, bad);
    }
    if (bad) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const T *mv = (const T *)M.val;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
        const int64_t r = rows[x];
        const int64_t so = M.off[r], d = rp[x];
        const int L = M.len[r];
        if (L <= SORT_SHORT) {
            const int32_t k0 = lane < L ? M.col[so + lane] : INT32_MAX;
            const int32_t k1 = lane + 32 < L ? M.col[so + lane + 32] : INT32_MAX;
            T v0 = T(0), v1 = T(0);
            if (out_val) {
                if (lane < L) v0 = mv[so + lane];
                if (lane + 32 < L) v1 = mv[so + lane + 32];
            }
            // entry e + 1 after entry e: the next lane's, across the halves at lane 31
            const int32_t up0 = __shfl_down_sync(0xffffffffu, k0, 1);
            const int32_t lo1 = __shfl_sync(0xffffffffu, k1, 0);
            const int32_t up1 = __shfl_down_sync(0xffffffffu, k1, 1);
            const int32_t n0 = lane == 31 ? lo1 : up0;
            const bool out_of_order = (lane + 1 < L && k0 > n0) || (lane + 33 < L && k1 > up1);
            int r0 = lane, r1 = lane + 32;
            if (__any_sync(0xffffffffu, out_of_order)) {  // rank among the row's (distinct) columns
                r0 = 0;
                r1 = 0;
                for (int j = 0; j < 32; j++) {
                    const int32_t a = __shfl_sync(0xffffffffu, k0, j), b = __shfl_sync(0xffffffffu, k1, j);
                    r0 += (a < k0) + (b < k0);
                    r1 += (a < k1) + (b < k1);
                }
            }
            if (lane < L) {
                out_col[d + r0] = k0;
                if (out_val) out_val[d + r0] = v0;
            }
            if (lane + 32 < L) {
                out_col[d + r1] = k1;
                if (out_val) out_val[d + r1] = v1;
            }
        } else {
            for (int e = lane; e < L; e += 32) {
                scr_col[d + e] = M.col[so + e];
                if (out_val) scr_val[d + e] = mv[so + e];
            }
            if (lane == 0) long_list[atomicAdd(&res->n_long, 1u)] = x;
        }
    }
}

// The listed rows of more than SORT_SHORT entries, a block each: put in
// column order in shared memory (unless in order already) and written from
// the scratch to the caller's buffers; rows over SORT_MAX entries are listed
// again (huge_list) and left for the host's radix sort of the scratch.
template <typename T>
__global__ void __launch_bounds__(512) k_long_rows_out(const int64_t *rp, const int64_t *long_list, const int32_t *scr_col,
                                                       const T *scr_val, int32_t *out_col, T *out_val,
                                                       int64_t *huge_list, ReadOut *res) {
    pdl_begin();
    extern __shared__ __align__(16) unsigned char smem[];
    T *sv = (T *)smem;
    int32_t *sk = (int32_t *)(sv + SORT_MAX);
    if (res->flags) return;
    const unsigned nl = res->n_long;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (unsigned j = blockIdx.x; j < nl; j += gridDim.x) {
        const int64_t x = long_list[j];
        const int64_t lo = rp[x];
        const int64_t len = rp[x + 1] - lo;
        int unsorted = 0;
        for (int64_t e = tid; e + 1 < len; e += nt) unsorted |= scr_col[lo + e] > scr_col[lo + e + 1];
        if (!__syncthreads_or(unsorted)) {
            for (int64_t e = tid; e < len; e += nt) {
                out_col[lo + e] = scr_col[lo + e];
                if (out_val) out_val[lo + e] = scr_val[lo + e];
            }
            continue;
        }
        if (len > SORT_MAX) {
            if (tid == 0) huge_list[atomicAdd(&res->n_huge, 1u)] = x;
            continue;
        }
        int N = 128;
        while (N < len) N <<= 1;
        for (int e = tid; e < N; e += nt) {
            sk[e] = e < len ? scr_col[lo + e] : INT32_MAX;
            if (out_val && e < len) sv[e] = scr_val[lo + e];
        }
        __syncthreads();
        block_sort_row<T>(sk, sv, N, out_val != nullptr);
        for (int e = tid; e < len; e += nt) {
            out_col[lo + e] = sk[e];
            if (out_val) out_val[lo + e] = sv[e];
        }
        __syncthreads();
    }
}

template <typename T>
static void read_rows_direct_t(const int32_t *rows, int64_t n, const long long *n_dev, const MatView &M,
                               const int64_t *rp, const int64_t *r_total, int64_t nnz_cap, int32_t *out_col, T *out_val,
                               int32_t *scr_col, T *scr_val, int64_t *long_list, int64_t *huge_list, ReadOut *res,
                               cudaStream_t s, int num_sms) {
    // n on the device: n is the host's bound on it, which sizes the grids
    launch_k(k_gather_sort_out<T>, blocks_for(std::max<int64_t>(n, 1) * 32, 256, (int64_t)num_sms * 16), 256, 0, s, rows,
             n, n_dev, M, rp, r_total, nnz_cap, out_col, out_val, scr_col, scr_val, long_list, res);
    const size_t smem = (size_t)SORT_MAX * (sizeof(T) + sizeof(int32_t));
    static bool set = false;
    if (!set) {
        cudaFuncSetAttribute(k_long_rows_out<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        set = true;
    }
    launch_k(k_long_rows_out<T>, (unsigned)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)num_sms * 2)), 512, smem,
             s, rp, long_list, scr_col, scr_val, out_col, out_val, huge_list, res);
}

void read_rows_direct(const int32_t *rows, int64_t n, const long long *n_dev, const MatView &M, int vsize,
                      const int64_t *rp, const int64_t *r_total, int64_t nnz_cap, int32_t *out_col, void *out_val,
                      int32_t *scr_col, void *scr_val, int64_t *long_list, int64_t *huge_list, ReadOut *res,
                      cudaStream_t s, int num_sms) {
    if (vsize == 8)
        read_rows_direct_t<double>(rows, n, n_dev, M, rp, r_total, nnz_cap, out_col, (double *)out_val, scr_col,
                                   (double *)scr_val, long_list, huge_list, res, s, num_sms);
    else
        read_rows_direct_t<int32_t>(rows, n, n_dev, M, rp, r_total, nnz_cap, out_col, (int32_t *)out_val, scr_col,
                                    (int32_t *)scr_val, long_list, huge_list, res, s, num_sms);
}

template <typename T>
static void sort_rows_t(const int64_t *rowptr, int64_t n, int32_t *col, T *val, unsigned *n_listed, int64_t *listed,
                        int64_t list_cap, cudaStream_t s, int num_sms) {
    launch_k(k_sort_short_rows<T>, blocks_for(n * 32, 256, (int64_t)num_sms * 16), 256, 0, s, rowptr, n, col, val);
    const size_t smem = (size_t)SORT_MAX * (sizeof(T) + sizeof(int32_t));
    static bool set = false;
    if (!set) {
        cudaFuncSetAttribute(k_sort_long_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        set = true;
    }
    const int64_t g = std::min<int64_t>(n, (int64_t)num_sms * 2);
    launch_k(k_sort_long_rows<T>, (unsigned)std::max<int64_t>(g, 1), 512, smem, s, rowptr, n, col, val, n_listed,
             listed, list_cap);
}

void sort_rows(const int64_t *rowptr, int64_t n, int32_t *col, void *val, int vsize, unsigned *n_listed,
               int64_t *listed, int64_t list_cap, cudaStream_t s, int num_sms) {
    if (n <= 0 || !col) return;
    if (vsize == 8) sort_rows_t<double>(rowptr, n, col, (double *)val, n_listed, listed, list_cap, s, num_sms);
    else sort_rows_t<int32_t>(rowptr, n, col, (int32_t *)val, n_listed, listed, list_cap, s, num_sms);
}

// Rows too long for a CTA's shared memory, sorted all at once: the packed
// key (list index << cb | column) of every entry of the listed rows goes
// through the LSD radix sort with its place in the rows' concatenation,
// then each entry is gathered into its sorted place and copied back.
// pre[k] = entries of the listed rows before row k (pre[nl] = their total).
__device__ __forceinline__ int list_of(const int64_t *pre, int nl, int64_t q) {
    int lo = 0, hi = nl;  // the k with pre[k] <= q < pre[k + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= q) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_listed_keys(const int64_t *rowptr, const int64_t *listed, const int64_t *pre, int nl, int cb,
                              const int32_t *col, uint64_t *keys, uint32_t *idx) {
    pdl_begin();
    const int64_t E = pre[nl];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < E; q += (int64_t)gridDim.x * blockDim.x) {
        const int k = list_of(pre, nl, q);
        const int64_t p = rowptr[listed[k]] + (q - pre[k]);
        keys[q] = ((uint64_t)k << cb) | (uint32_t)col[p];
        idx[q] = (uint32_t)q;
    }
}

template <typename T>
__global__ void k_listed_gather(const int64_t *rowptr, const int64_t *listed, const int64_t *pre, int nl,
                                const uint32_t *idx, const int32_t *col, const T *val, int32_t *tcol, T *tval) {
    pdl_begin();
    const int64_t E = pre[nl];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < E; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t src = idx[q];  // the same row as q: the keys sort by list index first
        const int k = list_of(pre, nl, src);
        const int64_t p = rowptr[listed[k]] + (src - pre[k]);
        tcol[q] = col[p];
        if (val) tval[q] = val[p];
    }
}

template <typename T>
__global__ void k_listed_back(const int64_t *rowptr, const int64_t *listed, const int64_t *pre, int nl,
                              const int32_t *tcol, const T *tval, int32_t *col, T *val) {
    pdl_begin();
    const int64_t E = pre[nl];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < E; q += (int64_t)gridDim.x * blockDim.x) {
        const int k = list_of(pre, nl, q);
        const int64_t p = rowptr[listed[k]] + (q - pre[k]);
        col[p] = tcol[q];
        if (val) val[p] = tval[q];
    }
}

void sort_listed_rows(const int64_t *rowptr, const int64_t *listed, const int64_t *pre, int nl, int64_t total,
                      int cb, int32_t *col, void *val, int vsize, const SortScratch &w, cudaStream_t s, int num_sms) {
    if (nl <= 0 || total <= 0) return;
    const unsigned g = blocks_for(total, 256, (int64_t)num_sms * 8);
    launch_k(k_listed_keys, g, 256, 0, s, rowptr, listed, pre, nl, cb, col, w.k0, w.i0);
    bool alt = false;
    radix_sort_pairs(w.k0, w.i0, w.k1, w.i1, total, bits_for(nl) + cb, w.counts, w.scan_tmp, w.scan_out, s, &alt);
    const uint32_t *idx = alt ? w.i1 : w.i0;
    if (vsize == 8) {
        launch_k(k_listed_gather<double>, g, 256, 0, s, rowptr, listed, pre, nl, idx, col, (const double *)val, w.tcol,
                 (double *)w.tval);
        launch_k(k_listed_back<double>, g, 256, 0, s, rowptr, listed, pre, nl, (const int32_t *)w.tcol,
                 (const double *)w.tval, col, (double *)val);
    } else {
        launch_k(k_listed_gather<int32_t>, g, 256, 0, s, rowptr, listed, pre, nl, idx, col, (const int32_t *)val,
                 w.tcol, (int32_t *)w.tval);
        launch_k(k_listed_back<int32_t>, g, 256, 0, s, rowptr, listed, pre, nl, (const int32_t *)w.tcol,
                 (const int32_t *)w.tval, col, (int32_t *)val);
    }
}

// Canonical-CSR check: rowptr[0] = 0 and non-decreasing, rowptr[n] = nnz,
// columns in range and strictly ascending per row, values valid for the
// semiring.  Sets *bad = 1 on the first violation seen.
__global__ void k_validate_rows(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *rowptr, unsigned *bad) {
    pdl_begin();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (r == 0 && rowptr[0] != 0) atomicOr(bad, 1u);
        if (r == nrows && rowptr[nrows] != nnz) atomicOr(bad, 1u);
        if (r < nrows && rowptr[r + 1] < rowptr[r]) atomicOr(bad, 1u);
    }
}

__global__ void k_validate_entries(int64_t nrows, int64_t ncols, const int64_t *rowptr, const int32_t *col,
                                   const void *val, int sr, unsigned *bad) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nwarps) {
        const int64_t lo = rowptr[r], hi = rowptr[r + 1];
        if (hi < lo) continue;
        for (int64_t p = lo + lane; p < hi; p += 32) {
            const int32_t c = col[p];
            bool ok = c >= 0 && (int64_t)c < ncols && (p == lo || col[p - 1] < c);
            if (sr == SR_PT) ok = ok && isfinite(((const double *)val)[p]);
            else {
                const int32_t v = ((const int32_t *)val)[p];
                ok = ok && v > -MP_LIMIT && v < MP_LIMIT;
            }
            if (!ok) atomicOr(bad, 1u);
        }
    }
}

// Entry check, run only after the row bounds have been verified on the host.
void validate_csr_entries(int64_t nrows, int64_t ncols, const int64_t *rowptr, const int32_t *col, const void *val,
                          int sr, unsigned *bad, cudaStream_t s) {
    if (nrows > 0)
        launch_k(k_validate_entries, blocks_for(nrows * 32, 256, 8192), 256, 0, s, nrows, ncols, rowptr, col, val, sr, bad);
}

void validate_rowptr(int64_t nrows, int64_t nnz, const int64_t *rowptr, unsigned *bad, cudaStream_t s) {
    launch_k(k_validate_rows, blocks_for(nrows + 1, 256, 4096), 256, 0, s, nrows, 0, nnz, rowptr, bad);
}

__global__ void k_hist_cols(const int32_t *col, int64_t nnz, int32_t *counts) {
    pdl_begin();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nnz; x += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&counts[col[x]], 1);
}
void hist_cols(const int32_t *col, int64_t nnz, int32_t *counts, cudaStream_t s) {
    if (nnz > 0) launch_k(k_hist_cols, blocks_for(nnz, 256, 8192), 256, 0, s, col, nnz, counts);
}

__global__ void k_rows_of_entries(const int64_t *rowptr, int64_t nrows, uint32_t *rows_out) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nwarps)
        for (int64_t p = rowptr[r] + lane; p < rowptr[r + 1]; p += 32) rows_out[p] = (uint32_t)r;
}
void rows_of_entries(const int64_t *rowptr, int64_t nrows, uint32_t *rows_out, cudaStream_t s, int num_sms) {
    if (nrows > 0)
        launch_k(k_rows_of_entries, blocks_for(nrows * 32, 256, (int64_t)num_sms * 16), 256, 0, s, rowptr, nrows, rows_out);
}

__global__ void k_keys_from_cols(const int32_t *col, int64_t nnz, uint64_t *keys) {
    pdl_begin();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nnz; x += (int64_t)gridDim.x * blockDim.x)
        keys[x] = (uint64_t)(uint32_t)col[x];
}
void keys_from_cols(const int32_t *col, int64_t nnz, uint64_t *keys, cudaStream_t s) {
    if (nnz > 0) launch_k(k_keys_from_cols, blocks_for(nnz, 256, 8192), 256, 0, s, col, nnz, keys);
}

__global__ void k_keys_from_i32(const int32_t *a, int64_t n, uint64_t *keys, uint32_t *idx) {
    pdl_begin();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        keys[x] = (uint64_t)(uint32_t)a[x];
        idx[x] = (uint32_t)x;
    }
}
__global__ void k_keys_to_i32(const uint64_t *keys, int64_t n, int32_t *a) {
    pdl_begin();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        a[x] = (int32_t)keys[x];
}
void sort_i32_values(int32_t *a, int64_t n, int bits, uint64_t *k0, uint64_t *k1, uint32_t *i0, uint32_t *i1,
                     uint32_t *counts, int64_t *scan_tmp, int64_t *scan_out, cudaStream_t s) {
    if (n <= 1) return;
    launch_k(k_keys_from_i32, blocks_for(n, 256, 8192), 256, 0, s, a, n, k0, i0);
    bool alt = false;
    radix_sort_pairs(k0, i0, k1, i1, n, bits, counts, scan_tmp, scan_out, s, &alt);
    launch_k(k_keys_to_i32, blocks_for(n, 256, 8192), 256, 0, s, alt ? k1 : k0, n, a);
}

}  // namespace dspg
