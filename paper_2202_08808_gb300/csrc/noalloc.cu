// noalloc.cu -- rows of C = A B computed without allocating device memory.
//
// Some callers cannot let a library allocate: their device memory is owned
// by another allocator (a framework's caching pool, a fixed arena sized at
// start-up), or their latency budget cannot absorb cudaMalloc/cudaFree,
// which synchronise the device.  dspg_multiply_rows_noalloc serves them: it
// reads A and B from the caller's device CSR arrays, writes the requested
// rows into the caller's output buffers, and keeps its working memory in a
// fixed array of device memory that belongs to this library image.
//
// The working memory is na_scratch below: NA_CTAS slices, each a dense
// accumulator of NA_MAX_COLS values plus a presence bitmap, and one status
// word.  Every GPU that loads the library holds these NA_SCRATCH_BYTES
// (about 4.1 MiB) until the process exits.  Host code must not pass the
// symbol itself to a kernel (in host code it names a host-side stand-in):
// its device address is taken once per device with cudaGetSymbolAddress.
//
// The kernel is a CTA-per-row variant of the dense global-memory
// accumulator used for the longest rows of the recompute: each CTA owns one
// slice, scatters the row's products into it (atomics), then reads the set
// bits in column order.  A first pass counts each row's entries into the
// caller's rowptr, one CTA scans them, and a second pass writes the rows.
#include <atomic>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace dspg {

namespace {

constexpr int64_t NA_MAX_COLS = 1 << 16;  // widest C the entry point accepts
constexpr int NA_CTAS = 8;                // CTAs (and scratch slices)
constexpr int NA_NT = 256;
constexpr size_t NA_WORDS = NA_MAX_COLS / 32;
constexpr size_t NA_SLICE_BYTES = NA_MAX_COLS * sizeof(double) + NA_WORDS * sizeof(uint32_t);
constexpr size_t NA_STATUS_OFF = NA_CTAS * NA_SLICE_BYTES;
constexpr size_t NA_SCRATCH_BYTES = NA_STATUS_OFF + 256;

static __device__ __align__(256) unsigned char na_scratch[NA_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
// Device address of na_scratch per device, looked up once (under the mutex;
// later calls read it without locking).
std::atomic<unsigned char *> g_na_ptr[NA_MAX_DEVICES] = {};
std::mutex g_na_mutex;

template <int SR>
struct NaSr;
template <>
struct NaSr<SR_PT> {
    using T = double;
    __device__ static T zero() { return 0.0; }
    __device__ static T mul(T a, T b) { return a * b; }
    __device__ static void acc(T *p, T v) { atomicAdd(p, v); }
};
template <>
struct NaSr<SR_MP> {
    using T = int32_t;
    __device__ static T zero() { return MP_INF; }
    __device__ static T mul(T a, T b) { return a + b; }
    __device__ static void acc(T *p, T v) { atomicMin(p, v); }
};

struct NaArgs {
    const int64_t *arp;
    const int32_t *acol;
    const void *aval;
    const int64_t *brp;
    const int32_t *bcol;
    const void *bval;
    int64_t a_rows, b_rows, m;
    const int32_t *rows;
    int64_t nr;
    int64_t *rowptr;
    int32_t *out_col;
    void *out_val;
};

// mode 0: rowptr[t+1] = entries of row rows[t]; mode 1: write row rows[t]
// at rowptr[t].  Bad row or column indices set the status word and are
// skipped.
template <int SR>
__global__ void __launch_bounds__(NA_NT) k_na_rows(NaArgs g, unsigned char *scratch, int mode) {
    pdl_begin();
    using T = typename NaSr<SR>::T;
    __shared__ int s_incl[NA_NT];
    __shared__ int s_wsum[NA_NT / 32];
    __shared__ int s_n;
    T *acc = (T *)(scratch + (size_t)blockIdx.x * NA_SLICE_BYTES);
    uint32_t *msk = (uint32_t *)(acc + NA_MAX_COLS);
    unsigned *status = (unsigned *)(scratch + NA_STATUS_OFF);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int words = (int)((g.m + 31) / 32);
    // the array keeps the previous call's contents: start from a clean slice
    for (int64_t x = tid; x < g.m; x += NA_NT) acc[x] = NaSr<SR>::zero();
    for (int x = tid; x < words; x += NA_NT) msk[x] = 0u;
    __syncthreads();
    const T *Av = (const T *)g.aval;
    const T *Bv = (const T *)g.bval;
    T *Ov = (T *)g.out_val;
    for (int64_t t = blockIdx.x; t < g.nr; t += gridDim.x) {
        const int32_t i = g.rows[t];
        if (i < 0 || (int64_t)i >= g.a_rows) {
            if (tid == 0) {
                atomicOr(status, 1u);
                if (mode == 0) g.rowptr[t + 1] = 0;
            }
            continue;
        }
        for (int64_t p = g.arp[i]; p < g.arp[i + 1]; p++) {
            const int32_t k = g.acol[p];
            if (k < 0 || (int64_t)k >= g.b_rows) {
                if (tid == 0) atomicOr(status, 1u);
                continue;
            }
            const T a = Av[p];
            for (int64_t q = g.brp[k] + tid; q < g.brp[k + 1]; q += NA_NT) {
                const int32_t j = g.bcol[q];
                if (j < 0 || (int64_t)j >= g.m) {
                    atomicOr(status, 1u);
                    continue;
                }
                atomicOr(&msk[j >> 5], 1u << (j & 31));
                NaSr<SR>::acc(&acc[j], NaSr<SR>::mul(a, Bv[q]));
            }
        }
        __syncthreads();
        if (mode == 0) {
            int c = 0;
            for (int x = tid; x < words; x += NA_NT) c += __popc(msk[x]);
            c = warp_sum<int>(c);
            if (tid == 0) s_n = 0;
            __syncthreads();
            if (lane == 0) atomicAdd(&s_n, c);
            __syncthreads();
            if (tid == 0) g.rowptr[t + 1] = s_n;
        }
        // read out (mode 1) and clear, in column order, NA_NT words at a time
        int64_t run = mode == 1 ? g.rowptr[t] : 0;
        for (int x0 = 0; x0 < words; x0 += NA_NT) {
            const int x = x0 + tid;
            const uint32_t word = x < words ? msk[x] : 0u;
            const int pc = __popc(word);
            int incl = warp_incl_scan<int>(pc);
            if (lane == 31) s_wsum[w] = incl;
            __syncthreads();
            if (w == 0) {
                const int v = lane < NA_NT / 32 ? s_wsum[lane] : 0;
                const int vi = warp_incl_scan<int>(v);
                if (lane < NA_NT / 32) s_wsum[lane] = vi - v;
            }
            __syncthreads();
            incl += s_wsum[w];
            s_incl[tid] = incl;
            __syncthreads();
            int64_t o = run + incl - pc;
            uint32_t bits = word;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int j = (x << 5) + b;
                if (mode == 1) {
                    g.out_col[o] = j;
                    Ov[o] = acc[j];
                }
                acc[j] = NaSr<SR>::zero();
                o++;
            }
            if (x < words) msk[x] = 0u;
            run += s_incl[NA_NT - 1];
            __syncthreads();
        }
    }
}

// rowptr[0] = 0 and rowptr[1..nr] = running sums of the counts (one CTA).
__global__ void __launch_bounds__(1024) k_na_scan(int64_t *rowptr, int64_t nr) {
    pdl_begin();
    __shared__ int64_t s_w[32];
    __shared__ int64_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        rowptr[0] = 0;
        s_carry = 0;
    }
    __syncthreads();
    for (int64_t b = 0; b < nr; b += 1024) {
        const int64_t x = b + tid;
        const int64_t v = x < nr ? rowptr[x + 1] : 0;
        int64_t incl = warp_incl_scan<int64_t>(v);
        if (lane == 31) s_w[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int64_t u = s_w[lane];
            const int64_t ui = warp_incl_scan<int64_t>(u);
            s_w[lane] = ui - u;
        }
        __syncthreads();
        incl += s_w[w] + s_carry;
        if (x < nr) rowptr[x + 1] = incl;
        __syncthreads();
        if (tid == 1023) s_carry = incl;
        __syncthreads();
    }
}

dspg_status fail_na(dspg_status st, const char *msg) {
    set_thread_error(msg);
    return st;
}

}  // namespace
}  // namespace dspg

using namespace dspg;

extern "C" dspg_status dspg_multiply_rows_noalloc(const dspg_csr *A, const dspg_csr *B, dspg_semiring sr,
                                                  const int32_t *rows, int64_t nrows, int64_t *rowptr, int32_t *col,
                                                  void *val, int64_t capacity, int64_t *nnz_out, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!A || !B || !nnz_out || nrows < 0 || (nrows > 0 && (!rows || !rowptr)))
        return fail_na(DSPG_ERR_INVALID, "NULL argument or negative row count");
    if (sr != DSPG_PLUS_TIMES_F64 && sr != DSPG_MIN_PLUS_I32) return fail_na(DSPG_ERR_INVALID, "unknown semiring");
    if (!A->on_device || !B->on_device) return fail_na(DSPG_ERR_INVALID, "A and B must be in device memory");
    if (A->ncols != B->nrows) return fail_na(DSPG_ERR_INVALID, "A.ncols != B.nrows");
    if (B->ncols > NA_MAX_COLS)
        return fail_na(DSPG_ERR_INVALID, "B has more than 65536 columns, the limit of the fixed scratch array");
    if (A->nrows >= INT32_MAX || B->nrows >= INT32_MAX) return fail_na(DSPG_ERR_INVALID, "too many rows");
    if (!A->rowptr || !B->rowptr || (A->nnz > 0 && (!A->col || !A->val)) || (B->nnz > 0 && (!B->col || !B->val)))
        return fail_na(DSPG_ERR_INVALID, "NULL CSR array");
    *nnz_out = 0;
    if (nrows == 0) return DSPG_OK;

    // set-up, once per device with that device current: the device address
    // of the scratch array.  The stream must belong to that device, or the
    // kernels would get another device's address.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
        return fail_na(DSPG_ERR_CUDA, "cudaGetDevice failed");
    int sdev = dev;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) {
        cudaGetLastError();
        return fail_na(DSPG_ERR_INVALID, "the stream is not a valid stream");
    }
    if (sdev != dev) return fail_na(DSPG_ERR_INVALID, "the stream belongs to another device than the current one");
    unsigned char *scratch = g_na_ptr[dev].load(std::memory_order_acquire);
    if (!scratch) {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        scratch = g_na_ptr[dev].load(std::memory_order_relaxed);
        if (!scratch) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail_na(DSPG_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
            }
            scratch = (unsigned char *)p;
            g_na_ptr[dev].store(scratch, std::memory_order_release);
        }
    }
    unsigned *status = (unsigned *)(scratch + NA_STATUS_OFF);

    NaArgs g{A->rowptr, A->col, A->val, B->rowptr, B->col, B->val, A->nrows, B->nrows, B->ncols,
             rows, nrows, rowptr, col, val};
    auto run = [&](int mode) {
        if (sr == DSPG_PLUS_TIMES_F64) launch_k(k_na_rows<SR_PT>, NA_CTAS, NA_NT, 0, s, g, scratch, mode);
        else launch_k(k_na_rows<SR_MP>, NA_CTAS, NA_NT, 0, s, g, scratch, mode);
    };
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), s) != cudaSuccess) return fail_na(DSPG_ERR_CUDA, "memset failed");
    run(0);
    launch_k(k_na_scan, 1, 1024, 0, s, rowptr, nrows);
    int64_t total = 0;
    unsigned st = 0;
    if (cudaMemcpyAsync(&total, rowptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&st, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail_na(DSPG_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    if (st) return fail_na(DSPG_ERR_INVALID, "row or column index out of range");
    *nnz_out = total;
    if (!col) return DSPG_OK;  // size query
    if (total > capacity) return fail_na(DSPG_ERR_INVALID, "output capacity is smaller than the result");
    if (total > 0 && !val) return fail_na(DSPG_ERR_INVALID, "NULL value buffer");
    run(1);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail_na(DSPG_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    return DSPG_OK;
}
