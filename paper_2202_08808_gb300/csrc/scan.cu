// scan.cu -- device-wide exclusive prefix sums (reduce, scan of partials, scan + add).
#include "common.cuh"

namespace dspg {

constexpr int SCAN_NT = 1024;
constexpr int SCAN_IPT = 4;
constexpr int64_t SCAN_CHUNK = SCAN_NT * SCAN_IPT;

int64_t scan_tmp_entries(int64_t n) { return (n + SCAN_CHUNK - 1) / SCAN_CHUNK + 1; }

template <typename T>
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_tot[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = warp_incl_scan<int64_t>(v);
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
        int64_t ti = warp_incl_scan<int64_t>(t);
        warp_tot[lane] = ti - t;
        if (lane == 31) *total = ti;
    }
    __syncthreads();
    int64_t r = warp_tot[w] + incl - v;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void k_scan_reduce(const T *in, int64_t n, int64_t *partial) {
    pdl_begin();
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    int64_t s = 0;
    for (int j = 0; j < SCAN_IPT; j++) {
        int64_t i = base + (int64_t)j * SCAN_NT + threadIdx.x;
        if (i < n) s += (int64_t)in[i];
    }
    s = warp_sum<int64_t>(s);
    __shared__ int64_t ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t t = ws[threadIdx.x];
        t = warp_sum<int64_t>(t);
        if (threadIdx.x == 0) partial[blockIdx.x] = t;
    }
}

__global__ void k_scan_partials(int64_t *partial, int64_t nb) {
    pdl_begin();
    __shared__ int64_t carry;
    __shared__ int64_t tot;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_NT) {
        int64_t i = b0 + threadIdx.x;
        int64_t v = i < nb ? partial[i] : 0;
        int64_t e = block_excl_scan<int64_t>(v, &tot);
        if (i < nb) partial[i] = carry + e;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[nb] = carry;
}

template <typename T>
__global__ void k_scan_final(const T *in, int64_t n, const int64_t *partial, int64_t *out) {
    pdl_begin();
    __shared__ int64_t tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    // blocked arrangement: thread t owns SCAN_IPT consecutive elements
    int64_t v[SCAN_IPT];
    int64_t s = 0;
    for (int j = 0; j < SCAN_IPT; j++) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_IPT + j;
        v[j] = i < n ? (int64_t)in[i] : 0;
        s += v[j];
    }
    int64_t e = block_excl_scan<int64_t>(s, &tot) + partial[blockIdx.x];
    for (int j = 0; j < SCAN_IPT; j++) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_IPT + j;
        if (i < n) out[i] = e;
        e += v[j];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = partial[gridDim.x];
}

template <typename T>
static void scan_impl(const T *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
    if (n == 0) {
        cudaMemsetAsync(out, 0, sizeof(int64_t), s);
        return;
    }
    int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    launch_k(k_scan_reduce<T>, (unsigned)nb, SCAN_NT, 0, s, in, n, tmp);
    launch_k(k_scan_partials, 1, SCAN_NT, 0, s, tmp, nb);
    launch_k(k_scan_final<T>, (unsigned)nb, SCAN_NT, 0, s, in, n, tmp, out);
}

void scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
    scan_impl<int32_t>(in, out, n, tmp, s);
}
void scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s) {
    scan_impl<int64_t>(in, out, n, tmp, s);
}

}  // namespace dspg
