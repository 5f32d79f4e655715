// spgemm.cu -- recompute of selected rows of C = A B over a semiring.
//
// Section 6.1: the local product is Gustavson's row-wise algorithm; each row
// C(i,:) = (+)_k A(i,k) (x) B(k,:) is formed in a sparse accumulator.  An
// output column is a non-zero iff some product reaches it (structural
// semantics, Section 3).  Here every affected row is first sized by the
// product bound ub_i = sum_k len(B_k) (capped at the column count), binned
// by that bound, and recomputed by the kernel of its bin:
//
//   bins 0-4   warp per row, open-addressing hash in shared memory
//              (64 .. 1024 slots, load <= 1/2);
//   bins 5-7   CTA per row, hash of 2048 .. 8192 slots in shared memory;
//   bin  8     CTA per row, dense accumulator over all columns in global
//              memory (L2) with a presence bitmap, for the longest rows;
//   bins 9-10  when C has at most 1024 columns: dense accumulators in shared
//              memory (warp per row, or CTA per row for long rows).
//
// Products of a row are flattened over its A entries: a scan of the B-row
// lengths of up to 32 (warp) or blockDim (CTA) A entries assigns product p
// to A entry s by a binary search in the scan, so all lanes stay busy even
// when B rows are short.  Each row's output is compacted, sorted by column
// (hash bins) or read out in column order (dense bins), and written to a
// staging buffer at an offset taken from a device counter; the splice then
// moves it into C.  (+,.) accumulates with double atomics (the summation
// order varies; the library's tolerance covers any order), (min,+) with
// atomicMin (order-free, bit-exact).
#include "internal.h"

namespace dspg {

template <int SR>
struct Sr;
template <>
struct Sr<SR_PT> {
    using T = double;
    __device__ static T zero() { return 0.0; }
    __device__ static T mul(T a, T b) { return a * b; }
    __device__ static void acc(T *p, T v) { atomicAdd(p, v); }
};
template <>
struct Sr<SR_MP> {
    using T = int32_t;
    __device__ static T zero() { return MP_INF; }
    __device__ static T mul(T a, T b) { return a + b; }
    __device__ static void acc(T *p, T v) { atomicMin(p, v); }
};

enum {
    BIN_W64 = 0, BIN_W128, BIN_W256, BIN_W512, BIN_W1024,
    BIN_C2048, BIN_C4096, BIN_C8192,
    BIN_GD,
    BIN_WDENSE, BIN_CDENSE,
    BIN_COUNT
};
static_assert(BIN_COUNT <= NBINS, "bin counters");

__device__ __forceinline__ long long atomic_add_ll2(long long *p, long long v) {
    return (long long)atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

// ------------------------------------------------------------- sizing

__device__ __forceinline__ int pick_bin(long long ubc, int dense_mode) {
    if (dense_mode) return ubc <= 4096 ? BIN_WDENSE : BIN_CDENSE;
    if (ubc <= 32) return BIN_W64;
    if (ubc <= 64) return BIN_W128;
    if (ubc <= 128) return BIN_W256;
    if (ubc <= 256) return BIN_W512;
    if (ubc <= 512) return BIN_W1024;
    if (ubc <= 1024) return BIN_C2048;
    if (ubc <= 2048) return BIN_C4096;
    if (ubc <= 4096) return BIN_C8192;
    return BIN_GD;
}

// A warp sizes 32 rows of R at a time (all lanes on one row, lane r keeping
// row r's bound ub), then hands out staging room (ub entries per row, so the
// numeric kernels need no allocation) and bin slots with one atomic per warp
// and counter.
__global__ void k_size_bins(MatView A, MatView B, CJob J, Ctl *ctl, unsigned mask) {
    if (failed(ctl, mask)) return;
    const long long nR = ctl->n_affected;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    long long prod_acc = 0, a_acc = 0;
    for (long long t0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; t0 < nR; t0 += nwarps * 32) {
        const long long my_t = t0 + lane;
        const bool valid = my_t < nR;
        const int32_t my_i = valid ? J.R[my_t] : 0;
        const int64_t my_aoff = valid ? A.off[my_i] : 0;
        const int my_alen = valid ? A.len[my_i] : 0;
        long long my_s = 0;
        const int cnt = (int)(nR - t0 < 32 ? nR - t0 : 32);
        for (int rr = 0; rr < cnt; rr++) {
            const int64_t aoff = __shfl_sync(0xffffffffu, my_aoff, rr);
            const int alen = __shfl_sync(0xffffffffu, my_alen, rr);
            long long s = 0;
            for (int a = lane; a < alen; a += 32) s += B.len[A.col[aoff + a]];
            s = warp_sum<long long>(s);
            if (lane == rr) my_s = s;
        }
        const long long ubc = my_s < J.m ? my_s : J.m;
        const long long so = warp_fetch_add(&ctl->c_stage_top, ubc);
        if (valid) {
            J.soff[my_t] = so;
            J.slen[my_t] = 0;
            if (so + ubc > J.st_cap) set_status(ctl, ST_C_STAGE);
        }
        const int b = (valid && my_s > 0) ? pick_bin(ubc, J.dense_mode) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        long long bb = 0;
        if (b >= 0 && lane == leader) bb = atomic_add_ll2(&ctl->bin_count[b], __popc(peers));
        bb = __shfl_sync(0xffffffffu, bb, leader);
        if (b >= 0) J.bins[(int64_t)b * J.bin_cap + bb + __popc(peers & lanemask_lt())] = (int32_t)my_t;
        prod_acc += warp_sum<long long>(valid ? my_s : 0);
        a_acc += warp_sum<long long>(my_alen);
    }
    if (lane == 0) {
        if (prod_acc) atomic_add_ll2(&ctl->products, prod_acc);
        if (a_acc) atomic_add_ll2(&ctl->a_entries, a_acc);
    }
}

// --------------------------------------------------- product generators

// Calls emit(j, a (x) b) for every product of row i, lanes of one warp
// sharing the work.
template <int SR, class F>
__device__ __forceinline__ void warp_products(const MatView &A, const MatView &B, int32_t i, F emit) {
    using T = typename Sr<SR>::T;
    const int lane = threadIdx.x & 31;
    const int64_t aoff = A.off[i];
    const int alen = A.len[i];
    const T *Av = (const T *)A.val;
    const T *Bv = (const T *)B.val;
    for (int a0 = 0; a0 < alen; a0 += 32) {
        const int ai = a0 + lane;
        int blen = 0;
        int64_t boff = 0;
        T av = T(0);
        if (ai < alen) {
            const int32_t k = A.col[aoff + ai];
            av = Av[aoff + ai];
            boff = B.off[k];
            blen = B.len[k];
        }
        const int incl = warp_incl_scan<int>(blen);
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int base = 0; base < total; base += 32) {
            const int p = base + lane;
            int s = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int v = __shfl_sync(0xffffffffu, incl, s + step - 1);
                if (v <= p) s += step;
            }
            const int64_t bo = __shfl_sync(0xffffffffu, boff, s);
            const T a = __shfl_sync(0xffffffffu, av, s);
            const int excl = __shfl_sync(0xffffffffu, incl, s) - __shfl_sync(0xffffffffu, blen, s);
            if (p < total) {
                const int64_t q = bo + (p - excl);
                emit(B.col[q], Sr<SR>::mul(a, Bv[q]));
            }
        }
    }
}

template <typename T>
struct BlockProdSmem {
    int64_t *boff;
    T *av;
    int *incl;
    int *blen;
    int *wsum;  // 32 entries
};

// Block-wide inclusive scan of v into incl[tid]; returns the total.
__device__ __forceinline__ int block_incl_scan(int v, int *incl, int *wsum) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = warp_incl_scan<int>(v);
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? wsum[lane] : 0;
        int ti = warp_incl_scan<int>(t);
        wsum[lane] = ti - t;
    }
    __syncthreads();
    x += wsum[w];
    incl[threadIdx.x] = x;
    __syncthreads();
    return incl[blockDim.x - 1];
}

// Calls emit(j, a (x) b) for every product of row i, all threads of the
// block sharing the work.  Must be called by the whole block.
template <int SR, class F>
__device__ __forceinline__ void block_products(const MatView &A, const MatView &B, int32_t i,
                                               BlockProdSmem<typename Sr<SR>::T> sm, F emit) {
    using T = typename Sr<SR>::T;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t aoff = A.off[i];
    const int alen = A.len[i];
    const T *Av = (const T *)A.val;
    const T *Bv = (const T *)B.val;
    for (int a0 = 0; a0 < alen; a0 += nt) {
        const int ai = a0 + tid;
        int blen = 0;
        if (ai < alen) {
            const int32_t k = A.col[aoff + ai];
            sm.av[tid] = Av[aoff + ai];
            sm.boff[tid] = B.off[k];
            blen = B.len[k];
        }
        sm.blen[tid] = blen;
        const int total = block_incl_scan(blen, sm.incl, sm.wsum);
        for (int base = 0; base < total; base += nt) {
            const int p = base + tid;
            if (p < total) {
                const int s = (int)upper_bound_dev<int>(sm.incl, 0, nt, p);
                const int excl = sm.incl[s] - sm.blen[s];
                const int64_t q = sm.boff[s] + (p - excl);
                emit(B.col[q], Sr<SR>::mul(sm.av[s], Bv[q]));
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------- hash table

template <int LOG_TS, typename T, int SR>
__device__ __forceinline__ bool hash_acc(int32_t *keys, T *vals, int32_t j, T v) {
    constexpr int TS = 1 << LOG_TS;
    uint32_t h = ((uint32_t)j * 2654435761u) >> (32 - LOG_TS);
    for (int probe = 0; probe < TS; probe++) {
        const int32_t k = ((volatile int32_t *)keys)[h];
        if (k == j) {
            Sr<SR>::acc(&vals[h], v);
            return true;
        }
        if (k == -1) {
            const int32_t old = atomicCAS(&keys[h], -1, j);
            if (old == -1 || old == j) {
                Sr<SR>::acc(&vals[h], v);
                return true;
            }
        }
        h = (h + 1) & (TS - 1);
    }
    return false;  // table full: cannot happen when the bin bound holds
}

template <typename T>
__device__ __forceinline__ void bitonic_step(int32_t *k, T *v, int i, int l, bool up) {
    const int32_t ki = k[i], kl = k[l];
    if ((ki > kl) == up) {
        k[i] = kl;
        k[l] = ki;
        const T t = v[i];
        v[i] = v[l];
        v[l] = t;
    }
}

// ------------------------------------------------------ warp hash kernel

template <int SR, int LOG_TS, int NW>
__global__ void __launch_bounds__(NW * 32)
k_num_warp_hash(MatView A, MatView B, CJob J, Ctl *ctl, unsigned mask, int bin) {
    using T = typename Sr<SR>::T;
    constexpr int TS = 1 << LOG_TS;
    constexpr int HC = TS / 2;  // compacted list capacity
    extern __shared__ __align__(16) unsigned char smem[];
    if (failed(ctl, mask)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T *vals = (T *)smem + (size_t)w * TS;
    T *cv = (T *)smem + (size_t)NW * TS + (size_t)w * HC;
    int32_t *keys = (int32_t *)((T *)smem + (size_t)NW * (TS + HC)) + (size_t)w * TS;
    int32_t *ck = (int32_t *)((T *)smem + (size_t)NW * (TS + HC)) + (size_t)NW * TS + (size_t)w * HC;
    T *sv = (T *)J.st_val;
    long long nnz_acc = 0;
    const long long cnt = ctl->bin_count[bin];
    for (long long it = (long long)blockIdx.x * NW + w; it < cnt; it += (long long)gridDim.x * NW) {
        const int t = J.bins[(int64_t)bin * J.bin_cap + it];
        const int32_t i = J.R[t];
        for (int s = lane; s < TS; s += 32) {
            keys[s] = -1;
            vals[s] = Sr<SR>::zero();
        }
        __syncwarp();
        bool ok = true;
        warp_products<SR>(A, B, i, [&](int32_t j, T v) { ok &= hash_acc<LOG_TS, T, SR>(keys, vals, j, v); });
        if (!__all_sync(0xffffffffu, ok) && lane == 0) set_status(ctl, ST_TIMEOUT);
        __syncwarp();
        int n = 0;
        for (int s0 = 0; s0 < TS; s0 += 32) {
            const int s = s0 + lane;
            const int32_t k = keys[s];
            const bool occ = k >= 0;
            const unsigned bal = __ballot_sync(0xffffffffu, occ);
            if (occ) {
                const int x = n + __popc(bal & lanemask_lt());
                if (x < HC) {
                    ck[x] = k;
                    cv[x] = vals[s];
                }
            }
            n += __popc(bal);
        }
        if (n > HC) n = HC;  // unreachable when ub <= HC
        __syncwarp();
        const long long so = J.soff[t];  // room for the row's product bound, from the sizing pass
        if (lane == 0) J.slen[t] = n;
        nnz_acc += n;
        const bool fits = true;
        if (n <= 32) {
            // rank of each entry among distinct column keys
            const int32_t myk = lane < n ? ck[lane] : 0x7fffffff;
            const T myv = lane < n ? cv[lane] : Sr<SR>::zero();
            int rank = 0;
            for (int s = 0; s < n; s++) rank += __shfl_sync(0xffffffffu, myk, s) < myk;
            if (lane < n && fits) {
                J.st_col[so + rank] = myk;
                sv[so + rank] = myv;
            }
        } else {
            int N = 64;
            while (N < n) N <<= 1;
            for (int s = n + lane; s < N; s += 32) ck[s] = 0x7fffffff;
            __syncwarp();
            for (int size = 2; size <= N; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int x = lane; x < N / 2; x += 32) {
                        const int a = 2 * x - (x & (stride - 1));
                        bitonic_step<T>(ck, cv, a, a + stride, (a & size) == 0);
                    }
                    __syncwarp();
                }
            }
            if (fits)
                for (int s = lane; s < n; s += 32) {
                    J.st_col[so + s] = ck[s];
                    sv[so + s] = cv[s];
                }
        }
        __syncwarp();
    }
    if (lane == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// ------------------------------------------------------- CTA hash kernel

template <int SR, int LOG_TS>
__global__ void __launch_bounds__(256)
k_num_cta_hash(MatView A, MatView B, CJob J, Ctl *ctl, unsigned mask, int bin) {
    using T = typename Sr<SR>::T;
    constexpr int TS = 1 << LOG_TS;
    constexpr int HC = TS / 2;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t p_boff[256];
    __shared__ T p_av[256];
    __shared__ int p_incl[256], p_blen[256], p_wsum[32];
    __shared__ int s_n;
    __shared__ long long s_so;
    __shared__ int s_ok;
    if (failed(ctl, mask)) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    T *vals = (T *)smem;
    T *cv = vals + TS;
    int32_t *keys = (int32_t *)(cv + HC);
    int32_t *ck = keys + TS;
    T *sv = (T *)J.st_val;
    BlockProdSmem<T> ps{p_boff, p_av, p_incl, p_blen, p_wsum};
    long long nnz_acc = 0;
    const long long cnt = ctl->bin_count[bin];
    for (long long it = blockIdx.x; it < cnt; it += gridDim.x) {
        const int t = J.bins[(int64_t)bin * J.bin_cap + it];
        const int32_t i = J.R[t];
        for (int s = tid; s < TS; s += 256) {
            keys[s] = -1;
            vals[s] = Sr<SR>::zero();
        }
        if (tid == 0) {
            s_n = 0;
            s_ok = 1;
        }
        __syncthreads();
        bool ok = true;
        block_products<SR>(A, B, i, ps, [&](int32_t j, T v) { ok &= hash_acc<LOG_TS, T, SR>(keys, vals, j, v); });
        if (!ok) s_ok = 0;
        __syncthreads();
        if (!s_ok && tid == 0) set_status(ctl, ST_TIMEOUT);
        // compact (unordered) through a shared counter per warp chunk
        for (int s0 = w * 32; s0 < TS; s0 += 256) {
            const int s = s0 + lane;
            const int32_t k = keys[s];
            const bool occ = k >= 0;
            const unsigned bal = __ballot_sync(0xffffffffu, occ);
            int base = 0;
            if (lane == 0 && bal) base = atomicAdd(&s_n, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (occ) {
                const int x = base + __popc(bal & lanemask_lt());
                if (x < HC) {
                    ck[x] = k;
                    cv[x] = vals[s];
                }
            }
        }
        __syncthreads();
        int n = s_n < HC ? s_n : HC;
        int N = 2;
        while (N < n) N <<= 1;
        for (int s = n + tid; s < N; s += 256) ck[s] = 0x7fffffff;
        if (tid == 0) {
            J.slen[t] = n;
            s_so = J.soff[t];
            nnz_acc += n;
        }
        __syncthreads();
        for (int size = 2; size <= N; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int x = tid; x < N / 2; x += 256) {
                    const int a = 2 * x - (x & (stride - 1));
                    bitonic_step<T>(ck, cv, a, a + stride, (a & size) == 0);
                }
                __syncthreads();
            }
        }
        const long long so = s_so;
        for (int s = tid; s < n; s += 256) {
            J.st_col[so + s] = ck[s];
            sv[so + s] = cv[s];
        }
        __syncthreads();
    }
    if (tid == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// ------------------------------------------------- global dense kernel

template <int SR>
__global__ void __launch_bounds__(512)
k_num_gdense(MatView A, MatView B, CJob J, Ctl *ctl, unsigned mask, int bin) {
    using T = typename Sr<SR>::T;
    __shared__ int64_t p_boff[512];
    __shared__ T p_av[512];
    __shared__ int p_incl[512], p_blen[512], p_wsum[32];
    __shared__ int s_lo, s_hi;
    __shared__ int s_n;
    if (failed(ctl, mask)) return;
    const int tid = threadIdx.x;
    T *acc = (T *)J.gd_acc + (int64_t)blockIdx.x * J.gd_w;
    uint32_t *msk = J.gd_mask + (int64_t)blockIdx.x * (J.gd_w / 32);
    T *sv = (T *)J.st_val;
    BlockProdSmem<T> ps{p_boff, p_av, p_incl, p_blen, p_wsum};
    long long nnz_acc = 0;
    const long long cnt = ctl->bin_count[bin];
    for (long long it = blockIdx.x; it < cnt; it += gridDim.x) {
        const int t = J.bins[(int64_t)bin * J.bin_cap + it];
        const int32_t i = J.R[t];
        if (tid == 0) {
            s_lo = 0x7fffffff;
            s_hi = -1;
            s_n = 0;
        }
        __syncthreads();
        int lo = 0x7fffffff, hi = -1;
        block_products<SR>(A, B, i, ps, [&](int32_t j, T v) {
            atomicOr(&msk[j >> 5], 1u << (j & 31));
            Sr<SR>::acc(&acc[j], v);
            lo = min(lo, j);
            hi = max(hi, j);
        });
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
        __syncthreads();
        const int w0 = s_lo >> 5, w1 = s_hi < 0 ? -1 : (s_hi >> 5);
        int c = 0;
        for (int x = w0 + tid; x <= w1; x += 512) c += __popc(msk[x]);
        c = warp_sum<int>(c);
        if ((tid & 31) == 0 && c) atomicAdd(&s_n, c);
        __syncthreads();
        const int n = s_n;
        if (tid == 0) {
            J.slen[t] = n;
            nnz_acc += n;
        }
        const long long so = J.soff[t];
        const bool fits = true;
        int run = 0;  // entries written by earlier chunks
        for (int x0 = w0; x0 <= w1; x0 += 512) {
            const int x = x0 + tid;
            const uint32_t word = x <= w1 ? msk[x] : 0u;
            const int pc = __popc(word);
            const int incl = block_incl_scan(pc, p_incl, p_wsum);
            int o = run + p_incl[tid] - pc;
            uint32_t bits = word;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int j = (x << 5) + b;
                if (fits) {
                    J.st_col[so + o] = j;
                    sv[so + o] = acc[j];
                }
                acc[j] = Sr<SR>::zero();
                o++;
            }
            if (x <= w1) msk[x] = 0u;
            run += incl;
            __syncthreads();
        }
    }
    if (tid == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// ----------------------------------------------------- dense small-m kernels

template <int SR, int NW>
__global__ void __launch_bounds__(NW * 32)
k_num_warp_dense(MatView A, MatView B, CJob J, Ctl *ctl, unsigned mask, int bin, int mp) {
    using T = typename Sr<SR>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    if (failed(ctl, mask)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = mp >> 5;  // presence words (<= 32)
    T *acc = (T *)smem + (size_t)w * mp;
    uint32_t *msk = (uint32_t *)((T *)smem + (size_t)NW * mp) + (size_t)w * 32;
    T *sv = (T *)J.st_val;
    for (int s = lane; s < mp; s += 32) acc[s] = Sr<SR>::zero();
    msk[lane] = 0u;
    __syncwarp();
    long long nnz_acc = 0;
    const long long cnt = ctl->bin_count[bin];
    for (long long it = (long long)blockIdx.x * NW + w; it < cnt; it += (long long)gridDim.x * NW) {
        const int t = J.bins[(int64_t)bin * J.bin_cap + it];
        const int32_t i = J.R[t];
        warp_products<SR>(A, B, i, [&](int32_t j, T v) {
            atomicOr(&msk[j >> 5], 1u << (j & 31));
            Sr<SR>::acc(&acc[j], v);
        });
        __syncwarp();
        const uint32_t word = lane < nw ? msk[lane] : 0u;
        const int pc = __popc(word);
        const int incl = warp_incl_scan<int>(pc);
        const int n = __shfl_sync(0xffffffffu, incl, 31);
        const long long so = J.soff[t];
        if (lane == 0) J.slen[t] = n;
        nnz_acc += n;
        int o = incl - pc;
        uint32_t bits = word;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int j = (lane << 5) + b;
            J.st_col[so + o] = j;
            sv[so + o] = acc[j];
            acc[j] = Sr<SR>::zero();
            o++;
        }
        msk[lane] = 0u;
        __syncwarp();
    }
    if (lane == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

template <int SR>
__global__ void __launch_bounds__(512)
k_num_cta_dense(MatView A, MatView B, CJob J, Ctl *ctl, unsigned mask, int bin, int mp) {
    using T = typename Sr<SR>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t p_boff[512];
    __shared__ T p_av[512];
    __shared__ int p_incl[512], p_blen[512], p_wsum[32];
    if (failed(ctl, mask)) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nw = mp >> 5;
    T *acc = (T *)smem;
    uint32_t *msk = (uint32_t *)(acc + mp);
    T *sv = (T *)J.st_val;
    for (int s = tid; s < mp; s += 512) acc[s] = Sr<SR>::zero();
    if (tid < 32) msk[tid] = 0u;
    __syncthreads();
    BlockProdSmem<T> ps{p_boff, p_av, p_incl, p_blen, p_wsum};
    long long nnz_acc = 0;
    const long long cnt = ctl->bin_count[bin];
    for (long long it = blockIdx.x; it < cnt; it += gridDim.x) {
        const int t = J.bins[(int64_t)bin * J.bin_cap + it];
        const int32_t i = J.R[t];
        block_products<SR>(A, B, i, ps, [&](int32_t j, T v) {
            atomicOr(&msk[j >> 5], 1u << (j & 31));
            Sr<SR>::acc(&acc[j], v);
        });
        __syncthreads();
        if (tid < 32) {
            const uint32_t word = lane < nw ? msk[lane] : 0u;
            const int pc = __popc(word);
            const int incl = warp_incl_scan<int>(pc);
            const int n = __shfl_sync(0xffffffffu, incl, 31);
            const long long so = J.soff[t];
            if (lane == 0) {
                J.slen[t] = n;
                nnz_acc += n;
            }
            int o = incl - pc;
            uint32_t bits = word;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int j = (lane << 5) + b;
                J.st_col[so + o] = j;
                sv[so + o] = acc[j];
                acc[j] = Sr<SR>::zero();
                o++;
            }
            msk[lane] = 0u;
        }
        __syncthreads();
    }
    if (tid == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// -------------------------------------------------------------- host

template <typename T>
__global__ void k_fill(T *p, int64_t n, T v) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        p[x] = v;
}

void init_dense_scratch(int sr, void *acc, uint32_t *mask, int64_t entries, int64_t words, cudaStream_t s) {
    if (entries > 0) {
        if (sr == SR_PT) launch_k(k_fill<double>, 1024, 256, 0, s, (double *)acc, entries, 0.0);
        else launch_k(k_fill<int32_t>, 1024, 256, 0, s, (int32_t *)acc, entries, MP_INF);
    }
    if (words > 0) cudaMemsetAsync(mask, 0, words * sizeof(uint32_t), s);
}

void run_size_bins(const MatView &A, const MatView &B, const CJob &J, int64_t max_rows, Ctl *ctl, unsigned mask,
                   cudaStream_t s, int num_sms) {
    if (max_rows <= 0) return;
    int64_t g = (max_rows * 32 + 255) / 256;
    if (g > num_sms * 16) g = num_sms * 16;
    if (g < 1) g = 1;
    launch_k(k_size_bins, (unsigned)g, 256, 0, s, A, B, J, ctl, mask);
}

template <int SR, int LOG_TS, int NW>
static void launch_warp_hash(const MatView &A, const MatView &B, const CJob &J, Ctl *ctl, unsigned mask, int bin,
                             cudaStream_t s, int num_sms) {
    using T = typename Sr<SR>::T;
    constexpr int TS = 1 << LOG_TS;
    const size_t smem = (size_t)NW * (TS + TS / 2) * (sizeof(T) + sizeof(int32_t));
    static bool set = false;
    if (!set) {
        cudaFuncSetAttribute(k_num_warp_hash<SR, LOG_TS, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        set = true;
    }
    int per_sm = (int)((200 * 1024) / (smem + 1024));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 2048 / (NW * 32)) per_sm = 2048 / (NW * 32);
    launch_k(k_num_warp_hash<SR, LOG_TS, NW>, num_sms * per_sm, NW * 32, smem, s, A, B, J, ctl, mask, bin);
}

template <int SR, int LOG_TS>
static void launch_cta_hash(const MatView &A, const MatView &B, const CJob &J, Ctl *ctl, unsigned mask, int bin,
                            cudaStream_t s, int num_sms) {
    using T = typename Sr<SR>::T;
    constexpr int TS = 1 << LOG_TS;
    const size_t smem = (size_t)(TS + TS / 2) * (sizeof(T) + sizeof(int32_t));
    static bool set = false;
    if (!set) {
        cudaFuncSetAttribute(k_num_cta_hash<SR, LOG_TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        set = true;
    }
    int per_sm = (int)((200 * 1024) / (smem + 8 * 1024));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    launch_k(k_num_cta_hash<SR, LOG_TS>, num_sms * per_sm, 256, smem, s, A, B, J, ctl, mask, bin);
}

template <int SR>
static void run_numeric_t(const MatView &A, const MatView &B, const CJob &J, Ctl *ctl, unsigned mask, cudaStream_t s,
                          int num_sms) {
    using T = typename Sr<SR>::T;
    if (J.dense_mode) {
        const int mp = (int)((J.m + 31) / 32 * 32);
        constexpr int NW = 8;
        const size_t smem_w = (size_t)NW * mp * sizeof(T) + NW * 32 * sizeof(uint32_t);
        static bool set_w = false;
        if (!set_w) {
            cudaFuncSetAttribute(k_num_warp_dense<SR, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
            set_w = true;
        }
        launch_k(k_num_warp_dense<SR, NW>, num_sms * 4, NW * 32, smem_w, s, A, B, J, ctl, mask, BIN_WDENSE, mp);
        const size_t smem_c = (size_t)mp * sizeof(T) + 32 * sizeof(uint32_t);
        launch_k(k_num_cta_dense<SR>, num_sms, 512, smem_c, s, A, B, J, ctl, mask, BIN_CDENSE, mp);
        return;
    }
    launch_warp_hash<SR, 6, 8>(A, B, J, ctl, mask, BIN_W64, s, num_sms);
    launch_warp_hash<SR, 7, 8>(A, B, J, ctl, mask, BIN_W128, s, num_sms);
    launch_warp_hash<SR, 8, 8>(A, B, J, ctl, mask, BIN_W256, s, num_sms);
    launch_warp_hash<SR, 9, 4>(A, B, J, ctl, mask, BIN_W512, s, num_sms);
    launch_warp_hash<SR, 10, 4>(A, B, J, ctl, mask, BIN_W1024, s, num_sms);
    launch_cta_hash<SR, 11>(A, B, J, ctl, mask, BIN_C2048, s, num_sms);
    launch_cta_hash<SR, 12>(A, B, J, ctl, mask, BIN_C4096, s, num_sms);
    launch_cta_hash<SR, 13>(A, B, J, ctl, mask, BIN_C8192, s, num_sms);
    launch_k(k_num_gdense<SR>, J.gd_ctas, 512, 0, s, A, B, J, ctl, mask, BIN_GD);
}

void run_numeric(int sr, const MatView &A, const MatView &B, const CJob &J, Ctl *ctl, unsigned mask, cudaStream_t s,
                 int num_sms) {
    if (sr == SR_PT) run_numeric_t<SR_PT>(A, B, J, ctl, mask, s, num_sms);
    else run_numeric_t<SR_MP>(A, B, J, ctl, mask, s, num_sms);
}

}  // namespace dspg
