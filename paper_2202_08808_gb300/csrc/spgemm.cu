// spgemm.cu -- recompute of selected rows of C = A B over a semiring.
//
// Section 6.1: the local product is Gustavson's row-wise algorithm; each row
// C(i,:) = (+)_k A(i,k) (x) B(k,:) is formed in a sparse accumulator.  An
// output column is a non-zero iff some product reaches it (structural
// semantics, Section 3).  Every row of R is first sized by its product bound
// ub_i = sum_k len(B_k) (capped at the column count), binned by that bound,
// and recomputed by the kernel of its bin:
//
//   bins 0-1   8 / 16 lanes per row, open-addressing hash in shared memory
//              (64 / 128 slots, load <= 1/2), several rows per warp in flight;
//   bins 2-4   a warp per row, hash of 256 .. 1024 slots;
//   bins 5-7   a CTA per row, hash of 2048 .. 8192 slots;
//   bin  8     a CTA per row, dense accumulator over all columns in global
//              memory (L2) with a presence bitmap, for the longest rows;
//   bins 9-10  when C has at most 1024 columns: dense accumulators in shared
//              memory (warp per row, or CTA per row for long rows).
//
// Products of a row are flattened over its A entries: a scan of the B-row
// lengths of the A entries held by the lanes assigns product p to A entry s
// by a binary search in the scan, so lanes stay busy even when B rows are
// short.  Each row is written straight into C (in place when it fits the
// row's capacity, otherwise at the arena tail) in whatever column order its
// kernel produces it: like the paper's local rows, C's rows carry no column
// order (the thread-merge, dense and small hash rows happen to come out
// sorted; longer hash rows come out in table order), and reads sort them.  For the static
// product the sizing pass lays C out afresh with room for the bound.
// (+,.) accumulates with double atomics (the summation order varies; the
// library's tolerance covers any order), (min,+) with atomicMin
// (order-free, bit-exact).
#include <algorithm>

#include <cooperative_groups.h>

#include "estimator.cuh"
#include "internal.h"

namespace dspg {

namespace cg = cooperative_groups;

template <int SR>
struct Sr;
// mul and add round each operation separately; fma(a, b, c) = c (+) a (x) b
// in one step, which for (+,.) is a fused multiply-add: one rounding instead
// of two, and one instruction of the double-precision pipe (whose rate on
// this GPU is 1/64 of single precision) instead of two.
template <>
struct Sr<SR_PT> {
    using T = double;
    __device__ static T zero() { return 0.0; }
    __device__ static T mul(T a, T b) { return __dmul_rn(a, b); }
    __device__ static T add(T a, T b) { return __dadd_rn(a, b); }
    __device__ static T fma(T a, T b, T c) { return __fma_rn(a, b, c); }
    __device__ static void acc(T *p, T v) { atomicAdd(p, v); }
};
template <>
struct Sr<SR_MP> {
    using T = int32_t;
    __device__ static T zero() { return MP_INF; }
    __device__ static T mul(T a, T b) { return a + b; }
    __device__ static T add(T a, T b) { return a < b ? a : b; }
    __device__ static T fma(T a, T b, T c) { return add(c, mul(a, b)); }
    __device__ static void acc(T *p, T v) { atomicMin(p, v); }
};

enum {
    BIN_T8 = 0, BIN_G8, BIN_G16, BIN_W128, BIN_W256, BIN_W512, BIN_W1024,
    BIN_C2048, BIN_C4096, BIN_C8192, BIN_C16384,
    BIN_GD,
    BIN_WDENSE, BIN_CDENSE, BIN_DSPLIT,
    BIN_T64,  // thread merge, rows whose bound is above the tuned staging bound (up to MERGE_UB)
    BIN_K2, BIN_K4, BIN_K8, BIN_K8L,  // cluster tables: 2, 4, 8 CTAs x 8192 slots, 8 x 16384
    BIN_S64, BIN_S128, BIN_S256,      // group sort: 8, 16, 32 lanes, up to 64, 128, 256 products
    BIN_COUNT
};
static_assert(BIN_COUNT <= NBINS, "bin counters");

__device__ __forceinline__ long long atomic_add_ll2(long long *p, long long v) {
    return (long long)atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

// ------------------------------------------------------------- sizing

constexpr int MERGE_K = 8;      // A rows up to this length can be merged by one thread
constexpr int MERGE_UB = 64;    // ... when their product bound is at most this (the tuning
                                // may lower it: the kernel stages the tuned bound per thread)

// The hash (or global dense) bin for a table of at least `need` slots under
// the job's thresholds.
// A table or staging area too small for a row although the sizing bound it:
// reported as ST_TIMEOUT, with the bin and a row for the error message.
__device__ __forceinline__ void report_overflow(Ctl *ctl, int bin, int32_t i, const MatView &A, const MatView &B) {
    long long ub = 0;
    for (int a = 0; a < A.len[i]; a++) ub += B.len[A.col[A.off[i] + a]];
    ctl->timeout_bin = bin + 1;
    ctl->timeout_row = i;
    ctl->timeout_ub = ub;
    set_status(ctl, ST_TIMEOUT);
}

// ub: the row's uncapped product bound.  Rows beyond a CTA's table go to a
// cluster's table only while their products are not far more than its
// slots (ub <= 2 * need) and the row is sparse (need <= m / 8): a row whose
// products collide many times over, or that fills much of C's width (as in
// small squares of skewed graphs), is cheaper in the global dense
// accumulator, which every CTA of a cluster would otherwise read the whole
// row's products for.
__device__ __forceinline__ int pick_table_bin(long long need, const CJob &J, long long ub) {
    need <<= J.table_shift;
    if (need <= 32 && J.lanes_min <= 8) return BIN_G8;
    if (need <= 64 && J.lanes_min <= 16) return BIN_G16;
    if (need <= J.warp_max) {
        if (need <= 128) return BIN_W128;
        if (need <= 256) return BIN_W256;
        if (need <= 512) return BIN_W512;
        return BIN_W1024;
    }
    if (need <= J.cta_max) {
        if (need <= 2048) return BIN_C2048;
        if (need <= 4096) return BIN_C4096;
        if (need <= 8192) return BIN_C8192;
        return BIN_C16384;
    }
    if (ub > 2 * need || need * 8 > J.m) return BIN_GD;
    if (need <= 2 * 8192) return BIN_K2;
    if (need <= 4 * 8192) return BIN_K4;
    if (need <= 8 * 8192) return BIN_K8;
    if (need <= 8 * 16384) return BIN_K8L;
    return BIN_GD;
}

// The bin of a row from its capped bound and A-row length (and, when the
// tables are sized by an exact count, that count).  A table is never smaller
// than the size it is given, so with the bound or an exact count no choice
// of thresholds can make a table overflow.
// With dense accumulators (few columns) the work of a row is its A entries
// (each gathers a B row) and its products, not the capped bound: a warp for
// short rows, else a CTA (rows with very many products are split later).
constexpr int DENSE_WARP_A = 64;
// Rows merged by one thread: at most tm_k A entries and at most MERGE_UB
// products (the uncapped bound: it is what the thread stages), in the first
// kernel while the bound is within the tuned staging size tm_ub.
__device__ __forceinline__ bool merge_row(int alen, long long ub, const CJob &J) {
    return alen <= J.tm_k && ub <= MERGE_UB;
}

// Rows sorted in registers by a group of lanes: at most sort_max products
// (the uncapped bound, which is what the group holds), in the smallest of
// the three group sizes that holds them.
// The group sort packs a column with a product index (up to 8 bits) into 32.
__device__ __forceinline__ bool sort_cols_ok(long long m) { return m < (1LL << 24) - 1; }
__device__ __forceinline__ bool sort_row(long long ub, const CJob &J) { return ub <= J.sort_max && sort_cols_ok(J.m); }

// Rows whose kernel holds all their products (no table to size).
__device__ __forceinline__ bool small_row(int alen, long long ub, const CJob &J) {
    return sort_row(ub, J) || merge_row(alen, ub, J);
}

__device__ __forceinline__ int pick_bin(long long ubc, int alen, const CJob &J, long long table_need,
                                        long long ub) {
    if (sort_row(ub, J)) return ub <= 64 ? BIN_S64 : (ub <= 128 ? BIN_S128 : BIN_S256);
    if (merge_row(alen, ub, J)) return ub <= J.tm_ub ? BIN_T8 : BIN_T64;
    if (J.dense_mode) return (alen <= DENSE_WARP_A && ub <= 4096) ? BIN_WDENSE : BIN_CDENSE;
    return pick_table_bin(table_need, J, ub);
}

// A row whose bin b is not launched by this pipeline goes to the global
// dense bin, which takes rows of any size and width; b is recorded so that
// the host launches it from the next captured pipeline on.
__device__ __forceinline__ int gate_bin(const CJob &J, Ctl *ctl, int b) {
    if (b < 0 || ((J.bin_on >> b) & 1ull)) return b;
    atomicOr(&ctl->bins_wanted, 1ull << b);
    return BIN_GD;
}

// Append the calling lanes' rows i (of C) to their bins b (b < 0: none), one
// atomic per distinct bin in the warp.
__device__ __forceinline__ void append_bins(const CJob &J, Ctl *ctl, int b, int32_t i) {
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    long long bb = 0;
    if (b >= 0 && lane == leader) bb = atomic_add_ll2(&ctl->bin_count[b], __popc(peers));
    bb = __shfl_sync(0xffffffffu, bb, leader);
    const long long slot = bb + __popc(peers & lanemask_lt());
    if (b >= 0 && dcheck(ctl, slot < J.bin_cap, DBG_BIN_SLOT, i)) J.bins[(int64_t)b * J.bin_cap + slot] = i;
}

constexpr int SIZE_SHORT = 64;   // A rows up to this length are sized by one thread,
constexpr int SIZE_LONG = 512;   // up to this by a warp, longer ones by the whole block
constexpr long long SPLIT_MIN = 8192;  // dense mode: rows with more products, or with more than
constexpr int SPLIT_A = 256;           // SPLIT_A A entries, are split in chunks (k_num_dsplit)
constexpr int SPLIT_CHUNK = 2048;      // A entries per work item of a split row
constexpr int DS_NT = 256;             // threads of a split-kernel block

// Dense mode: claim a split slot for a row with very many products; false
// when all slots are taken (the row then goes to the CTA dense bin).
__device__ __forceinline__ bool claim_split(const CJob &J, Ctl *ctl, int32_t i) {
    const long long slot = atomic_add_ll2(&ctl->bin_count[BIN_DSPLIT], 1);
    if (slot >= J.sp_rows) return false;
    J.bins[(int64_t)BIN_DSPLIT * J.bin_cap + slot] = i;
    return true;
}

__device__ __forceinline__ bool wants_est(const CJob &J, long long ub, long long ubc, bool t8) {
    return ub > 0 && J.sizing == SIZE_LEARNED && !t8 && !J.dense_mode && ubc > J.est_min;
}

__device__ __forceinline__ void push_est(const CJob &J, Ctl *ctl, int32_t i, int alen, long long bmax, long long ub) {
    const int4 e = make_int4(i, alen, (int)bmax, (int)(ub < 0x7fffffffLL ? ub : 0x7fffffffLL));
    J.est[atomic_add_ll2(&ctl->n_est, 1)] = e;
}

// A row of R with more than SIZE_LONG A entries, sized by the whole block:
// the B-row lengths summed with several loads in flight per thread, then
// the row is binned as in k_size_bins (by thread 0).  t indexes R.
__device__ __forceinline__ void size_long_row(const MatView &A, const MatView &B, const MatView &C, const CJob &J,
                                              Ctl *ctl, long long t, long long *s_sum, long long *s_max) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int nw = blockDim.x >> 5;
    const int32_t i = __ldcg(J.R + t);
    const int64_t aoff = __ldcg(A.off + i);
    const int alen = __ldcg(A.len + i);
    long long sm = 0, mx = 0;
    for (int a0 = 0; a0 < alen; a0 += (int)blockDim.x * 4) {
        long long l[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int a = a0 + u * (int)blockDim.x + tid;
            const int32_t k = a < alen ? __ldcg(A.col + aoff + a) : 0;
            l[u] = a < alen && dcheck(ctl, k >= 0 && k < B.nrows, DBG_B_ROW, aoff + a) ? (long long)__ldcg(B.len + k) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            sm += l[u];
            mx = l[u] > mx ? l[u] : mx;
        }
    }
    sm = warp_sum<long long>(sm);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const long long y = __shfl_xor_sync(0xffffffffu, mx, d);
        mx = y > mx ? y : mx;
    }
    if (lane == 0) {
        s_sum[w] = sm;
        s_max[w] = mx;
    }
    __syncthreads();
    if (tid == 0) {
        long long ub = 0, bmax = 0;
        for (int k = 0; k < nw; k++) {
            ub += s_sum[k];
            bmax = s_max[k] > bmax ? s_max[k] : bmax;
        }
        const long long ubc = ub < J.m ? ub : J.m;
        if (J.static_mode) {
            const int32_t c = slack_cap(ubc, J.slack_min, J.slack_div);
            const long long d = atomic_add_ll2(C.top, c);
            C.off[i] = d;
            C.cap[i] = c;
            C.len[i] = 0;
            if (d + c > C.arena_cap) set_status(ctl, ST_C_ARENA);
        } else if (J.sizing != SIZE_COUNT) {
            if (ub == 0) C.len[i] = 0;
        }
        const bool t8 = small_row(alen, ub, J);
        if (wants_est(J, ub, ubc, t8)) {
            push_est(J, ctl, i, alen, bmax, ub);
        } else if (ub > 0) {
            const long long need = J.sizing == SIZE_COUNT ? (long long)C.len[i] : ubc;
            const int b = gate_bin(J, ctl, pick_bin(ubc, alen, J, need, ub));
            if (!(b == BIN_CDENSE && (ub > SPLIT_MIN || alen > SPLIT_A) && claim_split(J, ctl, i)))
                J.bins[(int64_t)b * J.bin_cap + atomic_add_ll2(&ctl->bin_count[b], 1)] = i;
        }
        if (J.sizing != SIZE_COUNT) {
            atomic_add_ll2(&ctl->products, ub);
            atomic_add_ll2(&ctl->a_entries, alen);
        }
    }
    __syncthreads();
}

// One thread per row of R sums the B-row lengths of its A entries; rows
// longer than SIZE_SHORT are listed and summed by a whole warp each (the
// block's warps share the list), rows longer than SIZE_LONG by the whole
// block at the end of its round; then the warp hands out bin slots (and,
// for the static product, the row's place in a fresh C) with one atomic per
// counter.  A block takes 256 rows a round, or 32 when R has fewer than 32
// rows a block: a small R of long rows (the hubs a skewed graph's batch
// touches) then spreads over as many SMs as it can instead of queueing in a
// few warps (with 64 rows a block the 52 k rows of a stencil step took 21
// instead of 13 us: four times the blocks, each mostly idle).  With SIZE_COUNT the tables are sized by C.len (an exact count from
// a count_only pass); with SIZE_LEARNED rows whose bound exceeds est_min go
// to the estimate list instead of a bin.
__global__ void __launch_bounds__(256) k_size_bins(MatView A, MatView B, MatView C, CJob J, Ctl *ctl, unsigned mask) {
    pdl_begin();
    __shared__ long long s_long[256];  // this block's rows (indices into R) with long A rows
    __shared__ long long s_sum[8], s_max[8];
    __shared__ int s_nlong, s_nmid;
    __shared__ int s_mid[256];          // this round's rows (thread index) of more than SIZE_SHORT A entries
    __shared__ long long s_moff[256], s_mub[256], s_mmax[256];
    __shared__ int s_mlen[256];
    if (failed(ctl, mask)) return;
    const long long nR = ctl->n_affected;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long per = (nR + gridDim.x - 1) / gridDim.x;
    const int CH = per >= 32 ? 256 : 32;  // 32 rows a block only when R is small against the grid
    long long prod_acc = 0, a_acc = 0;
    if (threadIdx.x == 0) {
        s_nlong = 0;
        s_nmid = 0;
    }
    __syncthreads();
    for (long long base = (long long)blockIdx.x * CH; base < nR; base += (long long)gridDim.x * CH) {
        const long long t = base + threadIdx.x;
        bool valid = (int)threadIdx.x < CH && t < nR;
        // the row structure was just rewritten by the commit: read through L2
        // (ld.global.cg), not a possibly stale L1 line
        int32_t i = valid ? __ldcg(J.R + t) : 0;
        if (valid && !dcheck(ctl, i >= 0 && i < A.nrows, DBG_R_ROW, t)) {
            valid = false;
            i = 0;
        }
        int64_t aoff = valid ? __ldcg(A.off + i) : 0;
        int alen = valid ? __ldcg(A.len + i) : 0;
        if (valid && !dcheck(ctl, aoff >= 0 && alen >= 0 && aoff + alen <= A.arena_cap, DBG_R_ROW, i)) {
            valid = false;
            aoff = 0;
            alen = 0;
        }
        // dense accumulators: a row with more than SPLIT_A A entries is split,
        // whatever its product count, so it needs no sum (its products are
        // counted by the split kernel); its bound for the static layout is m
        const bool direct = valid && J.dense_mode && alen > SPLIT_A && claim_split(J, ctl, i);
        if (valid && !direct && alen > SIZE_LONG) {  // the whole block sizes this row below
            s_long[atomicAdd(&s_nlong, 1)] = t;
            valid = false;
        }
        const bool lng = alen > SIZE_SHORT && !direct;
        long long ub = direct ? J.m : 0, bmax = 0;
        if (valid && !lng && !direct)
#pragma unroll 8
            for (int a = 0; a < alen; a++) {
                const int32_t k = __ldcg(A.col + aoff + a);
                const long long l = dcheck(ctl, k >= 0 && k < B.nrows, DBG_B_ROW, aoff + a) ? __ldcg(B.len + k) : 0;
                ub += l;
                bmax = l > bmax ? l : bmax;
            }
        if (valid && lng) {
            const int k = atomicAdd(&s_nmid, 1);
            s_mid[k] = (int)threadIdx.x;
            s_moff[threadIdx.x] = aoff;
            s_mlen[threadIdx.x] = alen;
        }
        // the listed rows, a warp each, all of the block's warps at once (a
        // round without such rows skips the pass and its second barrier)
        const int nmid = __syncthreads_or(valid && lng) ? s_nmid : 0;
        for (int k = warp; k < nmid; k += (int)(blockDim.x >> 5)) {
            const int r = s_mid[k];
            const int64_t o = s_moff[r];
            const int l = s_mlen[r];
            long long sm = 0, mx = 0;
#pragma unroll 4
            for (int a = lane; a < l; a += 32) {
                const int32_t k = __ldcg(A.col + o + a);
                const long long x = dcheck(ctl, k >= 0 && k < B.nrows, DBG_B_ROW, o + a) ? __ldcg(B.len + k) : 0;
                sm += x;
                mx = x > mx ? x : mx;
            }
            sm = warp_sum<long long>(sm);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const long long y = __shfl_xor_sync(0xffffffffu, mx, d);
                mx = y > mx ? y : mx;
            }
            if (lane == 0) {
                s_mub[r] = sm;
                s_mmax[r] = mx;
            }
        }
        if (nmid > 0) __syncthreads();
        if (valid && lng) {
            ub = s_mub[threadIdx.x];
            bmax = s_mmax[threadIdx.x];
        }
        const long long ubc = ub < J.m ? ub : J.m;
        if (J.static_mode) {
            const int32_t c = valid ? slack_cap(ubc, J.slack_min, J.slack_div) : 0;
            const long long d = warp_fetch_add(C.top, c);
            if (valid) {
                C.off[i] = d;
                C.cap[i] = c;
                C.len[i] = 0;
                if (d + c > C.arena_cap) set_status(ctl, ST_C_ARENA);
            }
        } else if (valid && J.sizing != SIZE_COUNT) {
            if (ub == 0) C.len[i] = 0;  // no products: the row becomes empty
        }
        const bool t8 = small_row(alen, ub, J);
        const bool to_est = valid && wants_est(J, ub, ubc, t8);
        long long need = ubc;
        if (J.sizing == SIZE_COUNT && valid) need = C.len[i];
        int b = (valid && ub > 0 && !to_est && !direct) ? gate_bin(J, ctl, pick_bin(ubc, alen, J, need, ub)) : -1;
        if (b == BIN_CDENSE && (ub > SPLIT_MIN || alen > SPLIT_A) && claim_split(J, ctl, i)) b = -1;
        append_bins(J, ctl, b, i);
        if (to_est) push_est(J, ctl, i, alen, bmax, ub);
        if (J.sizing != SIZE_COUNT && valid) {
            if (!direct) prod_acc += ub;
            a_acc += alen;
        }
        __syncthreads();
        const int nl = s_nlong;
        for (int k = 0; k < nl; k++) size_long_row(A, B, C, J, ctl, s_long[k], s_sum, s_max);
        __syncthreads();
        if (threadIdx.x == 0) {
            s_nlong = 0;
            s_nmid = 0;
        }
        __syncthreads();
    }
    prod_acc = warp_sum<long long>(prod_acc);
    a_acc = warp_sum<long long>(a_acc);
    if (lane == 0) {
        if (prod_acc) atomic_add_ll2(&ctl->products, prod_acc);
        if (a_acc) atomic_add_ll2(&ctl->a_entries, a_acc);
    }
}

// The learned sizing: one thread per row of the estimate list evaluates the
// network (weights as floats in shared memory), sizes the row's table by the
// prediction times (1 + margin), clamped to [max len(B_k), bound], and bins it.
__global__ void __launch_bounds__(128) k_est_bins(CJob J, Ctl *ctl, unsigned mask) {
    pdl_begin();
    extern __shared__ __align__(16) float W[];
    if (failed(ctl, mask)) return;
    for (int k = threadIdx.x; k < EST_PARAMS; k += blockDim.x) W[k] = bf16_bits_to_float(J.est_w[k]);
    __syncthreads();
    const long long cnt = ctl->n_est;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < cnt; base += (long long)gridDim.x * blockDim.x) {
        const long long q = base + threadIdx.x;
        int b = -1;
        int32_t i = 0;
        if (q < cnt) {
            const int4 e = __ldcg(J.est + q);
            i = e.x;
            float x[EST_IN];
            est_features(x, e.y, e.w, e.z);
            const float o = est_forward(W, x);
            const float pred = exp2f(fminf(o, 40.0f)) - 1.0f;
            long long need = (long long)ceilf(pred * (1.0f + J.est_margin));
            const long long ubc = e.w < J.m ? e.w : J.m;
            if (need > ubc) need = ubc;
            if (need < e.z) need = e.z;
            if (need < 1) need = 1;
            b = gate_bin(J, ctl, pick_table_bin(need, J, (long long)e.w));
        }
        append_bins(J, ctl, b, i);
    }
}

// ------------------------------------------------------------ output

// Where row i of C goes when it has n entries: its own place when n fits
// its capacity (always in the static layout), else a fresh place at the
// arena tail.  Returns -1 when the tail is exhausted: the status bit makes
// the host rebuild C with more room and recompute R again.
__device__ __forceinline__ int64_t c_row_dest(const MatView &C, const CJob &J, Ctl *ctl, int32_t i, int n) {
    if (J.count_only) {  // exact sizing pass: record the length, write nothing
        C.len[i] = n;
        return -1;
    }
    const int32_t cap = C.cap[i];
    if (J.static_mode || n <= cap) {
        const int64_t o = C.off[i];
        if (!dcheck(ctl, o >= 0 && o + n <= C.arena_cap && (J.static_mode || n <= cap), DBG_C_ROOM, i)) return -1;
        return o;
    }
    const int32_t c = slack_cap(n, J.slack_min, J.slack_div);
    const long long d = atomic_add_ll2(C.top, c);
    if (d + c > C.arena_cap) {
        set_status(ctl, ST_C_ARENA);
        return -1;
    }
    C.off[i] = d;
    C.cap[i] = c;
    atomic_add_ll2(&ctl->c_reloc, 1);
    return d;
}

// --------------------------------------------------- product generators

constexpr int PU = 4;  // products per lane whose B loads are issued together

// Calls emit(j, a (x) b) for every product of row i; the G lanes of one
// group (G = 8, 16 or 32 consecutive lanes, mask gmask) share the work.
// (Only the A entries a_begin, a_begin + a_step, ... below a_end, in groups
// of G, when given: the warps of a CTA can share a row this way without
// block-wide barriers.)
template <int SR, int G, class F>
__device__ __forceinline__ void group_products(const MatView &A, const MatView &B, int32_t i, unsigned gmask,
                                               F emit, int a_begin = 0, int a_end = -1, int a_step = G) {
    using T = typename Sr<SR>::T;
    const int gl = threadIdx.x & (G - 1);
    const int64_t aoff = A.off[i];
    const int alen = a_end >= 0 ? a_end : A.len[i];
    const T *Av = (const T *)A.val;
    const T *Bv = (const T *)B.val;
    for (int a0 = a_begin; a0 < alen; a0 += a_step) {
        const int ai = a0 + gl;
        int blen = 0;
        int64_t boff = 0;
        T av = T(0);
        if (ai < alen) {
            const int32_t k = A.col[aoff + ai];
            av = Av[aoff + ai];
            boff = B.off[k];
            blen = B.len[k];
        }
        int incl = blen;
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const int o = __shfl_up_sync(gmask, incl, d, G);
            if (gl >= d) incl += o;
        }
        const int total = __shfl_sync(gmask, incl, G - 1, G);
        // PU products per lane per round: their B entries are all loaded
        // before any is accumulated, so PU loads per lane are in flight
        for (int base = 0; base < total; base += G * PU) {
            int64_t q[PU];
            T a[PU];
#pragma unroll
            for (int u = 0; u < PU; u++) {
                const int p = base + u * G + gl;
                int s = 0;
#pragma unroll
                for (int step = G / 2; step > 0; step >>= 1) {
                    const int v = __shfl_sync(gmask, incl, s + step - 1, G);
                    if (v <= p) s += step;
                }
                const int64_t bo = __shfl_sync(gmask, boff, s, G);
                a[u] = __shfl_sync(gmask, av, s, G);
                const int excl = __shfl_sync(gmask, incl, s, G) - __shfl_sync(gmask, blen, s, G);
                q[u] = p < total ? bo + (p - excl) : -1;
            }
            int32_t c[PU];
            T b[PU];
#pragma unroll
            for (int u = 0; u < PU; u++)
                if (q[u] >= 0) {
                    c[u] = __ldg(B.col + q[u]);
                    b[u] = __ldg(Bv + q[u]);
                }
#pragma unroll
            for (int u = 0; u < PU; u++)
                if (q[u] >= 0) emit(c[u], Sr<SR>::mul(a[u], b[u]));
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
// block sharing the work (with parts > 1: the share `part` of them, the
// CTAs of a cluster taking one part each), and of those only the ones whose
// column passes keep (the others load no value).  Must be called by the
// whole block.
struct KeepAll {
    __device__ bool operator()(int32_t) const { return true; }
};

template <int SR, class F, class K = KeepAll>
__device__ __forceinline__ void block_products(const MatView &A, const MatView &B, int32_t i,
                                               BlockProdSmem<typename Sr<SR>::T> sm, F emit, int part = 0,
                                               int parts = 1, K keep = K()) {
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
        // PU loads per thread in flight, as above; with parts > 1 the rounds
        // of a chunk's products are dealt out to the parts in turn
        for (int base = part * nt * PU; base < total; base += parts * nt * PU) {
            // each thread takes PU consecutive products: one search for the
            // first, then a step to the next B row where the run crosses one
            int64_t q[PU];
            T a[PU];
            const int p0 = base + tid * PU;
            int s = p0 < total ? (int)upper_bound_dev<int>(sm.incl, 0, nt, p0) : 0;
#pragma unroll
            for (int u = 0; u < PU; u++) {
                const int p = p0 + u;
                q[u] = -1;
                if (p < total) {
                    while (sm.incl[s] <= p) s++;  // past the B rows that end before p (empty ones too)
                    const int excl = sm.incl[s] - sm.blen[s];
                    q[u] = sm.boff[s] + (p - excl);
                    a[u] = sm.av[s];
                }
            }
            int32_t c[PU];
            T b[PU];
#pragma unroll
            for (int u = 0; u < PU; u++)
                if (q[u] >= 0) c[u] = __ldg(B.col + q[u]);
#pragma unroll
            for (int u = 0; u < PU; u++)
                if (q[u] >= 0) {
                    if (keep(c[u])) b[u] = __ldg(Bv + q[u]);
                    else q[u] = -1;  // another CTA's column: no value load, no product
                }
#pragma unroll
            for (int u = 0; u < PU; u++)
                if (q[u] >= 0) emit(c[u], Sr<SR>::mul(a[u], b[u]));
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------- hash table

// Accumulates v into the slot of column j: 1 when this call claimed the
// slot (a new column of the row), 0 when the column was there, -1 when the
// table is full.  Probing is triangular (steps 1, 2, 3, ...), which visits
// every slot of a power-of-two table and, unlike linear probing, does not
// build long runs of occupied slots as the table fills.
// With CAS_FIRST every probe is a compare-and-swap (one round trip per
// probe instead of a load and then a swap: for tables in another CTA's
// shared memory).  probe0 > 0 continues a probe sequence from that step.
template <int LOG_TS, typename T, int SR, bool CAS_FIRST = false>
__device__ __forceinline__ int hash_acc_from(int32_t *keys, T *vals, uint32_t h, int32_t j, T v, int probe0 = 0) {
    constexpr int TS = 1 << LOG_TS;
    h = (h + (uint32_t)(probe0 * (probe0 + 1) / 2)) & (TS - 1);
    for (int probe = probe0; probe < TS; probe++) {
        if constexpr (CAS_FIRST) {
            const int32_t old = atomicCAS(&keys[h], -1, j);
            if (old == -1 || old == j) {
                Sr<SR>::acc(&vals[h], v);
                return old == -1 ? 1 : 0;
            }
        } else {
            const int32_t k = ((volatile int32_t *)keys)[h];
            if (k == j) {
                Sr<SR>::acc(&vals[h], v);
                return 0;
            }
            if (k == -1) {
                const int32_t old = atomicCAS(&keys[h], -1, j);
                if (old == -1 || old == j) {
                    Sr<SR>::acc(&vals[h], v);
                    return old == -1 ? 1 : 0;
                }
            }
        }
        h = (h + probe + 1) & (TS - 1);
    }
    return -1;  // table full: cannot happen when the bin bound holds
}

template <int LOG_TS, typename T, int SR>
__device__ __forceinline__ int hash_acc(int32_t *keys, T *vals, int32_t j, T v) {
    return hash_acc_from<LOG_TS, T, SR>(keys, vals, ((uint32_t)j * 2654435761u) >> (32 - LOG_TS), j, v);
}

// ---------------------------------------------------- thread merge kernel

// One thread per row with at most MERGE_K A entries and at most MERGE_UB
// products.  The row's B entries (columns and values) are first copied into
// shared memory with asynchronous copies (cp.async: every copy of the row in
// flight at once, no registers held), then the ≤ MERGE_K sorted B rows are
// merged like sorted lists, a cursor each, entirely in shared memory: every
// output column comes out in ascending order with its products folded in
// ascending k, so no table and no sort are needed.  Shared memory is laid
// out [entry][thread], so the lanes of a warp never share a bank.  Writes go
// to the row's place while they fit its capacity; a row that outgrows it is
// counted to the end, moved to the arena tail and merged again (rare).
constexpr int TM_NT = 128;  // threads per block of the merge kernel

__device__ __forceinline__ void cp_async_4(void *dst_smem, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(void *dst_smem, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int SR, int K>
__device__ __forceinline__ int merge_rows_smem(const int32_t *scol, const typename Sr<SR>::T *sval,
                                               const typename Sr<SR>::T *av, const int *start, const int *blen,
                                               int alen, int32_t *out_col, typename Sr<SR>::T *out_val, int limit) {
    using T = typename Sr<SR>::T;
    int pos[K], end[K];
    int32_t head[K];
#pragma unroll
    for (int s = 0; s < K; s++) {
        pos[s] = start[s];
        end[s] = start[s] + (s < alen ? blen[s] : 0);
        head[s] = pos[s] < end[s] ? scol[pos[s] * TM_NT] : 0x7fffffff;
    }
    int n = 0;
    while (true) {
        int32_t j = head[0];
#pragma unroll
        for (int s = 1; s < K; s++) j = min(j, head[s]);
        if (j == 0x7fffffff) break;
        T acc = Sr<SR>::zero();
#pragma unroll
        for (int s = 0; s < K; s++) {
            if (head[s] == j) {
                acc = Sr<SR>::fma(av[s], sval[pos[s] * TM_NT], acc);
                pos[s]++;
                head[s] = pos[s] < end[s] ? scol[pos[s] * TM_NT] : 0x7fffffff;
            }
        }
        if (n < limit) {
            out_col[n] = j;
            out_val[n] = acc;
        }
        n++;
    }
    return n;
}

template <int SR, int K>
__global__ void __launch_bounds__(TM_NT)
k_num_thread_merge(MatView A, MatView B, MatView C, CJob J, Ctl *ctl, unsigned mask, int bin, int UB) {
    pdl_begin();
    using T = typename Sr<SR>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    if (failed(ctl, mask)) return;
    // UB: staged entries per thread (the bin's product bound)
    T *svals = (T *)smem + threadIdx.x;                              // [UB][TM_NT] values
    int32_t *scols = (int32_t *)((T *)smem + UB * TM_NT) + threadIdx.x;  // [UB][TM_NT] columns
    const T *Av = (const T *)A.val;
    const T *Bv = (const T *)B.val;
    T *Cv = (T *)C.val;
    long long nnz_acc = 0;
    const long long cnt = ctl->bin_count[bin];
    for (long long it = (long long)blockIdx.x * TM_NT + threadIdx.x; it < cnt; it += (long long)gridDim.x * TM_NT) {
        int32_t i = J.bins[(int64_t)bin * J.bin_cap + it];
        if (!dcheck(ctl, i >= 0 && i < A.nrows, DBG_R_ROW, it)) i = 0;  // debug build: a bad list entry fails the batch
        const int64_t aoff = A.off[i];
        const int alen = A.len[i];
        const int64_t off = C.off[i];  // independent of the A and B loads: issued with them
        const int cap = J.count_only ? 0 : (J.static_mode ? 0x7fffffff : C.cap[i]);
        T av[K];
        int64_t boff[K];
        int blen[K], start[K];
#pragma unroll
        for (int s = 0; s < K; s++) {
            av[s] = T(0);
            boff[s] = 0;
            blen[s] = 0;
            if (s < alen) {
                const int32_t k = A.col[aoff + s];
                if (dcheck(ctl, k >= 0 && k < B.nrows, DBG_B_ROW, aoff + s)) {
                    av[s] = Av[aoff + s];
                    boff[s] = B.off[k];
                    blen[s] = B.len[k];
                }
            }
        }
        int tot = 0;
#pragma unroll
        for (int s = 0; s < K; s++) {
            start[s] = tot;
            tot += blen[s];
        }
        if (tot > UB) {  // the sizing pass guarantees tot <= UB; guard the buffer anyway
            report_overflow(ctl, bin, i, A, B);
            continue;
        }
#pragma unroll
        for (int s = 0; s < K; s++)
            for (int q = 0; q < blen[s]; q++) {
                cp_async_4(&scols[(start[s] + q) * TM_NT], B.col + boff[s] + q);
                if (sizeof(T) == 8) cp_async_8(&svals[(start[s] + q) * TM_NT], Bv + boff[s] + q);
                else cp_async_4(&svals[(start[s] + q) * TM_NT], Bv + boff[s] + q);
            }
        cp_async_wait_all();
        const int n = merge_rows_smem<SR, K>(scols, svals, av, start, blen, alen, C.col + off, Cv + off, cap);
        bool ok = true;
        if (J.count_only) {
            C.len[i] = n;
            ok = false;
        } else if (n > cap) {
            const int64_t d = c_row_dest(C, J, ctl, i, n);
            if (d >= 0) merge_rows_smem<SR, K>(scols, svals, av, start, blen, alen, C.col + d, Cv + d, n);
            else ok = false;
        }
        if (ok) C.len[i] = n;
        nnz_acc += n;
    }
    nnz_acc = warp_sum<long long>(nnz_acc);
    if ((threadIdx.x & 31) == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// ---------------------------------------------------- group sort kernel

// G lanes per row (32 / G rows per warp) for rows of at most N = G * GS_EPL
// products.  Product p of the row (A entries in order, each B row in order)
// has slot p of the group's shared memory, filled by lane p % G: its B
// column and value arrive by asynchronous copies (all of the row's copies
// in flight at once, lane after lane along each B row), its A value by a
// store.  The lane then holds the word (column << log2 N | p) as its
// register p / G.  The group sorts its N words with a bitonic network of
// integer min/max (partners inside a lane's registers for the short
// strides, in another lane of the group, by shuffles, for the long ones; a
// run that descends is sorted ascending on complemented words), folds each
// run of equal columns (inside a lane, then across lanes with a segmented
// scan), multiplying out the slots that the sorted words name, and writes
// the row in column order.  The words are distinct, so the sort needs no
// tie rule, and it has no data-dependent branches.  Columns must leave room
// for the slot bits (sort_cols_ok).
constexpr int GS_EPL = 8;
constexpr int GS_NT = 256;

template <int SR, int G>
__global__ void __launch_bounds__(GS_NT, 4)
k_num_group_sort(MatView A, MatView B, MatView C, CJob J, Ctl *ctl, unsigned mask, int bin) {
    pdl_begin();
    using T = typename Sr<SR>::T;
    constexpr int N = G * GS_EPL;
    constexpr int LOGN = G == 8 ? 6 : (G == 16 ? 7 : 8);
    static_assert((1 << LOGN) == N, "words per group");
    constexpr uint32_t PAD = 0xffffffffu;  // empty word: sorts last, never written
    // the group's N product slots: B column, A value, B value
    __shared__ int32_t s_col[GS_NT / G * N];
    __shared__ T s_a[GS_NT / G * N];
    __shared__ T s_b[GS_NT / G * N];
    if (__any_sync(0xffffffffu, failed(ctl, mask))) return;  // a warp leaves as a whole
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1), gw = lane / G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (gw * G));
    int32_t *scol = s_col + (threadIdx.x / G) * N;
    T *sa = s_a + (threadIdx.x / G) * N;
    T *sb = s_b + (threadIdx.x / G) * N;
    const long long ngroups = ((long long)gridDim.x * GS_NT) / G;
    const T *Av = (const T *)A.val;
    const T *Bv = (const T *)B.val;
    T *Cv = (T *)C.val;
    long long nnz_acc = 0;
    const long long cnt = ctl->bin_count[bin];
    for (long long it = ((long long)blockIdx.x * GS_NT + threadIdx.x) / G; it < cnt; it += ngroups) {
        int32_t i = J.bins[(int64_t)bin * J.bin_cap + it];
        if (!dcheck(ctl, i >= 0 && i < A.nrows, DBG_R_ROW, it)) i = 0;  // debug build: a bad list entry fails the batch
        const int64_t aoff = A.off[i];
        const int alen = A.len[i];
        int base = 0;  // products placed so far (the same on every lane of the group)
        bool over = false;
        for (int a0 = 0; a0 < alen; a0 += G) {
            const int ai = a0 + gl;
            int blen = 0;
            int64_t boff = 0;
            T av = T(0);
            if (ai < alen) {
                const int32_t k = A.col[aoff + ai];
                if (dcheck(ctl, k >= 0 && k < B.nrows, DBG_B_ROW, aoff + ai)) {
                    av = Av[aoff + ai];
                    boff = B.off[k];
                    blen = B.len[k];
                }
            }
            int incl = blen;
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
                const int o = __shfl_up_sync(gmask, incl, d, G);
                if (gl >= d) incl += o;
            }
            const int total = __shfl_sync(gmask, incl, G - 1, G);
            if (base + total > N) {  // the bin's bound rules this out; guard the slots anyway
                over = true;
                break;
            }
#pragma unroll
            for (int e = 0; e < GS_EPL; e++) {
                // the same on every lane of the group: whether word e takes
                // a product of this chunk
                if ((e + 1) * G > base && e * G < base + total) {
                    const int p = e * G + gl - base;
                    const bool in = p >= 0 && p < total;
                    const int pc = in ? p : 0;
                    int s = 0;  // the A entry whose B row holds product pc of the chunk
#pragma unroll
                    for (int step = G / 2; step > 0; step >>= 1) {
                        const int v = __shfl_sync(gmask, incl, s + step - 1, G);
                        if (v <= pc) s += step;
                    }
                    const int64_t bo = __shfl_sync(gmask, boff, s, G);
                    const T as = __shfl_sync(gmask, av, s, G);
                    const int ex = __shfl_sync(gmask, incl, s, G) - __shfl_sync(gmask, blen, s, G);
                    if (in) {
                        // the B entry straight into the slot (no register
                        // waits for it): every copy of the row is in flight
                        const int slot = e * G + gl;
                        const int64_t q = bo + (pc - ex);
                        cp_async_4(&scol[slot], B.col + q);
                        if (sizeof(T) == 8) cp_async_8(&sb[slot], Bv + q);
                        else cp_async_4(&sb[slot], Bv + q);
                        sa[slot] = as;
                    }
                }
            }
            base += total;
        }
        cp_async_wait_all();  // this lane's copies (it reads only its own slots here)
        if (over) {
            if (gl == 0) report_overflow(ctl, bin, i, A, B);
            __syncwarp(gmask);
            continue;
        }
        uint32_t x[GS_EPL];
#pragma unroll
        for (int e = 0; e < GS_EPL; e++) {
            const int slot = e * G + gl;
            x[e] = slot < base ? ((uint32_t)scol[slot] << LOGN) | (uint32_t)slot : PAD;
        }
        // bitonic sort of the N words; word e of lane gl is position
        // gl * GS_EPL + e.  Merges of up to GS_EPL / 2 words lie inside a
        // lane with a direction fixed by e; a merge of size >= GS_EPL runs
        // one direction per lane, taken as ascending on complemented words.
        uint32_t flip = 0;
#pragma unroll
        for (int size = 2; size <= N; size <<= 1) {
            if (size >= GS_EPL) {
                const uint32_t f = ((gl * GS_EPL) & size) ? PAD : 0u;
#pragma unroll
                for (int e = 0; e < GS_EPL; e++) x[e] ^= f ^ flip;
                flip = f;
            }
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                if (stride >= GS_EPL) {
                    const int lm = stride / GS_EPL;
                    const bool lower = (gl & lm) == 0;
#pragma unroll
                    for (int e = 0; e < GS_EPL; e++) {
                        const uint32_t y = __shfl_xor_sync(gmask, x[e], lm, G);
                        const uint32_t lo = min(x[e], y), hi = max(x[e], y);
                        x[e] = lower ? lo : hi;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < GS_EPL; e++)
                        if ((e & stride) == 0) {
                            const uint32_t lo = min(x[e], x[e | stride]), hi = max(x[e], x[e | stride]);
                            const bool up = size >= GS_EPL || (e & size) == 0;
                            x[e] = up ? lo : hi;
                            x[e | stride] = up ? hi : lo;
                        }
                }
            }
        }
        __syncwarp(gmask);  // the slots, filled by the group's lanes
        // fold runs of equal columns: inside the lane, each word's value
        // becomes the fold of its run up to itself, one multiply-add per
        // product (c (+) a (x) b, with c the run so far or the neutral
        // element where a run starts; the double-precision pipe is the
        // scarce one on this GPU)
        int32_t col[GS_EPL];
        T v[GS_EPL];
#pragma unroll
        for (int e = 0; e < GS_EPL; e++) {
            const int slot = (int)(x[e] & (N - 1));
            const bool pad = x[e] == PAD;
            col[e] = pad ? -1 : (int32_t)(x[e] >> LOGN);
            const T a = pad ? T(0) : sa[slot], b = pad ? T(0) : sb[slot];
            const bool same = e > 0 && col[e] == col[e - 1];
            v[e] = Sr<SR>::fma(a, b, same ? v[e > 0 ? e - 1 : 0] : Sr<SR>::zero());
        }
        // across lanes: a lane's first run continues the previous lane's
        // last one when their columns agree; a segmented scan over the lanes
        // gives each lane the fold of the run that ends at its last word
        const int32_t first = col[0], last = col[GS_EPL - 1];
        const int32_t prev_last = __shfl_up_sync(gmask, last, 1, G);
        const bool link = gl > 0 && prev_last == first;
        T run = v[GS_EPL - 1];
        int head = !(link && first == last);  // the run ending here starts in this lane
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const T pr = __shfl_up_sync(gmask, run, d, G);
            const int ph = __shfl_up_sync(gmask, head, d, G);
            if (gl >= d && !head) {
                run = Sr<SR>::add(pr, run);
                head = ph;
            }
        }
        // the carry of a linked lane joins its first run, whose last word is
        // the only one of that run an output can come from
        const T carry = __shfl_up_sync(gmask, run, 1, G);
        if (link)
#pragma unroll
            for (int e = 0; e < GS_EPL; e++)
                if (col[e] == first && (e + 1 == GS_EPL || col[e + 1 < GS_EPL ? e + 1 : e] != first))
                    v[e] = Sr<SR>::add(carry, v[e]);
        // the last word of each run holds the entry; its rank among the
        // row's runs is its place in the output
        const int32_t next_first = __shfl_down_sync(gmask, first, 1, G);
        int nl = 0;
#pragma unroll
        for (int e = 0; e < GS_EPL; e++) {
            const int32_t nk = e + 1 < GS_EPL ? col[e + 1] : (gl + 1 < G ? next_first : -1);
            nl += col[e] >= 0 && nk != col[e];
        }
        int w = nl;
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const int o = __shfl_up_sync(gmask, w, d, G);
            if (gl >= d) w += o;
        }
        const int n = __shfl_sync(gmask, w, G - 1, G);
        w -= nl;
        int64_t dest = 0;
        if (gl == 0) dest = c_row_dest(C, J, ctl, i, n);
        dest = __shfl_sync(gmask, dest, 0, G);
        if (dest >= 0) {
#pragma unroll
            for (int e = 0; e < GS_EPL; e++) {
                const int32_t nk = e + 1 < GS_EPL ? col[e + 1] : (gl + 1 < G ? next_first : -1);
                if (col[e] >= 0 && nk != col[e]) {
                    C.col[dest + w] = col[e];
                    Cv[dest + w] = v[e];
                    w++;
                }
            }
            if (gl == 0) C.len[i] = n;
        }
        if (gl == 0) nnz_acc += n;
        __syncwarp(gmask);  // every lane has read the slots before the next row fills them
    }
    nnz_acc = warp_sum<long long>(nnz_acc);
    if (lane == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// ---------------------------------------------------- group hash kernel

// G lanes per row (32 / G rows per warp), TS hash slots per row.
template <int SR, int LOG_TS, int G, int NW>
__global__ void __launch_bounds__(NW * 32)
k_num_group_hash(MatView A, MatView B, MatView C, CJob J, Ctl *ctl, unsigned mask, int bin) {
    pdl_begin();
    using T = typename Sr<SR>::T;
    constexpr int TS = 1 << LOG_TS;
    // rows of tables up to 64 slots are compacted and ranked (column order,
    // cheap at that size); larger tables are written straight to C
    constexpr bool RANKED = TS <= 64;
    constexpr int HC = RANKED ? TS : 0;  // compacted list capacity
    constexpr int GPW = 32 / G;
    constexpr int NG = NW * GPW;  // groups per block
    extern __shared__ __align__(16) unsigned char smem[];
    if (failed(ctl, mask)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gl = lane & (G - 1), gw = lane / G;
    const int g = w * GPW + gw;  // group in block
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (gw * G));
    T *vals = (T *)smem + (size_t)g * TS;
    T *cv = (T *)smem + (size_t)NG * TS + (size_t)g * HC;
    int32_t *keys = (int32_t *)((T *)smem + (size_t)NG * (TS + HC)) + (size_t)g * TS;
    int32_t *ck = (int32_t *)((T *)smem + (size_t)NG * (TS + HC)) + (size_t)NG * TS + (size_t)g * HC;
    (void)cv;
    (void)ck;
    T *Cv = (T *)C.val;
    long long nnz_acc = 0;
    const long long cnt = ctl->bin_count[bin];
    if ((long long)blockIdx.x * NG >= cnt) return;  // no row for this block
    // the table is cleared once here; each row's read-out clears the slots
    // it used
    for (int s = gl; s < TS; s += G) {
        keys[s] = -1;
        vals[s] = Sr<SR>::zero();
    }
    __syncwarp(gmask);
    for (long long it = (long long)blockIdx.x * NG + g; it < cnt; it += (long long)gridDim.x * NG) {
        int32_t i = J.bins[(int64_t)bin * J.bin_cap + it];
        if (!dcheck(ctl, i >= 0 && i < A.nrows, DBG_R_ROW, it)) i = 0;  // debug build: a bad list entry fails the batch
        bool ok = true;
        unsigned fresh = 0;  // slots this lane claimed: the row's length, summed over the group
        group_products<SR, G>(A, B, i, gmask, [&](int32_t j, T v) {
            const int r = hash_acc<LOG_TS, T, SR>(keys, vals, j, v);
            ok &= r >= 0;
            fresh += r > 0;
        });
        const bool full = (__ballot_sync(gmask, !ok) & gmask) != 0u;
        if (full) {
            // a learned table too small: the row goes to the overflow list and
            // is counted and recomputed later; with a bound or exact size a
            // full table cannot happen, so it is reported as an error
            __syncwarp(gmask);
            for (int s = gl; s < TS; s += G) {
                keys[s] = -1;
                vals[s] = Sr<SR>::zero();
            }
            if (gl == 0) {
                if (J.sizing == SIZE_LEARNED) J.ovf[atomic_add_ll2(&ctl->n_ovf, 1)] = i;
                else report_overflow(ctl, bin, i, A, B);
            }
            __syncwarp(gmask);
            continue;
        }
        __syncwarp(gmask);
        const int n = (int)__reduce_add_sync(gmask, fresh);
        if constexpr (RANKED) {
            int x0 = 0;
            for (int s0 = 0; s0 < TS; s0 += G) {
                const int s = s0 + gl;
                const int32_t k = keys[s];
                const bool occ = k >= 0;
                const unsigned bal = (__ballot_sync(gmask, occ) & gmask) >> (gw * G);
                if (occ) {
                    const int x = x0 + __popc(bal & ((1u << gl) - 1u));
                    ck[x] = k;
                    cv[x] = vals[s];
                    keys[s] = -1;
                    vals[s] = Sr<SR>::zero();
                }
                x0 += __popc(bal);
            }
            __syncwarp(gmask);
        }
        int64_t dest = 0;
        if (gl == 0) dest = c_row_dest(C, J, ctl, i, n);
        dest = __shfl_sync(gmask, dest, 0, G);
        if constexpr (RANKED) {
            // rank of each entry among the row's distinct columns
            for (int e = gl; e < n; e += G) {
                const int32_t key = ck[e];
                int rank = 0;
                for (int x = 0; x < n; x++) rank += ck[x] < key;
                if (dest >= 0) {
                    C.col[dest + rank] = key;
                    Cv[dest + rank] = cv[e];
                }
            }
        } else {
            // straight from the table, in table order (C's rows need no column
            // order: the reads sort them), clearing the used slots
            int x0 = 0;
            for (int s0 = 0; s0 < TS; s0 += G) {
                const int s = s0 + gl;
                const int32_t k = keys[s];
                const bool occ = k >= 0;
                const unsigned bal = (__ballot_sync(gmask, occ) & gmask) >> (gw * G);
                if (occ) {
                    if (dest >= 0) {
                        const int x = x0 + __popc(bal & ((1u << gl) - 1u));
                        C.col[dest + x] = k;
                        Cv[dest + x] = vals[s];
                    }
                    keys[s] = -1;
                    vals[s] = Sr<SR>::zero();
                }
                x0 += __popc(bal);
            }
        }
        if (gl == 0 && dest >= 0) C.len[i] = n;
        nnz_acc += n;
        __syncwarp(gmask);
    }
    if (gl == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// ------------------------------------------------------- CTA hash kernel

// NT threads per CTA: more for the larger tables, whose shared memory leaves
// room for fewer CTAs per SM, so that an SM keeps as many warps in flight.
template <int SR, int LOG_TS, int NT>
__global__ void __launch_bounds__(NT)
k_num_cta_hash(MatView A, MatView B, MatView C, CJob J, Ctl *ctl, unsigned mask, int bin) {
    pdl_begin();
    using T = typename Sr<SR>::T;
    constexpr int TS = 1 << LOG_TS;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t p_boff[NT];
    __shared__ T p_av[NT];
    __shared__ int p_incl[NT], p_blen[NT], p_wsum[32];
    __shared__ int s_n, s_pos;
    __shared__ long long s_dest;
    if (failed(ctl, mask)) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    T *vals = (T *)smem;
    int32_t *keys = (int32_t *)(vals + TS);
    T *Cv = (T *)C.val;
    BlockProdSmem<T> ps{p_boff, p_av, p_incl, p_blen, p_wsum};
    long long nnz_acc = 0;
    const long long cnt = ctl->bin_count[bin];
    if (blockIdx.x >= cnt) return;  // no row for this CTA (an empty bin costs no table clear)
    // the table is cleared once here; each row's read-out clears the slots it used
    for (int s = tid; s < TS; s += NT) {
        keys[s] = -1;
        vals[s] = Sr<SR>::zero();
    }
    if (tid == 0) s_n = 0;
    __syncthreads();
    for (long long it = blockIdx.x; it < cnt; it += gridDim.x) {
        int32_t i = J.bins[(int64_t)bin * J.bin_cap + it];
        if (!dcheck(ctl, i >= 0 && i < A.nrows, DBG_R_ROW, it)) i = 0;  // debug build: a bad list entry fails the batch
        bool ok = true;
        int fresh = 0;  // slots this thread claimed; their sum is the row's length
        block_products<SR>(A, B, i, ps, [&](int32_t j, T v) {
            const int r = hash_acc<LOG_TS, T, SR>(keys, vals, j, v);
            ok &= r >= 0;
            fresh += r > 0;
        });
        fresh = warp_sum<int>(fresh);
        if (lane == 0 && fresh) atomicAdd(&s_n, fresh);
        const bool full = __syncthreads_or(!ok);
        const int n = s_n;
        if (full) {  // table too small: see the group kernel
            for (int s = tid; s < TS; s += NT) {
                keys[s] = -1;
                vals[s] = Sr<SR>::zero();
            }
            __syncthreads();  // every thread has read s_n
            if (tid == 0) {
                s_n = 0;
                if (J.sizing == SIZE_LEARNED) J.ovf[atomic_add_ll2(&ctl->n_ovf, 1)] = i;
                else report_overflow(ctl, bin, i, A, B);
            }
            __syncthreads();
            continue;
        }
        if (tid == 0) {
            s_dest = c_row_dest(C, J, ctl, i, n);
            s_pos = 0;
            nnz_acc += n;
        }
        __syncthreads();
        if (tid == 0) s_n = 0;  // every thread has read it
        const long long dest = s_dest;
        // one pass over the table: write straight to C (in table order; C's
        // rows need no column order) and clear the used slots
        for (int s0 = w * 32; s0 < TS; s0 += NT) {
            const int s = s0 + lane;
            const int32_t k = keys[s];
            const bool occ = k >= 0;
            const unsigned bal = __ballot_sync(0xffffffffu, occ);
            if (bal) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_pos, __popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (occ) {
                    if (dest >= 0) {
                        const int x = base + __popc(bal & lanemask_lt());
                        C.col[dest + x] = k;
                        Cv[dest + x] = vals[s];
                    }
                    keys[s] = -1;
                    vals[s] = Sr<SR>::zero();
                }
            }
        }
        if (tid == 0 && dest >= 0) C.len[i] = n;
        __syncthreads();
    }
    if (tid == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// --------------------------------------------------- cluster hash kernel
//
// Rows whose tables outgrow one CTA's shared memory: a thread-block cluster
// of CL CTAs holds one table of CL * TS slots in their shared memories
// together.  Each column belongs to one CTA (the top bits of its hash); every
// CTA goes through all of the row's products, keeps those of its own
// columns (loading no value for the others) and inserts them into its own
// shared memory, at the slot given by the next LOG_TS bits (triangular
// probing).  Only when a CTA's table is full does it pass a column on to the
// next CTA's table, with atomics through distributed shared memory, so the
// cluster's tables fill up together whatever the hash spread.  Then each CTA
// counts its slots, CTA 0 places the row (the sum) and hands every CTA its
// offset, and each writes its entries straight to C (in table order) and
// clears the slots it used.  Every CTA passes the same cluster barriers: the
// row loop and the status test are uniform.
template <int SR, int LOG_TS, int CL, int NT>
__global__ void __launch_bounds__(NT, LOG_TS == 13 ? 2 : 1)  // two 8192-slot tables fit an SM
k_num_cluster_hash(MatView A, MatView B, MatView C, CJob J, Ctl *ctl, unsigned early_mask, int bin) {
    pdl_begin();
    using T = typename Sr<SR>::T;
    constexpr int TS = 1 << LOG_TS;
    constexpr int LOG_CL = CL == 2 ? 1 : (CL == 4 ? 2 : 3);
    static_assert((1 << LOG_CL) == CL, "cluster size 2, 4 or 8");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t p_boff[NT];
    __shared__ T p_av[NT];
    __shared__ int p_incl[NT], p_blen[NT], p_wsum[32];
    __shared__ int s_cnt, s_full, s_pos;
    __shared__ long long s_dest;  // written by CTA 0: this row's place (-1: none)
    __shared__ int s_off;         // written by CTA 0: this CTA's offset in the row
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    T *vals = (T *)smem;
    int32_t *keys = (int32_t *)(vals + TS);
    T *Cv = (T *)C.val;
    BlockProdSmem<T> ps{p_boff, p_av, p_incl, p_blen, p_wsum};
    // early_mask holds only bits of the stages before the recompute, which
    // no sibling kernel sets meanwhile: every CTA reads the same answer
    const bool skip = failed(ctl, early_mask);
    const long long cnt = skip ? 0 : ctl->bin_count[bin];
    const long long nclusters = gridDim.x / CL;
    // a cluster without rows leaves before its first barrier: all of its CTAs
    // see the same count and cluster index, so they all leave together
    if ((long long)(blockIdx.x / CL) >= cnt) return;
    for (int s = tid; s < TS; s += NT) {
        keys[s] = -1;
        vals[s] = Sr<SR>::zero();
    }
    if (tid == 0) {
        s_cnt = 0;
        s_full = 0;
    }
    cl.sync();
    long long nnz_acc = 0;
    for (long long it = blockIdx.x / CL; it < cnt; it += nclusters) {
        int32_t i = J.bins[(int64_t)bin * J.bin_cap + it];
        if (!dcheck(ctl, i >= 0 && i < A.nrows, DBG_R_ROW, it)) i = 0;  // debug build: a bad list entry fails the batch
        if (tid == 0) s_pos = 0;
        bool ok = true;
        // every CTA goes through all of the row's products and keeps those
        // whose column it owns: inserts into its own shared memory, no remote
        // atomics; only a full table passes a column on to the next CTA's
        block_products<SR>(A, B, i, ps, [&](int32_t j, T v) {
            const uint32_t h = (uint32_t)j * 2654435761u;
            const uint32_t slot = (h << LOG_CL) >> (32 - LOG_TS);
            int r = hash_acc_from<LOG_TS, T, SR>(keys, vals, slot, j, v);
            for (int t = 1; t < CL && r < 0; t++) {
                const int o = (rank + t) & (CL - 1);
                r = hash_acc_from<LOG_TS, T, SR, true>(cl.map_shared_rank(keys, o), cl.map_shared_rank(vals, o), slot,
                                                        j, v);
            }
            ok &= r >= 0;
        }, 0, 1, [&](int32_t j) { return (int)(((uint32_t)j * 2654435761u) >> (32 - LOG_CL)) == rank; });
        if (!ok) s_full = 1;
        cl.sync();  // (1) every product of the row is in the tables
        int c = 0;
        for (int s0 = w * 32; s0 < TS; s0 += NT) c += __popc(__ballot_sync(0xffffffffu, keys[s0 + lane] >= 0));
        if (lane == 0 && c) atomicAdd(&s_cnt, c);
        cl.sync();  // (2) counts and overflow flags are final
        if (rank == 0 && tid == 0) {
            int full = 0, n = 0;
            for (int r = 0; r < CL; r++) {
                *cl.map_shared_rank(&s_off, r) = n;  // this CTA's entries follow those of the CTAs before it
                n += *cl.map_shared_rank(&s_cnt, r);
                full |= *cl.map_shared_rank(&s_full, r);
            }
            long long dest = -1;
            if (full) {  // a learned table too small: see the group kernel
                if (J.sizing == SIZE_LEARNED) J.ovf[atomic_add_ll2(&ctl->n_ovf, 1)] = i;
                else report_overflow(ctl, bin, i, A, B);
            } else {
                dest = c_row_dest(C, J, ctl, i, n);
                nnz_acc += n;
                if (dest >= 0) C.len[i] = n;
            }
            for (int r = 0; r < CL; r++) *cl.map_shared_rank(&s_dest, r) = dest;
        }
        cl.sync();  // (3) every CTA knows the row's place and its offset
        const long long dest = s_dest;
        const int off = s_off;
        for (int s0 = w * 32; s0 < TS; s0 += NT) {
            const int s = s0 + lane;
            const int32_t k = keys[s];
            const bool occ = k >= 0;
            const unsigned bal = __ballot_sync(0xffffffffu, occ);
            if (bal) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_pos, __popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (occ) {
                    if (dest >= 0) {
                        const int x = off + base + __popc(bal & lanemask_lt());
                        C.col[dest + x] = k;
                        Cv[dest + x] = vals[s];
                    }
                    keys[s] = -1;
                    vals[s] = Sr<SR>::zero();
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            s_cnt = 0;
            s_full = 0;
        }
        cl.sync();  // (4) the tables are clear before the next row's products arrive
    }
    if (tid == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// ------------------------------------------------- global dense kernel

// Up to this many mask words (512K columns) the read-out takes a thread per
// mask word; wider rows go through the summary of touched words.
constexpr int GD_DIRECT = 16384;

template <int SR>
__global__ void __launch_bounds__(512)
k_num_gdense(MatView A, MatView B, MatView C, CJob J, Ctl *ctl, unsigned mask, int bin) {
    pdl_begin();
    using T = typename Sr<SR>::T;
    __shared__ int64_t p_boff[512];
    __shared__ T p_av[512];
    __shared__ int p_incl[512], p_blen[512], p_wsum[32];
    __shared__ int s_n;
    __shared__ long long s_dest;
    if (failed(ctl, mask)) return;
    const int tid = threadIdx.x;
    const int nwords = (int)(J.gd_w / 32);
    const int nsum = (nwords + 31) / 32;
    const bool direct = nwords <= GD_DIRECT;
    T *acc = (T *)J.gd_acc + (int64_t)blockIdx.x * J.gd_w;
    uint32_t *msk = J.gd_mask + (int64_t)blockIdx.x * nwords;
    uint32_t *sum = J.gd_sum + (int64_t)blockIdx.x * nsum;  // bit w: mask word w was touched
    T *Cv = (T *)C.val;
    BlockProdSmem<T> ps{p_boff, p_av, p_incl, p_blen, p_wsum};
    long long nnz_acc = 0;
    const long long cnt = ctl->bin_count[bin];
    for (long long it = blockIdx.x; it < cnt; it += gridDim.x) {
        int32_t i = J.bins[(int64_t)bin * J.bin_cap + it];
        if (!dcheck(ctl, i >= 0 && i < A.nrows, DBG_R_ROW, it)) i = 0;  // debug build: a bad list entry fails the batch
        if (tid == 0) s_n = 0;
        __syncthreads();
        block_products<SR>(A, B, i, ps, [&](int32_t j, T v) {
            // the product that sets the first bit of a mask word marks the
            // word in the summary, so the read-out skips untouched words
            if (atomicOr(&msk[j >> 5], 1u << (j & 31)) == 0u && !direct)
                atomicOr(&sum[j >> 10], 1u << ((j >> 5) & 31));
            Sr<SR>::acc(&acc[j], v);
        });
        __syncthreads();
        if (direct) {
            // few columns: a thread per mask word, in order (a block scan per
            // 512 words gives each its offset); no summary needed
            int c = 0;
            for (int wd = tid; wd < nwords; wd += 512) c += __popc(__ldcg(msk + wd));
            c = warp_sum<int>(c);
            if ((tid & 31) == 0 && c) atomicAdd(&s_n, c);
            __syncthreads();
            const int n = s_n;
            if (tid == 0) {
                s_dest = c_row_dest(C, J, ctl, i, n);
                nnz_acc += n;
            }
            __syncthreads();
            const long long dest = s_dest;
            int run = 0;
            for (int w0 = 0; w0 < nwords; w0 += 512) {
                const int wd = w0 + tid;
                uint32_t bits = wd < nwords ? __ldcg(msk + wd) : 0u;
                const int e = __popc(bits);
                const int incl = block_incl_scan(e, p_incl, p_wsum);
                int o = run + p_incl[tid] - e;
                if (bits) msk[wd] = 0u;
                while (bits) {
                    const int bt = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int j = (wd << 5) + bt;
                    if (dest >= 0) {
                        C.col[dest + o] = j;
                        Cv[dest + o] = __ldcg(acc + j);
                    }
                    acc[j] = Sr<SR>::zero();
                    o++;
                }
                run += incl;
                __syncthreads();
            }
            if (tid == 0 && dest >= 0) C.len[i] = n;
            continue;
        }
        // entries under summary word x (its touched mask words)
        auto entries_of = [&](int x) {
            int c = 0;
            uint32_t sw = x < nsum ? __ldcg(sum + x) : 0u;
            while (sw) {
                const int b = __ffs(sw) - 1;
                sw &= sw - 1;
                c += __popc(__ldcg(msk + x * 32 + b));
            }
            return c;
        };
        int c = 0;
        for (int x = tid; x < nsum; x += 512) c += entries_of(x);
        c = warp_sum<int>(c);
        if ((tid & 31) == 0 && c) atomicAdd(&s_n, c);
        __syncthreads();
        const int n = s_n;
        if (tid == 0) {
            s_dest = c_row_dest(C, J, ctl, i, n);
            nnz_acc += n;
        }
        __syncthreads();
        const long long dest = s_dest;
        // the row in column order: summary words in order (a block scan gives
        // each its offset), then each summary word's mask words and bits in order
        int run = 0;
        for (int x0 = 0; x0 < nsum; x0 += 512) {
            const int x = x0 + tid;
            const int e = entries_of(x);
            const int incl = block_incl_scan(e, p_incl, p_wsum);
            int o = run + p_incl[tid] - e;
            uint32_t sw = x < nsum ? __ldcg(sum + x) : 0u;
            while (sw) {
                const int b = __ffs(sw) - 1;
                sw &= sw - 1;
                const int wd = x * 32 + b;
                uint32_t bits = __ldcg(msk + wd);
                while (bits) {
                    const int bt = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int j = (wd << 5) + bt;
                    if (dest >= 0) {
                        C.col[dest + o] = j;
                        Cv[dest + o] = __ldcg(acc + j);
                    }
                    acc[j] = Sr<SR>::zero();
                    o++;
                }
                msk[wd] = 0u;
            }
            if (x < nsum) sum[x] = 0u;
            run += incl;
            __syncthreads();
        }
        if (tid == 0 && dest >= 0) C.len[i] = n;
    }
    if (tid == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// ----------------------------------------------------- dense small-m kernels

template <int SR, int NW>
__global__ void __launch_bounds__(NW * 32)
k_num_warp_dense(MatView A, MatView B, MatView C, CJob J, Ctl *ctl, unsigned mask, int bin, int mp) {
    pdl_begin();
    using T = typename Sr<SR>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    if (failed(ctl, mask)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = mp >> 5;  // presence words (<= 32)
    T *acc = (T *)smem + (size_t)w * mp;
    uint32_t *msk = (uint32_t *)((T *)smem + (size_t)NW * mp) + (size_t)w * 32;
    T *Cv = (T *)C.val;
    const long long cnt = ctl->bin_count[bin];
    if ((long long)blockIdx.x * NW >= cnt) return;  // no row for this block
    for (int s = lane; s < mp; s += 32) acc[s] = Sr<SR>::zero();
    msk[lane] = 0u;
    __syncwarp();
    long long nnz_acc = 0;
    for (long long it = (long long)blockIdx.x * NW + w; it < cnt; it += (long long)gridDim.x * NW) {
        int32_t i = J.bins[(int64_t)bin * J.bin_cap + it];
        if (!dcheck(ctl, i >= 0 && i < A.nrows, DBG_R_ROW, it)) i = 0;  // debug build: a bad list entry fails the batch
        group_products<SR, 32>(A, B, i, 0xffffffffu, [&](int32_t j, T v) {
            atomicOr(&msk[j >> 5], 1u << (j & 31));
            Sr<SR>::acc(&acc[j], v);
        });
        __syncwarp();
        const uint32_t word = lane < nw ? msk[lane] : 0u;
        const int pc = __popc(word);
        const int incl = warp_incl_scan<int>(pc);
        const int n = __shfl_sync(0xffffffffu, incl, 31);
        int64_t dest = 0;
        if (lane == 0) dest = c_row_dest(C, J, ctl, i, n);
        dest = __shfl_sync(0xffffffffu, dest, 0);
        int o = incl - pc;
        uint32_t bits = word;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int j = (lane << 5) + b;
            if (dest >= 0) {
                C.col[dest + o] = j;
                Cv[dest + o] = acc[j];
            }
            acc[j] = Sr<SR>::zero();
            o++;
        }
        msk[lane] = 0u;
        if (lane == 0 && dest >= 0) C.len[i] = n;
        nnz_acc += n;
        __syncwarp();
    }
    if (lane == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

template <int SR>
__global__ void __launch_bounds__(512)
k_num_cta_dense(MatView A, MatView B, MatView C, CJob J, Ctl *ctl, unsigned mask, int bin, int mp) {
    pdl_begin();
    using T = typename Sr<SR>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    if (failed(ctl, mask)) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nw = mp >> 5;
    T *acc = (T *)smem;
    uint32_t *msk = (uint32_t *)(acc + mp);
    T *Cv = (T *)C.val;
    const long long cnt = ctl->bin_count[bin];
    if (blockIdx.x >= cnt) return;  // no row for this block
    for (int s = tid; s < mp; s += 512) acc[s] = Sr<SR>::zero();
    if (tid < 32) msk[tid] = 0u;
    __syncthreads();
    long long nnz_acc = 0;
    for (long long it = blockIdx.x; it < cnt; it += gridDim.x) {
        int32_t i = J.bins[(int64_t)bin * J.bin_cap + it];
        if (!dcheck(ctl, i >= 0 && i < A.nrows, DBG_R_ROW, it)) i = 0;  // debug build: a bad list entry fails the batch
        group_products<SR, 32>(A, B, i, 0xffffffffu, [&](int32_t j, T v) {
            atomicOr(&msk[j >> 5], 1u << (j & 31));
            Sr<SR>::acc(&acc[j], v);
        }, (tid >> 5) * 32, -1, 512);
        __syncthreads();
        if (tid < 32) {
            const uint32_t word = lane < nw ? msk[lane] : 0u;
            const int pc = __popc(word);
            const int incl = warp_incl_scan<int>(pc);
            const int n = __shfl_sync(0xffffffffu, incl, 31);
            int64_t dest = 0;
            if (lane == 0) dest = c_row_dest(C, J, ctl, i, n);
            dest = __shfl_sync(0xffffffffu, dest, 0);
            int o = incl - pc;
            uint32_t bits = word;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                const int j = (lane << 5) + b;
                if (dest >= 0) {
                    C.col[dest + o] = j;
                    Cv[dest + o] = acc[j];
                }
                acc[j] = Sr<SR>::zero();
                o++;
            }
            msk[lane] = 0u;
            if (lane == 0) {
                if (dest >= 0) C.len[i] = n;
                nnz_acc += n;
            }
        }
        __syncthreads();
    }
    if (tid == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// -------------------------------------------------------------- host

template <typename T>
__global__ void k_fill(T *p, int64_t n, T v) {
    pdl_begin();
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

void run_size_bins(const MatView &A, const MatView &B, const MatView &C, const CJob &J, int64_t max_rows, Ctl *ctl,
                   unsigned mask, cudaStream_t s, int num_sms) {
    if (max_rows <= 0) return;
    int64_t g = (max_rows + 255) / 256;
    if (g > num_sms * 8) g = num_sms * 8;
    if (g < 1) g = 1;
    launch_k(k_size_bins, (unsigned)g, 256, 0, s, A, B, C, J, ctl, mask);
    if (J.sizing == SIZE_LEARNED) {
        constexpr size_t smem = EST_PARAMS * sizeof(float) + 16;
        static bool set = false;
        if (!set) {
            cudaFuncSetAttribute(k_est_bins, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            set = true;
        }
        int64_t ge = (max_rows + 127) / 128;
        if (ge > num_sms * 4) ge = num_sms * 4;
        if (ge < 1) ge = 1;
        launch_k(k_est_bins, (unsigned)ge, 128, smem, s, J, ctl, mask);
    }
}

// ---------------------------------------------------- split dense rows

// Dense mode, rows with many A entries or products (the hubs of skewed
// graphs): each split row is cut into chunks of SPLIT_CHUNK A entries, and
// the chunks of all split rows form one work list (k_split_prep writes its
// prefix over the rows, sp_pre).  A CTA accumulates a chunk in shared memory
// and folds it into the row's global accumulator with atomics; the CTA that
// folds a row's last chunk (a per-row counter) writes the row into C in
// column order and resets the accumulator for the next launch.
__global__ void __launch_bounds__(1024) k_split_prep(MatView A, CJob J, Ctl *ctl, unsigned mask) {
    pdl_begin();
    __shared__ int incl[1024], wsum[32];
    if (failed(ctl, mask)) return;
    long long cnt = ctl->bin_count[BIN_DSPLIT];
    if (cnt > J.sp_rows) cnt = J.sp_rows;
    long long carry = 0;
    for (long long b0 = 0; b0 < cnt; b0 += 1024) {
        const long long slot = b0 + threadIdx.x;
        int nch = 0;
        if (slot < cnt) {
            const int32_t i = J.bins[(int64_t)BIN_DSPLIT * J.bin_cap + slot];
            nch = (A.len[i] + SPLIT_CHUNK - 1) / SPLIT_CHUNK;
        }
        const int tot = block_incl_scan(nch, incl, wsum);
        if (slot < cnt) J.sp_pre[slot] = carry + incl[threadIdx.x] - nch;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) J.sp_pre[cnt] = carry;
}

template <int SR, int NT>
__global__ void __launch_bounds__(NT)
k_num_dsplit(MatView A, MatView B, MatView C, CJob J, Ctl *ctl, unsigned mask, int mp) {
    pdl_begin();
    using T = typename Sr<SR>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_last;
    __shared__ long long s_dest;
    __shared__ int s_n;
    if (failed(ctl, mask)) return;
    const int tid = threadIdx.x;
    const int nw = mp >> 5;
    T *acc = (T *)smem;
    uint32_t *msk = (uint32_t *)(acc + mp);
    T *Cv = (T *)C.val;
    for (int s = tid; s < mp; s += NT) acc[s] = Sr<SR>::zero();
    if (tid < 32) msk[tid] = 0u;
    __syncthreads();
    long long cnt = ctl->bin_count[BIN_DSPLIT];
    if (cnt > J.sp_rows) cnt = J.sp_rows;
    const long long total = cnt > 0 ? J.sp_pre[cnt] : 0;
    long long nnz_acc = 0;
    // each CTA takes a contiguous range of work items: one search for its
    // first row, then forward; consecutive chunks of a row are accumulated
    // together and folded once
    const long long per = (total + gridDim.x - 1) / gridDim.x;
    const long long w0 = (long long)blockIdx.x * per, w1 = w0 + per < total ? w0 + per : total;
    long long slot = 0;
    if (w0 < w1) {
        long long lo = 0, hi = cnt;  // last slot with sp_pre[slot] <= w0
        while (hi - lo > 1) {
            const long long mid = (lo + hi) >> 1;
            if (J.sp_pre[mid] <= w0) lo = mid; else hi = mid;
        }
        slot = lo;
    }
    int pending = 0;  // chunks accumulated in shared memory, not yet folded
    long long prods = 0;  // products formed (the sizing pass does not sum split rows)
    for (long long w = w0; w < w1; w++) {
        while (J.sp_pre[slot + 1] <= w) slot++;
        const long long base = J.sp_pre[slot];
        const int nch = (int)(J.sp_pre[slot + 1] - base);
        const int c = (int)(w - base);
        const int32_t i = J.bins[(int64_t)BIN_DSPLIT * J.bin_cap + slot];
        const int alen = A.len[i];
        const int a_lo = c * SPLIT_CHUNK, a_hi = a_lo + SPLIT_CHUNK < alen ? a_lo + SPLIT_CHUNK : alen;
        // each warp takes groups of 32 A entries of the chunk (no block barriers)
        group_products<SR, 32>(A, B, i, 0xffffffffu, [&](int32_t j, T v) {
            atomicOr(&msk[j >> 5], 1u << (j & 31));
            Sr<SR>::acc(&acc[j], v);
            prods++;
        }, a_lo + (tid >> 5) * 32, a_hi, NT);
        pending++;
        if (c + 1 < nch && w + 1 < w1) continue;  // the next item is this row's next chunk: keep accumulating
        __syncthreads();
        T *gacc = (T *)J.sp_acc + slot * mp;
        uint32_t *gmsk = J.sp_mask + slot * nw;
        // fold: each present column into the global row, each mask word once;
        // then one barrier, the mask reset and the row's chunk counter
        for (int j = tid; j < mp; j += NT) {
            const uint32_t word = msk[j >> 5];
            if ((j & 31) == 0 && word) atomicOr(&gmsk[j >> 5], word);
            if (word & (1u << (j & 31))) {
                Sr<SR>::acc(&gacc[j], acc[j]);
                acc[j] = Sr<SR>::zero();
            }
        }
        __threadfence();
        __syncthreads();
        if (tid < 32) msk[tid] = 0u;
        if (tid == 0) s_last = atomicAdd(&J.sp_done[slot], pending) == nch - pending;
        pending = 0;
        __syncthreads();
        if (s_last) {  // every chunk of the row is folded: write the row
            __threadfence();
            if (tid < 32) {
                const int lane = tid;
                const uint32_t word = lane < nw ? __ldcg(gmsk + lane) : 0u;
                const int pc = __popc(word);
                const int incl = warp_incl_scan<int>(pc);
                const int n = __shfl_sync(0xffffffffu, incl, 31);
                int64_t dest = 0;
                if (lane == 0) dest = c_row_dest(C, J, ctl, i, n);
                dest = __shfl_sync(0xffffffffu, dest, 0);
                int o = incl - pc;
                uint32_t bits = word;
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const int j = (lane << 5) + b;
                    if (dest >= 0) {
                        C.col[dest + o] = j;
                        Cv[dest + o] = __ldcg(gacc + j);
                    }
                    o++;
                }
                if (lane == 0) {
                    s_dest = dest;
                    s_n = n;
                }
            }
            __syncthreads();
            for (int j = tid; j < mp; j += NT) gacc[j] = Sr<SR>::zero();
            if (tid < nw) gmsk[tid] = 0u;
            if (tid == 0) {
                if (s_dest >= 0) C.len[i] = s_n;
                nnz_acc += s_n;
                J.sp_done[slot] = 0;
            }
        }
        __syncthreads();
    }
    prods = warp_sum<long long>(prods);
    if ((tid & 31) == 0 && prods && !J.count_only) atomic_add_ll2(&ctl->products, prods);
    if (tid == 0 && nnz_acc) atomic_add_ll2(&ctl->nnz_written, nnz_acc);
}

// A persistent grid of `full` blocks, but no more blocks than it takes for
// `rows` rows at `per_block` rows per block (small matrices launch small).
static unsigned grid_for(int64_t full, int64_t rows, int64_t per_block) {
    const int64_t need = (std::max<int64_t>(rows, 1) + per_block - 1) / per_block;
    return (unsigned)std::max<int64_t>(1, std::min(full, need));
}

// Blocks of `kern` resident per SM at nt threads and smem dynamic bytes
// (registers, shared memory and the thread limit all counted), with the
// shared-memory carveout at its maximum: the hash tables live there.  The
// launchers keep the answer per kernel for the process, whose handles all
// run on one GPU model.
template <typename K>
static int resident_per_sm(K kern, int nt, size_t smem) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nt, smem) != cudaSuccess || nb < 1) {
        cudaGetLastError();  // the launch itself reports a kernel that cannot run
        nb = 1;
    }
    return nb;
}

template <int SR, int LOG_TS, int G, int NW>
static void launch_group_hash(const MatView &A, const MatView &B, const MatView &C, const CJob &J, Ctl *ctl,
                              unsigned mask, int bin, cudaStream_t s, int num_sms) {
    using T = typename Sr<SR>::T;
    constexpr int TS = 1 << LOG_TS;
    constexpr int NG = NW * (32 / G);
    const size_t smem = (size_t)NG * ((TS <= 64 ? 2 : 1) * TS) * (sizeof(T) + sizeof(int32_t));
    static const int per_sm = resident_per_sm(k_num_group_hash<SR, LOG_TS, G, NW>, NW * 32, smem);
    launch_k(k_num_group_hash<SR, LOG_TS, G, NW>, grid_for(num_sms * per_sm, J.rows_hint, NG), NW * 32, smem, s, A, B,
             C, J, ctl, mask, bin);
}

template <int SR, int G>
static void launch_group_sort(const MatView &A, const MatView &B, const MatView &C, const CJob &J, Ctl *ctl,
                              unsigned mask, int bin, cudaStream_t s, int num_sms) {
    static const int per_sm = resident_per_sm(k_num_group_sort<SR, G>, GS_NT, 0);
    launch_k(k_num_group_sort<SR, G>, grid_for(num_sms * per_sm, J.rows_hint, GS_NT / G), GS_NT, 0, s, A, B, C, J,
             ctl, mask, bin);
}

template <int SR, int LOG_TS>
static void launch_cta_hash(const MatView &A, const MatView &B, const MatView &C, const CJob &J, Ctl *ctl,
                            unsigned mask, int bin, cudaStream_t s, int num_sms) {
    using T = typename Sr<SR>::T;
    constexpr int TS = 1 << LOG_TS;
    constexpr int NT = LOG_TS <= 12 ? 256 : (LOG_TS == 13 ? 512 : 1024);
    const size_t smem = (size_t)TS * (sizeof(T) + sizeof(int32_t));
    // one wave of resident CTAs: a second, partial wave would only lengthen the tail
    static const int per_sm = std::min(8, resident_per_sm(k_num_cta_hash<SR, LOG_TS, NT>, NT, smem));
    launch_k(k_num_cta_hash<SR, LOG_TS, NT>, grid_for(num_sms * per_sm, J.rows_hint, 1), NT, smem, s, A, B, C, J, ctl,
             mask, bin);
}

// The bin kernels are independent; they are spread over the given streams
// (which the caller has ordered after the sizing pass) so that empty bins
// cost no time on the critical path.
template <int SR, int LOG_TS, int CL>
static void launch_cluster_hash(const MatView &A, const MatView &B, const MatView &C, const CJob &J, Ctl *ctl,
                                unsigned mask, int bin, cudaStream_t s, int num_sms) {
    using T = typename Sr<SR>::T;
    constexpr int TS = 1 << LOG_TS;
    constexpr int NT = LOG_TS == 13 ? 512 : 1024;  // as the CTA kernels: warps per SM for the larger tables
    const size_t smem = (size_t)TS * (sizeof(T) + sizeof(int32_t));
    // as many clusters as can be resident at once (the occupancy query for
    // this cluster shape), so the grid is one wave
    static long long max_clusters = 0;
    if (!max_clusters) {
        cudaFuncSetAttribute(k_num_cluster_hash<SR, LOG_TS, CL, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_num_cluster_hash<SR, LOG_TS, CL, NT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3((unsigned)(CL * num_sms));
        q.blockDim = dim3(NT);
        q.dynamicSmemBytes = smem;
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = CL;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        q.attrs = qa;
        q.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k_num_cluster_hash<SR, LOG_TS, CL, NT>, &q) != cudaSuccess || nc < 1) {
            cudaGetLastError();  // the launch reports a shape that cannot run
            nc = std::max(1, num_sms / CL);
        }
        max_clusters = nc;
    }
    long long clusters = max_clusters;
    if (clusters > J.rows_hint) clusters = J.rows_hint;
    if (clusters < 1) clusters = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * CL));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1] = pdl_attribute();
    cfg.attrs = at;
    cfg.numAttrs = 2;
    // every CTA must reach the kernel's cluster barriers, so it tests only the
    // status bits of the stages before the recompute (see the split kernel)
    const unsigned early = mask & (ST_INVALID | ST_AB_STAGE | ST_AB_ARENA);
    // a failed launch stays in the runtime's last error, which the caller checks
    cudaLaunchKernelEx(&cfg, k_num_cluster_hash<SR, LOG_TS, CL, NT>, A, B, C, J, ctl, early, bin);
    __atomic_fetch_add(&launch_counter(), 1ull, __ATOMIC_RELAXED);
}

template <int SR>
static void run_numeric_t(const MatView &A, const MatView &B, const MatView &C, const CJob &J, Ctl *ctl, unsigned mask,
                          const cudaStream_t *ss, int ns, int num_sms) {
    using T = typename Sr<SR>::T;
    // the first kernel (the bin of the bulk of the rows of sparse products)
    // has ss[0] to itself; the others take the remaining streams in turn,
    // so that a small bin never waits behind a large one of a stream it
    // shares unless there are more bins than streams
    int k = 0;
    auto on = [&](int b) { return ((J.bin_on >> b) & 1ull) != 0; };
    auto next = [&]() {
        const int j = k++;
        return (j == 0 || ns == 1) ? ss[0] : ss[1 + (j - 1) % (ns - 1)];
    };
    // with the group sort on, its 64-product bin takes the rows of sparse
    // products and the first stream.  Its grid is one resident wave that
    // fills every SM, so kernels launched after it wait for it: with dense
    // accumulators it is launched last, so that the split kernel of the
    // long rows (the longest kernel there) starts first (the R-MAT 20
    // step: 0.329 to 0.311 ms); on the hash path first, as the empty grids
    // of the small bins would otherwise be dispatched ahead of it (a
    // one-update stencil step: 0.070 to 0.075 ms)
    const bool s64 = J.sort_max > 0 && on(BIN_S64);
    const bool s64_last = s64 && J.dense_mode;
    if (s64_last) k = 1;
    auto launch_s64 = [&]() {
        if (s64_last) launch_group_sort<SR, 8>(A, B, C, J, ctl, mask, BIN_S64, ss[0], num_sms);
    };
    if (s64 && !s64_last) launch_group_sort<SR, 8>(A, B, C, J, ctl, mask, BIN_S64, next(), num_sms);
    if (J.sort_max > 64 && on(BIN_S128)) launch_group_sort<SR, 16>(A, B, C, J, ctl, mask, BIN_S128, next(), num_sms);
    if (J.sort_max > 128 && on(BIN_S256)) launch_group_sort<SR, 32>(A, B, C, J, ctl, mask, BIN_S256, next(), num_sms);
    {
        // shared memory for the bin's bound only: at a bound of 49 three
        // blocks of 128 threads fit an SM with double values (two at 64),
        // leaving less of the SM's memory to the L1 cache that catches the
        // B rows shared by neighbouring rows
        static bool set_m = false;
        if (!set_m) {
            cudaFuncSetAttribute(k_num_thread_merge<SR, MERGE_K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)MERGE_UB * TM_NT * (sizeof(int32_t) + sizeof(T))));
            set_m = true;
        }
        auto launch_merge = [&](int bin, int ub) {
            const size_t smem_m = (size_t)ub * TM_NT * (sizeof(int32_t) + sizeof(T));
            const int per_sm = (int)std::min<size_t>(8, std::max<size_t>(1, (227 * 1024) / (smem_m + 1024)));
            launch_k(k_num_thread_merge<SR, MERGE_K>, grid_for(num_sms * per_sm, J.rows_hint, TM_NT), TM_NT, smem_m,
                     next(), A, B, C, J, ctl, mask, bin, ub);
        };
        // rows the group sort takes leave the merge bins empty
        if (J.tm_k > 0 && J.sort_max < MERGE_UB) {
            if (on(BIN_T8)) launch_merge((int)BIN_T8, std::max(J.tm_ub, 1));
            if (J.tm_ub < MERGE_UB && on(BIN_T64)) launch_merge((int)BIN_T64, MERGE_UB);
        }
    }
    if (J.dense_mode) {
        const int mp = (int)((J.m + 31) / 32 * 32);
        constexpr int NW = 8;
        const size_t smem_w = (size_t)NW * mp * sizeof(T) + NW * 32 * sizeof(uint32_t);
        static bool set_w = false;
        if (!set_w) {
            cudaFuncSetAttribute(k_num_warp_dense<SR, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
            set_w = true;
        }
        launch_k(k_num_warp_dense<SR, NW>, grid_for(num_sms * 4, J.rows_hint, NW), NW * 32, smem_w, next(), A, B, C, J,
                 ctl, mask, (int)BIN_WDENSE, mp);
        const size_t smem_c = (size_t)mp * sizeof(T) + 32 * sizeof(uint32_t);
        launch_k(k_num_cta_dense<SR>, grid_for((int64_t)num_sms * 2, J.rows_hint, 1), 512, smem_c, next(), A, B, C, J,
                 ctl, mask, (int)BIN_CDENSE, mp);
        // every CTA of the split kernel must run to the end (the last one to
        // arrive at a row writes it), so it tests only the status bits of
        // the stages before the recompute, which no sibling kernel can set
        if (J.sp_rows > 0) {
            const cudaStream_t ss = next();
            const unsigned early = mask & (ST_INVALID | ST_AB_STAGE | ST_AB_ARENA);
            launch_k(k_split_prep, 1, 1024, 0, ss, A, J, ctl, early);
            // blocks of DS_NT threads, 1024 threads an SM: a row's fold waits for fewer warps
            launch_k(k_num_dsplit<SR, DS_NT>, (unsigned)((1024 / DS_NT) * num_sms), DS_NT, smem_c, ss, A, B, C, J,
                     ctl, early, mp);
        }
        launch_s64();
        return;
    }
    if (on(BIN_G16)) launch_group_hash<SR, 6, 16, 8>(A, B, C, J, ctl, mask, BIN_G16, next(), num_sms);
    if (on(BIN_G8)) launch_group_hash<SR, 5, 8, 8>(A, B, C, J, ctl, mask, BIN_G8, next(), num_sms);
    if (on(BIN_W128)) launch_group_hash<SR, 7, 32, 8>(A, B, C, J, ctl, mask, BIN_W128, next(), num_sms);
    if (on(BIN_W256)) launch_group_hash<SR, 8, 32, 8>(A, B, C, J, ctl, mask, BIN_W256, next(), num_sms);
    if (on(BIN_W512)) launch_group_hash<SR, 9, 32, 4>(A, B, C, J, ctl, mask, BIN_W512, next(), num_sms);
    if (on(BIN_W1024)) launch_group_hash<SR, 10, 32, 4>(A, B, C, J, ctl, mask, BIN_W1024, next(), num_sms);
    if (on(BIN_C2048)) launch_cta_hash<SR, 11>(A, B, C, J, ctl, mask, BIN_C2048, next(), num_sms);
    if (on(BIN_C4096)) launch_cta_hash<SR, 12>(A, B, C, J, ctl, mask, BIN_C4096, next(), num_sms);
    if (on(BIN_C8192)) launch_cta_hash<SR, 13>(A, B, C, J, ctl, mask, BIN_C8192, next(), num_sms);
    if (on(BIN_C16384)) launch_cta_hash<SR, 14>(A, B, C, J, ctl, mask, BIN_C16384, next(), num_sms);
    if (on(BIN_K2)) launch_cluster_hash<SR, 13, 2>(A, B, C, J, ctl, mask, BIN_K2, next(), num_sms);
    if (on(BIN_K4)) launch_cluster_hash<SR, 13, 4>(A, B, C, J, ctl, mask, BIN_K4, next(), num_sms);
    if (on(BIN_K8)) launch_cluster_hash<SR, 13, 8>(A, B, C, J, ctl, mask, BIN_K8, next(), num_sms);
    if (on(BIN_K8L)) launch_cluster_hash<SR, 14, 8>(A, B, C, J, ctl, mask, BIN_K8L, next(), num_sms);
    // the global dense bin is always launched: rows of bins that are off go there
    launch_k(k_num_gdense<SR>, grid_for(J.gd_ctas, J.rows_hint, 1), 512, 0, next(), A, B, C, J, ctl, mask, (int)BIN_GD);
    launch_s64();
}

int64_t bin_table_slots(int bin, int64_t m) {
    switch (bin) {
        case BIN_G8: return 32;
        case BIN_G16: return 64;
        case BIN_W128: return 128;
        case BIN_W256: return 256;
        case BIN_W512: return 512;
        case BIN_W1024: return 1024;
        case BIN_C2048: return 2048;
        case BIN_C4096: return 4096;
        case BIN_C8192: return 8192;
        case BIN_C16384: return 16384;
        case BIN_K2: return 2 * 8192;
        case BIN_K4: return 4 * 8192;
        case BIN_K8: return 8 * 8192;
        case BIN_K8L: return 8 * 16384;
        case BIN_GD: case BIN_WDENSE: case BIN_CDENSE: case BIN_DSPLIT: return m;
        default: return 0;  // the thread-merge bins stage the row's products, no table
    }
}

unsigned long long next_bin_mask(const Ctl &c, unsigned long long on, bool narrowed) {
    unsigned long long used = c.bins_wanted | (1ull << BIN_GD);
    for (int b = 0; b < BIN_COUNT; b++)
        if (c.bin_count[b] > 0) used |= 1ull << b;
    return narrowed ? (on | used) : used;
}

void run_numeric(int sr, const MatView &A, const MatView &B, const MatView &C, const CJob &J, Ctl *ctl, unsigned mask,
                 const cudaStream_t *ss, int ns, int num_sms) {
    if (sr == SR_PT) run_numeric_t<SR_PT>(A, B, C, J, ctl, mask, ss, ns, num_sms);
    else run_numeric_t<SR_MP>(A, B, C, J, ctl, mask, ss, ns, num_sms);
}

}  // namespace dspg
