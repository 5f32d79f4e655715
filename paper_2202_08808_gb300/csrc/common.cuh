// common.cuh -- types and device helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dspg.h"

namespace dspg {

constexpr int SR_PT = 0;  // (+,.) on double
constexpr int SR_MP = 1;  // (min,+) on int32

constexpr int32_t MP_INF = 0x7fffffff;     // (min,+) additive neutral element
constexpr int32_t MP_LIMIT = 1 << 30;      // |value| bound for (min,+)

// Device status bits (Ctl::status).  A kernel returns at entry when any bit
// of the mask it depends on is set, so nothing is mutated after a failed
// check.  Overflow bits are not errors: the host grows the buffer named by
// the bit and re-runs the stage that set it.
enum : unsigned {
    ST_INVALID = 1u << 0,     // batch failed validation
    ST_AB_STAGE = 1u << 1,    // A/B merge staging too small
    ST_AB_ARENA = 1u << 2,    // A/B arena cannot take relocated rows
    ST_AT_STAGE = 1u << 3,    // transposed-pattern staging too small
    ST_AT_ARENA = 1u << 4,    // transposed-pattern arena exhausted
    ST_C_STAGE = 1u << 5,     // C staging too small
    ST_C_ARENA = 1u << 6,     // C arena exhausted
    ST_C_SCRATCH = 1u << 7,   // accumulator scratch too small
    ST_TIMEOUT = 1u << 8,     // a bounded probe loop gave up
    ST_ALG_FULL = 1u << 9,    // the delta path's list of new C entries is full: recompute the touched rows
    ST_MASK_FULL = 1u << 10,  // the masked path's contribution or kept-entry list is full: grow it, run again
    ST_DEBUG = 1u << 11,      // a check of the debug build failed (code and index in the control block)
};
constexpr unsigned M_AB = ST_INVALID | ST_AB_STAGE | ST_AB_ARENA | ST_TIMEOUT;
constexpr unsigned M_AT = M_AB | ST_AT_STAGE | ST_AT_ARENA;
constexpr unsigned M_C = M_AB | ST_C_STAGE | ST_C_ARENA | ST_C_SCRATCH;

// Update operation codes as received, plus DEAD for an earlier duplicate of
// a key (only the last write of a key in a batch takes effect).
enum : uint8_t { OP_INSERT = 0, OP_DELETE = 1, OP_SET = 2, OP_DEAD = 3 };

// Classification of a unique update against the row it targets.
enum : uint8_t { K_NOP = 0, K_INS = 1, K_UPD = 2, K_DEL = 3 };

// Counters of one matrix update (sort -> classify -> merge -> commit).
struct UpdCtl {
    long long n_seg;      // row segments of the sorted batch
    long long n_merge;    // rows with at least one effective change
    long long n_chunk;    // merge copy work items
    long long stage_top;  // staging entries handed out
    long long n_cchunk;   // commit copy work items
    long long ins, upd, del, nop;
    long long reloc;      // rows moved to the arena tail
    long long pad[5];
};

constexpr int NBINS = 24;

struct Ctl {
    unsigned status;
    unsigned pad0;
    UpdCtl u[3];               // 0: A, 1: B, 2: transposed pattern of A
    long long n_affected;      // |R|
    long long c_stage_top;     // C staging entries handed out
    long long c_chunk;         // C commit copy items
    long long c_reloc;
    long long products;
    long long nnz_written;
    long long scratch_top;     // accumulator scratch handed out
    long long n_K;             // rows of B* (detection)
    long long bin_count[NBINS];
    long long ubc_total;       // sum over rows of min(product bound, columns)
    long long a_entries;       // A' entries read by the recompute
    long long n_est;           // rows sized by the learned estimator
    long long n_ovf;           // of those, rows whose table overflowed
    long long timeout_bin;     // 1 + the bin whose table or staging overflowed (ST_TIMEOUT)
    long long timeout_row;     // a row it happened on
    long long timeout_ub;      // that row's product bound, summed again when it happened
    long long alg_new;         // delta path: new entries of C listed
    long long alg_contrib;     // delta path: contributions formed (products of Eq. 1's two terms)
    long long mask_n;          // masked path: contributions to the pattern of C* formed
    long long mask_kept;       // masked path: entries of A' kept by the Bloom filter (A^R)
    long long mask_u;          // masked path: entries of C*
    long long dbg_code;        // debug build: the first failed check's code (0: none) and index
    long long dbg_idx;
    unsigned long long bins_wanted;  // bins (bit b) whose rows went to the global dense bin instead
};

// A row-slack CSR ("slack-CSR") on the device: row i occupies
// col[off[i] .. off[i]+len[i]) with room for cap[i] entries; rows are kept
// column-sorted.  Rows that outgrow their room move to the arena tail
// (top), and the whole arena is rebuilt when the tail is exhausted.
struct MatView {
    int64_t nrows, ncols;
    int64_t *off;
    int32_t *len;
    int32_t *cap;
    int32_t *col;
    void *val;            // double* or int32_t*, nullptr for a pattern
    long long *top;       // arena high-water mark (device)
    int64_t arena_cap;    // entries
};

__host__ __device__ inline int32_t slack_cap(int64_t len, int slack_min, int slack_div) {
    int64_t extra = len / slack_div;
    if (extra < slack_min) extra = slack_min;
    int64_t c = len + extra;
    c = (c + 3) & ~int64_t(3);  // 16-byte aligned rows for int32 columns
    return (int32_t)c;
}

__host__ __device__ inline int bits_for(int64_t x) {  // bits to hold values in [0, x)
    int b = 1;
    while (b < 63 && (int64_t(1) << b) < x) b++;
    return b;
}

#ifdef __CUDACC__

// Programmatic dependent launch: every kernel is launched so that it may
// start while the kernel before it on the stream is finishing (launch_k).
// Its first step waits until that kernel has completed and its writes are
// visible (griddepcontrol.wait, a no-op without such a predecessor), then
// lets its own successor start launching (launch_dependents), which will in
// turn wait for this kernel's completion before reading anything.  So every
// kernel calls pdl_begin() before its first access to global memory.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" :::);
}

__device__ __forceinline__ bool failed(const Ctl *ctl, unsigned mask) {
    return (*(volatile const unsigned *)&ctl->status & mask) != 0u;
}

__device__ __forceinline__ void set_status(Ctl *ctl, unsigned bit) { atomicOr(&ctl->status, bit); }

// The debug build (DSPG_DEBUG=1) checks indices and room before its
// accesses: a failed check records its code and the offending index (the
// first one only), sets ST_DEBUG, and returns false so that the caller
// skips the access; the batch then fails with the code in its message.
// Without DSPG_DEBUG the checks compile to nothing (always true).
#ifndef DSPG_DEBUG
#define DSPG_DEBUG 0
#endif
enum : int {
    DBG_B_ROW = 1,      // a column of A is not a row of B
    DBG_C_ROOM = 2,     // a row of C written past its capacity or the arena
    DBG_BIN_SLOT = 3,   // a bin list written past its capacity
    DBG_STAGE = 4,      // merge staging written past its capacity
    DBG_ARENA = 5,      // a committed row of A, B or the pattern past its arena
    DBG_MASK_ROOM = 6,  // the masked merge wrote a row of C past its room
    DBG_R_ROW = 7,      // a row of R is not a row of A, or its entries lie outside A's arena
};
__device__ __forceinline__ bool dcheck(Ctl *ctl, bool ok, int code, long long idx) {
#if DSPG_DEBUG
    if (!ok) {
        if (atomicCAS((unsigned long long *)&ctl->dbg_code, 0ull, (unsigned long long)code) == 0ull) ctl->dbg_idx = idx;
        set_status(ctl, ST_DEBUG);
    }
    return ok;
#else
    (void)ctl; (void)code; (void)idx;
    return ok || true;
#endif
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Warp-aggregated fetch-and-add on a device counter: all 32 lanes call it,
// each with its own amount (0 allowed); lane l gets the counter value plus
// the amounts of lanes < l.  One atomic per warp instead of one per lane, so
// a counter shared by the whole grid does not serialise the kernel.
__device__ __forceinline__ long long warp_fetch_add(long long *ctr, long long amount) {
    const int lane = threadIdx.x & 31;
    const long long incl = warp_incl_scan<long long>(amount);
    const long long tot = __shfl_sync(0xffffffffu, incl, 31);
    long long base = 0;
    if (lane == 31 && tot != 0) base = (long long)atomicAdd((unsigned long long *)ctr, (unsigned long long)tot);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + incl - amount;
}

// First index in [lo, hi) with a[idx] >= x (a ascending).
template <typename T>
__device__ __forceinline__ int64_t lower_bound_dev(const T *a, int64_t lo, int64_t hi, T x) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// lower_bound_dev with fewer loads in a row: while more than eight entries
// remain, seven pivots loaded together split the range into eight; the last
// eight at most are loaded together and counted.  A search in a row of
// thousands of entries then waits for about four loads one after another
// instead of a dozen.
template <typename T>
__device__ __forceinline__ int64_t lower_bound_wide(const T *a, int64_t lo, int64_t hi, T x) {
    while (hi - lo > 8) {
        const int64_t len = hi - lo;
        T v[7];  // pivot j at lo + len (j + 1) / 8
#pragma unroll
        for (int j = 0; j < 7; j++) v[j] = a[lo + (len * (j + 1)) / 8];
        int c = 0;  // pivots below x: a prefix of them, a being ascending
#pragma unroll
        for (int j = 0; j < 7; j++) c += v[j] < x;
        const int64_t nlo = c == 0 ? lo : lo + (len * c) / 8 + 1;
        const int64_t nhi = c == 7 ? hi : lo + (len * (c + 1)) / 8;
        lo = nlo;
        hi = nhi;
    }
    int c = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) c += (lo + j < hi) && (a[lo + j] < x);
    return lo + c;
}

// First index in [lo, hi) with a[idx] > x.
template <typename T>
__device__ __forceinline__ int64_t upper_bound_dev(const T *a, int64_t lo, int64_t hi, T x) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// End of the run of x that starts at s in the sorted array a[0, n) (a[s] ==
// x): the first index past it.  Galloping forward (1, 2, 4, ... entries)
// before the binary search makes a short run cost a load or two instead of
// a search over the whole array.
template <typename T>
__device__ __forceinline__ int64_t run_end_dev(const T *a, int64_t s, int64_t n, T x) {
    int64_t lo = s, step = 1, hi = s + 1 < n ? s + 1 : n;
    while (hi < n && a[hi] == x) {
        lo = hi;
        step <<= 1;
        hi = lo + step < n ? lo + step : n;
    }
    return upper_bound_dev<T>(a, lo + 1, hi, x);
}

#endif  // __CUDACC__

// ---------------------------------------------------------------- host side

// Every kernel of the library is launched through launch_k, which counts
// launches (process-wide) so that callers can audit the work of a call.
unsigned long long &launch_counter();

#ifdef __CUDACC__
// The launch attribute that lets a kernel start before its predecessor on
// the stream has finished (it waits in pdl_begin); in a captured graph it
// becomes a programmatic dependency between the two kernel nodes.
inline cudaLaunchAttribute pdl_attribute() {
    cudaLaunchAttribute a;
    a.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a.val.programmaticStreamSerializationAllowed = 1;
    return a;
}

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1] = {pdl_attribute()};
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);  // errors surface through cudaGetLastError
    __atomic_fetch_add(&launch_counter(), 1ull, __ATOMIC_RELAXED);
}
#endif

// Device scan: out[i] = sum_{j<i} in[j] for i <= n (out has n+1 entries).
void scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);
void scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t s);
int64_t scan_tmp_entries(int64_t n);

// Where a batch's arrays are: a small device-side block the pipeline reads,
// so that a captured pipeline can take new input pointers on every launch.
struct InArgs {
    const int32_t *row;
    const int32_t *col;
    const void *val;
    const uint8_t *op;
    int64_t n;  // entries; launches are sized for a bucket of at least n, kernels stop at n
};

// Launch size of a batch of n entries: n rounded up to a multiple of 1024
// (the batch sort's tile) up to 16384, the next power of two beyond (0 for
// an empty batch).  One captured pipeline serves every batch of the same
// launch size: its kernels read the true length from the argument block.
inline int64_t batch_bucket(int64_t n) {
    if (n <= 0) return 0;
    if (n <= 16384) return (n + 1023) / 1024 * 1024;
    int64_t b = 32768;
    while (b < n) b <<= 1;
    return b;
}

// Sort a batch of updates by (row, col), keep the last write of each key:
// see sort.cu.
struct SortOut {
    int32_t *row, *col;
    void *val;
    uint8_t *op;
};
struct SortTmp {
    uint64_t *k0, *k1;
    uint32_t *i0, *i1;
    uint32_t *counts;
    int64_t *scan_tmp;
    int64_t *scan_out;
    int64_t cap;      // entries
    int64_t cnt_cap;  // count entries
};
int64_t sort_small_max();
void sort_tmp_sizes(int64_t n, int64_t *count_entries);
// Validate + sort + dedupe the in->n updates of a matrix with the given shape;
// n is the launch size (at least in->n, e.g. batch_bucket(in->n)).
// Sets ST_INVALID in ctl on a bad entry.
// Kernels return at entry when a bit of skip_mask is set in ctl->status.
void sort_updates(const InArgs *in, int64_t n, int64_t nrows, int64_t ncols, int sr, bool check_values, SortOut out,
                  SortTmp tmp, Ctl *ctl, unsigned skip_mask, cudaStream_t s);
// Stable sort of (key, value) pairs by the low `bits` bits of key (multi-CTA).
void radix_sort_pairs(uint64_t *k, uint32_t *v, uint64_t *k_alt, uint32_t *v_alt, int64_t n, int bits,
                      uint32_t *counts, int64_t *scan_tmp, int64_t *scan_out, cudaStream_t s, bool *result_in_alt);

}  // namespace dspg
