// sort.cu -- batch sort by (row, col) with last-writer-wins de-duplication.
//
// The paper groups updates by destination with counting sorts before the
// local insertion (Section 4.2); on one GPU the same grouping is an LSD
// radix sort of the 64-bit key (row << cb | col).  Equal keys keep arrival
// order (the sort is stable), so the last entry of each run of equal keys is
// the write that takes effect; earlier ones are marked OP_DEAD.
//
// Two paths:
//  * small batches (<= 8192 entries, key + index bits <= 64): one CTA does
//    validation, key packing, all radix passes in shared memory, and the
//    de-duplicating gather in a single launch;
//  * larger batches: a key kernel, then per 8-bit digit a histogram kernel,
//    a device scan of the digit counts, and a stable scatter kernel, then a
//    gather kernel.
//
// Stable ranking inside a CTA: each warp owns a contiguous segment of the
// tile and walks it 32 entries at a time; __match_any_sync groups lanes
// with equal digits, the rank inside the group is a popcount, and a per-warp
// shared-memory counter per digit carries ranks across rounds.  Per-digit
// prefixes over warps (in warp order) then give each entry its position.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace dspg {

// ------------------------------------------------------------ validation

__device__ __forceinline__ bool entry_ok(int32_t r, int32_t c, uint8_t o, const void *val, int64_t i,
                                         int64_t nrows, int64_t ncols, int sr, bool check_values) {
    if (r < 0 || (int64_t)r >= nrows || c < 0 || (int64_t)c >= ncols || o > OP_SET) return false;
    if (check_values && o != OP_DELETE) {
        if (sr == SR_PT) {
            double v = ((const double *)val)[i];
            if (!isfinite(v)) return false;
        } else {
            int32_t v = ((const int32_t *)val)[i];
            if (v <= -MP_LIMIT || v >= MP_LIMIT) return false;
        }
    }
    return true;
}

__device__ __forceinline__ void write_sorted(SortOut out, int64_t s, uint64_t key, uint64_t idx, bool dead,
                                             int cb, const void *val, const uint8_t *op, int sr) {
    out.row[s] = (int32_t)(key >> cb);
    out.col[s] = (int32_t)(key & ((uint64_t(1) << cb) - 1));
    if (out.val != nullptr) {  // pattern batches carry no values
        if (sr == SR_PT) ((double *)out.val)[s] = ((const double *)val)[idx];
        else ((int32_t *)out.val)[s] = ((const int32_t *)val)[idx];
    }
    out.op[s] = dead ? OP_DEAD : op[idx];
}

// ---------------------------------------------------- cluster-sort path
//
// Batches up to 16384 entries whose packed word (key << ib | arrival index)
// fits 64 bits are sorted by one launch: a thread-block cluster with a CTA
// per tile of 1024 words (512 threads; up to 16 CTAs where the device allows
// clusters that large, else tiles of 2048 words in up to 8 CTAs of 1024
// threads).  Each CTA sorts its tile with a bitonic network held in
// registers (CS_EPT consecutive words per thread: strides below CS_EPT
// inside a thread, strides up to a warp's span by shuffles, longer ones
// through shared memory; the words are distinct, so no stability is
// needed).  The CTAs then copy each other's sorted tiles through
// distributed shared memory, and every word's global rank is its rank in
// its own tile plus the number of smaller words in each other tile (a
// thread's words are consecutive, so each search starts where the previous
// one ended).  A word is dead when a word with the same key and a later
// index exists: the next word of its own tile or, in another tile, the
// first word above it.

constexpr int CS_EPT = 2;   // words per thread
constexpr int CS_MAXT = 8;  // the portable cluster size

int64_t sort_small_max() { return (int64_t)2048 * CS_MAXT; }

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a < b ? b : a; }

// number of words of t[lo, hi) below x (t sorted)
__device__ __forceinline__ int count_below(const uint64_t *t, int lo, int hi, uint64_t x) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (t[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Compare-exchange of x (at position i) with its partner y at distance
// stride in a bitonic merge of size `size`: the lower position keeps the
// smaller word when the run ascends.
__device__ __forceinline__ uint64_t bitonic_keep(uint64_t x, uint64_t y, int i, int stride, int size) {
    const bool keep_min = ((i & stride) == 0) == ((i & size) == 0);
    return keep_min ? umin64(x, y) : umax64(x, y);
}

// Steps of distance 4, 2, 1 of a merge of size >= 8: inside the thread, in
// one direction (asc) for all of its words.
__device__ __forceinline__ void bitonic_in_thread(uint64_t (&x)[CS_EPT], bool asc) {
#pragma unroll
    for (int stride = CS_EPT / 2; stride > 0; stride >>= 1)
#pragma unroll
        for (int e = 0; e < CS_EPT; e++)
            if ((e & stride) == 0) {
                const uint64_t a = x[e], b = x[e | stride];
                x[e] = asc ? umin64(a, b) : umax64(a, b);
                x[e | stride] = asc ? umax64(a, b) : umin64(a, b);
            }
}

// Bitonic sort of the tile, word e of thread tid at position tid * CS_EPT + e.
// Merges up to CS_EPT words run inside the thread (unrolled); the larger ones
// are loops whose steps reach the partner by shuffle (within a warp's span)
// or through shared memory, so the code stays small.  Only the first `span`
// positions (a power of two, the same across the CTA) hold words: the rest
// is padding, which sorts last and is already in place, so the merges stop
// at size span (a one-entry batch then skips the network).
template <int TILE>
__device__ __forceinline__ void bitonic_sort_tile(uint64_t (&x)[CS_EPT], uint64_t *own, int tid, int span) {
#pragma unroll
    for (int size = 2; size <= CS_EPT; size <<= 1)
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
            for (int e = 0; e < CS_EPT; e++)
                if ((e & stride) == 0) {
                    const int i = tid * CS_EPT + e;
                    const uint64_t a = x[e], b = x[e | stride];
                    const bool asc = (i & size) == 0;
                    x[e] = asc ? umin64(a, b) : umax64(a, b);
                    x[e | stride] = asc ? umax64(a, b) : umin64(a, b);
                }
#pragma unroll 1
    for (int size = 2 * CS_EPT; size <= span; size <<= 1) {
#pragma unroll 1
        for (int stride = size >> 1; stride >= CS_EPT; stride >>= 1) {
            if (stride >= CS_EPT * 32) {  // partner in another warp
#pragma unroll
                for (int e = 0; e < CS_EPT; e++) own[tid * CS_EPT + e] = x[e];
                __syncthreads();
#pragma unroll
                for (int e = 0; e < CS_EPT; e++) {
                    const int i = tid * CS_EPT + e;
                    x[e] = bitonic_keep(x[e], own[i ^ stride], i, stride, size);
                }
                __syncthreads();
            } else {  // partner in another lane
                const int lm = stride / CS_EPT;
#pragma unroll
                for (int e = 0; e < CS_EPT; e++) {
                    const uint64_t y = __shfl_xor_sync(0xffffffffu, (unsigned long long)x[e], lm);
                    x[e] = bitonic_keep(x[e], y, tid * CS_EPT + e, stride, size);
                }
            }
        }
        bitonic_in_thread(x, ((tid * CS_EPT) & size) == 0);
    }
}

template <int NT>
__global__ void __launch_bounds__(NT)
k_cluster_sort(const InArgs *in, int64_t nrows, int64_t ncols, int sr, bool check_values, SortOut out, Ctl *ctl,
               unsigned skip_mask, int cb, int ib) {
    pdl_begin();
    const int n = (int)in->n;  // the launch covers a bucket of at least n words
    constexpr int TILE = NT * CS_EPT;
    extern __shared__ uint64_t tiles[];  // slot u: the sorted tile of CTA u
    cg::cluster_group cl = cg::this_cluster();
    // no early return: every CTA of the cluster must reach both cluster barriers
    const bool skip = failed(ctl, skip_mask);
    const int tid = threadIdx.x;
    const int me = blockIdx.x, nt = gridDim.x;
    const int lo = me * TILE;
    const int cnt = min(TILE, n - lo);
    uint64_t *own = tiles + (size_t)me * TILE;
    uint64_t x[CS_EPT];
    if (!skip) {
        const int32_t *row = in->row, *col = in->col;
        const void *val = in->val;
        const uint8_t *op = in->op;
#pragma unroll
        for (int e = 0; e < CS_EPT; e++) {
            const int i = tid * CS_EPT + e;
            uint64_t w = ~uint64_t(0);  // padding sorts last
            if (i < cnt) {
                const int gi = lo + i;
                const int32_t r = row[gi], c = col[gi];
                const uint8_t o = op[gi];
                const bool ok = entry_ok(r, c, o, val, gi, nrows, ncols, sr, check_values);
                if (!ok) set_status(ctl, ST_INVALID);
                const uint64_t key = ok ? (((uint64_t)(uint32_t)r << cb) | (uint32_t)c) : 0;
                w = (key << ib) | (uint64_t)gi;
            }
            x[e] = w;
        }
    } else {
#pragma unroll
        for (int e = 0; e < CS_EPT; e++) x[e] = ~uint64_t(0);
    }
    // bitonic sort of the tile: position of x[e] is tid * CS_EPT + e; the
    // merges cover the smallest power of two that holds the tile's words
    int span = CS_EPT;
    while (span < cnt) span <<= 1;
    bitonic_sort_tile<TILE>(x, own, tid, span);
#pragma unroll
    for (int e = 0; e < CS_EPT; e++) own[tid * CS_EPT + e] = x[e];
    cl.sync();
    // the other tiles into this CTA's shared memory (16-byte loads)
    for (int u = 0; u < nt; u++) {
        if (u == me) continue;
        const uint4 *src = (const uint4 *)cl.map_shared_rank(tiles + (size_t)u * TILE, u);
        uint4 *dst = (uint4 *)(tiles + (size_t)u * TILE);
        for (int k = tid; k < TILE / 2; k += NT) dst[k] = src[k];
    }
    cl.sync();  // no CTA leaves while another still reads its tile
    if (skip) return;
    const uint64_t imask = (uint64_t(1) << ib) - 1;
    int rank[CS_EPT];
    bool dead[CS_EPT];
    const int nv = max(0, min(CS_EPT, cnt - tid * CS_EPT));  // this thread's real words
#pragma unroll
    for (int e = 0; e < CS_EPT; e++) {
        rank[e] = tid * CS_EPT + e;
        const int nx = tid * CS_EPT + e + 1;
        dead[e] = nx < cnt && ((own[nx] >> ib) == (x[e] >> ib));
    }
    if (nv > 0)
        for (int u = 0; u < nt; u++) {
            if (u == me) continue;
            const uint64_t *t = tiles + (size_t)u * TILE;
            const int cu = min(TILE, n - u * TILE);
            int p = count_below(t, 0, cu, x[0]);
#pragma unroll
            for (int e = 0; e < CS_EPT; e++) {
                const uint64_t xe = x[e];  // padding words (e >= nv) leave p where it is
                const bool real = e < nv;
                // a few steps forward, then a search over the rest
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (real && p < cu && t[p] < xe) p++;
                if (real && p < cu && t[p] < xe) p = count_below(t, p, cu, xe);
                rank[e] += p;
                dead[e] |= real && p < cu && ((t[p] >> ib) == (xe >> ib));
            }
        }
    const void *val = in->val;
    const uint8_t *op = in->op;
#pragma unroll
    for (int e = 0; e < CS_EPT; e++)
        if (e < nv) write_sorted(out, rank[e], x[e] >> ib, x[e] & imask, dead[e], cb, val, op, sr);
}

// ------------------------------------------------- cluster radix path
//
// Batches of more than 8192 entries (up to 16384) where clusters of 16 CTAs
// are allowed: the same one-launch contract as k_cluster_sort, but an LSD
// radix sort across the cluster instead of the bitonic network and the
// cross-tile rank searches, whose work grows with the number of tiles.  The
// words start in arrival order (word p of the batch in slot p mod 1024 of
// CTA p / 1024) and go through passes over the key's digits (at most 8 bits
// each, as few passes as the key's width needs).  Each pass:
//  * every warp ranks its 2 x 32 slots by digit: the lanes holding the same
//    digit are found with one ballot per digit bit, and a per-warp
//    shared-memory counter per digit carries ranks from the first 32 slots
//    to the next, which keeps slot order among equal digits;
//  * the CTA turns the warps' counts into per-warp offsets and its digit
//    totals, which the other CTAs read through distributed shared memory
//    (one cluster barrier);
//  * each CTA derives, per digit, the words of smaller digits in the whole
//    cluster plus those of the same digit in lower CTAs, and every word is
//    stored straight into the slot of its new position, in the CTA that
//    owns it (distributed shared memory; a second barrier).
// The sort is stable, so equal keys keep arrival order; a word is dead when
// the word after it (in the next CTA for a tile's last slot) has its key.
// The output is written at the words' final positions, consecutive across a
// warp's lanes.  On GB300 it takes a 10^4-entry batch in about 26 us against
// 31 us for k_cluster_sort (16384 entries: 29 against 43 us), and is slower
// below about 8192 entries.

constexpr int CS_DIG = 256;  // digit counters (at most 8-bit digits)
constexpr int CS_MAXC = 16;  // CTAs of the radix path's cluster

// dynamic shared memory of k_cluster_radix<NT>: the tile, the per-warp digit
// counters, the CTA's digit totals, the digit bases and the scan's warp sums
static size_t cluster_radix_smem(int nt) {
    return (size_t)nt * CS_EPT * sizeof(uint64_t) + ((size_t)(nt / 32) * CS_DIG + 2 * CS_DIG + 32) * sizeof(uint32_t);
}

template <int NT>
__global__ void __launch_bounds__(NT)
k_cluster_radix(const InArgs *in, int64_t nrows, int64_t ncols, int sr, bool check_values, SortOut out, Ctl *ctl,
                unsigned skip_mask, int cb, int ib, int kb) {
    pdl_begin();
    constexpr int TILE = NT * CS_EPT;
    constexpr int NW = NT / 32;
    extern __shared__ uint64_t cr_smem[];
    uint64_t *tile = cr_smem;                          // TILE words: this CTA's slots
    uint32_t *wc = (uint32_t *)(cr_smem + TILE);      // NW x CS_DIG per-warp counts, then offsets
    uint32_t *tot = wc + NW * CS_DIG;                  // this CTA's count per digit (read by the cluster)
    uint32_t *base = tot + CS_DIG;                     // first position of each digit's words of this CTA
    uint32_t *wsum = base + CS_DIG;                    // warp sums of the digit scan
    cg::cluster_group cl = cg::this_cluster();
    // no early return: every CTA of the cluster must reach every cluster barrier
    const bool skip = failed(ctl, skip_mask);
    const int n = (int)in->n;  // the launch covers a bucket of at least n words
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int me = blockIdx.x, nt = gridDim.x;
    // slot of word e of this thread: w * 64 + e * 32 + lane
    uint64_t x[CS_EPT];
#pragma unroll
    for (int e = 0; e < CS_EPT; e++) {
        const int gi = me * TILE + w * 32 * CS_EPT + e * 32 + lane;
        uint64_t word = ~uint64_t(0);  // padding sorts last
        if (!skip && gi < n) {
            const int32_t r = in->row[gi], c = in->col[gi];
            const uint8_t o = in->op[gi];
            const bool ok = entry_ok(r, c, o, in->val, gi, nrows, ncols, sr, check_values);
            if (!ok) set_status(ctl, ST_INVALID);
            const uint64_t key = ok ? (((uint64_t)(uint32_t)r << cb) | (uint32_t)c) : 0;
            word = (key << ib) | (uint64_t)gi;
        }
        x[e] = word;
    }
    const int passes = (kb + 7) / 8;
    const int width = passes > 0 ? (kb + passes - 1) / passes : 0;
    const int nd = 1 << width;
    uint32_t *mine = wc + w * CS_DIG;
    for (int p = 0; p < passes; p++) {
        const int shift = ib + p * width;
        for (int d = lane; d < nd; d += 32) mine[d] = 0;
        __syncwarp();
        unsigned dg[CS_EPT];
        uint32_t lr[CS_EPT];
#pragma unroll
        for (int e = 0; e < CS_EPT; e++) {
            dg[e] = (unsigned)(x[e] >> shift) & (unsigned)(nd - 1);
            unsigned peers = 0xffffffffu;
#pragma unroll
            for (int b = 0; b < 8; b++)
                if (b < width) {
                    const bool bit = (dg[e] >> b) & 1u;
                    const unsigned bal = __ballot_sync(0xffffffffu, bit);
                    peers &= bit ? bal : ~bal;
                }
            const uint32_t before = mine[dg[e]];
            __syncwarp();  // every lane has read the counter before the group's last lane bumps it
            lr[e] = before + __popc(peers & lanemask_lt());
            if (lane == 31 - __clz(peers)) mine[dg[e]] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        for (int d = tid; d < nd; d += NT) {  // per-warp offsets inside the CTA, warp order
            uint32_t c[NW];
#pragma unroll
            for (int ww = 0; ww < NW; ww++) c[ww] = wc[ww * CS_DIG + d];
            uint32_t run = 0;
#pragma unroll
            for (int ww = 0; ww < NW; ww++) {
                wc[ww * CS_DIG + d] = run;
                run += c[ww];
            }
            tot[d] = run;
        }
        cl.sync();  // every CTA's totals are complete
        if (tid < CS_DIG) {  // warps 0..7: the digit bases (an exclusive scan over digits)
            const int d = tid;
            uint32_t t[CS_MAXC];  // the other CTAs' counts, loaded together
#pragma unroll
            for (int u = 0; u < CS_MAXC; u++) t[u] = (d < nd && u < nt) ? *cl.map_shared_rank(tot + d, u) : 0u;
            uint32_t all = 0, lower = 0;
#pragma unroll
            for (int u = 0; u < CS_MAXC; u++) {
                all += t[u];
                lower += u < me ? t[u] : 0u;
            }
            uint32_t inc = all;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) wsum[w] = inc;
            asm volatile("bar.sync 1, %0;" ::"r"(CS_DIG));  // the scanning warps only
            uint32_t off = 0;
            for (int ww = 0; ww < w; ww++) off += wsum[ww];
            base[d] = off + inc - all + lower;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < CS_EPT; e++) {
            const uint32_t pos = base[dg[e]] + mine[dg[e]] + lr[e];
            *cl.map_shared_rank(tile + (pos % TILE), (int)(pos / TILE)) = x[e];
        }
        cl.sync();  // every word is in its new slot
#pragma unroll
        for (int e = 0; e < CS_EPT; e++) x[e] = tile[w * 32 * CS_EPT + e * 32 + lane];
    }
    if (passes == 0) {  // one key: the slots still hold arrival order
#pragma unroll
        for (int e = 0; e < CS_EPT; e++) tile[w * 32 * CS_EPT + e * 32 + lane] = x[e];
        cl.sync();
    }
    // a word is dead when the next position holds its key
    bool dead[CS_EPT];
#pragma unroll
    for (int e = 0; e < CS_EPT; e++) {
        const int slot = w * 32 * CS_EPT + e * 32 + lane;
        const int pos = me * TILE + slot;
        uint64_t nx = ~uint64_t(0);
        if (pos + 1 < n) nx = slot + 1 < TILE ? tile[slot + 1] : *cl.map_shared_rank(tile, me + 1);
        dead[e] = pos + 1 < n && (nx >> ib) == (x[e] >> ib);
    }
    cl.sync();  // no CTA leaves while another still reads its first slot
    if (skip) return;
    const uint64_t imask = (uint64_t(1) << ib) - 1;
#pragma unroll
    for (int e = 0; e < CS_EPT; e++) {
        const int pos = me * TILE + w * 32 * CS_EPT + e * 32 + lane;
        if (pos < n) write_sorted(out, pos, x[e] >> ib, x[e] & imask, dead[e], cb, in->val, in->op, sr);
    }
}

// ------------------------------------------------------- multi-CTA path

constexpr int MS_NT = 512;
constexpr int MS_NW = MS_NT / 32;
constexpr int MS_IPT = 8;
constexpr int MS_TILE = MS_NT * MS_IPT;
constexpr int MS_ROUNDS = MS_TILE / MS_NT;

void sort_tmp_sizes(int64_t n, int64_t *count_entries) {
    int64_t nb = (n + MS_TILE - 1) / MS_TILE;
    *count_entries = 256 * (nb > 0 ? nb : 1);
}

__global__ void k_make_keys(const InArgs *in, int64_t n, int64_t nrows, int64_t ncols, int sr, bool check_values,
                            Ctl *ctl, unsigned skip_mask, int cb, uint64_t *k, uint32_t *v) {
    pdl_begin();
    if (failed(ctl, skip_mask)) return;
    const int32_t *row = in->row, *col = in->col;
    const void *val = in->val;
    const uint8_t *op = in->op;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i >= in->n) {  // padding up to the launch size: sorts after every entry
        k[i] = ~uint64_t(0);
        v[i] = (uint32_t)i;
        return;
    }
    int32_t r = row[i], c = col[i];
    bool ok = entry_ok(r, c, op[i], val, i, nrows, ncols, sr, check_values);
    if (!ok) set_status(ctl, ST_INVALID);
    k[i] = ok ? (((uint64_t)(uint32_t)r << cb) | (uint32_t)c) : 0;
    v[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(MS_NT)
k_hist(const uint64_t *k, int64_t n, int shift, uint32_t *counts, int64_t nb) {
    pdl_begin();
    __shared__ uint32_t h[256];
    for (int j = threadIdx.x; j < 256; j += MS_NT) h[j] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * MS_TILE;
    for (int j = 0; j < MS_IPT; j++) {
        int64_t i = base + (int64_t)j * MS_NT + threadIdx.x;
        if (i < n) atomicAdd(&h[(k[i] >> shift) & 255], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += MS_NT) counts[(int64_t)d * nb + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(MS_NT)
k_scatter(const uint64_t *k, const uint32_t *v, int64_t n, int shift, const int64_t *offs, int64_t nb,
          uint64_t *k_out, uint32_t *v_out) {
    pdl_begin();
    __shared__ uint32_t wc[MS_NW * 256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int j = tid; j < MS_NW * 256; j += MS_NT) wc[j] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * MS_TILE;
    const int seg = MS_TILE / MS_NW;
    const int64_t seg_lo = base + (int64_t)w * seg;
    const int64_t seg_hi = min(n, seg_lo + seg);
    uint32_t lr[MS_ROUNDS];
    unsigned dd[MS_ROUNDS];
#pragma unroll
    for (int r = 0; r < MS_ROUNDS; r++) {
        int64_t idx = seg_lo + r * 32 + lane;
        bool valid = idx < seg_hi;
        unsigned d = valid ? (unsigned)((k[idx] >> shift) & 255) : 0xffffffffu;
        dd[r] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = valid ? wc[w * 256 + d] : 0;
        __syncwarp();
        lr[r] = before + __popc(peers & lanemask_lt());
        if (valid && lane == 31 - __clz(peers)) wc[w * 256 + d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    if (tid < 256) {
        uint32_t s = 0;
        for (int ww = 0; ww < MS_NW; ww++) {
            uint32_t c = wc[ww * 256 + tid];
            wc[ww * 256 + tid] = s;
            s += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < MS_ROUNDS; r++) {
        int64_t idx = seg_lo + r * 32 + lane;
        if (idx < seg_hi) {
            unsigned d = dd[r];
            int64_t pos = offs[(int64_t)d * nb + blockIdx.x] + wc[w * 256 + d] + lr[r];
            k_out[pos] = k[idx];
            v_out[pos] = v[idx];
        }
    }
}

__global__ void k_finalize(const uint64_t *k, const uint32_t *v, int64_t n, int cb, const InArgs *in, int sr,
                           SortOut out, const Ctl *ctl, unsigned skip_mask) {
    pdl_begin();
    if (failed(ctl, skip_mask)) return;
    const void *val = in->val;
    const uint8_t *op = in->op;
    n = in->n;  // the entries; the sort covered padding after them
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    uint64_t key = k[s];
    bool dead = (s + 1 < n) && (k[s + 1] == key);
    write_sorted(out, s, key, v[s], dead, cb, val, op, sr);
}

void radix_sort_pairs(uint64_t *k, uint32_t *v, uint64_t *k_alt, uint32_t *v_alt, int64_t n, int bits,
                      uint32_t *counts, int64_t *scan_tmp, int64_t *scan_out, cudaStream_t s, bool *in_alt) {
    int64_t nb = (n + MS_TILE - 1) / MS_TILE;
    bool alt = false;
    for (int shift = 0; shift < bits; shift += 8) {
        const uint64_t *ki = alt ? k_alt : k;
        const uint32_t *vi = alt ? v_alt : v;
        uint64_t *ko = alt ? k : k_alt;
        uint32_t *vo = alt ? v : v_alt;
        launch_k(k_hist, (unsigned)nb, MS_NT, 0, s, ki, n, shift, counts, nb);
        scan_i32_to_i64((const int32_t *)counts, scan_out, 256 * nb, scan_tmp, s);
        launch_k(k_scatter, (unsigned)nb, MS_NT, 0, s, ki, vi, n, shift, scan_out, nb, ko, vo);
        alt = !alt;
    }
    *in_alt = alt;
}

void sort_updates(const InArgs *in, int64_t n, int64_t nrows, int64_t ncols, int sr, bool check_values, SortOut out,
                  SortTmp tmp, Ctl *ctl, unsigned skip_mask, cudaStream_t s) {
    if (n <= 0) return;
    const int cb = bits_for(ncols), rb = bits_for(nrows), ib = bits_for(n);
    const int kb = cb + rb;
    if (n <= sort_small_max() && kb + ib <= 64) {
        // tiles of 1024 words (512 threads) where the cluster may hold as
        // many CTAs as there are tiles (8 portably, 16 where the device
        // allows it), else tiles of 2048 words (1024 threads)
        static int small_tiles_max = 0;  // most 1024-word tiles per cluster
        if (small_tiles_max == 0) {
            const size_t smem16 = (size_t)16 * 1024 * sizeof(uint64_t);
            cudaFuncSetAttribute(k_cluster_sort<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem16);
            cudaFuncSetAttribute(k_cluster_sort<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((size_t)CS_MAXT * 2048 * sizeof(uint64_t)));
            small_tiles_max = 8;
            if (cudaFuncSetAttribute(k_cluster_sort<512>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess) {
                cudaLaunchConfig_t q = {};
                q.gridDim = dim3(16);
                q.blockDim = dim3(512);
                q.dynamicSmemBytes = smem16;
                int cs = 0;
                if (cudaOccupancyMaxPotentialClusterSize(&cs, k_cluster_sort<512>, &q) == cudaSuccess && cs >= 16)
                    small_tiles_max = 16;
            }
            cudaGetLastError();  // the queries' errors are not the pipeline's
        }
        static int radix_ok = -1;  // clusters of 16 CTAs of the radix kernel allowed
        if (radix_ok < 0) {
            radix_ok = 0;
            if (small_tiles_max == 16 &&
                cudaFuncSetAttribute(k_cluster_radix<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cluster_radix_smem(512)) == cudaSuccess &&
                cudaFuncSetAttribute(k_cluster_radix<512>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                    cudaSuccess) {
                cudaLaunchConfig_t q = {};
                q.gridDim = dim3(CS_MAXC);
                q.blockDim = dim3(512);
                q.dynamicSmemBytes = cluster_radix_smem(512);
                int cs = 0;
                if (cudaOccupancyMaxPotentialClusterSize(&cs, k_cluster_radix<512>, &q) == cudaSuccess && cs >= CS_MAXC)
                    radix_ok = 1;
            }
            cudaGetLastError();
        }
        if (radix_ok && n > 8192) {
            const int tiles = (int)((n + 1023) / 1024);
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)tiles);
            cfg.blockDim = dim3(512);
            cfg.dynamicSmemBytes = cluster_radix_smem(512);
            cfg.stream = s;
            cudaLaunchAttribute at[2];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = (unsigned)tiles;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            at[1] = pdl_attribute();
            cfg.attrs = at;
            cfg.numAttrs = 2;
            cudaLaunchKernelEx(&cfg, k_cluster_radix<512>, in, nrows, ncols, sr, check_values, out, ctl, skip_mask, cb,
                               ib, kb);
            __atomic_fetch_add(&launch_counter(), 1ull, __ATOMIC_RELAXED);
            return;
        }
        const bool small = n <= (int64_t)1024 * small_tiles_max;
        const int tile = small ? 1024 : 2048;
        const int tiles = (int)((n + tile - 1) / tile);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)tiles);
        cfg.blockDim = dim3(small ? 512 : 1024);
        cfg.dynamicSmemBytes = (size_t)tiles * tile * sizeof(uint64_t);
        cfg.stream = s;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)tiles;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1] = pdl_attribute();
        cfg.attrs = at;
        cfg.numAttrs = 2;
        // a failed launch stays in the runtime's last error, which the caller checks
        if (small)
            cudaLaunchKernelEx(&cfg, k_cluster_sort<512>, in, nrows, ncols, sr, check_values, out, ctl, skip_mask, cb,
                               ib);
        else
            cudaLaunchKernelEx(&cfg, k_cluster_sort<1024>, in, nrows, ncols, sr, check_values, out, ctl, skip_mask, cb,
                               ib);
        __atomic_fetch_add(&launch_counter(), 1ull, __ATOMIC_RELAXED);
        return;
    }
    unsigned nblk = (unsigned)((n + 255) / 256);
    launch_k(k_make_keys, nblk, 256, 0, s, in, n, nrows, ncols, sr, check_values, ctl, skip_mask, cb, tmp.k0, tmp.i0);
    bool in_alt = false;
    radix_sort_pairs(tmp.k0, tmp.i0, tmp.k1, tmp.i1, n, kb, tmp.counts, tmp.scan_tmp, tmp.scan_out, s, &in_alt);
    launch_k(k_finalize, nblk, 256, 0, s, in_alt ? tmp.k1 : tmp.k0, in_alt ? tmp.i1 : tmp.i0, n, cb, in, sr, out, ctl,
                                    skip_mask);
}

}  // namespace dspg
