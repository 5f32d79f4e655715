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
#include "common.cuh"

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

// ---------------------------------------------------- tile-sort path
//
// Batches up to TS_TILE * TS_MAXT entries whose packed word
// (key << ib | arrival index) fits 64 bits: each CTA sorts one tile of
// TS_TILE words in shared memory with a bitonic network (the words are
// distinct, so no stability is needed), and one merge kernel places every
// word at its global rank = its rank in its own tile + the number of smaller
// words in each other tile (binary searches in a shared-memory copy of all
// tiles).  An entry is dead when a word with the same key and a later index
// exists.  A single tile finishes (de-duplicates and gathers) in the sort
// kernel itself.

constexpr int TS_NT = 256;
constexpr int TS_TILE = 1024;
constexpr int TS_MAXT = 16;
constexpr size_t TS_SMEM = TS_TILE * sizeof(uint64_t);
constexpr size_t TM_SMEM = (size_t)TS_TILE * TS_MAXT * sizeof(uint64_t);

int64_t sort_small_max() { return (int64_t)TS_TILE * TS_MAXT; }

__global__ void __launch_bounds__(TS_NT)
k_tile_sort(const InArgs *in, int n, int64_t nrows, int64_t ncols, int sr, bool check_values, SortOut out, Ctl *ctl,
            unsigned skip_mask, int cb, int ib, uint64_t *words_out) {
    extern __shared__ uint64_t sm[];
    if (failed(ctl, skip_mask)) return;
    const int32_t *row = in->row, *col = in->col;
    const void *val = in->val;
    const uint8_t *op = in->op;
    const int tid = threadIdx.x;
    const int lo = blockIdx.x * TS_TILE;
    const int cnt = min(TS_TILE, n - lo);
    int N = 64;
    while (N < cnt) N <<= 1;
    for (int i = tid; i < N; i += TS_NT) {
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
        sm[i] = w;
    }
    __syncthreads();
    for (int size = 2; size <= N; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int x = tid; x < N / 2; x += TS_NT) {
                const int a = 2 * x - (x & (stride - 1));
                const int b = a + stride;
                const uint64_t wa = sm[a], wb = sm[b];
                if ((wa > wb) == ((a & size) == 0)) {
                    sm[a] = wb;
                    sm[b] = wa;
                }
            }
            __syncthreads();
        }
    }
    if (gridDim.x == 1) {
        const uint64_t imask = (uint64_t(1) << ib) - 1;
        for (int s = tid; s < cnt; s += TS_NT) {
            const uint64_t x = sm[s];
            const uint64_t key = x >> ib;
            const bool dead = (s + 1 < cnt) && ((sm[s + 1] >> ib) == key);
            write_sorted(out, s, key, x & imask, dead, cb, val, op, sr);
        }
    } else {
        for (int s = tid; s < cnt; s += TS_NT) words_out[lo + s] = sm[s];
    }
}

__device__ __forceinline__ int count_less(const uint64_t *a, int n, uint64_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int count_le(const uint64_t *a, int n, uint64_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(1024)
k_tile_merge(const uint64_t *words, int n, int ib, int cb, const InArgs *in, int sr, SortOut out, const Ctl *ctl,
             unsigned skip_mask) {
    extern __shared__ uint64_t sw[];
    if (failed(ctl, skip_mask)) return;
    const void *val = in->val;
    const uint8_t *op = in->op;
    for (int x = threadIdx.x; x < n; x += blockDim.x) sw[x] = words[x];
    __syncthreads();
    const int ntiles = (n + TS_TILE - 1) / TS_TILE;
    const uint64_t imask = (uint64_t(1) << ib) - 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int t = e / TS_TILE;
        const uint64_t w = sw[e];
        const uint64_t key = w >> ib;
        int rank = e - t * TS_TILE;
        int le = 0;  // words with a key <= key
        for (int u = 0; u < ntiles; u++) {
            const int ulo = u * TS_TILE;
            const int ucnt = min(TS_TILE, n - ulo);
            if (u != t) rank += count_less(sw + ulo, ucnt, w);
            le += count_le(sw + ulo, ucnt, w | imask);
        }
        const bool dead = rank != le - 1;
        write_sorted(out, rank, key, w & imask, dead, cb, val, op, sr);
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
    if (failed(ctl, skip_mask)) return;
    const int32_t *row = in->row, *col = in->col;
    const void *val = in->val;
    const uint8_t *op = in->op;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t r = row[i], c = col[i];
    bool ok = entry_ok(r, c, op[i], val, i, nrows, ncols, sr, check_values);
    if (!ok) set_status(ctl, ST_INVALID);
    k[i] = ok ? (((uint64_t)(uint32_t)r << cb) | (uint32_t)c) : 0;
    v[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(MS_NT)
k_hist(const uint64_t *k, int64_t n, int shift, uint32_t *counts, int64_t nb) {
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
    if (failed(ctl, skip_mask)) return;
    const void *val = in->val;
    const uint8_t *op = in->op;
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
    if (n <= (int64_t)TS_TILE * TS_MAXT && kb + ib <= 64) {
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TS_SMEM);
            cudaFuncSetAttribute(k_tile_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TM_SMEM);
            attr_set = true;
        }
        const int tiles = (int)((n + TS_TILE - 1) / TS_TILE);
        launch_k(k_tile_sort, tiles, TS_NT, TS_SMEM, s, in, (int)n, nrows, ncols, sr, check_values, out, ctl, skip_mask,
                 cb, ib, tmp.k0);
        if (tiles > 1)
            launch_k(k_tile_merge, (unsigned)((n + 1023) / 1024), 1024, (size_t)n * sizeof(uint64_t), s,
                     (const uint64_t *)tmp.k0, (int)n, ib, cb, in, sr, out, (const Ctl *)ctl, skip_mask);
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
