// masked.cu -- general updates by the entry-level masked recompute
// (Section 5.2, Algorithm 2), and the Bloom filter F that it keeps.
//
// F has C's pattern and a 64-bit word per entry: bit (k mod 64) of F(i,j)
// is set when the term A(i,k) B(k,j) contributes to C(i,j) (Section 5.2,
// l = 64).  On one GPU the words sit beside C's values in C's arena (same
// offsets), so every move of a row of C moves its words too.
//
// A batch of general updates (inserts, deletes, value changes of A and B)
// is applied in the paper's order:
//
//  1. computePattern: the pattern of C* = A* B' + A B* (Eq. 1), with F*:
//     each changed entry (i,k) of A meets the row k of B' (contribution
//     (i, j, bit k)); each changed entry (k,j) of B meets the rows i with
//     A(i,k) != 0 before the batch, read from the transposed pattern of A
//     before it is updated (contribution (i, j, bit k)).  The contributions
//     are sorted by (i, j) with the radix sort of the batch and equal keys
//     are merged (bits OR-ed): C* as sorted runs, one run per row.
//  2. E = (F | F*) at the entries of C*, and R_i = OR of E over row i
//     (k_mask_scan: the row of C is scanned once, each of its columns looked
//     up in the row's run of C*).
//  3. A^R: the entries (i,k) of A' whose bit (k mod 64) is set in R_i
//     (k_mask_keep).
//  4. Z, H = A^R B' masked at C* (k_mask_product): each kept (i,k,a) meets
//     row k of B'; a product whose column j is in row i's run of C* is
//     folded into Z(i,j) and sets bit k of H(i,j).
//  5. Merge Z into C and H into F at C*'s entries (k_mask_plan,
//     k_mask_splice): an entry of C* that received a product takes its new
//     value and word (written in place, or appended when C had no entry
//     there); one that received none leaves C (the row is compacted).
//     Entries of C outside C* are not touched.
//
// Every k that contributes to an entry of C* at the end has its bit in E
// (it contributed before, or one of its two factors changed), so A^R keeps
// every term of every masked entry; terms it keeps beyond those (bits
// shared modulo 64) reach no masked column or are genuine terms anyway.
//
// The static product's F comes from k_bloom_warp (a warp per row, the
// row's columns in a shared-memory table) and k_bloom_cta (rows longer than
// BL_WARP entries, a CTA with a dense column-to-place map in global memory).
#include "internal.h"

namespace dspg {

namespace {

constexpr int BL_WARP = 512;    // rows up to this many entries: the warp kernel
constexpr int BL_SLOTS = 1024;  // its table: at most half full
constexpr int BL_NW = 2;        // warps per block of the warp kernel (static shared memory)

__device__ __forceinline__ unsigned long long kbit(int32_t k) { return 1ull << (k & 63); }

__device__ __forceinline__ unsigned long long warp_or(unsigned long long v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Slot of column j in a warp's table (inserting it when absent and
// insert is set); -1 when absent (or the table is full, which the row
// bound rules out).
__device__ __forceinline__ int bl_slot(int32_t *keys, int32_t j, bool insert) {
    uint32_t h = ((uint32_t)j * 2654435761u) >> (32 - 10);
    for (int probe = 0; probe < BL_SLOTS; probe++) {
        const int32_t k = ((volatile int32_t *)keys)[h];
        if (k == j) return (int)h;
        if (k == -1) {
            if (!insert) return -1;
            const int32_t old = atomicCAS(&keys[h], -1, j);
            if (old == -1 || old == j) return (int)h;
        }
        h = (h + probe + 1) & (BL_SLOTS - 1);
    }
    return -1;
}

__global__ void __launch_bounds__(BL_NW * 32)
k_bloom_warp(MatView A, MatView B, MatView C, unsigned long long *F, int32_t *rows_long, long long *n_long,
             long long cap_long) {
    pdl_begin();
    __shared__ int32_t s_key[BL_NW][BL_SLOTS];
    __shared__ unsigned long long s_bits[BL_NW][BL_SLOTS];
    __shared__ int16_t s_slot[BL_NW][BL_WARP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *keys = s_key[w];
    unsigned long long *bits = s_bits[w];
    int16_t *slot = s_slot[w];
    for (int q = lane; q < BL_SLOTS; q += 32) {
        keys[q] = -1;
        bits[q] = 0ull;
    }
    __syncwarp();
    const long long nw = (long long)gridDim.x * BL_NW;
    for (long long i = (long long)blockIdx.x * BL_NW + w; i < C.nrows; i += nw) {
        const int L = C.len[i];
        if (L == 0) continue;
        if (L > BL_WARP) {
            if (lane == 0) {
                const long long t = atomicAdd((unsigned long long *)n_long, 1ull);
                if (t < cap_long) rows_long[t] = (int32_t)i;
            }
            continue;
        }
        const int64_t coff = C.off[i];
        for (int p = lane; p < L; p += 32) slot[p] = (int16_t)bl_slot(keys, C.col[coff + p], true);
        __syncwarp();
        const int64_t aoff = A.off[i];
        const int alen = A.len[i];
        for (int a = 0; a < alen; a++) {
            const int32_t k = A.col[aoff + a];
            const unsigned long long b = kbit(k);
            const int64_t bo = B.off[k];
            const int bl = B.len[k];
            for (int q = lane; q < bl; q += 32) {
                const int h = bl_slot(keys, B.col[bo + q], false);
                if (h >= 0) atomicOr(&bits[h], b);
            }
        }
        __syncwarp();
        for (int p = lane; p < L; p += 32) {
            const int h = slot[p];
            if (h >= 0) {
                F[coff + p] = bits[h];
                keys[h] = -1;
                bits[h] = 0ull;
            }
        }
        __syncwarp();
    }
}

// Rows longer than BL_WARP: a CTA per row, with pos[j] = the place of
// column j in the row (this CTA's m entries of posmap, -1 elsewhere).
__global__ void __launch_bounds__(512)
k_bloom_cta(MatView A, MatView B, MatView C, unsigned long long *F, const int32_t *rows_long, const long long *n_long,
            long long cap_long, int32_t *posmap) {
    pdl_begin();
    int32_t *pos = posmap + (int64_t)blockIdx.x * C.ncols;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    const long long n = *n_long < cap_long ? *n_long : cap_long;
    for (long long t = blockIdx.x; t < n; t += gridDim.x) {
        const int32_t i = rows_long[t];
        const int64_t coff = C.off[i];
        const int L = C.len[i];
        for (int p = tid; p < L; p += blockDim.x) {
            pos[C.col[coff + p]] = p;
            F[coff + p] = 0ull;
        }
        __syncthreads();
        const int64_t aoff = A.off[i];
        const int alen = A.len[i];
        for (int a = w; a < alen; a += nw) {
            const int32_t k = A.col[aoff + a];
            const unsigned long long b = kbit(k);
            const int64_t bo = B.off[k];
            const int bl = B.len[k];
            for (int q = lane; q < bl; q += 32) {
                const int32_t p = pos[B.col[bo + q]];
                if (p >= 0) atomicOr(&F[coff + p], b);
            }
        }
        __syncthreads();
        for (int p = tid; p < L; p += blockDim.x) pos[C.col[coff + p]] = -1;
        __syncthreads();
    }
}

// ------------------------------------------------------- computePattern

__device__ __forceinline__ void pat_emit(const PatJob &J, Ctl *ctl, bool ok, int32_t i, int32_t j, int32_t k) {
    const long long t = warp_fetch_add(&ctl->mask_n, ok ? 1 : 0);
    if (ok) {
        if (t < J.cap) {
            J.key[t] = ((uint64_t)(uint32_t)i << J.cb) | (uint32_t)j;
            J.bits[t] = kbit(k);
        } else {
            set_status(ctl, ST_MASK_FULL);
        }
    }
}

// A warp per batch entry that changes its matrix: the X term (A batch
// against B') and the Y term (B batch against the old pattern of A).
__global__ void k_pat_contrib(PatJob J, MatView B, MatView AT, Ctl *ctl, unsigned mask) {
    pdl_begin();
    if (__any_sync(0xffffffffu, failed(ctl, mask))) return;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (long long e = w0; e < J.xn; e += nwarps) {
        if (J.xk[e] == K_NOP) continue;  // the same e on every lane
        const int32_t i = J.xr[e], k = J.xc[e];
        const int64_t bo = B.off[k];
        const int bl = B.len[k];
        for (int q0 = 0; q0 < bl; q0 += 32) {
            const int q = q0 + lane;
            const bool ok = q < bl;
            pat_emit(J, ctl, ok, i, ok ? B.col[bo + q] : 0, k);
        }
    }
    for (long long e = w0; e < J.yn; e += nwarps) {
        if (J.yk[e] == K_NOP) continue;
        const int32_t k = J.yr[e], j = J.yc[e];
        const int64_t to = AT.off[k];
        const int tl = AT.len[k];
        for (int q0 = 0; q0 < tl; q0 += 32) {
            const int q = q0 + lane;
            const bool ok = q < tl;
            pat_emit(J, ctl, ok, ok ? AT.col[to + q] : 0, j, k);
        }
    }
}

__global__ void k_iota(uint32_t *v, int64_t n) {
    pdl_begin();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        v[t] = (uint32_t)t;
}

// flag[s] = 1 where a run of equal keys starts.
__global__ void k_pat_heads(const uint64_t *K, int64_t n, int32_t *flag) {
    pdl_begin();
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        flag[s] = (s == 0 || K[s] != K[s - 1]) ? 1 : 0;
}

// Each run of equal keys becomes entry u = ex[s] of C*: its row and
// column, and F* = OR of the run's bits; rflag[u] = 1 where a row starts.
__global__ void k_pat_unique(const uint64_t *K, const uint32_t *I, const uint64_t *bits, int64_t n,
                             const int64_t *ex, int cb, MaskJob M, int32_t *rflag) {
    pdl_begin();
    const uint64_t cmask = (uint64_t(1) << cb) - 1;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = K[s];
        if (s > 0 && K[s - 1] == key) continue;
        unsigned long long f = 0;
        for (int64_t t = s; t < n && K[t] == key; t++) f |= bits[I[t]];
        const int64_t u = ex[s];
        M.urow[u] = (int32_t)(key >> cb);
        M.ucol[u] = (int32_t)(key & cmask);
        M.ufs[u] = f;
        rflag[u] = (s == 0 || (K[s - 1] >> cb) != (key >> cb)) ? 1 : 0;
    }
}

// Runs of C* per row: start and row of run r = rex[u]; the row's bit in
// bm; and the end of the last run.
__global__ void k_pat_runs(MaskJob M, const int32_t *rflag, const int64_t *rex, uint32_t *bm) {
    pdl_begin();
    const int64_t nu = *M.nu_dev;
    if (blockIdx.x == 0 && threadIdx.x == 0) M.run_start[*M.nruns_dev] = nu;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += (int64_t)gridDim.x * blockDim.x) {
        if (!rflag[u]) continue;
        const int64_t r = rex[u];
        const int32_t i = M.urow[u];
        M.run_start[r] = u;
        M.run_row[r] = i;
        atomicOr(&bm[i >> 5], 1u << (i & 31));
    }
}

// --------------------------------------------------- E, R and A^R

// A warp per run: each entry of the row of C is looked up in the run; a
// hit records its place in the row and its word of F.  Then R_i = OR over
// the run of (F | F*).
__global__ void k_mask_scan(MaskJob M, MatView C, const unsigned long long *F) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long nr = *M.nruns_dev;
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nr; r += nwarps) {
        const int64_t u0 = M.run_start[r], u1 = M.run_start[r + 1];
        const int32_t i = M.run_row[r];
        const int64_t coff = C.off[i];
        const int L = C.len[i];
        for (int p = lane; p < L; p += 32) {
            const int32_t j = C.col[coff + p];
            const int64_t t = lower_bound_dev<int32_t>(M.ucol, u0, u1, j);
            if (t < u1 && M.ucol[t] == j) {
                M.upos[t] = p;
                M.ue[t] = F[coff + p];
            }
        }
        __syncwarp();
        unsigned long long rb = 0;
        for (int64_t t = u0 + lane; t < u1; t += 32) rb |= M.ue[t] | M.ufs[t];
        rb = warp_or(rb);
        if (lane == 0) M.rbits[r] = rb;
        __syncwarp();
    }
}

// A warp per run: the entries of row i of A' whose bit is set in R_i.
__global__ void k_mask_keep(MaskJob M, MatView A, Ctl *ctl) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long nr = *M.nruns_dev;
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nr; r += nwarps) {
        const int32_t i = M.run_row[r];
        const unsigned long long rb = M.rbits[r];
        const int64_t aoff = A.off[i];
        const int alen = A.len[i];
        for (int q0 = 0; q0 < alen; q0 += 32) {
            const int q = q0 + lane;
            const bool keep = q < alen && ((rb & kbit(A.col[aoff + q])) != 0ull);
            const long long t = warp_fetch_add(&ctl->mask_kept, keep ? 1 : 0);
            if (keep) {
                if (t < M.kcap) {
                    M.kept_run[t] = (int32_t)r;
                    M.kept_a[t] = aoff + q;
                } else {
                    set_status(ctl, ST_MASK_FULL);
                }
            }
        }
    }
}

// ------------------------------------------------ the masked product

template <int SR>
struct MSr;
template <>
struct MSr<SR_PT> {
    using T = double;
    __device__ static T mul(T a, T b) { return __dmul_rn(a, b); }
    __device__ static void acc(T *p, T v) { atomicAdd(p, v); }
};
template <>
struct MSr<SR_MP> {
    using T = int32_t;
    __device__ static T mul(T a, T b) { return a + b; }
    __device__ static void acc(T *p, T v) { atomicMin(p, v); }
};

// A warp per kept entry (i, k, a): the products with row k of B' whose
// column is in row i's run of C*.
template <int SR>
__global__ void k_mask_product(MaskJob M, MatView A, MatView B, Ctl *ctl, unsigned mask) {
    pdl_begin();
    using T = typename MSr<SR>::T;
    if (failed(ctl, mask)) return;  // no barrier or shuffle below
    const int lane = threadIdx.x & 31;
    const long long nk = *M.nkept_dev < M.kcap ? *M.nkept_dev : M.kcap;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const T *Av = (const T *)A.val;
    const T *Bv = (const T *)B.val;
    T *z = (T *)M.z;
    long long prods = 0;
    for (long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nk; t += nwarps) {
        const int32_t r = M.kept_run[t];
        const int64_t ae = M.kept_a[t];
        const int32_t k = A.col[ae];
        const T a = Av[ae];
        const unsigned long long b = kbit(k);
        const int64_t u0 = M.run_start[r], u1 = M.run_start[r + 1];
        const int64_t bo = B.off[k];
        const int bl = B.len[k];
        for (int q = lane; q < bl; q += 32) {
            const int32_t j = B.col[bo + q];
            const int64_t u = lower_bound_dev<int32_t>(M.ucol, u0, u1, j);
            if (u < u1 && M.ucol[u] == j) {
                MSr<SR>::acc(z + u, MSr<SR>::mul(a, Bv[bo + q]));
                atomicOr(&M.h[u], b);
                M.hit[u] = 1;
            }
        }
        prods += bl;
    }
    if (lane == 0 && prods) atomicAdd((unsigned long long *)&ctl->products, (unsigned long long)prods);
}

// ------------------------------------------------------------ merge

// A warp per run: the row's length after the merge (deleted entries out,
// new entries in); a row that outgrows its capacity gets a place at the
// arena tail (nothing is written when the arena is exhausted).
__global__ void k_mask_plan(MaskJob M, MatView C, Ctl *ctl, unsigned mask, int slack_min, int slack_div) {
    pdl_begin();
    if (__any_sync(0xffffffffu, failed(ctl, mask))) return;  // a warp leaves as a whole
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long nr = *M.nruns_dev;
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nr; r += nwarps) {
        const int64_t u0 = M.run_start[r], u1 = M.run_start[r + 1];
        int ndel = 0, nins = 0;
        for (int64_t u = u0 + lane; u < u1; u += 32) {
            const bool in_c = M.upos[u] >= 0, hit = M.hit[u] != 0;
            ndel += in_c && !hit;
            nins += !in_c && hit;
        }
        ndel = warp_sum<int>(ndel);
        nins = warp_sum<int>(nins);
        if (lane == 0) {
            const int32_t i = M.run_row[r];
            const int64_t L2 = (int64_t)C.len[i] - ndel + nins;
            int64_t dest = -1;
            int32_t cap = C.cap[i];
            if (L2 > cap) {
                cap = slack_cap(L2, slack_min, slack_div);
                dest = (int64_t)atomicAdd((unsigned long long *)C.top, (unsigned long long)cap);
                if (dest + cap > C.arena_cap) set_status(ctl, ST_C_ARENA);
                atomicAdd((unsigned long long *)&ctl->c_reloc, 1ull);
            }
            M.dest[r] = dest;
            M.dcap[r] = cap;
        }
    }
}

// A warp per run: (moves the row to its new place first, when it has one)
// writes the new values and words in place, removes the entries that
// received no product (a compaction of the row in order), and appends the
// new entries.
template <int SR>
__global__ void k_mask_splice(MaskJob M, MatView C, unsigned long long *F, Ctl *ctl, unsigned mask) {
    pdl_begin();
    using T = typename MSr<SR>::T;
    if (__any_sync(0xffffffffu, failed(ctl, mask))) return;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    T *Cv = (T *)C.val;
    const T *z = (const T *)M.z;
    long long written = 0;
    const long long nr = *M.nruns_dev;
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nr; r += nwarps) {
        const int64_t u0 = M.run_start[r], u1 = M.run_start[r + 1];
        const int32_t i = M.run_row[r];
        const int L = C.len[i];
        int64_t base = C.off[i];
        const int64_t dest = M.dest[r];
        if (dest >= 0) {
            for (int p = lane; p < L; p += 32) {
                C.col[dest + p] = C.col[base + p];
                Cv[dest + p] = Cv[base + p];
                F[dest + p] = F[base + p];
            }
            base = dest;
            __syncwarp();
        }
        int ndel = 0;
        for (int64_t u = u0 + lane; u < u1; u += 32) {
            const int p = M.upos[u];
            if (p < 0) continue;
            if (M.hit[u]) {
                Cv[base + p] = z[u];
                F[base + p] = M.h[u];
                written++;
            } else {
                C.col[base + p] = -1;  // leaves the row below
                ndel++;
            }
        }
        ndel = warp_sum<int>(ndel);
        __syncwarp();
        int len = L;
        if (ndel > 0) {
            // in order, chunk by chunk: a kept entry moves down to the count of
            // kept entries before it, never above a place still to be read
            int w = 0;
            for (int p0 = 0; p0 < L; p0 += 32) {
                const int p = p0 + lane;
                const int32_t c = p < L ? C.col[base + p] : -1;
                const bool keep = c >= 0;
                T v = T(0);
                unsigned long long f = 0ull;
                if (keep) {
                    v = Cv[base + p];
                    f = F[base + p];
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                __syncwarp();
                if (keep) {
                    const int d = w + __popc(bal & lanemask_lt());
                    C.col[base + d] = c;
                    Cv[base + d] = v;
                    F[base + d] = f;
                }
                w += __popc(bal);
                __syncwarp();
            }
            len = w;
        }
        for (int64_t u0c = u0; u0c < u1; u0c += 32) {
            const int64_t u = u0c + lane;
            const bool ins = u < u1 && M.upos[u] < 0 && M.hit[u];
            const unsigned bal = __ballot_sync(0xffffffffu, ins);
            if (ins) {
                const int d = len + __popc(bal & lanemask_lt());
                C.col[base + d] = M.ucol[u];
                Cv[base + d] = z[u];
                F[base + d] = M.h[u];
                written++;
            }
            len += __popc(bal);
        }
        __syncwarp();
        if (lane == 0) {
            dcheck(ctl, base + len <= C.arena_cap && len <= (dest >= 0 ? M.dcap[r] : C.cap[i]), DBG_MASK_ROOM, i);
            C.len[i] = len;
            if (dest >= 0) {
                C.off[i] = dest;
                C.cap[i] = M.dcap[r];
            }
        }
    }
    written = warp_sum<long long>(written);
    if (lane == 0 && written) atomicAdd((unsigned long long *)&ctl->nnz_written, (unsigned long long)written);
}

template <typename T>
__global__ void k_fill_val(T *p, int64_t n, T v) {
    pdl_begin();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        p[t] = v;
}

unsigned grid_of(int64_t items, int per_block, int num_sms, int waves = 16) {
    int64_t g = (items + per_block - 1) / per_block;
    if (g > (int64_t)num_sms * waves) g = (int64_t)num_sms * waves;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

void bloom_rows(const MatView &A, const MatView &B, const MatView &C, unsigned long long *F, int32_t *rows_long,
                long long *n_long, long long cap_long, cudaStream_t s, int num_sms) {
    if (C.nrows <= 0) return;
    launch_k(k_bloom_warp, grid_of(C.nrows, BL_NW, num_sms, 8), BL_NW * 32, 0, s, A, B, C, F, rows_long, n_long,
             cap_long);
}

void bloom_long_rows(const MatView &A, const MatView &B, const MatView &C, unsigned long long *F,
                     const int32_t *rows_long, const long long *n_long, long long cap_long, int32_t *posmap,
                     int ctas, cudaStream_t s) {
    launch_k(k_bloom_cta, (unsigned)std::max(ctas, 1), 512, 0, s, A, B, C, F, rows_long, n_long, cap_long, posmap);
}

void pat_contrib(const PatJob &J, const MatView &B, const MatView &AT, Ctl *ctl, unsigned mask, cudaStream_t s,
                 int num_sms) {
    const int64_t warps = std::max(J.xn, J.yn);
    if (warps <= 0) return;
    launch_k(k_pat_contrib, grid_of(warps, 8, num_sms, 8), 256, 0, s, J, B, AT, ctl, mask);
}

void iota_u32(uint32_t *v, int64_t n, cudaStream_t s, int num_sms) {
    if (n <= 0) return;
    launch_k(k_iota, grid_of(n, 256, num_sms), 256, 0, s, v, n);
}

void pat_heads(const uint64_t *K, int64_t n, int32_t *flag, cudaStream_t s, int num_sms) {
    if (n <= 0) return;
    launch_k(k_pat_heads, grid_of(n, 256, num_sms), 256, 0, s, K, n, flag);
}

void pat_unique(const uint64_t *K, const uint32_t *I, const uint64_t *bits, int64_t n, const int64_t *ex, int cb,
                const MaskJob &M, int32_t *rflag, cudaStream_t s, int num_sms) {
    if (n <= 0) return;
    launch_k(k_pat_unique, grid_of(n, 256, num_sms), 256, 0, s, K, I, bits, n, ex, cb, M, rflag);
}

void pat_runs(const MaskJob &M, const int32_t *rflag, const int64_t *rex, int64_t max_u, uint32_t *bm, cudaStream_t s,
              int num_sms) {
    if (max_u <= 0) return;
    launch_k(k_pat_runs, grid_of(max_u, 256, num_sms), 256, 0, s, M, rflag, rex, bm);
}

void mask_scan(const MaskJob &M, const MatView &C, const unsigned long long *F, cudaStream_t s, int num_sms) {
    if (M.max_runs <= 0) return;
    launch_k(k_mask_scan, grid_of(M.max_runs, 8, num_sms), 256, 0, s, M, C, F);
}

void mask_keep(const MaskJob &M, const MatView &A, Ctl *ctl, cudaStream_t s, int num_sms) {
    if (M.max_runs <= 0) return;
    launch_k(k_mask_keep, grid_of(M.max_runs, 8, num_sms), 256, 0, s, M, A, ctl);
}

void mask_product(int sr, const MaskJob &M, const MatView &A, const MatView &B, Ctl *ctl, unsigned mask,
                  cudaStream_t s, int num_sms) {
    if (M.kcap <= 0) return;
    if (sr == SR_PT)
        launch_k(k_mask_product<SR_PT>, grid_of(M.kcap, 8, num_sms), 256, 0, s, M, A, B, ctl, mask);
    else
        launch_k(k_mask_product<SR_MP>, grid_of(M.kcap, 8, num_sms), 256, 0, s, M, A, B, ctl, mask);
}

void mask_init_acc(int sr, const MaskJob &M, int64_t nu, cudaStream_t s, int num_sms) {
    if (nu <= 0) return;
    if (sr == SR_PT) launch_k(k_fill_val<double>, grid_of(nu, 256, num_sms), 256, 0, s, (double *)M.z, nu, 0.0);
    else launch_k(k_fill_val<int32_t>, grid_of(nu, 256, num_sms), 256, 0, s, (int32_t *)M.z, nu, MP_INF);
}

void mask_plan(const MaskJob &M, const MatView &C, Ctl *ctl, unsigned mask, int slack_min, int slack_div,
               cudaStream_t s, int num_sms) {
    if (M.max_runs <= 0) return;
    launch_k(k_mask_plan, grid_of(M.max_runs, 8, num_sms), 256, 0, s, M, C, ctl, mask, slack_min, slack_div);
}

void mask_splice(int sr, const MaskJob &M, const MatView &C, unsigned long long *F, Ctl *ctl, unsigned mask,
                 cudaStream_t s, int num_sms) {
    if (M.max_runs <= 0) return;
    if (sr == SR_PT) launch_k(k_mask_splice<SR_PT>, grid_of(M.max_runs, 8, num_sms), 256, 0, s, M, C, F, ctl, mask);
    else launch_k(k_mask_splice<SR_MP>, grid_of(M.max_runs, 8, num_sms), 256, 0, s, M, C, F, ctl, mask);
}

}  // namespace dspg
