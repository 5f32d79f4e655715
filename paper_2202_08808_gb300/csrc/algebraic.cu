// algebraic.cu -- the delta path of Eq. 1 for batches that only insert.
//
// Section 5 ("algebraic updates"): when A' = A (+) A* and B' = B (+) B* with
// the semiring's own addition, C' = C (+) C* with C* = A* B' (+) A B*
// (Eq. 1), so C can be brought up to date by adding the products of the
// update matrices instead of recomputing whole rows.  A batch whose every
// effective change writes an absent entry (an insertion) is such an update
// in both semirings: A'(i,k) = A*(i,k) where A had no entry, and A' = A
// elsewhere.  On one GPU the two terms are formed entry by entry:
//
//   X = A* B':  an inserted A entry (i, k, a) meets every entry (k, j, b) of
//               B' (the rows of B after the batch): contribution (i, j, a b);
//   Y = A B*:   an inserted B entry (k, j, b) meets every row i with
//               A(i,k) != 0 before the batch, read from the transposed
//               pattern of A before it is updated: contribution
//               (i, j, A(i,k) b).
//
// Each contribution is folded into C'(i, j) where row i of C already holds
// column j (an atomic add, or min, on the value: Section 5.1's local step
// C (+)= C*), and otherwise joins a list of new entries of C.  The new
// entries are sorted by (row, column) with the batch sort, equal keys are
// combined, and each row of C takes its new entries at its end (C's rows
// carry no column order) or moves to the arena tail when they do not fit
// (plan, then copy: a plan that finds the arena exhausted writes nothing).
// Rows of C longer than ALG_SCAN entries are not searched: they are marked
// and recomputed by the row path afterwards, which is exact from A', B'
// whatever contributions a row received before.
#include "internal.h"

namespace dspg {

namespace {

template <int SR>
struct AlgSr;
template <>
struct AlgSr<SR_PT> {
    using T = double;
    __device__ static T mul(T a, T b) { return __dmul_rn(a, b); }
    __device__ static T add(T a, T b) { return __dadd_rn(a, b); }
    __device__ static void acc(T *p, T v) { atomicAdd(p, v); }
};
template <>
struct AlgSr<SR_MP> {
    using T = int32_t;
    __device__ static T mul(T a, T b) { return a + b; }
    __device__ static T add(T a, T b) { return a < b ? a : b; }
    __device__ static void acc(T *p, T v) { atomicMin(p, v); }
};

__device__ __forceinline__ void set_row_bit(uint32_t *bm, int32_t i) {
    const uint32_t bit = 1u << (i & 31);
    if (!(((volatile uint32_t *)bm)[i >> 5] & bit)) atomicOr(&bm[i >> 5], bit);
}

// Contribution (i, j, v) of lane `want` into C (every lane of the warp calls
// it: the new-entry list is handed out with one atomic per warp).
template <int SR>
__device__ __forceinline__ void alg_apply(const MatView &C, const AlgJob &J, Ctl *ctl, bool want, int32_t i,
                                          int32_t j, typename AlgSr<SR>::T v) {
    using T = typename AlgSr<SR>::T;
    bool fresh = false;
    if (want) {
        set_row_bit(J.bm_touch, i);
        const int L = C.len[i];
        if (L > ALG_SCAN) {
            set_row_bit(J.bm_long, i);
        } else {
            const int64_t o = C.off[i];
            int p = 0;
            while (p < L && C.col[o + p] != j) p++;
            if (p < L) AlgSr<SR>::acc((T *)C.val + o + p, v);
            else fresh = true;
        }
    }
    const long long t = warp_fetch_add(&ctl->alg_new, fresh ? 1 : 0);
    if (fresh) {
        if (t < J.ncap) {
            J.nr[t] = i;
            J.nc[t] = j;
            ((T *)J.nv)[t] = v;
            J.nop[t] = OP_SET;
        } else {
            set_status(ctl, ST_ALG_FULL);
        }
    }
}

// A warp per batch entry: the inserted entries of the A batch form X's
// contributions, those of the B batch (the A batch again when B is A) Y's.
template <int SR>
__global__ void k_alg_contrib(AlgJob J, MatView A, MatView B, MatView AT, MatView C, Ctl *ctl, unsigned mask) {
    pdl_begin();
    using T = typename AlgSr<SR>::T;
    if (__any_sync(0xffffffffu, failed(ctl, mask))) return;  // a warp leaves as a whole
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const T *Av = (const T *)A.val;
    const T *Bv = (const T *)B.val;
    long long ncon = 0;
    for (long long e = w0; e < J.xn; e += nwarps) {
        if (J.xk[e] != K_INS) continue;  // the same e on every lane
        const int32_t i = J.xr[e], k = J.xc[e];
        const T a = ((const T *)J.xv)[e];
        const int64_t bo = B.off[k];
        const int bl = B.len[k];
        for (int q0 = 0; q0 < bl; q0 += 32) {
            const int q = q0 + lane;
            const bool ok = q < bl;
            const int32_t j = ok ? B.col[bo + q] : 0;
            const T v = ok ? AlgSr<SR>::mul(a, Bv[bo + q]) : T(0);
            alg_apply<SR>(C, J, ctl, ok, i, j, v);
            ncon += ok;
        }
    }
    for (long long e = w0; e < J.yn; e += nwarps) {
        if (J.yk[e] != K_INS) continue;
        const int32_t k = J.yr[e], j = J.yc[e];
        const T b = ((const T *)J.yv)[e];
        const int64_t to = AT.off[k];
        const int tl = AT.len[k];
        for (int q0 = 0; q0 < tl; q0 += 32) {
            const int q = q0 + lane;
            const bool ok = q < tl;
            int32_t i = 0;
            T v = T(0);
            bool found = false;
            if (ok) {
                // (i, k) is an entry of A before the batch, so A' holds it
                // with the same value (the batch only inserts)
                i = AT.col[to + q];
                const int64_t ao = A.off[i], ae = ao + A.len[i];
                const int64_t p = lower_bound_dev<int32_t>(A.col, ao, ae, k);
                found = p < ae && A.col[p] == k;
                if (found) v = AlgSr<SR>::mul(Av[p], b);
            }
            alg_apply<SR>(C, J, ctl, found, i, j, v);
            ncon += found;
        }
    }
    ncon = warp_sum<long long>(ncon);
    if (lane == 0 && ncon) atomicAdd((unsigned long long *)&ctl->alg_contrib, (unsigned long long)ncon);
}

// The new entries, sorted by (row, column) with equal keys adjacent: the
// first entry of each row's run plans where the row goes (its own place if
// the combined new entries fit its capacity, else the arena tail).
__global__ void k_alg_plan(AlgNew N, MatView C, Ctl *ctl, unsigned mask, int slack_min, int slack_div) {
    pdl_begin();
    if (failed(ctl, mask)) return;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N.n; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = N.row[s];
        if (s > 0 && N.row[s - 1] == r) continue;
        const int64_t hi = run_end_dev<int32_t>(N.row, s, N.n, r);
        int u = 0;
        for (int64_t x = s; x < hi; x++) u += (x == s || N.col[x] != N.col[x - 1]);
        const int L = C.len[r];
        int32_t cap = C.cap[r];
        int64_t dest = C.off[r];
        if (L + u > cap) {
            cap = slack_cap(L + u, slack_min, slack_div);
            dest = (int64_t)atomicAdd((unsigned long long *)C.top, (unsigned long long)cap);
            if (dest + cap > C.arena_cap) set_status(ctl, ST_C_ARENA);
            atomicAdd((unsigned long long *)&ctl->c_reloc, 1ull);
        }
        N.dest[s] = dest;
        N.cap[s] = cap;
    }
}

// Each planned row: move the old entries if the row relocates, then write
// the combined new entries after them.
template <int SR>
__global__ void k_alg_copy(AlgNew N, MatView C, Ctl *ctl, unsigned mask) {
    pdl_begin();
    using T = typename AlgSr<SR>::T;
    if (failed(ctl, mask)) return;
    T *Cv = (T *)C.val;
    const T *nv = (const T *)N.val;
    long long written = 0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N.n; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = N.row[s];
        if (s > 0 && N.row[s - 1] == r) continue;
        const int64_t hi = run_end_dev<int32_t>(N.row, s, N.n, r);
        const int L = C.len[r];
        const int64_t o = C.off[r];
        const int64_t d = N.dest[s];
        if (d != o)
            for (int p = 0; p < L; p++) {
                C.col[d + p] = C.col[o + p];
                Cv[d + p] = Cv[o + p];
            }
        int n = L;
        for (int64_t x = s; x < hi;) {
            const int32_t j = N.col[x];
            T v = nv[x];
            int64_t y = x + 1;
            for (; y < hi && N.col[y] == j; y++) v = AlgSr<SR>::add(v, nv[y]);
            C.col[d + n] = j;
            Cv[d + n] = v;
            n++;
            x = y;
        }
        C.off[r] = d;
        C.len[r] = n;
        C.cap[r] = N.cap[s];
        written += n - L;
    }
    written = warp_sum<long long>(written);
    if ((threadIdx.x & 31) == 0 && written) atomicAdd((unsigned long long *)&ctl->nnz_written, (unsigned long long)written);
}

unsigned alg_grid(int64_t items, int per_block, int num_sms) {
    int64_t g = (items + per_block - 1) / per_block;
    if (g > (int64_t)num_sms * 8) g = (int64_t)num_sms * 8;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

void run_alg_contrib(int sr, const AlgJob &J, const MatView &A, const MatView &B, const MatView &AT, const MatView &C,
                     Ctl *ctl, unsigned mask, cudaStream_t s, int num_sms) {
    const int64_t warps = J.xn > J.yn ? J.xn : J.yn;
    if (warps <= 0) return;
    const unsigned g = alg_grid(warps, 8, num_sms);  // 8 warps per block of 256
    if (sr == SR_PT) launch_k(k_alg_contrib<SR_PT>, g, 256, 0, s, J, A, B, AT, C, ctl, mask);
    else launch_k(k_alg_contrib<SR_MP>, g, 256, 0, s, J, A, B, AT, C, ctl, mask);
}

void run_alg_append(int sr, const AlgNew &N, const MatView &C, Ctl *ctl, unsigned plan_mask, unsigned copy_mask,
                    int slack_min, int slack_div, bool plan, cudaStream_t s, int num_sms) {
    if (N.n <= 0) return;
    const unsigned g = alg_grid(N.n, 256, num_sms);
    if (plan) {
        launch_k(k_alg_plan, g, 256, 0, s, N, C, ctl, plan_mask, slack_min, slack_div);
        return;
    }
    if (sr == SR_PT) launch_k(k_alg_copy<SR_PT>, g, 256, 0, s, N, C, ctl, copy_mask);
    else launch_k(k_alg_copy<SR_MP>, g, 256, 0, s, N, C, ctl, copy_mask);
}

}  // namespace dspg
