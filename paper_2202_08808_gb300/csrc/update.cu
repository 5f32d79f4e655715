// update.cu -- applying a sorted batch to a slack-CSR, and affected-row detection.
//
// Section 4.1: an insert or value change is the paper's merge(A, A*) (write
// the entry, adding it when absent); a delete is mask(A, A*) (remove the
// entry when present).  The paper keeps a hash table per row for O(1)
// lookups; here rows stay column-sorted so that one sorted batch merges into
// a row with binary searches and no per-row table.
//
// A row with updates is rebuilt in a staging buffer and then committed:
//
//   classify  (warp per row segment of the batch): binary-search each update
//             in the old row -> kind (INS: write of an absent column, UPD:
//             write of a present one, DEL: delete of a present one, NOP),
//             its lower-bound position pos, and exclusive prefix counts of
//             INS and DEL within the segment.  New length
//             L' = L + #INS - #DEL.  INS/UPD entries are written straight to
//             their final slot  pos - DEL_before + INS_before.
//   copy      (warp per 256 old entries): a kept old entry p lands at
//             p - #DEL(pos < p) + #INS(pos <= p); found by two binary
//             searches over the segment's pos array.
//   commit    (staged rows -> matrix): a row that fits its capacity is
//             copied in place, a longer one moves to the arena tail.  All
//             destinations are planned before anything is written, so an
//             exhausted arena leaves the matrix untouched.
#include "internal.h"

namespace dspg {

constexpr int CH = 256;  // entries per copy work item

__device__ __forceinline__ long long atomic_add_ll(long long *p, long long v) {
    return (long long)atomicAdd((unsigned long long *)p, (unsigned long long)v);
}

// ------------------------------------------------------------- classify

constexpr int SEG_SHORT = 16;  // row segments up to this many updates are classified by one thread

__device__ __forceinline__ uint8_t kind_of(uint8_t op, bool present) {
    if (op == OP_DEAD) return K_NOP;
    if (op == OP_DELETE) return present ? K_DEL : K_NOP;
    return present ? K_UPD : K_INS;
}

// Rows of C* (Section 5, Eq. 1) at row granularity: R = rows(A*) u
// {i : A(i,k) != 0, k in rows(B*)}.  A* and B* hold the batch entries that
// change their matrix (kind INS, UPD or DEL).  The second set is read from
// the transposed pattern of A *before* this batch; it equals the set taken
// over A' because a pattern difference at (i,k) already puts i in rows(A*).
// Sets bit i of bm; the lanes that set a fresh bit append i to list with one
// atomic per warp.  All 32 lanes must call it (want = false to abstain).
__device__ __forceinline__ void mark_bit(uint32_t *bm, int32_t i) {
    const uint32_t bit = 1u << (i & 31);
    if (!(((volatile uint32_t *)bm)[i >> 5] & bit)) atomicOr(&bm[i >> 5], bit);
}

__device__ __forceinline__ void mark_warp(uint32_t *bm, bool want, int32_t i, int32_t *list, long long *cnt) {
    bool fresh = false;
    if (want) {
        const uint32_t bit = 1u << (i & 31);
        if (!(((volatile uint32_t *)bm)[i >> 5] & bit)) fresh = !(atomicOr(&bm[i >> 5], bit) & bit);
    }
    const long long t = warp_fetch_add(cnt, fresh ? 1 : 0);
    if (fresh) list[t] = i;
}

// The thread at the first entry of each row segment of the sorted batch
// owns the segment: it classifies the segment's updates against the old row
// (binary search), keeps running INS/DEL counts, and writes the INS/UPD
// entries of a changed row to their final staging slots; merge items,
// staging and copy items are handed out with one atomic per warp.
// Segments with more than SEG_SHORT updates are classified by the whole warp
// afterwards, one at a time.
template <typename T>
__global__ void k_classify(UpdJob J, MatView M, Ctl *ctl, unsigned mask, unsigned stage_bit, DetectBufs D,
                           int mark_rows, int mark_cols) {
    pdl_begin();
    if (failed(ctl, mask)) return;
    UpdCtl *u = &ctl->u[J.which];
    const int64_t n = *J.n_dev;  // the launch covers a bucket of at least n entries
    const int lane = threadIdx.x & 31;
    const T *bval = (const T *)J.val;
    T *sval = (T *)J.st_val;
    long long s_ins = 0, s_del = 0, s_upd = 0, s_nop = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = base + threadIdx.x;
        int32_t r = 0;
        bool head = false;
        int hi = 0;
        if (s < n) {
            r = J.row[s];
            // padding entries of a forwarded batch sit in a row past the end
            head = (int64_t)r < M.nrows && (s == 0 || J.row[s - 1] != r);
        }
        if (head) hi = (int)run_end_dev<int32_t>(J.row, s, n, r);
        const bool lng = head && (hi - s > SEG_SHORT);
        const bool mine = head && !lng;
        int L = 0, cins = 0, cdel = 0, cupd = 0, cnop = 0;
        if (mine) {
            const int64_t mb = M.off[r];
            L = M.len[r];
            const int32_t *rc = M.col + mb;
            for (int x = (int)s; x < hi; x++) {
                const int32_t c = J.col[x];
                const uint8_t op = J.op[x];
                const int p = (int)lower_bound_wide<int32_t>(rc, 0, L, c);
                const uint8_t k = kind_of(op, p < L && rc[p] == c);
                J.kind[x] = k;
                J.pos[x] = p;
                J.insx[x] = cins;
                J.delx[x] = cdel;
                cins += k == K_INS;
                cdel += k == K_DEL;
                cupd += k == K_UPD;
                cnop += (k == K_NOP && op == OP_DELETE);
            }
        }
        s_ins += cins;
        s_del += cdel;
        s_upd += cupd;
        s_nop += cnop;
        const bool changed = mine && (cins + cdel + cupd) > 0;
        // the first step of the affected-row detection: a row with an
        // effective change is in rows(A*) (and, for C = A A, in rows(B*))
        if (mark_rows && changed) mark_bit(D.bmR, r);
        if (mark_cols) mark_warp(D.bmK, changed, r, D.K, D.nK);
        const int nl = L + cins - cdel;
        const int nch = changed ? (L + CH - 1) / CH : 0;
        const long long m = warp_fetch_add(&u->n_merge, changed ? 1 : 0);
        const long long soff = warp_fetch_add(&u->stage_top, changed ? nl : 0);
        const long long cb = warp_fetch_add(&u->n_chunk, nch);
        if (changed) {
            if (soff + nl > J.st_cap || cb + nch > J.ch_cap) {
                set_status(ctl, stage_bit);
            } else {
                J.m_row[m] = r;
                J.m_lo[m] = (int32_t)s;
                J.m_hi[m] = hi;
                J.m_len[m] = nl;
                J.m_soff[m] = soff;
                J.m_nins[m] = cins;
                J.m_ndel[m] = cdel;
                for (int c = 0; c < nch; c++) {
                    J.ch_item[cb + c] = (int32_t)m;
                    J.ch_part[cb + c] = c;
                }
                for (int x = (int)s; x < hi; x++) {
                    const uint8_t k = J.kind[x];
                    if (k == K_INS || k == K_UPD) {
                        const int o = J.pos[x] - J.delx[x] + J.insx[x];
                        J.st_col[soff + o] = J.col[x];
                        if (sval) sval[soff + o] = bval[x];
                    }
                }
            }
        }
        // long segments of this warp: all lanes on one segment at a time
        unsigned lm = __ballot_sync(0xffffffffu, lng);
        while (lm) {
            const int src = __ffs(lm) - 1;
            lm &= lm - 1;
            const int lo = (int)__shfl_sync(0xffffffffu, (long long)s, src);
            const int hi2 = __shfl_sync(0xffffffffu, hi, src);
            const int32_t r2 = __shfl_sync(0xffffffffu, r, src);
            const int64_t mb = M.off[r2];
            const int L2 = M.len[r2];
            const int32_t *rc = M.col + mb;
            int ti = 0, td = 0, tu = 0, tn = 0;
            for (int u0 = lo; u0 < hi2; u0 += 32) {
                const int x = u0 + lane;
                int ins = 0, del = 0;
                if (x < hi2) {
                    const int32_t c = J.col[x];
                    const uint8_t op = J.op[x];
                    const int p = (int)lower_bound_wide<int32_t>(rc, 0, L2, c);
                    const uint8_t k = kind_of(op, p < L2 && rc[p] == c);
                    J.kind[x] = k;
                    J.pos[x] = p;
                    ins = k == K_INS;
                    del = k == K_DEL;
                    tu += k == K_UPD;
                    tn += (k == K_NOP && op == OP_DELETE);
                }
                const int ii = warp_incl_scan<int>(ins), di = warp_incl_scan<int>(del);
                if (x < hi2) {
                    J.insx[x] = ti + ii - ins;
                    J.delx[x] = td + di - del;
                }
                ti += __shfl_sync(0xffffffffu, ii, 31);
                td += __shfl_sync(0xffffffffu, di, 31);
            }
            tu = warp_sum<int>(tu);
            tn = warp_sum<int>(tn);
            if (lane == 0) {
                s_ins += ti;
                s_del += td;
                s_upd += tu;
                s_nop += tn;
            }
            if (ti + td + tu == 0) continue;
            if (mark_rows && lane == 0) mark_bit(D.bmR, r2);
            if (mark_cols) mark_warp(D.bmK, lane == 0, r2, D.K, D.nK);
            const int nl2 = L2 + ti - td;
            const int nch2 = (L2 + CH - 1) / CH;
            long long m2 = 0, so2 = 0, cb2 = 0;
            int ok = 1;
            if (lane == 0) {
                m2 = atomic_add_ll(&u->n_merge, 1);
                so2 = atomic_add_ll(&u->stage_top, nl2);
                cb2 = atomic_add_ll(&u->n_chunk, nch2);
                ok = (so2 + nl2 <= J.st_cap) && (cb2 + nch2 <= J.ch_cap);
                if (!ok) set_status(ctl, stage_bit);
                else {
                    J.m_row[m2] = r2;
                    J.m_lo[m2] = lo;
                    J.m_hi[m2] = hi2;
                    J.m_len[m2] = nl2;
                    J.m_soff[m2] = so2;
                    J.m_nins[m2] = ti;
                    J.m_ndel[m2] = td;
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) continue;
            m2 = __shfl_sync(0xffffffffu, m2, 0);
            so2 = __shfl_sync(0xffffffffu, so2, 0);
            cb2 = __shfl_sync(0xffffffffu, cb2, 0);
            for (int c = lane; c < nch2; c += 32) {
                J.ch_item[cb2 + c] = (int32_t)m2;
                J.ch_part[cb2 + c] = c;
            }
            __syncwarp();
            for (int x = lo + lane; x < hi2; x += 32) {
                const uint8_t k = J.kind[x];
                if (k == K_INS || k == K_UPD) {
                    const int o = J.pos[x] - J.delx[x] + J.insx[x];
                    J.st_col[so2 + o] = J.col[x];
                    if (sval) sval[so2 + o] = bval[x];
                }
            }
        }
    }
    s_ins = warp_sum<long long>(s_ins);
    s_del = warp_sum<long long>(s_del);
    s_upd = warp_sum<long long>(s_upd);
    s_nop = warp_sum<long long>(s_nop);
    if (lane == 0) {
        if (s_ins) atomic_add_ll(&u->ins, s_ins);
        if (s_del) atomic_add_ll(&u->del, s_del);
        if (s_upd) atomic_add_ll(&u->upd, s_upd);
        if (s_nop) atomic_add_ll(&u->nop, s_nop);
    }
}

// ------------------------------------------------------------ merge copy

// The work of the merge copy for block `blk` of `nblk` (a kernel of its own,
// or a share of the grid of k_detect_merge).
// BATCHED: a row of at most 32 updates takes them a lane each and loads
// its chunk before any store (rows of thousands of entries and few updates,
// the hubs of skewed graphs); the fused kernels, whose registers the
// detection shares, keep a search per entry.
template <typename T, bool BATCHED>
__device__ __forceinline__ void merge_copy_blocks(const UpdJob &J, const MatView &M, const Ctl *ctl, long long blk,
                                                  long long nblk) {
    const long long nch = ctl->u[J.which].n_chunk;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (nblk * blockDim.x) >> 5;
    const T *mval = (const T *)M.val;
    T *sval = (T *)J.st_val;
    for (long long x = (blk * blockDim.x + threadIdx.x) >> 5; x < nch; x += nwarps) {
        const int m = J.ch_item[x], part = J.ch_part[x];
        const int32_t r = J.m_row[m];
        const int lo = J.m_lo[m], hi = J.m_hi[m];
        const int64_t base = M.off[r];
        const int L = M.len[r];
        const int64_t soff = J.m_soff[m];
        const int tins = J.m_nins[m], tdel = J.m_ndel[m];
        const int p0 = part * CH;
        const int p1 = min(L, p0 + CH);
        const int nu = hi - lo;  // the row's updates (warp-uniform)
        if (BATCHED && nu <= 32) {
            // the row's updates a lane each (position, kind, the deletions
            // and insertions before it), the chunk's entries loaded together
            // first; each entry's place then comes from shuffles over the
            // updates instead of a search in global memory per entry
            const int upos = lane < nu ? J.pos[lo + lane] : 0;
            const uint8_t ukind = lane < nu ? J.kind[lo + lane] : (uint8_t)K_NOP;
            const int udel = lane < nu ? J.delx[lo + lane] : 0;
            const int uins = lane < nu ? J.insx[lo + lane] : 0;
            constexpr int PER = CH / 32;
            const int nit = (p1 - p0 + 31) >> 5;  // rounds of 32 entries in this chunk (warp-uniform)
            int32_t cc[PER];
            T vv[PER];
#pragma unroll
            for (int u = 0; u < PER; u++) {
                const int p = p0 + u * 32 + lane;
                cc[u] = p < p1 ? M.col[base + p] : 0;
                vv[u] = (sval && p < p1) ? mval[base + p] : T(0);
            }
#pragma unroll
            for (int u = 0; u < PER; u++) {
                if (u >= nit) break;
                const int p = p0 + u * 32 + lane;
                int lt = 0, le = 0;  // updates at positions below p, and at or below p
                for (int j = 0; j < nu; j++) {
                    const int pj = __shfl_sync(0xffffffffu, upos, j);
                    lt += pj < p;
                    le += pj <= p;
                }
                const uint8_t klast = (uint8_t)__shfl_sync(0xffffffffu, (int)ukind, le > 0 ? le - 1 : 0);
                const int dsh = __shfl_sync(0xffffffffu, udel, lt < 32 ? lt : 31);
                const int ish = __shfl_sync(0xffffffffu, uins, le < 32 ? le : 31);
                const bool hit = le > lt && (klast == K_UPD || klast == K_DEL);
                if (p >= p1 || hit) continue;  // past the row, deleted, or rewritten by the classify kernel
                const int dbefore = lt < nu ? dsh : tdel;
                const int ibefore = le < nu ? ish : tins;
                const int o = p - dbefore + ibefore;
                J.st_col[soff + o] = cc[u];
                if (sval) sval[soff + o] = vv[u];
            }
            continue;
        }
        for (int p = p0 + lane; p < p1; p += 32) {
            const int q = (int)lower_bound_dev<int32_t>(J.pos, lo, hi, p);
            const int q2 = (int)upper_bound_dev<int32_t>(J.pos, q, hi, p);
            const bool hit = q2 > q && (J.kind[q2 - 1] == K_UPD || J.kind[q2 - 1] == K_DEL);
            if (hit) continue;  // deleted, or rewritten by the classify kernel
            const int dbefore = q < hi ? J.delx[q] : tdel;
            const int ibefore = q2 < hi ? J.insx[q2] : tins;
            const int o = p - dbefore + ibefore;
            J.st_col[soff + o] = M.col[base + p];
            if (sval) sval[soff + o] = mval[base + p];
        }
    }
}

template <typename T>
__global__ void k_merge_copy(UpdJob J, MatView M, const Ctl *ctl, unsigned mask) {
    pdl_begin();
    if (failed(ctl, mask)) return;
    merge_copy_blocks<T, true>(J, M, ctl, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- commit

__device__ __forceinline__ void commit_plan_blocks(const CommitJob &J, const MatView &M, Ctl *ctl, int slack_min,
                                                   int slack_div, long long blk, long long nblk) {
    const long long n = *J.count;
    for (long long base = blk * blockDim.x; base < n; base += nblk * blockDim.x) {
        const long long m = base + threadIdx.x;
        const bool valid = m < n;
        int32_t r = 0, nl = 0, c = 0;
        bool reloc = false;
        if (valid) {
            r = J.rows[m];
            nl = J.lens[m];
            c = M.cap[r];
            if (nl > c) {
                reloc = true;
                c = slack_cap(nl, slack_min, slack_div);
            }
        }
        const long long dr = warp_fetch_add(M.top, reloc ? c : 0);
        const unsigned nrel = __popc(__ballot_sync(0xffffffffu, reloc));
        if ((threadIdx.x & 31) == 0 && nrel) atomic_add_ll(J.reloc, nrel);
        const int nch = valid ? (nl > 0 ? (nl + CH - 1) / CH : 1) : 0;
        const long long cb = warp_fetch_add(J.cc_count, nch);
        if (!valid) continue;
        int64_t d = reloc ? (int64_t)dr : M.off[r];
        if (reloc && d + c > M.arena_cap) set_status(ctl, J.arena_bit);
        J.dest[m] = d;
        J.ncap[m] = c;
        if (cb + nch > J.cc_cap) {
            set_status(ctl, J.stage_bit);
            continue;
        }
        for (int k = 0; k < nch; k++) {
            J.cc_item[cb + k] = (int32_t)m;
            J.cc_part[cb + k] = k;
        }
    }
}

__global__ void k_commit_plan(CommitJob J, MatView M, Ctl *ctl, unsigned mask, int slack_min, int slack_div) {
    pdl_begin();
    if (failed(ctl, mask)) return;
    commit_plan_blocks(J, M, ctl, slack_min, slack_div, blockIdx.x, gridDim.x);
}

template <typename T>
__device__ __forceinline__ void commit_copy_blocks(const CommitJob &J, const MatView &M, long long blk,
                                                   long long nblk, Ctl *ctl) {
    const long long n = *J.cc_count;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (nblk * blockDim.x) >> 5;
    const T *sv = (const T *)J.st_val;
    T *mv = (T *)M.val;
    for (long long x = (blk * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
        const int m = J.cc_item[x], part = J.cc_part[x];
        const int32_t r = J.rows[m];
        const int32_t nl = J.lens[m];
        const int64_t d = J.dest[m];
        const int64_t so = J.soff[m];
        const int e0 = part * CH;
        const int e1 = min(nl, e0 + CH);
        if (!dcheck(ctl, d >= 0 && d + nl <= M.arena_cap, DBG_ARENA, r)) continue;
        // the chunk's entries loaded together, then stored
        constexpr int PER = CH / 32;
        int32_t cc[PER];
        T vv[PER];
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int e = e0 + u * 32 + lane;
            cc[u] = e < e1 ? J.st_col[so + e] : 0;
            vv[u] = (mv && e < e1) ? sv[so + e] : T(0);
        }
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int e = e0 + u * 32 + lane;
            if (e < e1) {
                M.col[d + e] = cc[u];
                if (mv) mv[d + e] = vv[u];
            }
        }
        if (part == 0 && lane == 0) {
            M.off[r] = d;
            M.len[r] = nl;
            M.cap[r] = J.ncap[m];
        }
    }
}

template <typename T>
__global__ void k_commit_copy(CommitJob J, MatView M, const Ctl *ctl, unsigned mask) {
    pdl_begin();
    if (failed(ctl, mask)) return;
    commit_copy_blocks<T>(J, M, blockIdx.x, gridDim.x, const_cast<Ctl *>(ctl));
}

// ---------------------------------------------------------- detection

__device__ __forceinline__ void detect_cols_blocks(const MatView &AT, const DetectBufs &D, Ctl *ctl, long long blk,
                                                   long long nblk) {
    const long long nk = *D.nK;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (nblk * blockDim.x) >> 5;
    for (long long x = (blk * blockDim.x + threadIdx.x) >> 5; x < nk; x += nwarps) {
        const int32_t k = D.K[x];
        if (lane == 0) D.bmK[k >> 5] = 0u;  // marks of B* rows are not needed any more
        const int64_t base = AT.off[k];
        const int L = AT.len[k];
        for (int p0 = 0; p0 < L; p0 += 32) {
            const int p = p0 + lane;
            if (p < L) mark_bit(D.bmR, AT.col[base + p]);
        }
    }
}

__global__ void k_detect_cols(MatView AT, DetectBufs D, Ctl *ctl, unsigned mask) {
    pdl_begin();
    if (failed(ctl, mask)) return;
    detect_cols_blocks(AT, D, ctl, blockIdx.x, gridDim.x);
}

// The detection's second step and the merge copy of one matrix in one
// launch (they read and write disjoint data): the first `detect_blocks`
// blocks detect, the others copy.
template <typename T>
__global__ void k_detect_merge(MatView AT, DetectBufs D, long long detect_blocks, UpdJob J, MatView M, Ctl *ctl,
                               unsigned mask) {
    pdl_begin();
    if (failed(ctl, mask)) return;
    if (blockIdx.x < detect_blocks) detect_cols_blocks(AT, D, ctl, blockIdx.x, detect_blocks);
    else merge_copy_blocks<T, false>(J, M, ctl, blockIdx.x - detect_blocks, gridDim.x - detect_blocks);
}

// The affected rows R from their bitmap: a thread per bitmap word, a block
// per 256 words (8192 rows), one atomic per block for its place in R.  R
// comes out in row order within each block's range, so the recompute's
// neighbouring lanes work on neighbouring rows (shared B rows stay in L1).
// The words are cleared for the next batch.
// chunk (may be NULL): per 256-word chunk of the bitmap, where its rows went
// in R and how many (R is ascending within a chunk; chunks land in any order)
__device__ __forceinline__ void collect_blocks(uint32_t *bm, int64_t words, int32_t *R, Ctl *ctl, long long blk,
                                               long long nblk, long long *chunk) {
    __shared__ int s_wsum[8];
    __shared__ long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int64_t b0 = blk * 256; b0 < words; b0 += nblk * 256) {
        const int64_t x = b0 + tid;
        uint32_t bits = x < words ? bm[x] : 0u;
        const int c = __popc(bits);
        int incl = warp_incl_scan<int>(c);
        if (lane == 31) s_wsum[w] = incl;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int k = 0; k < 8; k++) {
                const int v = s_wsum[k];
                s_wsum[k] = t;
                t += v;
            }
            s_base = t ? atomic_add_ll(&ctl->n_affected, t) : 0;
            if (chunk) {
                chunk[2 * (b0 / 256)] = s_base;
                chunk[2 * (b0 / 256) + 1] = t;
            }
        }
        __syncthreads();
        long long o = s_base + s_wsum[w] + incl - c;
        if (bits) {
            bm[x] = 0u;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                R[o++] = (int32_t)(x * 32 + b);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_collect_rows(uint32_t *bm, int64_t words, int32_t *R, long long *chunk,
                                                      Ctl *ctl, unsigned mask) {
    pdl_begin();
    if (failed(ctl, mask)) return;
    collect_blocks(bm, words, R, ctl, blockIdx.x, gridDim.x, chunk);
}

// When B is A the update needs two launches between the classification and
// the sizing: the detection's column step, the merge copy and the commit
// plan (disjoint data: the transposed pattern, A's old rows into staging,
// A's row places) in one, then the collection of R and the commit copy in
// the next.  The first launch's blocks are dealt out to the three jobs; the
// plan may set the arena bit, which none of the others depends on.
template <typename T>
__global__ void __launch_bounds__(256)
k_detect_merge_plan(MatView AT, DetectBufs D, long long nd, UpdJob J, MatView M, CommitJob CJ, long long nm, Ctl *ctl,
                    unsigned mask, int slack_min, int slack_div) {
    pdl_begin();
    if (failed(ctl, mask)) return;
    if (blockIdx.x < nd) detect_cols_blocks(AT, D, ctl, blockIdx.x, nd);
    else if (blockIdx.x < nd + nm) merge_copy_blocks<T, false>(J, M, ctl, blockIdx.x - nd, nm);
    else commit_plan_blocks(CJ, M, ctl, slack_min, slack_div, blockIdx.x - nd - nm, gridDim.x - nd - nm);
}

// R is collected whatever the plan decided (a recovery after an exhausted
// arena re-runs the commit, not the detection); the copy waits for a plan
// that did not fail.
template <typename T>
__global__ void __launch_bounds__(256)
k_collect_copy(uint32_t *bm, int64_t words, int32_t *R, long long *chunk, long long nc, CommitJob CJ, MatView M,
               Ctl *ctl, unsigned collect_mask, unsigned copy_mask) {
    pdl_begin();
    if (blockIdx.x < nc) {
        if (failed(ctl, collect_mask)) return;
        collect_blocks(bm, words, R, ctl, blockIdx.x, nc, chunk);
    } else {
        if (failed(ctl, copy_mask)) return;
        commit_copy_blocks<T>(CJ, M, blockIdx.x - nc, gridDim.x - nc, const_cast<Ctl *>(ctl));
    }
}

void run_detect_merge_plan(const MatView &AT, const DetectBufs &D, const UpdJob &J, const MatView &M,
                           const CommitJob &CJ, int vsize, Ctl *ctl, unsigned mask, int slack_min, int slack_div,
                           int64_t max_items, cudaStream_t s, int num_sms) {
    const long long nd = (long long)num_sms * 4, nm = (long long)num_sms * 8;
    long long np = (max_items + 255) / 256;
    if (np > (long long)num_sms * 4) np = (long long)num_sms * 4;
    if (np < 1) np = 1;
    const unsigned g = (unsigned)(nd + nm + np);
    if (vsize == 8)
        launch_k(k_detect_merge_plan<double>, g, 256, 0, s, AT, D, nd, J, M, CJ, nm, ctl, mask, slack_min, slack_div);
    else
        launch_k(k_detect_merge_plan<int32_t>, g, 256, 0, s, AT, D, nd, J, M, CJ, nm, ctl, mask, slack_min, slack_div);
}

void run_collect_copy(uint32_t *bm, int64_t words, int32_t *R, long long *chunk, const CommitJob &CJ, const MatView &M,
                      int vsize, Ctl *ctl, unsigned collect_mask, unsigned copy_mask, cudaStream_t s, int num_sms) {
    long long nc = (words + 255) / 256;
    if (nc > (long long)num_sms * 8) nc = (long long)num_sms * 8;
    if (nc < 1) nc = 1;
    const unsigned g = (unsigned)(nc + (long long)num_sms * 8);
    if (vsize == 8)
        launch_k(k_collect_copy<double>, g, 256, 0, s, bm, words, R, chunk, nc, CJ, M, ctl, collect_mask, copy_mask);
    else
        launch_k(k_collect_copy<int32_t>, g, 256, 0, s, bm, words, R, chunk, nc, CJ, M, ctl, collect_mask, copy_mask);
}

void run_collect_rows(uint32_t *bm, int64_t words, int32_t *R, long long *chunk, Ctl *ctl, unsigned mask,
                      cudaStream_t s, int num_sms) {
    int64_t g = (words + 255) / 256;
    if (g > (int64_t)num_sms * 8) g = (int64_t)num_sms * 8;
    if (g < 1) g = 1;
    launch_k(k_collect_rows, (unsigned)g, 256, 0, s, bm, words, R, chunk, ctl, mask);
}

// Structural changes of A, forwarded to its transposed pattern: INS (i,k)
// inserts (k,i), DEL (i,k) deletes (k,i).  Other entries become padding in a
// row past the end (dropped by k_segments), so the forwarded batch keeps the
// host-known length of the A batch.
__global__ void k_transpose_feed(const int32_t *srow, const int32_t *scol, const uint8_t *kind, const int64_t *n_dev,
                                 int32_t pad_row, int32_t *trow, int32_t *tcol, uint8_t *top, const Ctl *ctl,
                                 unsigned mask) {
    pdl_begin();
    if (failed(ctl, mask)) return;
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= *n_dev) return;
    const uint8_t k = kind[s];
    if (k == K_INS || k == K_DEL) {
        trow[s] = scol[s];
        tcol[s] = srow[s];
        top[s] = k == K_INS ? OP_INSERT : OP_DELETE;
    } else {
        trow[s] = pad_row;
        tcol[s] = 0;
        top[s] = OP_DELETE;
    }
}

// ------------------------------------------------------------ host glue

static unsigned grid_for(int64_t n, int nt) {
    int64_t g = (n + nt - 1) / nt;
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    return (unsigned)g;
}

void run_classify(const UpdJob &J, const MatView &M, int vsize, Ctl *ctl, unsigned mask, unsigned stage_bit,
                  const DetectBufs &D, bool mark_rows, bool mark_cols, cudaStream_t s, int num_sms) {
    if (J.n <= 0) return;
    unsigned g = grid_for(J.n, 256);
    if (g > (unsigned)num_sms * 8) g = num_sms * 8;
    if (vsize == 8) launch_k(k_classify<double>, g, 256, 0, s, J, M, ctl, mask, stage_bit, D, (int)mark_rows, (int)mark_cols);
    else launch_k(k_classify<int32_t>, g, 256, 0, s, J, M, ctl, mask, stage_bit, D, (int)mark_rows, (int)mark_cols);
}

void run_merge_copy(const UpdJob &J, const MatView &M, int vsize, Ctl *ctl, unsigned mask, cudaStream_t s,
                    int num_sms) {
    if (J.n <= 0) return;
    unsigned g = num_sms * 8;
    if (vsize == 8) launch_k(k_merge_copy<double>, g, 256, 0, s, J, M, ctl, mask);
    else launch_k(k_merge_copy<int32_t>, g, 256, 0, s, J, M, ctl, mask);
}

void run_commit(const CommitJob &J, const MatView &M, int vsize, int64_t max_items, Ctl *ctl, unsigned plan_mask,
                unsigned copy_mask, int slack_min, int slack_div, cudaStream_t s, int num_sms) {
    if (max_items <= 0) return;
    unsigned gp = grid_for(max_items, 256);
    if (gp > (unsigned)num_sms * 4) gp = num_sms * 4;
    launch_k(k_commit_plan, gp, 256, 0, s, J, M, ctl, plan_mask, slack_min, slack_div);
    unsigned g = num_sms * 8;
    if (vsize == 8) launch_k(k_commit_copy<double>, g, 256, 0, s, J, M, ctl, copy_mask);
    else launch_k(k_commit_copy<int32_t>, g, 256, 0, s, J, M, ctl, copy_mask);
}

void run_detect_merge(const MatView &AT, const DetectBufs &D, const UpdJob &J, const MatView &M, int vsize, Ctl *ctl,
                      unsigned mask, cudaStream_t s, int num_sms) {
    if (J.n <= 0) {
        run_detect_cols(AT, D, ctl, mask, s, num_sms);
        return;
    }
    const long long nd = (long long)num_sms * 4;
    const unsigned g = (unsigned)(nd + (long long)num_sms * 8);
    if (vsize == 8) launch_k(k_detect_merge<double>, g, 256, 0, s, AT, D, nd, J, M, ctl, mask);
    else launch_k(k_detect_merge<int32_t>, g, 256, 0, s, AT, D, nd, J, M, ctl, mask);
}

void run_detect_cols(const MatView &AT, const DetectBufs &D, Ctl *ctl, unsigned mask, cudaStream_t s, int num_sms) {
    launch_k(k_detect_cols, num_sms * 4, 256, 0, s, AT, D, ctl, mask);
}

void run_transpose_feed(const UpdJob &J, int32_t pad_row, int32_t *trow, int32_t *tcol, uint8_t *top, Ctl *ctl,
                        unsigned mask, cudaStream_t s) {
    if (J.n <= 0) return;
    launch_k(k_transpose_feed, (unsigned)((J.n + 255) / 256), 256, 0, s, J.row, J.col, J.kind, J.n_dev, pad_row, trow,
             tcol, top, ctl, mask);
}

// ------------------------------------------------------------ footprints

// The rows of C a batch of A updates can touch, as bits over the rows of A:
// its rows (and, when B is A, its columns and every row i with A(i,k) != 0
// for a row k of the batch: the rows of A* B' + A B* of Eq. 1, on the
// current pattern).  A warp per batch entry walks the transposed pattern.
__global__ void k_footprint(const int32_t *row, const int32_t *col, int64_t n, int64_t nrows, int64_t ncols,
                            int b_is_a, MatView AT, uint32_t *bm, unsigned *bad) {
    pdl_begin();
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = w0; e < n; e += nw) {
        const int32_t r = row[e], c = col[e];
        if (r < 0 || r >= nrows || c < 0 || c >= ncols) {
            if (lane == 0) atomicOr(bad, 1u);
            continue;
        }
        if (lane == 0) {
            atomicOr(&bm[r >> 5], 1u << (r & 31));
            if (b_is_a) atomicOr(&bm[c >> 5], 1u << (c & 31));
        }
        if (!b_is_a) continue;
        const int64_t off = AT.off[r];
        const int len = AT.len[r];
        for (int x = lane; x < len; x += 32) {
            const int32_t i = AT.col[off + x];
            atomicOr(&bm[i >> 5], 1u << (i & 31));
        }
    }
}

// cnt[0] = number of words where f and u share a bit (u may be null),
// cnt[1] = number of bits set in f.
__global__ void k_bitmap_overlap(const uint32_t *f, const uint32_t *u, int64_t words, unsigned long long *cnt) {
    pdl_begin();
    unsigned long long c = 0, b = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < words; x += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = f[x];
        b += __popc(w);
        if (u) c += (w & u[x]) != 0u;
    }
    c = warp_sum<unsigned long long>(c);
    b = warp_sum<unsigned long long>(b);
    if ((threadIdx.x & 31) == 0) {
        if (c) atomicAdd(&cnt[0], c);
        if (b) atomicAdd(&cnt[1], b);
    }
}

// u |= f when nothing overlapped (cnt[0] == 0) or always (or_anyway).  With
// `stopped` (a run of admissions in one stream): nothing once an earlier
// footprint overlapped without or_anyway, and such an overlap sets it.  The
// blocks of one launch agree: the flag changes only when cnt says overlap,
// and then every block leaves without writing.
__global__ void k_bitmap_or(const uint32_t *f, uint32_t *u, int64_t words, const unsigned long long *cnt,
                            int or_anyway, unsigned *stopped) {
    pdl_begin();
    if (stopped && *(volatile unsigned *)stopped) return;
    const bool hit = *(volatile const unsigned long long *)cnt != 0ull;
    if (hit && !or_anyway) {
        if (stopped && blockIdx.x == 0 && threadIdx.x == 0) *stopped = 1u;
        return;
    }
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < words; x += (int64_t)gridDim.x * blockDim.x)
        u[x] |= f[x];
}

void run_footprint(const int32_t *row, const int32_t *col, int64_t n, int64_t nrows, int64_t ncols, bool b_is_a,
                   const MatView &AT, uint32_t *bm, unsigned *bad, cudaStream_t s, int num_sms) {
    if (n <= 0) return;
    int64_t g = (n * 32 + 255) / 256;
    if (g > num_sms * 16) g = num_sms * 16;
    launch_k(k_footprint, (unsigned)g, 256, 0, s, row, col, n, nrows, ncols, b_is_a ? 1 : 0, AT, bm, bad);
}

void run_bitmap_overlap(const uint32_t *f, const uint32_t *u, int64_t words, unsigned long long *cnt, cudaStream_t s,
                        int num_sms) {
    int64_t g = (words + 255) / 256;
    if (g > num_sms * 8) g = num_sms * 8;
    if (g < 1) g = 1;
    launch_k(k_bitmap_overlap, (unsigned)g, 256, 0, s, f, u, words, cnt);
}

void run_bitmap_or(const uint32_t *f, uint32_t *u, int64_t words, const unsigned long long *cnt, int or_anyway,
                   cudaStream_t s, int num_sms, unsigned *stopped) {
    int64_t g = (words + 255) / 256;
    if (g > num_sms * 8) g = num_sms * 8;
    if (g < 1) g = 1;
    launch_k(k_bitmap_or, (unsigned)g, 256, 0, s, f, u, words, cnt, or_anyway, stopped);
}

}  // namespace dspg
