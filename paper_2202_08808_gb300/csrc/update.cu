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

// ------------------------------------------------------------- segments

__global__ void k_segments(const int32_t *srow, int64_t n, int64_t nrows, int32_t *seg_lo, int32_t *seg_hi,
                           long long *n_seg, const Ctl *ctl, unsigned mask) {
    if (failed(ctl, mask)) return;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = base + threadIdx.x;
        int32_t r = 0;
        bool head = false;
        if (s < n) {
            r = srow[s];
            // padding entries of a forwarded batch sit in a row past the end
            head = (int64_t)r < nrows && (s == 0 || srow[s - 1] != r);
        }
        const long long t = warp_fetch_add(n_seg, head ? 1 : 0);
        if (head) {
            seg_lo[t] = (int32_t)s;
            seg_hi[t] = (int32_t)upper_bound_dev<int32_t>(srow, s, n, r);
        }
    }
}

// ------------------------------------------------------------- classify

// A warp takes 32 segments at a time: it classifies them one after the
// other (all lanes on one segment), lane r keeping segment r's totals; then
// it allocates merge items, staging and copy items for the 32 segments with
// one atomic per counter, and finally writes the INS/UPD entries.
template <typename T>
__global__ void k_classify(UpdJob J, MatView M, Ctl *ctl, unsigned mask, unsigned stage_bit) {
    if (failed(ctl, mask)) return;
    UpdCtl *u = &ctl->u[J.which];
    const long long nseg = u->n_seg;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const T *bval = (const T *)J.val;
    T *sval = (T *)J.st_val;
    long long s_ins = 0, s_del = 0, s_upd = 0, s_nop = 0;
    for (long long t0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; t0 < nseg; t0 += nwarps * 32) {
        int my_L = 0, my_ins = 0, my_del = 0, my_changed = 0;
        int32_t my_row = 0;
        for (int rr = 0; rr < 32; rr++) {
            const long long t = t0 + rr;
            if (t >= nseg) break;
            const int lo = J.seg_lo[t], hi = J.seg_hi[t];
            const int32_t r = J.row[lo];
            const int64_t base = M.off[r];
            const int L = M.len[r];
            const int32_t *rc = M.col + base;
            int cins = 0, cdel = 0, cupd = 0, cnop = 0;
            for (int u0 = lo; u0 < hi; u0 += 32) {
                const int x = u0 + lane;
                int ins = 0, del = 0;
                if (x < hi) {
                    const int32_t c = J.col[x];
                    const uint8_t op = J.op[x];
                    const int p = (int)lower_bound_dev<int32_t>(rc, 0, L, c);
                    const bool present = p < L && rc[p] == c;
                    uint8_t k;
                    if (op == OP_DEAD) k = K_NOP;
                    else if (op == OP_DELETE) k = present ? K_DEL : K_NOP;
                    else k = present ? K_UPD : K_INS;
                    J.kind[x] = k;
                    J.pos[x] = p;
                    ins = k == K_INS;
                    del = k == K_DEL;
                    cupd += k == K_UPD;
                    cnop += (k == K_NOP && op == OP_DELETE);
                }
                const int ii = warp_incl_scan<int>(ins), di = warp_incl_scan<int>(del);
                if (x < hi) {
                    J.insx[x] = cins + ii - ins;
                    J.delx[x] = cdel + di - del;
                }
                cins += __shfl_sync(0xffffffffu, ii, 31);
                cdel += __shfl_sync(0xffffffffu, di, 31);
            }
            cupd = warp_sum<int>(cupd);
            cnop = warp_sum<int>(cnop);
            s_ins += cins;
            s_del += cdel;
            s_upd += cupd;
            s_nop += cnop;
            if (lane == rr) {
                my_L = L;
                my_ins = cins;
                my_del = cdel;
                my_changed = (cins + cdel + cupd) > 0;
                my_row = r;
            }
        }
        const int my_nl = my_L + my_ins - my_del;
        const int my_nch = my_changed ? (my_L + CH - 1) / CH : 0;
        const long long m = warp_fetch_add(&u->n_merge, my_changed);
        const long long soff = warp_fetch_add(&u->stage_top, my_changed ? my_nl : 0);
        const long long cb = warp_fetch_add(&u->n_chunk, my_nch);
        int ok = 1;
        if (my_changed) {
            ok = (soff + my_nl <= J.st_cap) && (cb + my_nch <= J.ch_cap);
            if (!ok) set_status(ctl, stage_bit);
            else {
                J.m_row[m] = my_row;
                J.m_seg[m] = (int32_t)(t0 + lane);
                J.m_len[m] = my_nl;
                J.m_soff[m] = soff;
                J.m_nins[m] = my_ins;
                J.m_ndel[m] = my_del;
                for (int c = 0; c < my_nch; c++) {
                    J.ch_item[cb + c] = (int32_t)m;
                    J.ch_part[cb + c] = c;
                }
            }
        }
        __syncwarp();
        for (int rr = 0; rr < 32; rr++) {
            const long long t = t0 + rr;
            if (t >= nseg) break;
            const int write = __shfl_sync(0xffffffffu, my_changed && ok, rr);
            const long long so = __shfl_sync(0xffffffffu, soff, rr);
            if (!write) continue;
            const int lo = J.seg_lo[t], hi = J.seg_hi[t];
            for (int x = lo + lane; x < hi; x += 32) {
                const uint8_t k = J.kind[x];
                if (k == K_INS || k == K_UPD) {
                    const int o = J.pos[x] - J.delx[x] + J.insx[x];
                    J.st_col[so + o] = J.col[x];
                    if (sval) sval[so + o] = bval[x];
                }
            }
        }
    }
    if (lane == 0) {
        if (s_ins) atomic_add_ll(&u->ins, s_ins);
        if (s_del) atomic_add_ll(&u->del, s_del);
        if (s_upd) atomic_add_ll(&u->upd, s_upd);
        if (s_nop) atomic_add_ll(&u->nop, s_nop);
    }
}

// ------------------------------------------------------------ merge copy

template <typename T>
__global__ void k_merge_copy(UpdJob J, MatView M, const Ctl *ctl, unsigned mask) {
    if (failed(ctl, mask)) return;
    const long long nch = ctl->u[J.which].n_chunk;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const T *mval = (const T *)M.val;
    T *sval = (T *)J.st_val;
    for (long long x = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < nch; x += nwarps) {
        const int m = J.ch_item[x], part = J.ch_part[x];
        const int32_t r = J.m_row[m];
        const int t = J.m_seg[m];
        const int lo = J.seg_lo[t], hi = J.seg_hi[t];
        const int64_t base = M.off[r];
        const int L = M.len[r];
        const int64_t soff = J.m_soff[m];
        const int tins = J.m_nins[m], tdel = J.m_ndel[m];
        const int p1 = min(L, (part + 1) * CH);
        for (int p = part * CH + lane; p < p1; p += 32) {
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

// ---------------------------------------------------------------- commit

__global__ void k_commit_plan(CommitJob J, MatView M, Ctl *ctl, unsigned mask, int slack_min, int slack_div) {
    if (failed(ctl, mask)) return;
    const long long n = *J.count;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
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

template <typename T>
__global__ void k_commit_copy(CommitJob J, MatView M, const Ctl *ctl, unsigned mask) {
    if (failed(ctl, mask)) return;
    const long long n = *J.cc_count;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const T *sv = (const T *)J.st_val;
    T *mv = (T *)M.val;
    for (long long x = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n; x += nwarps) {
        const int m = J.cc_item[x], part = J.cc_part[x];
        const int32_t r = J.rows[m];
        const int32_t nl = J.lens[m];
        const int64_t d = J.dest[m];
        const int64_t so = J.soff[m];
        const int e1 = min(nl, (part + 1) * CH);
        for (int e = part * CH + lane; e < e1; e += 32) {
            M.col[d + e] = J.st_col[so + e];
            if (mv) mv[d + e] = sv[so + e];
        }
        if (part == 0 && lane == 0) {
            M.off[r] = d;
            M.len[r] = nl;
            M.cap[r] = J.ncap[m];
        }
    }
}

// ---------------------------------------------------------- detection

// Rows of C* (Section 5, Eq. 1) at row granularity: R = rows(A*) u
// {i : A(i,k) != 0, k in rows(B*)}.  A* and B* hold the batch entries that
// change their matrix (kind INS, UPD or DEL).  The second set is read from
// the transposed pattern of A *before* this batch; it equals the set taken
// over A' because a pattern difference at (i,k) already puts i in rows(A*).
// Sets bit i of bm; the lanes that set a fresh bit append i to list with one
// atomic per warp.  All 32 lanes must call it (want = false to abstain).
__device__ __forceinline__ void mark_warp(uint32_t *bm, bool want, int32_t i, int32_t *list, long long *cnt) {
    bool fresh = false;
    if (want) {
        const uint32_t bit = 1u << (i & 31);
        if (!(((volatile uint32_t *)bm)[i >> 5] & bit)) fresh = !(atomicOr(&bm[i >> 5], bit) & bit);
    }
    const long long t = warp_fetch_add(cnt, fresh ? 1 : 0);
    if (fresh) list[t] = i;
}

__global__ void k_detect_entries(const int32_t *srow, const uint8_t *kind, int64_t n, int mark_rows, int mark_cols,
                                 DetectBufs D, Ctl *ctl, unsigned mask) {
    if (failed(ctl, mask)) return;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = base + threadIdx.x;
        const bool ch = s < n && kind[s] != K_NOP;
        const int32_t r = ch ? srow[s] : 0;
        if (mark_rows) mark_warp(D.bmR, ch, r, D.R, &ctl->n_affected);
        if (mark_cols) mark_warp(D.bmK, ch, r, D.K, D.nK);
    }
}

__global__ void k_detect_cols(MatView AT, DetectBufs D, Ctl *ctl, unsigned mask) {
    if (failed(ctl, mask)) return;
    const long long nk = *D.nK;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long x = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < nk; x += nwarps) {
        const int32_t k = D.K[x];
        const int64_t base = AT.off[k];
        const int L = AT.len[k];
        for (int p0 = 0; p0 < L; p0 += 32) {
            const int p = p0 + lane;
            mark_warp(D.bmR, p < L, p < L ? AT.col[base + p] : 0, D.R, &ctl->n_affected);
        }
    }
}

__global__ void k_clear_marks(uint32_t *bm, const int32_t *list, const long long *cnt) {
    const long long n = *cnt;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        bm[list[t] >> 5] = 0u;
}

// Structural changes of A, forwarded to its transposed pattern: INS (i,k)
// inserts (k,i), DEL (i,k) deletes (k,i).  Other entries become padding in a
// row past the end (dropped by k_segments), so the forwarded batch keeps the
// host-known length of the A batch.
__global__ void k_transpose_feed(const int32_t *srow, const int32_t *scol, const uint8_t *kind, int64_t n,
                                 int32_t pad_row, int32_t *trow, int32_t *tcol, uint8_t *top, const Ctl *ctl,
                                 unsigned mask) {
    if (failed(ctl, mask)) return;
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
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

void run_segments(const UpdJob &J, int64_t nrows, Ctl *ctl, unsigned mask, cudaStream_t s) {
    if (J.n <= 0) return;
    launch_k(k_segments, (unsigned)((J.n + 255) / 256), 256, 0, s, J.row, J.n, nrows, J.seg_lo, J.seg_hi,
                                                            &ctl->u[J.which].n_seg, ctl, mask);
}

void run_classify(const UpdJob &J, const MatView &M, int vsize, Ctl *ctl, unsigned mask, unsigned stage_bit,
                  cudaStream_t s, int num_sms) {
    if (J.n <= 0) return;
    unsigned g = grid_for(J.n * 32, 256);
    if (g > (unsigned)num_sms * 8) g = num_sms * 8;
    if (vsize == 8) launch_k(k_classify<double>, g, 256, 0, s, J, M, ctl, mask, stage_bit);
    else launch_k(k_classify<int32_t>, g, 256, 0, s, J, M, ctl, mask, stage_bit);
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

void run_detect_entries(const int32_t *srow, const uint8_t *kind, int64_t n, bool mark_rows, bool mark_cols,
                        const DetectBufs &D, Ctl *ctl, unsigned mask, cudaStream_t s) {
    if (n <= 0) return;
    launch_k(k_detect_entries, (unsigned)((n + 255) / 256), 256, 0, s, srow, kind, n, mark_rows, mark_cols, D, ctl, mask);
}

void run_detect_cols(const MatView &AT, const DetectBufs &D, Ctl *ctl, unsigned mask, cudaStream_t s, int num_sms) {
    launch_k(k_detect_cols, num_sms * 4, 256, 0, s, AT, D, ctl, mask);
}

void run_clear_marks(uint32_t *bm, const int32_t *list, const long long *cnt, int64_t max_n, cudaStream_t s) {
    if (max_n <= 0) return;
    launch_k(k_clear_marks, grid_for(max_n, 256), 256, 0, s, bm, list, cnt);
}

void run_transpose_feed(const UpdJob &J, int32_t pad_row, int32_t *trow, int32_t *tcol, uint8_t *top, Ctl *ctl,
                        unsigned mask, cudaStream_t s) {
    if (J.n <= 0) return;
    launch_k(k_transpose_feed, (unsigned)((J.n + 255) / 256), 256, 0, s, J.row, J.col, J.kind, J.n, pad_row, trow, tcol,
                                                                  top, ctl, mask);
}

}  // namespace dspg
