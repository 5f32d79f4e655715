// handle.cu -- the C ABI: handle lifecycle, build, apply_batch and reads.
//
// apply_batch enqueues the whole pipeline on the caller's stream without a
// host round trip and synchronises once at the end to read the status:
//
//   S1 sort + de-duplicate the A (and B) batch        (sort.cu)
//   S2 segment by row, classify against the old rows  (update.cu)
//   S3 affected rows R from the classification and the transposed pattern
//   S4 merge copy, S5 commit into A (and B)
//   S6 forward structural changes to the transposed pattern of A, apply them
//   S7 size and bin the rows of R, S8 recompute them  (spgemm.cu)
//   S9 splice the recomputed rows into C
//
// Buffers whose need is only known on the device (staging, arena tails) are
// checked there; an overflow sets a status bit, later kernels that depend on
// it return at entry, and the host grows the buffer and re-runs the stages
// from the failed one.  Nothing is mutated before the stage that overflowed
// has succeeded, so the handle always stays consistent.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "estimator.cuh"
#include "internal.h"

using namespace dspg;

unsigned long long &dspg::launch_counter() {
    static unsigned long long count = 0;
    return count;
}

namespace {

struct Err : std::runtime_error {
    dspg_status st;
    Err(dspg_status s, const std::string &m) : std::runtime_error(m), st(s) {}
};

#define CK(x)                                                                                      \
    do {                                                                                           \
        cudaError_t e_ = (x);                                                                      \
        if (e_ != cudaSuccess) throw Err(DSPG_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Host-side fault injection (testing aid; DSPG_FAULT in the environment or
// dspg_fault_inject): "alloc@N" makes the N-th device allocation from then
// on fail as out of memory, "validate@N" the N-th batch check fail as an
// invalid batch.  Counted process-wide.
struct FaultPlan {
    std::atomic<long long> alloc_at{0}, alloc_seen{0}, validate_at{0}, validate_seen{0};
};
FaultPlan &faults() {
    static FaultPlan f;
    return f;
}
bool parse_faults(const char *spec, long long *alloc_at, long long *validate_at) {
    *alloc_at = 0;
    *validate_at = 0;
    if (!spec) return true;
    std::string s(spec);
    size_t p = 0;
    while (p < s.size()) {
        size_t q = s.find(',', p);
        if (q == std::string::npos) q = s.size();
        const std::string item = s.substr(p, q - p);
        const size_t at = item.find('@');
        if (!item.empty()) {
            if (at == std::string::npos) return false;
            const std::string site = item.substr(0, at);
            char *end = nullptr;
            const long long n = strtoll(item.c_str() + at + 1, &end, 10);
            if (!end || *end != '\0' || n < 1) return false;
            if (site == "alloc") *alloc_at = n;
            else if (site == "validate") *validate_at = n;
            else return false;
        }
        p = q + 1;
    }
    return true;
}
void arm_faults(long long alloc_at, long long validate_at) {
    FaultPlan &f = faults();
    f.alloc_seen = 0;
    f.validate_seen = 0;
    f.alloc_at = alloc_at;
    f.validate_at = validate_at;
}
void faults_from_env() {
    static bool done = false;
    if (done) return;
    done = true;
    long long a = 0, v = 0;
    if (const char *env = getenv("DSPG_FAULT"))
        if (parse_faults(env, &a, &v)) arm_faults(a, v);
}
bool fault_fires(std::atomic<long long> &at, std::atomic<long long> &seen) {
    faults_from_env();
    if (at.load() <= 0) return false;
    return ++seen == at.load();
}

void *dmalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (fault_fires(faults().alloc_at, faults().alloc_seen))
        throw Err(DSPG_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected fault)");
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Err(DSPG_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return p;
}

template <typename T>
struct DBuf {
    T *p = nullptr;
    int64_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    // Ensure room for `need` elements; contents are discarded on growth.
    // Returns true when the buffer moved.
    bool reserve(int64_t need) {
        if (need <= n) return false;
        T *q = (T *)dmalloc(sizeof(T) * (size_t)need);
        release();
        p = q;
        n = need;
        return true;
    }
    void swap(DBuf &o) {
        std::swap(p, o.p);
        std::swap(n, o.n);
    }
};

struct DevMat {
    int64_t nrows = 0, ncols = 0;
    int vsize = 0;  // 8, 4, or 0 for a pattern
    DBuf<int64_t> off;
    DBuf<int32_t> len, cap, col;
    DBuf<char> val;
    DBuf<unsigned long long> fb;  // C with its Bloom filter: a word per arena entry (else empty)
    DBuf<long long> top;
    int64_t arena_cap = 0;
    MatView view() {
        return MatView{nrows, ncols, off.p, len.p, cap.p, col.p, vsize ? (void *)val.p : nullptr, top.p, arena_cap};
    }
};

// Work buffers of one matrix update (A, B, or the transposed pattern).
struct UpdWs {
    int which = 0;
    int vsize = 0;
    const int64_t *n_dev = nullptr;  // the batch's length in the device argument block
    int64_t ncap = 0;
    DBuf<int32_t> in_row, in_col;
    DBuf<char> in_val;
    DBuf<uint8_t> in_op;
    DBuf<int32_t> row, col;
    DBuf<char> val;
    DBuf<uint8_t> op, kind;
    DBuf<int32_t> pos, insx, delx, m_lo, m_hi, m_row, m_len, m_nins, m_ndel, m_cap;
    DBuf<int64_t> m_soff, m_dest;
    DBuf<int32_t> ch_item, ch_part, cc_item, cc_part;
    DBuf<int32_t> st_col;
    DBuf<char> st_val;
    int64_t st_cap = 0;
    DBuf<uint64_t> k0, k1;
    DBuf<uint32_t> i0, i1, counts;
    DBuf<int64_t> scan_tmp, scan_out;

    bool ensure(int64_t n, int64_t arena_cap) {
        bool moved = false;
        if (n > ncap) {
            moved = true;
            int64_t c = std::max<int64_t>(n, std::max<int64_t>(2 * ncap, 1024));
            in_row.reserve(c); in_col.reserve(c); in_val.reserve(c * std::max(vsize, 1)); in_op.reserve(c);
            row.reserve(c); col.reserve(c); val.reserve(c * std::max(vsize, 1)); op.reserve(c); kind.reserve(c);
            pos.reserve(c); insx.reserve(c); delx.reserve(c); m_lo.reserve(c); m_hi.reserve(c);
            m_row.reserve(c); m_len.reserve(c); m_nins.reserve(c); m_ndel.reserve(c);
            m_cap.reserve(c); m_soff.reserve(c); m_dest.reserve(c);
            k0.reserve(c); k1.reserve(c); i0.reserve(c); i1.reserve(c);
            int64_t cnt;
            sort_tmp_sizes(c, &cnt);
            counts.reserve(cnt);
            scan_out.reserve(cnt + 1);
            scan_tmp.reserve(scan_tmp_entries(cnt) + 1);
            ncap = c;
        }
        if (st_cap < 16 * n + 65536) moved |= grow_stage(16 * n + 65536);
        moved |= ch_item.reserve(ncap + arena_cap / 256 + 64);
        moved |= ch_part.reserve(ncap + arena_cap / 256 + 64);
        return moved;
    }
    bool grow_stage(int64_t need) {
        if (need <= st_cap) return false;
        int64_t c = std::max<int64_t>(need, st_cap + st_cap / 2);
        st_col.reserve(c);
        if (vsize) st_val.reserve(c * vsize);
        st_cap = c;
        cc_item.reserve(ncap * 2 + c / 256 + 64);
        cc_part.reserve(ncap * 2 + c / 256 + 64);
        return true;
    }
    SortOut sort_out() { return SortOut{row.p, col.p, vsize ? (void *)val.p : nullptr, op.p}; }
    SortTmp sort_tmp() {
        return SortTmp{k0.p, k1.p, i0.p, i1.p, counts.p, scan_tmp.p, scan_out.p, k0.n, counts.n};
    }
    UpdJob job(int64_t n) {  // n: the launch size (at least the batch's length)
        UpdJob J{};
        J.which = which;
        J.n = n;
        J.n_dev = n_dev;
        J.row = row.p; J.col = col.p; J.val = vsize ? (void *)val.p : nullptr; J.op = op.p;
        J.kind = kind.p; J.pos = pos.p; J.insx = insx.p; J.delx = delx.p;
        J.m_row = m_row.p; J.m_lo = m_lo.p; J.m_hi = m_hi.p; J.m_len = m_len.p; J.m_nins = m_nins.p; J.m_ndel = m_ndel.p;
        J.m_soff = m_soff.p; J.m_dest = m_dest.p; J.m_cap = m_cap.p;
        J.ch_item = ch_item.p; J.ch_part = ch_part.p; J.ch_cap = ch_item.n;
        J.cc_item = cc_item.p; J.cc_part = cc_part.p; J.cc_cap = cc_item.n;
        J.st_col = st_col.p; J.st_val = vsize ? (void *)st_val.p : nullptr; J.st_cap = st_cap;
        return J;
    }
};

// Work buffers of the recompute of C rows.
struct CWs {
    int64_t nrows = 0;
    DBuf<int32_t> R, iota, bins;
    DBuf<char> gd_acc;
    DBuf<uint32_t> gd_mask;
    DBuf<uint32_t> gd_sum;
    int64_t gd_w = 0;
    int gd_ctas = 0;
    // detection
    DBuf<uint32_t> bmR, bmK;
    // per 256-word chunk of bmR: the offset in R of its rows and their count
    // (R is ascending within a chunk), so R can be read back in order
    DBuf<long long> rchunk;
    DBuf<int32_t> K;
    int64_t nrows_b = 0;
    // learned sizing: rows waiting for an estimate, rows whose table overflowed
    DBuf<int4> est;
    DBuf<int32_t> ovf;
    // split rows (dense mode): global accumulators
    int64_t sp_rows = 0;
    DBuf<char> sp_acc;
    DBuf<uint32_t> sp_mask;
    DBuf<int> sp_done;
    DBuf<int64_t> sp_pre;
};

// Working memory of dspg_footprint (kept, so a serving loop allocates nothing).
struct FpWs {
    DBuf<int32_t> row, col;
    DBuf<unsigned long long> cnt;
    struct Pinned {
        unsigned long long *p = nullptr;
        int64_t n = 0;
        void reserve_host(int64_t need) {
            if (need <= n) return;
            if (p) cudaFreeHost(p);
            p = nullptr;
            n = 0;
            if (cudaMallocHost((void **)&p, sizeof(unsigned long long) * need) != cudaSuccess) {
                cudaGetLastError();
                p = nullptr;
                throw Err(DSPG_ERR_OOM, "pinned host allocation failed");
            }
            n = need;
        }
        ~Pinned() {
            if (p) cudaFreeHost(p);
        }
    } hcnt;
};

// Working memory of the delta path (algebraic updates, Eq. 1): the list of
// new entries of C, its sorted copy and sort buffers, the rows' plan, and the
// bitmap of rows of C too long to take contributions in place.
struct AlgWs {
    int64_t ncap = 0;
    DBuf<int32_t> nr, nc, srow, scol;
    DBuf<char> nv, sval;
    DBuf<uint8_t> nop, sop;
    DBuf<uint64_t> k0, k1;
    DBuf<uint32_t> i0, i1, counts;
    DBuf<int64_t> scan_tmp, scan_out, dest;
    DBuf<int32_t> cap;
    DBuf<uint32_t> bm_long;
    DBuf<InArgs> args;  // device: where the new-entry list is, for the sort
    bool ensure(int64_t need, int64_t nrows, int vsize, cudaStream_t s) {
        bool moved = false;
        if (need > ncap) {
            const int64_t c = std::max<int64_t>(need, 2 * ncap);
            nr.reserve(c); nc.reserve(c); nv.reserve(c * vsize); nop.reserve(c);
            srow.reserve(c); scol.reserve(c); sval.reserve(c * vsize); sop.reserve(c);
            k0.reserve(c); k1.reserve(c); i0.reserve(c); i1.reserve(c);
            int64_t cnt;
            sort_tmp_sizes(c, &cnt);
            counts.reserve(cnt);
            scan_out.reserve(cnt + 1);
            scan_tmp.reserve(scan_tmp_entries(cnt) + 1);
            dest.reserve(c);
            cap.reserve(c);
            ncap = c;
            moved = true;
        }
        if (bm_long.reserve(nrows / 32 + 2)) {
            CK(cudaMemsetAsync(bm_long.p, 0, sizeof(uint32_t) * bm_long.n, s));
            moved = true;
        }
        if (moved || !args.p) {
            args.reserve(1);
            const InArgs a{nr.p, nc.p, nv.p, nop.p};
            CK(cudaMemcpyAsync(args.p, &a, sizeof(InArgs), cudaMemcpyHostToDevice, s));
        }
        return moved;
    }
    SortOut sort_out() { return SortOut{srow.p, scol.p, (void *)sval.p, sop.p}; }
    SortTmp sort_tmp() { return SortTmp{k0.p, k1.p, i0.p, i1.p, counts.p, scan_tmp.p, scan_out.p, k0.n, counts.n}; }
};

struct BatchIn {
    const int32_t *row = nullptr, *col = nullptr;
    const void *val = nullptr;
    const uint8_t *op = nullptr;
    int64_t n = 0;
    int64_t cap = 0;  // launch size: batch_bucket(n)
};

thread_local std::string g_err;

}  // namespace

void dspg::set_thread_error(const char *msg) { g_err = msg; }

// Side streams of the recompute: the bin kernels run as parallel branches
// (the first, the thread-merge bin, alone on the handle's stream).  More
// branches than the device's hardware queues (8 by default) made the
// launches share queues and wait on each other: three side streams.
constexpr int NUM_SIDE = 3;

// The masked path's work buffers (Algorithm 2), grown to each batch's
// counts: contributions to C*, their sort, C* itself with its runs, the
// kept entries of A', and the Bloom build's long-row list and place maps.
struct MaskWs {
    int64_t ccap = 0;  // contributions
    DBuf<uint64_t> key, key_alt, bits;
    DBuf<uint32_t> idx, idx_alt, counts;
    DBuf<int64_t> scan_tmp, scan_out, ex;
    DBuf<int32_t> flag;
    int64_t ucap = 0;  // entries of C*
    DBuf<int32_t> urow, ucol, rflag, upos, run_row, dcap;
    DBuf<unsigned long long> ufs, ue, rbits, h;
    DBuf<int64_t> rex, run_start, dest, uscan;
    DBuf<char> z;
    DBuf<uint8_t> hit;
    int64_t kcap = 0;  // kept entries of A'
    DBuf<int32_t> kept_run;
    DBuf<int64_t> kept_a;
    DBuf<int32_t> rows_long, posmap;
    DBuf<long long> n_long;
    int64_t posmap_ctas = 0, posmap_m = 0;

    void ensure_contrib(int64_t n) {
        if (n <= ccap) return;
        const int64_t c = std::max<int64_t>(n, 2 * ccap);
        key.reserve(c); key_alt.reserve(c); bits.reserve(c);
        idx.reserve(c); idx_alt.reserve(c);
        flag.reserve(c); ex.reserve(c + 1);
        int64_t cnt = 0;
        sort_tmp_sizes(c, &cnt);
        counts.reserve(cnt);
        scan_out.reserve(cnt + 1);
        scan_tmp.reserve(scan_tmp_entries(std::max(cnt, c)) + 1);
        ccap = c;
    }
    void ensure_unique(int64_t nu, int vsize) {
        if (nu <= ucap) return;
        const int64_t c = std::max<int64_t>(nu, 2 * ucap);
        urow.reserve(c); ucol.reserve(c); rflag.reserve(c); upos.reserve(c); run_row.reserve(c); dcap.reserve(c);
        ufs.reserve(c); ue.reserve(c); rbits.reserve(c); h.reserve(c);
        rex.reserve(c + 1); run_start.reserve(c + 1); dest.reserve(c);
        uscan.reserve(scan_tmp_entries(c) + 1);
        z.reserve(c * vsize); hit.reserve(c);
        ucap = c;
    }
    void ensure_kept(int64_t n) {
        if (n <= kcap) return;
        const int64_t c = std::max<int64_t>(n, 2 * kcap);
        kept_run.reserve(c); kept_a.reserve(c);
        kcap = c;
    }
};

struct dspg_handle {
    int sr = 0, vsize = 8, num_sms = 148, dev = 0;
    dspg_options opt{};
    DevMat A, B, AT, C;
    bool b_is_a = true;
    bool has_at = false;
    Ctl *ctl = nullptr;   // device
    Ctl *hctl = nullptr;      // pinned, mapped host mirror
    Ctl *hctl_dev = nullptr;  // its device address
    UpdWs wA, wB, wAT;
    CWs wc;
    // grow-only scratch of the read calls (row list, lengths, row pointers,
    // gathered rows, the affected-row sort), so that reading results between
    // batches allocates nothing; a read larger than kReadKeep bytes per
    // buffer allocates for the call instead of holding that memory
    struct ReadWs {
        DBuf<int32_t> rows, lens, c, r;
        DBuf<int64_t> rp, scan, listed, st, so, chunk_cnt, chunk_ex, chunk_tmp, long_l, huge_l;
        DBuf<ReadOut> res;
        DBuf<unsigned> n_listed;
        DBuf<char> v;
        DBuf<uint64_t> k0, k1;
        DBuf<uint32_t> i0, i1, counts;
        std::vector<int32_t> h_r;     // R as collected (host)
        std::vector<long long> h_ch;  // its chunk table (host)
    } rd;
    // C's generation (bumped by every call that may change C) and the row
    // list whose row pointers rd.rp holds, so the fill call of a two-call
    // read of C's rows reuses what its count call computed
    uint64_t c_serial = 0;
    struct ReadKey {
        bool valid = false;
        uint64_t serial = 0;
        int64_t nnz = 0;
        std::vector<int32_t> rows;
    } rd_key;
    BatchIn inA, inB;
    InArgs *d_args = nullptr;  // device: where the A, B and forwarded batches are (read by the sorts)
    InArgs *h_args = nullptr;  // pinned, mapped host mirror, fetched by the pipeline's first step
    InArgs *h_args_dev = nullptr;
    int64_t last_nR = 0;
    bool prof = false;
    cudaEvent_t pev[10] = {};  // stage boundaries (profiling)
    float stage_ms[DSPG_NSTAGES] = {};
    // streams and events of the pipeline's branches
    cudaStream_t gs = nullptr;       // graphs run here
    cudaStream_t side = nullptr;     // transposed-pattern branch
    cudaStream_t nstr[NUM_SIDE] = {};  // numeric bin branches
    cudaEvent_t evIn = nullptr, evFork = nullptr, evDetect = nullptr, evSide = nullptr, evSize = nullptr;
    cudaEvent_t evNum[NUM_SIDE] = {};
    // captured pipelines, keyed by batch sizes and the buffer epoch
    struct Graph {
        int64_t nA, nB;
        uint64_t epoch;
        bool prof;
        cudaGraphExec_t exec;
        unsigned long long kernels;  // kernel nodes, added to the launch counter per replay
    };
    std::vector<Graph> graphs;
    std::vector<Graph> seen;  // keys run once eagerly (exec unused)
    uint64_t epoch = 1;       // bumped whenever a persistent buffer moves
    bool use_graphs = true;
    // recompute bins launched (bit b); a row of a bin that is off goes to the
    // global dense bin and turns the bin on for the next batch (learn_bins)
    unsigned long long bin_on = ~0ull;
    bool bins_narrowed = false;  // bin_on has been cut to the bins the first batch used
    bool gate_bins = true;       // DSPG_ALL_BINS=1: every bin, always
    bool direct_read = true;     // DSPG_NO_DIRECT_READ=1: reads always stage on the device and copy
    dspg_tuning tune{8, 64, 8, 0, 1024, 16384, 64};  // row bins of the recompute
    int sizing = DSPG_SIZE_BOUND;               // how the recompute's tables are sized
    int est_min = 128;
    float est_margin = 0.25f;
    DBuf<uint16_t> est_w;                       // estimator weights (bfloat16 bits)
    FpWs fp;                                    // footprints (serving)
    AlgWs alg;                                  // the delta path (algebraic updates)
    bool last_alg = false;                      // the last batch took the delta path
    int64_t grp_cap_a = 0, grp_cap_b = 0;       // in a group: launch sizes reserved so far (grow-only)
    int64_t runs_replayed = 0, runs_captured = 0, runs_eager = 0;  // how batches ran (dspg_run_counts)
    bool pending = false;                       // an asynchronous apply is in flight (dspg_apply_batch_async)
    int64_t pending_comp0 = 0;
    // the product form (Section 3): C = alpha op(A) op(B) (+) beta X
    bool trans_a = false, trans_b = false;      // op = transpose: the operand is stored transposed
    bool b_alias = false;                       // the caller's B is A, stored apart (one side transposed)
    bool form = false;                          // reads apply alpha, beta and X
    FormScalars fs{1.0, 1.0, 0, 0};
    bool has_x = false;
    DBuf<int64_t> xrp;                          // X (canonical CSR, library-owned)
    DBuf<int32_t> xcol;
    DBuf<char> xval;
    int64_t extra_slots = 0;                    // table slots of the last batch's overflow recompute
    bool bloom = false;                         // C keeps its Bloom filter; batches take Algorithm 2
    bool broken = false;                        // a batch failed after A, B or C began to change
    MaskWs mw;                                  // the masked path's buffers
    int64_t last_masked = 0;                    // entries of C* of the last batch
    int64_t compactions = 0;
    std::string err;

    DevMat &Bm() { return b_is_a ? A : B; }
};

// A group: the members' pipelines as branches of one graph.
struct dspg_group {
    std::vector<dspg_handle *> hs;
    cudaStream_t gs = nullptr;  // graphs run here
    cudaEvent_t evIn = nullptr, evFork = nullptr;
    struct Graph {
        std::vector<int64_t> key;  // per member: nA, nB, buffer epoch
        cudaGraphExec_t exec;
        unsigned long long kernels;
    };
    std::vector<Graph> graphs;
    std::vector<std::vector<int64_t>> seen;
    std::string err;
};

namespace {

// An NVTX range over a host call (shown by profilers that record NVTX; a
// push and a pop of a string otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// DSPG_TRACE=<file>: one JSON line per applied batch (its statistics, the
// stage times when profiling is on), appended to the file.
void trace_batch(const dspg_handle *h, const dspg_batch_stats &st, const char *path_kind);

void set_defaults(dspg_options *o) {
    o->slack_min = 4;
    o->slack_div = 4;
    o->arena_headroom = 1.5;
    o->keep_transpose = -1;
    o->exact_static = 0;
    o->bloom = 0;
}

// A failed check of the debug build (ST_DEBUG) as an error.
void check_debug(const Ctl *c) {
    if (c->status & ST_DEBUG)
        throw Err(DSPG_ERR_CUDA, "debug build: check " + std::to_string(c->dbg_code) + " failed at index " +
                                     std::to_string(c->dbg_idx));
}

std::string overflow_message(const Ctl *c) {
    return "accumulator probe limit reached (bin " + std::to_string(c->timeout_bin - 1) + ", row " +
           std::to_string(c->timeout_row) + ", product bound " + std::to_string(c->timeout_ub) + ")";
}

void read_ctl(dspg_handle *h, cudaStream_t s) {
    CK(cudaMemcpyAsync(h->hctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
}

int64_t read_i64(const int64_t *dptr, cudaStream_t s) {
    int64_t v = 0;
    CK(cudaMemcpyAsync(&v, dptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return v;
}

// Build a slack-CSR from rows given as (start, length) in source arrays
// (which must not be M's own).  M's buffers are reused when large enough.
void make_slack(dspg_handle *h, DevMat &M, int64_t nrows, int64_t ncols, int vsize, const int64_t *src_off,
                const int32_t *len, const int32_t *src_col, const void *src_val, cudaStream_t s) {
    M.nrows = nrows;
    M.ncols = ncols;
    M.vsize = vsize;
    M.len.reserve(std::max<int64_t>(nrows, 1));
    M.cap.reserve(std::max<int64_t>(nrows, 1));
    M.off.reserve(nrows + 1);
    M.top.reserve(1);
    if (nrows > 0) CK(cudaMemcpyAsync(M.len.p, len, sizeof(int32_t) * nrows, cudaMemcpyDeviceToDevice, s));
    caps_from_lens(M.len.p, M.cap.p, nrows, h->opt.slack_min, h->opt.slack_div, s);
    DBuf<int64_t> tmp;
    tmp.reserve(scan_tmp_entries(nrows) + 1);
    scan_i32_to_i64(M.cap.p, M.off.p, nrows, tmp.p, s);
    const int64_t total = read_i64(M.off.p + nrows, s);
    const int64_t need = std::max<int64_t>((int64_t)(total * h->opt.arena_headroom), total + 4096);
    if (M.col.n < need) {
        M.col.release();
        M.val.release();
        M.col.reserve(need);
    }
    M.arena_cap = M.col.n;
    if (vsize) M.val.reserve(M.arena_cap * vsize);
    copy_rows(nullptr, nrows, src_off, M.len.p, src_col, src_val, M.off.p, M.col.p, vsize ? (void *)M.val.p : nullptr,
              vsize, s, h->num_sms);
    long long t = total;
    CK(cudaMemcpyAsync(M.top.p, &t, sizeof(long long), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    h->epoch++;
}

// Rebuild M's arena with fresh slack for every row and at least twice the
// room of the old arena (growth after the tail ran out).
void regrow(dspg_handle *h, DevMat &M, cudaStream_t s) {
    DBuf<int32_t> ncap;
    DBuf<int64_t> noff, tmp;
    ncap.reserve(M.nrows);
    noff.reserve(M.nrows + 1);
    tmp.reserve(scan_tmp_entries(M.nrows) + 1);
    caps_from_lens(M.len.p, ncap.p, M.nrows, h->opt.slack_min, h->opt.slack_div, s);
    scan_i32_to_i64(ncap.p, noff.p, M.nrows, tmp.p, s);
    const int64_t total = read_i64(noff.p + M.nrows, s);
    const int64_t cap = std::max<int64_t>(std::max<int64_t>((int64_t)(total * h->opt.arena_headroom), 2 * M.arena_cap),
                                          total + 4096);
    DBuf<int32_t> ncol;
    DBuf<char> nval;
    ncol.reserve(cap);
    if (M.vsize) nval.reserve(cap * M.vsize);
    copy_rows(nullptr, M.nrows, M.off.p, M.len.p, M.col.p, M.vsize ? (void *)M.val.p : nullptr, noff.p, ncol.p,
              M.vsize ? (void *)nval.p : nullptr, M.vsize, s, h->num_sms);
    DBuf<unsigned long long> nfb;
    if (M.fb.n > 0) {  // the Bloom words move with their entries (bit patterns copied as 8-byte values)
        nfb.reserve(cap);
        copy_rows(nullptr, M.nrows, M.off.p, M.len.p, M.col.p, (const void *)M.fb.p, noff.p, ncol.p, (void *)nfb.p,
                  8, s, h->num_sms);
    }
    long long t = total;
    CK(cudaMemcpyAsync(M.top.p, &t, sizeof(long long), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    M.off.swap(noff);
    M.cap.swap(ncap);
    M.col.swap(ncol);
    M.val.swap(nval);
    if (M.fb.n > 0) M.fb.swap(nfb);
    M.arena_cap = cap;
    h->compactions++;
    h->epoch++;
}

// Canonical CSR copy of M's rows (all rows when rows == nullptr) into device
// buffers; returns nnz.  rowptr_out has n+1 entries.
constexpr int64_t kReadKeep = int64_t(256) << 20;  // bytes per kept read buffer

// Room for `need` elements: the handle's kept buffer while it stays within
// kReadKeep bytes, else `local` (freed when the caller returns).
template <typename T>
T *read_scratch(DBuf<T> &keep, DBuf<T> &local, int64_t need) {
    need = std::max<int64_t>(need, 1);
    if ((int64_t)sizeof(T) * need <= kReadKeep) {
        keep.reserve(need);
        return keep.p;
    }
    local.reserve(need);
    return local.p;
}

// Row pointers of rows[n] of M (every row when rows is NULL) into rowptr
// (room for n + 1); returns their total length.
int64_t mat_rowptr(dspg_handle *h, DevMat &M, const int32_t *rows, int64_t n, int64_t *rowptr, cudaStream_t s) {
    DBuf<int32_t> lens_l;
    DBuf<int64_t> tmp_l;
    const int32_t *lp = M.len.p;
    if (rows) {
        int32_t *lens = read_scratch(h->rd.lens, lens_l, n);
        lens_of_rows(rows, n, M.len.p, lens, s);
        lp = lens;
    }
    int64_t *tmp = read_scratch(h->rd.scan, tmp_l, scan_tmp_entries(n) + 1);
    scan_i32_to_i64(lp, rowptr, n, tmp, s);
    return read_i64(rowptr + n, s);
}

void ensure_c_ws(dspg_handle *h, cudaStream_t s) {
    CWs &w = h->wc;
    const int64_t n = h->A.nrows;
    if (w.nrows == n && w.R.p) return;
    h->epoch++;
    w.nrows = n;
    const int64_t nn = std::max<int64_t>(n, 1);
    w.R.reserve(nn);
    w.iota.reserve(nn);
    fill_iota(w.iota.p, n, s);
    w.bins.reserve((int64_t)NBINS * nn);
    w.bmR.reserve(nn / 32 + 2);
    CK(cudaMemsetAsync(w.bmR.p, 0, sizeof(uint32_t) * w.bmR.n, s));
    w.rchunk.reserve(2 * ((nn + 31) / 32 / 256 + 1));
    w.est.reserve(nn);
    w.ovf.reserve(nn);
    const int64_t nb = std::max<int64_t>(h->Bm().nrows, 1);
    w.nrows_b = nb;
    w.bmK.reserve(nb / 32 + 2);
    CK(cudaMemsetAsync(w.bmK.p, 0, sizeof(uint32_t) * w.bmK.n, s));
    w.K.reserve(nb);
    const int64_t m = h->Bm().ncols;
    if (m <= DENSE_M_MAX) {  // split rows: as many as 256 MiB of accumulators hold, at most 65536
        const int64_t mp = (m + 31) / 32 * 32;
        w.sp_rows = std::min<int64_t>(65536, (256LL << 20) / (mp * h->vsize + mp / 8));
        w.sp_pre.reserve(w.sp_rows + 1);
        w.sp_acc.reserve(w.sp_rows * mp * h->vsize);
        w.sp_mask.reserve(w.sp_rows * mp / 32);
        w.sp_done.reserve(w.sp_rows);
        init_dense_scratch(h->sr, w.sp_acc.p, w.sp_mask.p, w.sp_rows * mp, w.sp_rows * mp / 32, s);
        CK(cudaMemsetAsync(w.sp_done.p, 0, sizeof(int) * w.sp_rows, s));
    }
    if (m > DENSE_M_MAX) {
        w.gd_w = (m + 31) / 32 * 32;
        // per-CTA dense accumulators for the longest rows: up to two CTAs per
        // SM, within a budget of 1/32 of the free memory (256 MiB .. 4 GiB)
        const double per = (double)w.gd_w * (h->vsize + 0.13);
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        const double budget = std::min(4.0 * (1 << 30), std::max(256.0 * (1 << 20), (double)free_b / 32.0));
        int ctas = (int)std::min<double>(2.0 * h->num_sms, std::max(4.0, budget / per));
        w.gd_ctas = std::max(1, ctas);
        w.gd_acc.reserve(w.gd_w * w.gd_ctas * h->vsize);
        w.gd_mask.reserve(w.gd_w / 32 * w.gd_ctas);
        const int64_t nsum = (w.gd_w / 32 + 31) / 32;
        w.gd_sum.reserve(nsum * w.gd_ctas);
        CK(cudaMemsetAsync(w.gd_sum.p, 0, sizeof(uint32_t) * nsum * w.gd_ctas, s));
        init_dense_scratch(h->sr, w.gd_acc.p, w.gd_mask.p, w.gd_w * w.gd_ctas, w.gd_w / 32 * w.gd_ctas, s);
    }
}

CJob c_job(dspg_handle *h, const int32_t *R, bool static_mode) {
    CWs &w = h->wc;
    CJob J{};
    J.R = R;
    J.bins = w.bins.p;
    J.bin_cap = std::max<int64_t>(w.nrows, 1);
    J.gd_acc = w.gd_acc.p;
    J.gd_mask = w.gd_mask.p;
    J.gd_sum = w.gd_sum.p;
    J.gd_w = w.gd_w;
    J.gd_ctas = std::max(w.gd_ctas, 1);
    J.m = h->Bm().ncols;
    J.dense_mode = J.m <= DENSE_M_MAX ? 1 : 0;
    J.static_mode = static_mode ? 1 : 0;
    J.slack_min = h->opt.slack_min;
    J.slack_div = h->opt.slack_div;
    J.rows_hint = h->A.nrows;
    J.tm_k = h->tune.merge_k;
    J.tm_ub = h->tune.merge_ub;
    J.lanes_min = h->tune.lanes_min;
    J.table_shift = h->tune.table_shift;
    J.warp_max = h->tune.warp_max;
    J.cta_max = h->tune.cta_max;
    J.sort_max = h->tune.sort_max;
    J.bin_on = (J.dense_mode || static_mode || !h->gate_bins) ? ~0ull : h->bin_on;
    J.sizing = (!static_mode && h->sizing == DSPG_SIZE_LEARNED) ? SIZE_LEARNED : SIZE_BOUND;
    J.est_min = h->est_min;
    J.est_margin = h->est_margin;
    J.est_w = h->est_w.p;
    J.est = w.est.p;
    J.ovf = w.ovf.p;
    J.sp_rows = J.dense_mode ? w.sp_rows : 0;
    J.sp_acc = w.sp_acc.p;
    J.sp_mask = w.sp_mask.p;
    J.sp_done = w.sp_done.p;
    J.sp_pre = w.sp_pre.p;
    return J;
}

CommitJob upd_commit_job(dspg_handle *h, UpdWs &w, unsigned arena_bit, unsigned stage_bit) {
    CommitJob J{};
    J.rows = w.m_row.p;
    J.lens = w.m_len.p;
    J.soff = w.m_soff.p;
    J.count = &h->ctl->u[w.which].n_merge;
    J.st_col = w.st_col.p;
    J.st_val = w.vsize ? (const void *)w.st_val.p : nullptr;
    J.dest = w.m_dest.p;
    J.ncap = w.m_cap.p;
    J.cc_item = w.cc_item.p;
    J.cc_part = w.cc_part.p;
    J.cc_count = &h->ctl->u[w.which].n_cchunk;
    J.cc_cap = w.cc_item.n;
    J.reloc = &h->ctl->u[w.which].reloc;
    J.arena_bit = arena_bit;
    J.stage_bit = stage_bit;
    return J;
}

// The bin kernels of the recompute run on four branches that join s again.
void numeric_branches(dspg_handle *h, cudaStream_t s, const CJob &J) {
    CK(cudaEventRecord(h->evSize, s));
    for (int k = 0; k < NUM_SIDE; k++) CK(cudaStreamWaitEvent(h->nstr[k], h->evSize, 0));
    cudaStream_t ss[NUM_SIDE + 1] = {s};
    for (int k = 0; k < NUM_SIDE; k++) ss[k + 1] = h->nstr[k];
    run_numeric(h->sr, h->A.view(), h->Bm().view(), h->C.view(), J, h->ctl, M_C, ss, NUM_SIDE + 1, h->num_sms);
    for (int k = 0; k < NUM_SIDE; k++) {
        CK(cudaEventRecord(h->evNum[k], h->nstr[k]));
        CK(cudaStreamWaitEvent(s, h->evNum[k], 0));
    }
}

// Full recompute of C from A, B (the static product).  The sizing pass lays
// C out afresh with room for each row's product bound and the numeric
// kernels write every row in place.  When that layout would take more than a
// quarter of the free device memory (bounds far above the true row sizes,
// as in squares of skewed graphs), an exact pass first counts every row and
// C is laid out from the counts instead.  The arena is reused when large
// enough.
void bloom_build(dspg_handle *h, cudaStream_t s);

void static_recompute(dspg_handle *h, cudaStream_t s) {
    NvtxRange r("dspg/static_recompute");
    h->c_serial++;
    ensure_c_ws(h, s);
    DevMat &C = h->C;
    const int64_t n = h->A.nrows;
    C.nrows = n;
    C.ncols = h->Bm().ncols;
    C.vsize = h->vsize;
    C.len.reserve(std::max<int64_t>(n, 1));
    C.cap.reserve(std::max<int64_t>(n, 1));
    C.off.reserve(n + 1);
    C.top.reserve(1);
    h->epoch++;
    MatView Av = h->A.view(), Bv = h->Bm().view();
    CK(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), s));
    CK(cudaMemsetAsync(C.top.p, 0, sizeof(long long), s));
    long long nn = n;
    CK(cudaMemcpyAsync(&h->ctl->n_affected, &nn, sizeof(long long), cudaMemcpyHostToDevice, s));
    run_size_bins(Av, Bv, C.view(), c_job(h, h->wc.iota.p, true), n, h->ctl, M_AB, s, h->num_sms);
    read_ctl(h, s);
    if (h->hctl->status & ~ST_C_ARENA)
        throw Err(DSPG_ERR_CUDA, "static sizing failed with status " + std::to_string(h->hctl->status));
    long long need = 0;
    CK(cudaMemcpyAsync(&need, C.top.p, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const double entry_b = 4.0 + h->vsize;
    const bool exact = h->opt.exact_static == 1 ||
                       (double)need * entry_b * h->opt.arena_headroom > 0.25 * (double)(free_b + C.col.n * entry_b);
    CK(cudaMemsetAsync(&h->ctl->status, 0, sizeof(unsigned), s));
    if (exact) {
        CJob Jc = c_job(h, h->wc.iota.p, true);
        Jc.count_only = 1;
        numeric_branches(h, s, Jc);
        read_ctl(h, s);
        if (h->hctl->status) throw Err(DSPG_ERR_CUDA, "exact sizing failed with status " + std::to_string(h->hctl->status));
        caps_from_lens(C.len.p, C.cap.p, n, h->opt.slack_min, h->opt.slack_div, s);
        DBuf<int64_t> tmp;
        tmp.reserve(scan_tmp_entries(n) + 1);
        scan_i32_to_i64(C.cap.p, C.off.p, n, tmp.p, s);
        need = read_i64(C.off.p + n, s);
        CK(cudaMemcpyAsync(C.top.p, &need, sizeof(long long), cudaMemcpyHostToDevice, s));
    }
    const int64_t cap = std::max<int64_t>((int64_t)(need * h->opt.arena_headroom), need + 4096);
    if (C.col.n < need + 1) {
        C.col.release();
        C.val.release();
        C.col.reserve(cap);
        C.val.reserve(cap * h->vsize);
    }
    C.arena_cap = C.col.n;
    C.val.reserve(C.arena_cap * h->vsize);
    CK(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), s));
    CK(cudaMemcpyAsync(&h->ctl->n_affected, &nn, sizeof(long long), cudaMemcpyHostToDevice, s));
    // the bins of the sizing pass are still in place; restore their counts
    CK(cudaMemcpyAsync(h->ctl->bin_count, h->hctl->bin_count, sizeof(h->hctl->bin_count), cudaMemcpyHostToDevice, s));
    numeric_branches(h, s, c_job(h, h->wc.iota.p, true));
    read_ctl(h, s);
    check_debug(h->hctl);
    if (h->hctl->status & ST_TIMEOUT) throw Err(DSPG_ERR_TIMEOUT, overflow_message(h->hctl));
    if (h->hctl->status) throw Err(DSPG_ERR_CUDA, "static recompute failed with status " + std::to_string(h->hctl->status));
    if (h->bloom) bloom_build(h, s);
    h->epoch++;
}

// Transposed pattern of A (rows of A^T = columns of A), built from A's rows.
void build_transpose(dspg_handle *h, cudaStream_t s) {
    DevMat &A = h->A;
    DBuf<int64_t> rowptr;
    rowptr.reserve(A.nrows + 1);
    const int64_t nnz = mat_rowptr(h, A, nullptr, A.nrows, rowptr.p, s);
    DBuf<int32_t> col;
    col.reserve(nnz + 1);
    gather_rows_out(nullptr, A.nrows, A.view(), rowptr.p, col.p, nullptr, 0, s, h->num_sms);
    DBuf<uint64_t> k0, k1;
    DBuf<uint32_t> v0, v1, counts;
    DBuf<int64_t> scan_tmp, scan_out;
    k0.reserve(nnz + 1); k1.reserve(nnz + 1); v0.reserve(nnz + 1); v1.reserve(nnz + 1);
    int64_t cnt;
    sort_tmp_sizes(nnz, &cnt);
    counts.reserve(cnt);
    scan_out.reserve(cnt + 1);
    scan_tmp.reserve(scan_tmp_entries(cnt) + 1);
    keys_from_cols(col.p, nnz, k0.p, s);
    rows_of_entries(rowptr.p, A.nrows, v0.p, s, h->num_sms);
    bool alt = false;
    if (nnz > 0) radix_sort_pairs(k0.p, v0.p, k1.p, v1.p, nnz, bits_for(A.ncols), counts.p, scan_tmp.p, scan_out.p, s, &alt);
    DBuf<int32_t> tlen;
    tlen.reserve(std::max<int64_t>(A.ncols, 1));
    CK(cudaMemsetAsync(tlen.p, 0, sizeof(int32_t) * tlen.n, s));
    hist_cols(col.p, nnz, tlen.p, s);
    DBuf<int64_t> toff, tmp;
    toff.reserve(A.ncols + 1);
    tmp.reserve(scan_tmp_entries(A.ncols) + 1);
    scan_i32_to_i64(tlen.p, toff.p, A.ncols, tmp.p, s);
    make_slack(h, h->AT, A.ncols, A.nrows, 0, toff.p, tlen.p, (const int32_t *)(alt ? v1.p : v0.p), nullptr, s);
    h->has_at = true;
    h->epoch++;
}

// ------------------------------------------------------------ pipeline

void stage_sort(dspg_handle *h, cudaStream_t s) {
    if (h->inA.cap > 0)
        sort_updates(h->d_args + 0, h->inA.cap, h->A.nrows, h->A.ncols, h->sr, true, h->wA.sort_out(), h->wA.sort_tmp(),
                     h->ctl, 0u, s);
    if (!h->b_is_a && h->inB.cap > 0)
        sort_updates(h->d_args + 1, h->inB.cap, h->B.nrows, h->B.ncols, h->sr, true, h->wB.sort_out(), h->wB.sort_tmp(),
                     h->ctl, 0u, s);
}

DetectBufs detect_bufs(dspg_handle *h) {
    CWs &w = h->wc;
    return DetectBufs{w.bmR.p, w.bmK.p, w.R.p, w.K.p, &h->ctl->n_K};
}

// Classification of the sorted batches against the stored rows; it also
// marks the rows with an effective change, the first step of the
// affected-row detection (rows of the A batch are rows of C; rows of the B
// batch, or of the A batch when B is A, are rows of B* whose columns are
// followed next).
void stage_classify(dspg_handle *h, cudaStream_t s) {
    const DetectBufs D = detect_bufs(h);
    if (h->inA.cap > 0) {
        UpdJob J = h->wA.job(h->inA.cap);
        run_classify(J, h->A.view(), h->vsize, h->ctl, M_AB & ~ST_AB_STAGE, ST_AB_STAGE, D, true,
                     h->b_is_a && h->has_at, s, h->num_sms);
    }
    if (!h->b_is_a && h->inB.cap > 0) {
        UpdJob J = h->wB.job(h->inB.cap);
        run_classify(J, h->B.view(), h->vsize, h->ctl, M_AB & ~ST_AB_STAGE, ST_AB_STAGE, D, false, true, s,
                     h->num_sms);
    }
}

// Second step of the detection: rows i with A(i,k) != 0 for the marked
// rows k of B*, read from the transposed pattern of A.  It shares its launch
// with the merge copy of the matrix whose batch marked B* (B, or A when B
// is A); returns which (0: A, 1: B, -1: none).
int stage_detect(dspg_handle *h, cudaStream_t s) {
    const DetectBufs D = detect_bufs(h);
    const bool any_cols = h->has_at && (h->b_is_a ? h->inA.cap > 0 : h->inB.cap > 0);
    if (!any_cols) return -1;
    if (h->b_is_a) {
        run_detect_merge(h->AT.view(), D, h->wA.job(h->inA.cap), h->A.view(), h->vsize, h->ctl, M_AB, s, h->num_sms);
        return 0;
    }
    run_detect_merge(h->AT.view(), D, h->wB.job(h->inB.cap), h->B.view(), h->vsize, h->ctl, M_AB, s, h->num_sms);
    return 1;
}

// The merge copies not done with the detection.
void stage_merge(dspg_handle *h, cudaStream_t s, int merged) {
    if (h->inA.cap > 0 && merged != 0)
        run_merge_copy(h->wA.job(h->inA.cap), h->A.view(), h->vsize, h->ctl, M_AB, s, h->num_sms);
    if (!h->b_is_a && h->inB.cap > 0 && merged != 1)
        run_merge_copy(h->wB.job(h->inB.cap), h->B.view(), h->vsize, h->ctl, M_AB, s, h->num_sms);
}

void stage_commit_ab(dspg_handle *h, cudaStream_t s) {
    if (h->inA.cap > 0)
        run_commit(upd_commit_job(h, h->wA, ST_AB_ARENA, ST_AB_STAGE), h->A.view(), h->vsize, h->inA.cap, h->ctl,
                   M_AB & ~ST_AB_ARENA, M_AB, h->opt.slack_min, h->opt.slack_div, s, h->num_sms);
    if (!h->b_is_a && h->inB.cap > 0)
        run_commit(upd_commit_job(h, h->wB, ST_AB_ARENA, ST_AB_STAGE), h->B.view(), h->vsize, h->inB.cap, h->ctl,
                   M_AB & ~ST_AB_ARENA, M_AB, h->opt.slack_min, h->opt.slack_div, s, h->num_sms);
}

// Transposed pattern of A, first part: forward the structural changes of
// the A batch, sort them by (column, row) and rebuild the changed rows in
// staging.  These only read the transposed pattern.
void transpose_front(dspg_handle *h, cudaStream_t s) {
    const int64_t n = h->inA.cap;
    UpdWs &w = h->wAT;
    run_transpose_feed(h->wA.job(n), (int32_t)h->AT.nrows, w.in_row.p, w.in_col.p, w.in_op.p, h->ctl, M_AB, s);
    sort_updates(h->d_args + 2, n, h->AT.nrows + 1, h->AT.ncols, h->sr, false, w.sort_out(), w.sort_tmp(), h->ctl, M_AT,
                 s);
    UpdJob J = w.job(n);
    run_classify(J, h->AT.view(), 0, h->ctl, M_AT & ~ST_AT_STAGE, ST_AT_STAGE, DetectBufs{}, false, false, s,
                 h->num_sms);
    run_merge_copy(J, h->AT.view(), 0, h->ctl, M_AT, s, h->num_sms);
}

// Second part: write the rebuilt rows into the transposed pattern (only
// after the affected-row detection has finished reading it).
void transpose_commit(dspg_handle *h, cudaStream_t s) {
    run_commit(upd_commit_job(h, h->wAT, ST_AT_ARENA, ST_AT_STAGE), h->AT.view(), 0, h->inA.cap, h->ctl,
               M_AT & ~ST_AT_ARENA, M_AT, h->opt.slack_min, h->opt.slack_div, s, h->num_sms);
}

// Exact sizing of rows R (count of `n_max` rows at most): bins by the bound,
// a count_only pass writes each row's exact size into C.len, then the rows
// are binned again by that count for the numeric pass (whose job is returned).
CJob size_exact(dspg_handle *h, const int32_t *R, int64_t n_max, cudaStream_t s) {
    CJob J = c_job(h, R, false);
    J.sizing = SIZE_BOUND;
    run_size_bins(h->A.view(), h->Bm().view(), h->C.view(), J, n_max, h->ctl, M_AB, s, h->num_sms);
    CJob Jc = J;
    Jc.count_only = 1;
    numeric_branches(h, s, Jc);
    CK(cudaMemsetAsync(h->ctl->bin_count, 0, sizeof(h->ctl->bin_count), s));
    CK(cudaMemsetAsync(&h->ctl->nnz_written, 0, sizeof(long long), s));
    CJob J2 = J;
    J2.sizing = SIZE_COUNT;
    run_size_bins(h->A.view(), h->Bm().view(), h->C.view(), J2, n_max, h->ctl, M_AB, s, h->num_sms);
    return J2;
}

void stage_size(dspg_handle *h, cudaStream_t s) {
    if (h->sizing == DSPG_SIZE_EXACT) {
        size_exact(h, h->wc.R.p, h->A.nrows, s);
        return;
    }
    run_size_bins(h->A.view(), h->Bm().view(), h->C.view(), c_job(h, h->wc.R.p, false), h->A.nrows, h->ctl, M_AB, s,
                  h->num_sms);
}

void stage_numeric(dspg_handle *h, cudaStream_t s) { numeric_branches(h, s, c_job(h, h->wc.R.p, false)); }

void rec_event(cudaEvent_t e, cudaStream_t st, bool capturing) {
    if (capturing) CK(cudaEventRecordWithFlags(e, st, cudaEventRecordExternal));
    else CK(cudaEventRecord(e, st));
}

// The whole batch on stream s.  The transposed-pattern update runs on a side
// branch (its commit waits for the detection, which reads the old pattern);
// s waits for it at the end.  With `timed`, events mark the stage bounds.
void pipeline(dspg_handle *h, cudaStream_t s, bool timed, bool capturing) {
    auto mark = [&](int k, cudaStream_t st) {
        if (timed) rec_event(h->pev[k], st, capturing);
    };
    mark(0, s);
    stage_sort(h, s);
    mark(1, s);
    stage_classify(h, s);
    const bool side_on = h->has_at && h->inA.cap > 0;
    if (side_on) {
        CK(cudaEventRecord(h->evFork, s));
        CK(cudaStreamWaitEvent(h->side, h->evFork, 0));
        mark(8, h->side);
        transpose_front(h, h->side);
    }
    mark(2, s);
    // when B is A: the detection's column step, A's merge copy and commit
    // plan share one launch, the collection of R and the commit copy the
    // next (the merge and commit stage times are then part of the detection's)
    const bool fused = h->b_is_a && h->has_at && h->inA.cap > 0;
    const int64_t words = (h->A.nrows + 31) / 32;
    const CommitJob cjA = upd_commit_job(h, h->wA, ST_AB_ARENA, ST_AB_STAGE);
    int merged = -1;
    if (fused)
        run_detect_merge_plan(h->AT.view(), detect_bufs(h), h->wA.job(h->inA.cap), h->A.view(), cjA, h->vsize, h->ctl,
                              M_AB & ~ST_AB_ARENA, h->opt.slack_min, h->opt.slack_div, h->inA.cap, s, h->num_sms);
    else
        merged = stage_detect(h, s);
    if (side_on) {
        CK(cudaEventRecord(h->evDetect, s));
        CK(cudaStreamWaitEvent(h->side, h->evDetect, 0));
        transpose_commit(h, h->side);
        mark(9, h->side);
        CK(cudaEventRecord(h->evSide, h->side));
    }
    if (fused) {
        // R from the detection's bitmap, in row order within each block's range
        run_collect_copy(h->wc.bmR.p, words, h->wc.R.p, h->wc.rchunk.p, cjA, h->A.view(), h->vsize, h->ctl,
                         M_AB & ~ST_AB_ARENA, M_AB, s, h->num_sms);
        mark(3, s);
        mark(4, s);
    } else {
        run_collect_rows(h->wc.bmR.p, words, h->wc.R.p, h->wc.rchunk.p, h->ctl, M_AB, s, h->num_sms);
        mark(3, s);
        stage_merge(h, s, merged);
        mark(4, s);
        stage_commit_ab(h, s);
    }
    mark(5, s);
    stage_size(h, s);
    mark(6, s);
    stage_numeric(h, s);
    mark(7, s);
    if (side_on) CK(cudaStreamWaitEvent(s, h->evSide, 0));
}

void stage_times_from_events(dspg_handle *h) {
    const int a[DSPG_NSTAGES] = {0, 1, 2, 3, 4, 8, 5, 6};
    const int b[DSPG_NSTAGES] = {1, 2, 3, 4, 5, 9, 6, 7};
    const bool side_on = h->has_at && h->inA.cap > 0;
    for (int k = 0; k < DSPG_NSTAGES; k++) {
        h->stage_ms[k] = 0.f;
        if (k == DSPG_STAGE_TRANSPOSE && !side_on) continue;
        CK(cudaEventElapsedTime(&h->stage_ms[k], h->pev[a[k]], h->pev[b[k]]));
    }
}

void reset_range(dspg_handle *h, void *first, size_t bytes, cudaStream_t s) {
    CK(cudaMemsetAsync(first, 0, bytes, s));
}

void reset_c_counters(dspg_handle *h, cudaStream_t s) {
    Ctl *c = h->ctl;
    char *from = (char *)&c->c_stage_top;
    reset_range(h, from, sizeof(Ctl) - (size_t)(from - (char *)c), s);
}

// Host batches are copied to the device; device batches are read where
// they are.  Either way the pointers go to the argument block slot k.
// A transposed operand takes the caller's (i, j) as (j, i): the row and
// column arrays trade places (swap).
void upload(dspg_handle *h, UpdWs &w, const dspg_updates *u, BatchIn &in, int k, cudaStream_t s, bool swap = false) {
    in.n = u ? u->n : 0;
    in.cap = batch_bucket(in.n);
    h->h_args[k] = InArgs{nullptr, nullptr, nullptr, nullptr, 0};
    if (in.n <= 0) return;
    const int32_t *ur = swap ? u->col : u->row, *uc = swap ? u->row : u->col;
    if (u->on_device) {
        in.row = ur;
        in.col = uc;
        in.val = u->val;
        in.op = u->op;
    } else {
        CK(cudaMemcpyAsync(w.in_row.p, ur, sizeof(int32_t) * in.n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(w.in_col.p, uc, sizeof(int32_t) * in.n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(w.in_val.p, u->val, (size_t)h->vsize * in.n, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(w.in_op.p, u->op, sizeof(uint8_t) * in.n, cudaMemcpyHostToDevice, s));
        in.row = w.in_row.p;
        in.col = w.in_col.p;
        in.val = w.in_val.p;
        in.op = w.in_op.p;
    }
    h->h_args[k] = InArgs{in.row, in.col, in.val, in.op, in.n};
}

// Runs the pipeline once and reads the status.  A batch shape (sizes of the
// A and B batches) seen before with unchanged buffers runs as a captured
// CUDA graph on the handle's own stream (ordered after s); the first time a
// shape is seen it runs eagerly on s, the second time it is captured.
// With sync false the call returns once the work is enqueued (s is ordered
// after it); the control block reaches h->hctl when s completes.
void run_first(dspg_handle *h, cudaStream_t s, bool sync = true) {
    // a captured pipeline serves every batch of the same launch sizes
    const int64_t nA = h->inA.cap, nB = h->inB.cap;
    if (h->use_graphs) {
        for (auto &g : h->graphs) {
            if (g.nA == nA && g.nB == nB && g.epoch == h->epoch && g.prof == h->prof) {
                CK(cudaEventRecord(h->evIn, s));
                CK(cudaStreamWaitEvent(h->gs, h->evIn, 0));
                CK(cudaGraphLaunch(g.exec, h->gs));
                __atomic_fetch_add(&launch_counter(), g.kernels, __ATOMIC_RELAXED);
                h->runs_replayed++;
                CK(cudaEventRecord(h->evIn, h->gs));
                CK(cudaStreamWaitEvent(s, h->evIn, 0));
                if (sync) CK(cudaStreamSynchronize(h->gs));
                return;
            }
        }
        bool seen = false;
        for (auto &g : h->seen) seen |= (g.nA == nA && g.nB == nB && g.epoch == h->epoch && g.prof == h->prof);
        if (seen) {
            cudaGraph_t graph = nullptr;
            CK(cudaEventRecord(h->evIn, s));
            CK(cudaStreamWaitEvent(h->gs, h->evIn, 0));
            const unsigned long long k0 = launch_counter();
            CK(cudaStreamBeginCapture(h->gs, cudaStreamCaptureModeThreadLocal));
            begin_batch(h->h_args_dev, h->d_args, h->ctl, h->gs);
            pipeline(h, h->gs, h->prof, true);
            end_batch(h->ctl, h->hctl_dev, h->gs);
            CK(cudaStreamEndCapture(h->gs, &graph));
            cudaGraphExec_t exec = nullptr;
            const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            CK(e);
            if (h->graphs.size() >= 8) {
                cudaGraphExecDestroy(h->graphs.front().exec);
                h->graphs.erase(h->graphs.begin());
            }
            const unsigned long long nk = launch_counter() - k0;
            h->graphs.push_back(dspg_handle::Graph{nA, nB, h->epoch, h->prof, exec, nk});
            h->runs_captured++;
            CK(cudaGraphLaunch(exec, h->gs));
            CK(cudaEventRecord(h->evIn, h->gs));
            CK(cudaStreamWaitEvent(s, h->evIn, 0));
            if (sync) CK(cudaStreamSynchronize(h->gs));
            return;
        }
        if (h->seen.size() >= 16) h->seen.erase(h->seen.begin());
        h->seen.push_back(dspg_handle::Graph{nA, nB, h->epoch, h->prof, nullptr, 0});
    }
    h->runs_eager++;
    begin_batch(h->h_args_dev, h->d_args, h->ctl, s);
    pipeline(h, s, h->prof, false);
    CK(cudaGetLastError());
    if (sync) read_ctl(h, s);
    else CK(cudaMemcpyAsync(h->hctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
}

dspg_status fail(dspg_handle *h, const Err &e) {
    if (h) h->err = e.what();
    else g_err = e.what();
    return e.st;
}

void check_csr_arg(const dspg_csr *m, const char *name) {
    if (!m) throw Err(DSPG_ERR_INVALID, std::string(name) + " is NULL");
    if (m->nrows < 0 || m->ncols < 0 || m->nnz < 0) throw Err(DSPG_ERR_INVALID, std::string(name) + ": negative size");
    if (m->nrows >= INT32_MAX || m->ncols >= INT32_MAX) throw Err(DSPG_ERR_INVALID, std::string(name) + ": too many rows or columns");
    if (!m->rowptr || (m->nnz > 0 && (!m->col || !m->val))) throw Err(DSPG_ERR_INVALID, std::string(name) + ": NULL array");
}

// Device copy of an input CSR, validated.  Fills rowptr/col/val device buffers.
void load_csr(dspg_handle *h, const dspg_csr *m, DBuf<int64_t> &rp, DBuf<int32_t> &col, DBuf<char> &val,
              const int64_t **rp_d, const int32_t **col_d, const void **val_d, cudaStream_t s) {
    if (m->on_device) {
        *rp_d = m->rowptr;
        *col_d = m->col;
        *val_d = m->val;
    } else {
        rp.reserve(m->nrows + 1);
        col.reserve(std::max<int64_t>(m->nnz, 1));
        val.reserve(std::max<int64_t>(m->nnz, 1) * h->vsize);
        CK(cudaMemcpyAsync(rp.p, m->rowptr, sizeof(int64_t) * (m->nrows + 1), cudaMemcpyHostToDevice, s));
        if (m->nnz > 0) {
            CK(cudaMemcpyAsync(col.p, m->col, sizeof(int32_t) * m->nnz, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(val.p, m->val, (size_t)h->vsize * m->nnz, cudaMemcpyHostToDevice, s));
        }
        *rp_d = rp.p;
        *col_d = col.p;
        *val_d = val.p;
    }
    DBuf<unsigned> bad;
    bad.reserve(1);
    CK(cudaMemsetAsync(bad.p, 0, sizeof(unsigned), s));
    validate_rowptr(m->nrows, m->nnz, *rp_d, bad.p, s);
    unsigned hb = 0;
    CK(cudaMemcpyAsync(&hb, bad.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hb) throw Err(DSPG_ERR_INVALID, "row pointers are not a valid CSR");
    validate_csr_entries(m->nrows, m->ncols, *rp_d, *col_d, *val_d, h->sr, bad.p, s);
    CK(cudaMemcpyAsync(&hb, bad.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hb) throw Err(DSPG_ERR_INVALID, "columns out of range, not strictly ascending, or invalid values");
}

void init_slack_from_csr(dspg_handle *h, DevMat &M, const dspg_csr *m, cudaStream_t s) {
    DBuf<int64_t> rp;
    DBuf<int32_t> col;
    DBuf<char> val;
    const int64_t *rp_d;
    const int32_t *col_d;
    const void *val_d;
    load_csr(h, m, rp, col, val, &rp_d, &col_d, &val_d, s);
    DBuf<int32_t> len;
    len.reserve(std::max<int64_t>(m->nrows, 1));
    lens_from_rowptr(rp_d, len.p, m->nrows, s);
    make_slack(h, M, m->nrows, m->ncols, h->vsize, rp_d, len.p, col_d, val_d, s);
}

// Transpose of a canonical CSR on the device (nrows x ncols, nnz entries):
// the entries are sorted by column with a stable radix sort of their
// indices, which keeps each column's rows ascending, then gathered with
// their row and value.  Outputs: trp (ncols + 1 row pointers), tlen (ncols
// row lengths), tcol, tval.
void transpose_device(dspg_handle *h, int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *rp, const int32_t *col,
                      const void *val, int vsize, DBuf<int64_t> &trp, DBuf<int32_t> &tlen, DBuf<int32_t> &tcol,
                      DBuf<char> &tval, cudaStream_t s) {
    trp.reserve(ncols + 1);
    tlen.reserve(std::max<int64_t>(ncols, 1));
    tcol.reserve(std::max<int64_t>(nnz, 1));
    tval.reserve(std::max<int64_t>(nnz, 1) * std::max(vsize, 1));
    CK(cudaMemsetAsync(tlen.p, 0, sizeof(int32_t) * tlen.n, s));
    if (nnz > 0) {
        if (nnz >= (int64_t(1) << 32)) throw Err(DSPG_ERR_INVALID, "too many entries to transpose");
        DBuf<uint64_t> k0, k1;
        DBuf<uint32_t> i0, i1, counts, row_of;
        DBuf<int64_t> scan_tmp, scan_out;
        k0.reserve(nnz); k1.reserve(nnz); i0.reserve(nnz); i1.reserve(nnz); row_of.reserve(nnz);
        int64_t cnt;
        sort_tmp_sizes(nnz, &cnt);
        counts.reserve(cnt);
        scan_out.reserve(cnt + 1);
        scan_tmp.reserve(scan_tmp_entries(cnt) + 1);
        keys_from_cols(col, nnz, k0.p, s);
        fill_iota((int32_t *)i0.p, nnz, s);
        bool alt = false;
        radix_sort_pairs(k0.p, i0.p, k1.p, i1.p, nnz, bits_for(std::max<int64_t>(ncols, 2)), counts.p, scan_tmp.p,
                         scan_out.p, s, &alt);
        rows_of_entries(rp, nrows, row_of.p, s, h->num_sms);
        permute_entries(alt ? i1.p : i0.p, row_of.p, val, nnz, tcol.p, vsize ? (void *)tval.p : nullptr, vsize, s,
                        h->num_sms);
        hist_cols(col, nnz, tlen.p, s);
    }
    DBuf<int64_t> tmp;
    tmp.reserve(scan_tmp_entries(ncols) + 1);
    scan_i32_to_i64(tlen.p, trp.p, ncols, tmp.p, s);
    CK(cudaStreamSynchronize(s));  // the temporaries are freed on return
}

// An operand of the product from the caller's CSR: as given, or stored
// transposed when the product uses its transpose.
void load_operand(dspg_handle *h, DevMat &M, const dspg_csr *m, bool trans, cudaStream_t s) {
    if (!trans) {
        init_slack_from_csr(h, M, m, s);
        return;
    }
    DBuf<int64_t> rp;
    DBuf<int32_t> col;
    DBuf<char> val;
    const int64_t *rp_d;
    const int32_t *col_d;
    const void *val_d;
    load_csr(h, m, rp, col, val, &rp_d, &col_d, &val_d, s);
    DBuf<int64_t> trp;
    DBuf<int32_t> tlen, tcol;
    DBuf<char> tval;
    transpose_device(h, m->nrows, m->ncols, m->nnz, rp_d, col_d, val_d, h->vsize, trp, tlen, tcol, tval, s);
    make_slack(h, M, m->ncols, m->nrows, h->vsize, trp.p, tlen.p, tcol.p, tval.p, s);
}

// The fill of a read: rows (device, n of them; NULL = all) of M whose
// row pointers rp (device, n + 1) and total nnz are known, gathered, sorted
// by column and copied out (V, vs: the view and value size read).
// The device address of page-locked host memory the GPU can reach (over the
// C2C link on this system), or null for any other pointer.
void *device_view(void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The listed rows (lh: indices into the row list, rph: its row pointers on
// the host) of oc/ov, sorted by column on the device with the LSD radix sort,
// in groups of at most 2^28 entries (the radix sort's indices are 32-bit).
void sort_listed_host(dspg_handle *h, const DevMat &M, const int64_t *rp, const std::vector<int64_t> &lh,
                      const int64_t *rph, int32_t *oc, void *ov, int vs, cudaStream_t s) {
    const size_t nl = lh.size();
    std::vector<int64_t> lo(nl), hi(nl);
    for (size_t k = 0; k < nl; k++) {
        lo[k] = rph[lh[k]];
        hi[k] = rph[lh[k] + 1];
    }
    const int cb = bits_for(std::max<int64_t>(M.ncols, 2));
    size_t k0 = 0;
    while (k0 < nl) {
        std::vector<int64_t> pre(1, 0);
        size_t k1 = k0;
        while (k1 < nl && (k1 == k0 || pre.back() + (hi[k1] - lo[k1]) <= (int64_t(1) << 28))) {
            pre.push_back(pre.back() + (hi[k1] - lo[k1]));
            k1++;
        }
        const int nk = (int)(k1 - k0);
        const int64_t total = pre.back();
        DBuf<int64_t> d_pre, d_list, scan_tmp, scan_out;
        DBuf<uint64_t> kk0, kk1;
        DBuf<uint32_t> ii0, ii1, counts;
        DBuf<int32_t> tcol;
        DBuf<char> tval;
        d_pre.reserve(nk + 1);
        d_list.reserve(nk);
        kk0.reserve(total); kk1.reserve(total); ii0.reserve(total); ii1.reserve(total);
        int64_t cnt;
        sort_tmp_sizes(total, &cnt);
        counts.reserve(cnt);
        scan_out.reserve(cnt + 1);
        scan_tmp.reserve(scan_tmp_entries(cnt) + 1);
        tcol.reserve(total);
        tval.reserve(total * std::max(vs, 1));
        CK(cudaMemcpyAsync(d_pre.p, pre.data(), sizeof(int64_t) * (nk + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_list.p, lh.data() + k0, sizeof(int64_t) * nk, cudaMemcpyHostToDevice, s));
        SortScratch w{kk0.p, kk1.p, ii0.p, ii1.p, counts.p, scan_tmp.p, scan_out.p, tcol.p, (void *)tval.p};
        sort_listed_rows(rp, d_list.p, d_pre.p, nk, total, cb, oc, ov, vs, w, s, h->num_sms);
        CK(cudaStreamSynchronize(s));
        k0 = k1;
    }
}

void fill_rows_out(dspg_handle *h, DevMat &M, const MatView &V, int vs, const int32_t *rows, int64_t n, int64_t *rp,
                   int64_t nnz, int64_t *rowptr, int32_t *col, void *val, int on_device, cudaStream_t s) {
    // rows too long to sort in shared memory are listed, then sorted together
    const int64_t list_cap = nnz / 16385 + 1;
    DBuf<int64_t> listed_l;
    h->rd.n_listed.reserve(1);
    unsigned *n_listed = h->rd.n_listed.p;
    int64_t *listed = read_scratch(h->rd.listed, listed_l, list_cap);
    CK(cudaMemsetAsync(n_listed, 0, sizeof(unsigned), s));
    auto sort_out = [&](int32_t *oc, void *ov) {
        sort_rows(rp, n, oc, ov, vs, n_listed, listed, list_cap, s, h->num_sms);
        unsigned nl = 0;
        CK(cudaMemcpyAsync(&nl, n_listed, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (nl == 0) return;
        if ((int64_t)nl > list_cap) throw Err(DSPG_ERR_CUDA, "more long rows than the read can hold");
        std::vector<int64_t> lh(nl), rph(n + 1);
        CK(cudaMemcpyAsync(lh.data(), listed, sizeof(int64_t) * nl, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(rph.data(), rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        sort_listed_host(h, M, rp, lh, rph.data(), oc, ov, vs, s);
    };
    if (on_device) {
        CK(cudaMemcpyAsync(rowptr, rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
        gather_rows_out(rows, n, V, rp, col, val, vs, s, h->num_sms);
        sort_out(col, val);
    } else {
        DBuf<int32_t> c_l;
        DBuf<char> v_l;
        int32_t *c = read_scratch(h->rd.c, c_l, nnz);
        char *v = read_scratch(h->rd.v, v_l, nnz * std::max(vs, 1));
        gather_rows_out(rows, n, V, rp, c, v, vs, s, h->num_sms);
        sort_out(c, vs ? (void *)v : nullptr);
        CK(cudaMemcpyAsync(rowptr, rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
        if (nnz > 0) {
            if (col) CK(cudaMemcpyAsync(col, c, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, s));
            if (val) CK(cudaMemcpyAsync(val, v, (size_t)vs * nnz, cudaMemcpyDeviceToHost, s));
        }
        CK(cudaStreamSynchronize(s));
    }
}

int64_t read_mat(dspg_handle *h, DevMat &M, const int32_t *rows_in, int64_t nr, int64_t *rowptr, int32_t *col,
                 void *val, int on_device, cudaStream_t s, bool bloom = false) {
    NvtxRange nr_("dspg/read");
    // with bloom the values read are C's Bloom words (8 bytes each) instead
    MatView V = M.view();
    int vs = M.vsize;
    if (bloom) {
        V.val = (void *)M.fb.p;
        vs = 8;
    }
    DBuf<int32_t> rows_l;
    const int32_t *rows = nullptr;
    int64_t n = M.nrows;
    if (rows_in) n = nr;
    // host rows of C that the last read of this generation of C listed too:
    // their row pointers are still in the kept buffer
    dspg_handle::ReadKey &key = h->rd_key;
    const bool keyed = rows_in && !on_device && &M == &h->C;
    const bool hit = keyed && key.valid && key.serial == h->c_serial && (int64_t)key.rows.size() == n &&
                     (n == 0 || std::memcmp(key.rows.data(), rows_in, sizeof(int32_t) * (size_t)n) == 0);
    key.valid = false;  // the kept row list and row pointers are rewritten below unless this is a hit
    DBuf<int64_t> rp_l;
    int64_t *rp;
    int64_t nnz;
    if (hit) {
        rows = h->rd.rows.p;
        rp = h->rd.rp.p;
        nnz = key.nnz;
    } else {
        if (rows_in) {
            if (on_device) rows = rows_in;
            else {
                int32_t *rows_d = read_scratch(h->rd.rows, rows_l, n);
                if (n > 0) CK(cudaMemcpyAsync(rows_d, rows_in, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
                rows = rows_d;
            }
        }
        rp = read_scratch(h->rd.rp, rp_l, n + 1);
        nnz = mat_rowptr(h, M, rows, n, rp, s);
    }
    if (keyed && rows == h->rd.rows.p && rp == h->rd.rp.p) {
        if (!hit) key.rows.assign(rows_in, rows_in + n);
        key.serial = h->c_serial;
        key.nnz = nnz;
        key.valid = true;
    }
    if (!rowptr) return nnz;
    fill_rows_out(h, M, V, vs, rows, n, rp, nnz, rowptr, col, val, on_device, s);
    return nnz;
}

// Rows of C = alpha P (+) beta X, where P = op(A) op(B) is what the handle
// keeps (all rows when rows_in is NULL): sized by form_count, then P's rows
// are read canonically into scratch and merged with X's rows.
int64_t read_form(dspg_handle *h, const int32_t *rows_in, int64_t nr, int64_t *rowptr, int32_t *col, void *val,
                  int on_device, cudaStream_t s) {
    const int64_t n = rows_in ? nr : h->C.nrows;
    DBuf<int32_t> rows_d;
    const int32_t *rows = nullptr;
    if (rows_in) {
        if (on_device) rows = rows_in;
        else {
            rows_d.reserve(std::max<int64_t>(n, 1));
            if (n > 0) CK(cudaMemcpyAsync(rows_d.p, rows_in, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
            rows = rows_d.p;
        }
    }
    DBuf<int64_t> cnt, orp, tmp;
    cnt.reserve(std::max<int64_t>(n, 1));
    orp.reserve(n + 1);
    tmp.reserve(scan_tmp_entries(n) + 1);
    const int64_t *xrp = h->has_x ? h->xrp.p : nullptr;
    DBuf<int64_t> zrp;  // no X: empty rows
    if (!xrp) {
        zrp.reserve(h->C.nrows + 1);
        CK(cudaMemsetAsync(zrp.p, 0, sizeof(int64_t) * (h->C.nrows + 1), s));
        xrp = zrp.p;
    }
    form_count(rows, n, h->C.view(), xrp, h->xcol.p, cnt.p, s, h->num_sms);
    scan_i64(cnt.p, orp.p, n, tmp.p, s);
    const int64_t nnz = read_i64(orp.p + n, s);
    if (!rowptr) return nnz;
    // P's rows, canonical, into scratch
    DBuf<int64_t> prp;
    DBuf<int32_t> pcol;
    DBuf<char> pval;
    prp.reserve(n + 1);
    const int64_t pn = read_mat(h, h->C, rows, rows ? n : 0, nullptr, nullptr, nullptr, 1, s);
    pcol.reserve(std::max<int64_t>(pn, 1));
    pval.reserve(std::max<int64_t>(pn, 1) * h->vsize);
    read_mat(h, h->C, rows, rows ? n : 0, prp.p, pcol.p, pval.p, 1, s);
    DBuf<int32_t> ocol_l;
    DBuf<char> oval_l;
    int32_t *ocol = col;
    void *oval = val;
    if (!on_device) {
        ocol_l.reserve(std::max<int64_t>(nnz, 1));
        oval_l.reserve(std::max<int64_t>(nnz, 1) * h->vsize);
        ocol = ocol_l.p;
        oval = oval_l.p;
    }
    form_merge(h->sr, rows, n, prp.p, pcol.p, pval.p, xrp, h->xcol.p, h->xval.p, orp.p, ocol, oval, h->fs, s,
               h->num_sms);
    if (on_device) {
        CK(cudaMemcpyAsync(rowptr, orp.p, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
    } else {
        CK(cudaMemcpyAsync(rowptr, orp.p, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
        if (nnz > 0) {
            if (col) CK(cudaMemcpyAsync(col, ocol, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, s));
            if (val) CK(cudaMemcpyAsync(val, oval, (size_t)h->vsize * nnz, cudaMemcpyDeviceToHost, s));
        }
    }
    CK(cudaStreamSynchronize(s));
    return nnz;
}

// A as the caller gave it (its stored transpose turned back when the
// product uses A^T).
int64_t read_operand_a(dspg_handle *h, int64_t *rowptr, int32_t *col, void *val, int on_device, cudaStream_t s) {
    if (!h->trans_a) return read_mat(h, h->A, nullptr, 0, rowptr, col, val, on_device, s);
    const int64_t nnz = read_mat(h, h->A, nullptr, 0, nullptr, nullptr, nullptr, 1, s);
    if (!rowptr) return nnz;
    DBuf<int64_t> srp;
    DBuf<int32_t> scol;
    DBuf<char> sval;
    srp.reserve(h->A.nrows + 1);
    scol.reserve(std::max<int64_t>(nnz, 1));
    sval.reserve(std::max<int64_t>(nnz, 1) * h->vsize);
    read_mat(h, h->A, nullptr, 0, srp.p, scol.p, sval.p, 1, s);
    DBuf<int64_t> trp;
    DBuf<int32_t> tlen, tcol;
    DBuf<char> tval;
    transpose_device(h, h->A.nrows, h->A.ncols, nnz, srp.p, scol.p, sval.p, h->vsize, trp, tlen, tcol, tval, s);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(rowptr, trp.p, sizeof(int64_t) * (h->A.ncols + 1), k, s));
    if (nnz > 0) {
        if (col) CK(cudaMemcpyAsync(col, tcol.p, sizeof(int32_t) * nnz, k, s));
        if (val) CK(cudaMemcpyAsync(val, tval.p, (size_t)h->vsize * nnz, k, s));
    }
    CK(cudaStreamSynchronize(s));
    return nnz;
}

// Checks one batch pair and gets the handle's buffers and inputs ready.
void prepare_batch_impl(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB, cudaStream_t s);

// The host checks and the growth of the batch's buffers, before anything of
// A, B or C changes: a failure here leaves the handle as it was (buffers that
// moved before it bump the epoch, so no captured graph keeps their old places).
void prepare_batch(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB, cudaStream_t s) {
    try {
        if (fault_fires(faults().validate_at, faults().validate_seen))
            throw Err(DSPG_ERR_INVALID, "batch check failed (injected fault)");
        prepare_batch_impl(h, dA, dB, s);
    } catch (...) {
        h->epoch++;
        throw;
    }
}

void prepare_batch_impl(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB, cudaStream_t s) {
    h->c_serial++;
    h->extra_slots = 0;
    if ((h->b_is_a || h->b_alias) && dB && dB->n > 0) throw Err(DSPG_ERR_INVALID, "B is A: pass the batch as dA only");
    if (h->b_alias) dB = dA;  // the caller's B is A: its stored copy takes the same batch
    const int64_t nA = dA ? dA->n : 0, nB = dB ? dB->n : 0;
    if (nA < 0 || nB < 0) throw Err(DSPG_ERR_INVALID, "negative batch size");
    if (nA > INT32_MAX / 2 || nB > INT32_MAX / 2) throw Err(DSPG_ERR_INVALID, "batch too large");
    if (nA > 0 && (!dA->row || !dA->col || !dA->val || !dA->op)) throw Err(DSPG_ERR_INVALID, "NULL array in dA");
    if (nB > 0 && (!dB->row || !dB->col || !dB->val || !dB->op)) throw Err(DSPG_ERR_INVALID, "NULL array in dB");
    if (!h->b_is_a && nB > 0 && !h->has_at) build_transpose(h, s);
    ensure_c_ws(h, s);
    if (h->wA.ensure(batch_bucket(nA), h->A.arena_cap)) h->epoch++;
    if (!h->b_is_a && h->wB.ensure(batch_bucket(nB), h->B.arena_cap)) h->epoch++;
    if (h->has_at && h->wAT.ensure(batch_bucket(nA), h->AT.arena_cap)) h->epoch++;
    upload(h, h->wA, dA, h->inA, 0, s, h->trans_a);
    upload(h, h->wB, dB, h->inB, 1, s, h->trans_b);
    if (h->b_is_a) {
        h->inB = BatchIn{};
        h->h_args[1] = InArgs{nullptr, nullptr, nullptr, nullptr, 0};
    }
    h->h_args[2] = InArgs{h->wAT.in_row.p, h->wAT.in_col.p, nullptr, h->wAT.in_op.p, h->inA.n};
}

// After a run: grow what overflowed and re-run the failed stages (eagerly,
// on s) until the status is clean; errors become exceptions.
void recover(dspg_handle *h, cudaStream_t s) {
    const int64_t nA = h->inA.cap, nB = h->inB.cap;  // the stages that ran
    for (int iter = 0; iter < 8 && h->hctl->status; iter++) {
        const unsigned st = h->hctl->status;
        check_debug(h->hctl);
        if (st & ST_INVALID) throw Err(DSPG_ERR_INVALID, "batch entry out of range or with an invalid value/op");
        if (st & ST_TIMEOUT) throw Err(DSPG_ERR_TIMEOUT, overflow_message(h->hctl));
        if (st & ST_AB_STAGE) {
            if (h->wA.grow_stage(h->hctl->u[0].stage_top + 1024)) h->epoch++;
            if (h->wB.grow_stage(h->hctl->u[1].stage_top + 1024)) h->epoch++;
            CK(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), s));
            // the failed classification marked rows for the detection
            CK(cudaMemsetAsync(h->wc.bmR.p, 0, sizeof(uint32_t) * h->wc.bmR.n, s));
            CK(cudaMemsetAsync(h->wc.bmK.p, 0, sizeof(uint32_t) * h->wc.bmK.n, s));
            pipeline(h, s, false, false);
            read_ctl(h, s);
            continue;
        }
        const bool side_on = h->has_at && nA > 0;
        if (st & ST_AB_ARENA) {
            regrow(h, h->A, s);
            if (!h->b_is_a && nB > 0) regrow(h, h->B, s);
            for (int k = 0; k < 2; k++) {
                reset_range(h, &h->ctl->u[k].n_cchunk, sizeof(long long), s);
                reset_range(h, &h->ctl->u[k].reloc, sizeof(long long), s);
            }
            reset_range(h, &h->ctl->u[2], sizeof(UpdCtl), s);
            reset_c_counters(h, s);
            reset_range(h, &h->ctl->status, sizeof(unsigned), s);
            stage_commit_ab(h, s);
            if (side_on) {
                transpose_front(h, s);
                transpose_commit(h, s);
            }
            stage_size(h, s);
            stage_numeric(h, s);
            read_ctl(h, s);
            continue;
        }
        const bool at = side_on && (st & (ST_AT_STAGE | ST_AT_ARENA));
        const bool cc = st & ST_C_ARENA;
        if ((st & ST_AT_STAGE) && h->wAT.grow_stage(h->hctl->u[2].stage_top + 1024)) h->epoch++;
        if (st & ST_AT_ARENA) regrow(h, h->AT, s);
        if (st & ST_C_ARENA) regrow(h, h->C, s);
        reset_range(h, &h->ctl->status, sizeof(unsigned), s);
        if (at) {
            reset_range(h, &h->ctl->u[2], sizeof(UpdCtl), s);
            transpose_front(h, s);
            transpose_commit(h, s);
        }
        if (cc) {
            reset_c_counters(h, s);
            stage_size(h, s);
            stage_numeric(h, s);
        }
        read_ctl(h, s);
    }
    if (h->hctl->status) throw Err(DSPG_ERR_CUDA, "apply_batch did not converge, status " + std::to_string(h->hctl->status));
}

// After a row-path batch: which bins the recompute launches from now on.
// After the first batch that bins rows, only the bins it used (and the
// global dense bin, which takes rows of any size); later, also every bin
// whose rows a batch sent to the global dense bin instead.  A captured
// pipeline is right under any mask (its sizing pass and its launches share
// the mask it was captured with), so the narrowing keeps the captured
// pipelines (later captures take the narrower mask); turning a bin on bumps
// the epoch, so that the next batch is captured anew with it.  The mask
// only grows after the narrowing, so a handle is captured anew at most once
// per bin.
void learn_bins(dspg_handle *h) {
    if (!h->gate_bins || h->bloom) return;
    const Ctl &c = *h->hctl;
    bool any = c.bins_wanted != 0;
    for (int b = 0; b < NBINS; b++) any |= c.bin_count[b] > 0;
    if (!any) return;  // nothing was binned (no affected rows, or the delta path)
    const unsigned long long next = next_bin_mask(c, h->bin_on, h->bins_narrowed);
    const bool widened = h->bins_narrowed && next != h->bin_on;
    h->bins_narrowed = true;
    h->bin_on = next;
    if (widened) h->epoch++;
}

// Every bin on again (the thresholds or the sizing changed which bins rows
// take), and the next batch narrows them anew.
void reset_bins(dspg_handle *h) {
    h->bin_on = ~0ull;
    h->bins_narrowed = false;
    h->epoch++;
}

void fill_stats(dspg_handle *h, dspg_batch_stats *stats, int64_t compactions0) {
    const int64_t nA = h->inA.n, nB = h->inB.n;
    learn_bins(h);
    h->last_nR = h->hctl->n_affected;
    if (!h->bloom) h->last_masked = 0;
    if (stats) {
        const Ctl &c = *h->hctl;
        std::memset(stats, 0, sizeof(*stats));
        stats->n_updates = nA + nB;
        for (int k = 0; k < 2; k++) {
            stats->n_insert += c.u[k].ins;
            stats->n_update += c.u[k].upd;
            stats->n_delete += c.u[k].del;
            stats->n_noop += c.u[k].nop;
            stats->touched_rows += c.u[k].n_merge;
            stats->relocations += c.u[k].reloc;
        }
        stats->n_unique = stats->n_insert + stats->n_update + stats->n_delete + stats->n_noop;
        stats->relocations += c.u[2].reloc + c.c_reloc;
        stats->affected_rows = c.n_affected;
        stats->products = c.products;
        stats->nnz_written = c.nnz_written;
        stats->compactions = h->compactions - compactions0;
        stats->a_entries = c.a_entries;
        stats->est_rows = c.n_est;
        stats->est_overflows = c.n_ovf;
        const int64_t m = h->Bm().ncols;
        for (int b = 0; b < NBINS; b++) stats->table_slots += c.bin_count[b] * bin_table_slots(b, m);
        stats->table_slots += h->extra_slots;
        stats->masked_entries = h->last_masked;
    }
}

void trace_batch(const dspg_handle *h, const dspg_batch_stats &st, const char *path_kind) {
    const char *path = getenv("DSPG_TRACE");
    if (!path || !path[0]) return;
    FILE *f = fopen(path, "a");
    if (!f) return;  // tracing never fails a batch
    static const char *stage_names[DSPG_NSTAGES] = {"sort", "classify", "detect", "merge",
                                                    "commit", "transpose", "size", "numeric"};
    fprintf(f,
            "{\"handle\": \"%p\", \"path\": \"%s\", \"n_updates\": %lld, \"n_unique\": %lld, \"n_insert\": %lld, "
            "\"n_update\": %lld, \"n_delete\": %lld, \"n_noop\": %lld, \"touched_rows\": %lld, \"affected_rows\": %lld, "
            "\"products\": %lld, \"nnz_written\": %lld, \"relocations\": %lld, \"compactions\": %lld, "
            "\"a_entries\": %lld, \"est_rows\": %lld, \"est_overflows\": %lld, \"table_slots\": %lld, "
            "\"masked_entries\": %lld",
            (const void *)h, path_kind, (long long)st.n_updates, (long long)st.n_unique, (long long)st.n_insert,
            (long long)st.n_update, (long long)st.n_delete, (long long)st.n_noop, (long long)st.touched_rows,
            (long long)st.affected_rows, (long long)st.products, (long long)st.nnz_written,
            (long long)st.relocations, (long long)st.compactions, (long long)st.a_entries, (long long)st.est_rows,
            (long long)st.est_overflows, (long long)st.table_slots, (long long)st.masked_entries);
    if (h->prof && !h->bloom) {
        fprintf(f, ", \"stage_ms\": {");
        for (int k = 0; k < DSPG_NSTAGES; k++) fprintf(f, "%s\"%s\": %.5f", k ? ", " : "", stage_names[k], h->stage_ms[k]);
        fprintf(f, "}");
    }
    fprintf(f, "}\n");
    fclose(f);
}


// Rows whose learned table overflowed were left as they were; they are
// counted exactly and recomputed here (eagerly; only when there are any).
// The statistics of the main pass are kept.
void est_fallback(dspg_handle *h, cudaStream_t s) {
    const long long n_ovf = h->hctl->n_ovf;
    if (n_ovf <= 0) return;
    const Ctl main = *h->hctl;
    for (int iter = 0;; iter++) {
        CK(cudaMemsetAsync(&h->ctl->status, 0, sizeof(unsigned), s));
        reset_c_counters(h, s);
        CK(cudaMemcpyAsync(&h->ctl->n_affected, &main.n_ovf, sizeof(long long), cudaMemcpyHostToDevice, s));
        numeric_branches(h, s, size_exact(h, h->wc.ovf.p, n_ovf, s));
        read_ctl(h, s);
        if ((h->hctl->status & ST_C_ARENA) && iter < 4) {
            regrow(h, h->C, s);
            continue;
        }
        if (h->hctl->status) throw Err(DSPG_ERR_CUDA, "overflow recompute failed, status " + std::to_string(h->hctl->status));
        break;
    }
    CK(cudaMemcpyAsync(&h->ctl->n_affected, &main.n_affected, sizeof(long long), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    const long long reloc = h->hctl->c_reloc;
    // the overflow rows' second tables count too (the estimator's cost)
    for (int b = 0; b < NBINS; b++) h->extra_slots += h->hctl->bin_count[b] * bin_table_slots(b, h->Bm().ncols);
    *h->hctl = main;
    h->hctl->c_reloc += reloc;
}

// One batch on one handle, as dspg_apply_batch (errors as exceptions).
void masked_apply(dspg_handle *h, cudaStream_t s);

void apply_one(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB, dspg_batch_stats *stats,
               cudaStream_t s) {
    NvtxRange r(h->bloom ? "dspg/apply_batch (Algorithm 2)" : "dspg/apply_batch");
    dspg_batch_stats local;
    if (!stats) stats = &local;
    prepare_batch(h, dA, dB, s);
    const int64_t compactions0 = h->compactions;
    try {
        if (h->bloom) {
            masked_apply(h, s);
            fill_stats(h, stats, compactions0);
            trace_batch(h, *stats, "masked");
            return;
        }
        run_first(h, s);
        if (h->prof) stage_times_from_events(h);
        recover(h, s);
        est_fallback(h, s);
        fill_stats(h, stats, compactions0);
        trace_batch(h, *stats, "rows");
    } catch (const Err &e) {
        // an invalid batch is found before anything changes (every stage
        // after the check skips on its status bit); any other failure may
        // have left A', B' and C part-way
        if (e.st != DSPG_ERR_INVALID) h->broken = true;
        throw;
    }
}

// Calls on a handle whose earlier batch failed part-way are refused.
void check_usable(const dspg_handle *h) {
    if (h->broken)
        throw Err(DSPG_ERR_STATE, "an earlier batch failed part-way; the handle's matrices are undefined: rebuild it");
}

// ------------------------------------------------- the delta path (Eq. 1)

// Size and recompute the rows of R (ctl->n_affected of them) by the row
// path, growing C's arena until they fit (rows of the delta path that are
// too long to search, or every touched row when the new-entry list was full).
void alg_recompute_rows(dspg_handle *h, cudaStream_t s) {
    for (int iter = 0;; iter++) {
        stage_size(h, s);
        stage_numeric(h, s);
        read_ctl(h, s);
        const unsigned st = h->hctl->status & ~ST_ALG_FULL;
        if ((st & ST_C_ARENA) && iter < 4) {
            regrow(h, h->C, s);
            CK(cudaMemsetAsync(h->ctl->bin_count, 0, sizeof(h->ctl->bin_count), s));
            CK(cudaMemsetAsync(&h->ctl->status, 0, sizeof(unsigned), s));
            continue;
        }
        if (st & ST_TIMEOUT) throw Err(DSPG_ERR_TIMEOUT, overflow_message(h->hctl));
        if (st) throw Err(DSPG_ERR_CUDA, "row recompute of the delta path failed, status " + std::to_string(st));
        return;
    }
}

// Collect a row bitmap into R (clearing it) with n_affected starting at 0.
void alg_collect(dspg_handle *h, uint32_t *bm, cudaStream_t s) {
    CK(cudaMemsetAsync(&h->ctl->n_affected, 0, sizeof(long long), s));
    CK(cudaMemsetAsync(h->ctl->bin_count, 0, sizeof(h->ctl->bin_count), s));
    run_collect_rows(bm, (h->A.nrows + 31) / 32, h->wc.R.p, h->wc.rchunk.p, h->ctl, 0u, s, h->num_sms);
}

// One batch by Eq. 1 when every effective change of it inserts an absent
// entry (Section 5, algebraic updates): returns false, having changed
// nothing, for any other batch (a write to a present entry or a delete),
// which the caller then applies by the row path.  Runs eagerly on s and
// reads the control block between its steps.
bool apply_algebraic(dspg_handle *h, cudaStream_t s) {
    NvtxRange r("dspg/apply_batch_algebraic");
    const int64_t nA = h->inA.n, nB = h->b_is_a ? 0 : h->inB.n;
    begin_batch(h->h_args_dev, h->d_args, h->ctl, s);
    stage_sort(h, s);
    if (nA > 0)
        run_classify(h->wA.job(nA), h->A.view(), h->vsize, h->ctl, M_AB & ~ST_AB_STAGE, ST_AB_STAGE, DetectBufs{},
                     false, false, s, h->num_sms);
    if (nB > 0)
        run_classify(h->wB.job(nB), h->B.view(), h->vsize, h->ctl, M_AB & ~ST_AB_STAGE, ST_AB_STAGE, DetectBufs{},
                     false, false, s, h->num_sms);
    CK(cudaGetLastError());
    read_ctl(h, s);
    {
        const Ctl &c = *h->hctl;
        if (c.status & ST_INVALID) throw Err(DSPG_ERR_INVALID, "batch entry out of range or with an invalid value/op");
        if (c.status || c.u[0].upd || c.u[0].del || c.u[1].upd || c.u[1].del) return false;
    }
    // A' (and B'): the merge and the commit of the row path
    stage_merge(h, s, -1);
    stage_commit_ab(h, s);
    // the contributions read the transposed pattern before this batch
    const int64_t need = std::max<int64_t>(int64_t(1) << 20, 64 * (nA + nB));
    if (h->alg.ensure(need, h->A.nrows, h->vsize, s)) h->epoch++;
    AlgJob J{};
    const UpdJob ja = h->wA.job(nA);
    const UpdJob jb = h->b_is_a ? ja : h->wB.job(nB);
    J.xr = ja.row; J.xc = ja.col; J.xv = ja.val; J.xk = ja.kind; J.xn = nA;
    J.yr = jb.row; J.yc = jb.col; J.yv = jb.val; J.yk = jb.kind; J.yn = h->b_is_a ? nA : nB;
    if (!h->has_at) J.yn = 0;  // no B batch reaches C without the pattern (B is never updated then)
    J.nr = h->alg.nr.p; J.nc = h->alg.nc.p; J.nv = h->alg.nv.p; J.nop = h->alg.nop.p; J.ncap = h->alg.ncap;
    J.bm_touch = h->wc.bmR.p;
    J.bm_long = h->alg.bm_long.p;
    const bool side_on = h->has_at && nA > 0;
    for (int iter = 0;; iter++) {
        run_alg_contrib(h->sr, J, h->A.view(), h->Bm().view(), h->AT.view(), h->C.view(), h->ctl, M_AB, s,
                        h->num_sms);
        if (side_on) {
            transpose_front(h, s);
            transpose_commit(h, s);
        }
        CK(cudaGetLastError());
        read_ctl(h, s);
        const unsigned st = h->hctl->status;
        if (!(st & ST_AB_ARENA) || iter >= 4) break;
        // A's arena ran out in the commit: nothing after it ran; grow it and
        // commit again (the staged rows are still in place)
        regrow(h, h->A, s);
        if (nB > 0) regrow(h, h->B, s);
        for (int k = 0; k < 2; k++) {
            reset_range(h, &h->ctl->u[k].n_cchunk, sizeof(long long), s);
            reset_range(h, &h->ctl->u[k].reloc, sizeof(long long), s);
        }
        reset_range(h, &h->ctl->u[2], sizeof(UpdCtl), s);
        reset_range(h, &h->ctl->status, sizeof(unsigned), s);
        stage_commit_ab(h, s);
    }
    // the transposed pattern's staging or arena: grow and redo its update
    for (int iter = 0; iter < 8 && (h->hctl->status & (ST_AT_STAGE | ST_AT_ARENA)); iter++) {
        const unsigned st = h->hctl->status;
        if ((st & ST_AT_STAGE) && h->wAT.grow_stage(h->hctl->u[2].stage_top + 1024)) h->epoch++;
        if (st & ST_AT_ARENA) regrow(h, h->AT, s);
        reset_range(h, &h->ctl->status, sizeof(unsigned), s);
        reset_range(h, &h->ctl->u[2], sizeof(UpdCtl), s);
        transpose_front(h, s);
        transpose_commit(h, s);
        read_ctl(h, s);
    }
    check_debug(h->hctl);
    if (h->hctl->status & ~ST_ALG_FULL)
        throw Err(DSPG_ERR_CUDA, "delta path update failed, status " + std::to_string(h->hctl->status));
    const long long n_new = h->hctl->alg_new, n_con = h->hctl->alg_contrib;
    const bool full = h->hctl->status & ST_ALG_FULL;
    CK(cudaMemsetAsync(&h->ctl->status, 0, sizeof(unsigned), s));
    long long long_rows = 0;
    if (full) {
        // too many new entries: every touched row is recomputed from A', B'
        // instead (exact whatever contributions it took)
        CK(cudaMemsetAsync(h->alg.bm_long.p, 0, sizeof(uint32_t) * h->alg.bm_long.n, s));
        alg_collect(h, h->wc.bmR.p, s);
        read_ctl(h, s);
        long_rows = h->hctl->n_affected;
        alg_recompute_rows(h, s);
    } else {
        if (n_new > 0) {
            const InArgs na{h->alg.nr.p, h->alg.nc.p, h->alg.nv.p, h->alg.nop.p, n_new};
            CK(cudaMemcpyAsync(h->alg.args.p, &na, sizeof(InArgs), cudaMemcpyHostToDevice, s));
            CK(cudaStreamSynchronize(s));  // na leaves scope
            sort_updates(h->alg.args.p, n_new, h->C.nrows, h->C.ncols, h->sr, false, h->alg.sort_out(),
                         h->alg.sort_tmp(), h->ctl, 0u, s);
            const AlgNew N{h->alg.srow.p, h->alg.scol.p, h->alg.sval.p, n_new, h->alg.dest.p, h->alg.cap.p};
            for (int iter = 0;; iter++) {
                run_alg_append(h->sr, N, h->C.view(), h->ctl, 0u, 0u, h->opt.slack_min, h->opt.slack_div, true, s,
                               h->num_sms);
                read_ctl(h, s);
                if (!(h->hctl->status & ST_C_ARENA) || iter >= 4) break;
                regrow(h, h->C, s);  // the plan wrote nothing but places: plan again in the new arena
                CK(cudaMemsetAsync(&h->ctl->status, 0, sizeof(unsigned), s));
            }
            if (h->hctl->status) throw Err(DSPG_ERR_CUDA, "delta path: C's arena cannot take the new entries");
            run_alg_append(h->sr, N, h->C.view(), h->ctl, 0u, 0u, h->opt.slack_min, h->opt.slack_div, false, s,
                           h->num_sms);
        }
        // rows too long to search: recomputed by the row path
        alg_collect(h, h->alg.bm_long.p, s);
        read_ctl(h, s);
        long_rows = h->hctl->n_affected;
        if (long_rows > 0) alg_recompute_rows(h, s);
        // the touched rows, for the statistics and dspg_last_affected
        alg_collect(h, h->wc.bmR.p, s);
    }
    read_ctl(h, s);
    h->hctl->products += n_con;
    h->hctl->alg_new = n_new;
    h->hctl->alg_contrib = n_con;
    (void)long_rows;
    return true;
}

// ------------------------------------- general updates by Algorithm 2

// F for every entry of C from A and B (after a static recompute): rows up
// to 512 entries by the warp kernel, which lists the longer ones for the
// CTA kernel and its per-CTA column-to-place maps (m entries each, at most
// about 1 GiB of them).
void bloom_build(dspg_handle *h, cudaStream_t s) {
    DevMat &C = h->C;
    MaskWs &w = h->mw;
    if (C.fb.n < C.arena_cap) {
        C.fb.release();
        C.fb.reserve(std::max<int64_t>(C.arena_cap, 1));
    }
    const int64_t n = C.nrows;
    const long long cap_long = std::max<int64_t>(n, 1);
    w.rows_long.reserve(cap_long);
    w.n_long.reserve(1);
    CK(cudaMemsetAsync(w.n_long.p, 0, sizeof(long long), s));
    bloom_rows(h->A.view(), h->Bm().view(), C.view(), C.fb.p, w.rows_long.p, w.n_long.p, cap_long, s, h->num_sms);
    long long nl = 0;
    CK(cudaMemcpyAsync(&nl, w.n_long.p, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (nl > 0) {
        const int64_t m = std::max<int64_t>(C.ncols, 1);
        int64_t ctas = std::min<int64_t>(2 * h->num_sms, std::max<int64_t>(1, (int64_t(1) << 28) / m));
        ctas = std::min<int64_t>(ctas, nl);
        if (w.posmap_ctas < ctas || w.posmap_m != m) {
            w.posmap.release();
            w.posmap.reserve(ctas * m);
            CK(cudaMemsetAsync(w.posmap.p, 0xff, sizeof(int32_t) * ctas * m, s));  // -1: no place
            w.posmap_ctas = ctas;
            w.posmap_m = m;
        }
        bloom_long_rows(h->A.view(), h->Bm().view(), C.view(), C.fb.p, w.rows_long.p, w.n_long.p, cap_long,
                        w.posmap.p, (int)ctas, s);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
}

// One batch of general updates by Algorithm 2 (the handle keeps F): the
// merge of A' and B' as on the row path, then computePattern, E and R,
// A^R, the masked product and the merge into C and F.  Runs eagerly on s
// and reads the control block between its steps, growing what overflowed.
void masked_apply(dspg_handle *h, cudaStream_t s) {
    const int64_t nA = h->inA.n, nB = h->b_is_a ? 0 : h->inB.n;
    MaskWs &w = h->mw;
    const int cb = bits_for(std::max<int64_t>(h->C.ncols, 2));
    const int rb = bits_for(std::max<int64_t>(h->C.nrows, 2));
    w.ensure_contrib(std::max<int64_t>(int64_t(1) << 16, 16 * (nA + nB)));
    // sort, classify, merge and commit A' (and B'), then computePattern,
    // which reads B' and the transposed pattern of A before this batch; one
    // read of the control block after it (the later kernels skip on the
    // status bits, so a failed step is redone from where it stopped)
    bool restart = true;
    for (int iter = 0;; iter++) {
        // the jobs point at the staging, which a grown stage moves: built afresh each pass
        const UpdJob ja = h->wA.job(nA);
        const UpdJob jb = h->b_is_a ? ja : h->wB.job(nB);
        if (restart) {
            begin_batch(h->h_args_dev, h->d_args, h->ctl, s);
            stage_sort(h, s);
            if (nA > 0)
                run_classify(ja, h->A.view(), h->vsize, h->ctl, M_AB & ~ST_AB_STAGE, ST_AB_STAGE, DetectBufs{}, false,
                             false, s, h->num_sms);
            if (nB > 0)
                run_classify(jb, h->B.view(), h->vsize, h->ctl, M_AB & ~ST_AB_STAGE, ST_AB_STAGE, DetectBufs{}, false,
                             false, s, h->num_sms);
            stage_merge(h, s, -1);
            stage_commit_ab(h, s);
            restart = false;
        }
        PatJob J{};
        J.xr = ja.row; J.xc = ja.col; J.xk = ja.kind; J.xn = nA;
        J.yr = jb.row; J.yc = jb.col; J.yk = jb.kind; J.yn = h->b_is_a ? nA : nB;
        if (!h->has_at) J.yn = 0;  // B is never updated without the pattern
        J.key = w.key.p; J.bits = w.bits.p; J.cap = w.ccap; J.cb = cb;
        pat_contrib(J, h->Bm().view(), h->AT.view(), h->ctl, M_AB, s, h->num_sms);
        CK(cudaGetLastError());
        read_ctl(h, s);
        const unsigned st = h->hctl->status;
        if (st & ST_INVALID) throw Err(DSPG_ERR_INVALID, "batch entry out of range or with an invalid value/op");
        if ((st & ST_AB_STAGE) && iter < 6) {
            if (h->wA.grow_stage(h->hctl->u[0].stage_top + 1024)) h->epoch++;
            if (h->wB.grow_stage(h->hctl->u[1].stage_top + 1024)) h->epoch++;
            restart = true;
            continue;
        }
        if ((st & ST_AB_ARENA) && iter < 6) {
            // A's arena ran out in the commit: nothing after it ran; grow it
            // and commit again (the staged rows are still in place)
            regrow(h, h->A, s);
            if (nB > 0) regrow(h, h->B, s);
            for (int k = 0; k < 2; k++) {
                reset_range(h, &h->ctl->u[k].n_cchunk, sizeof(long long), s);
                reset_range(h, &h->ctl->u[k].reloc, sizeof(long long), s);
            }
            reset_range(h, &h->ctl->status, sizeof(unsigned), s);
            reset_range(h, &h->ctl->mask_n, sizeof(long long), s);
            stage_commit_ab(h, s);
            continue;
        }
        if ((st & ST_MASK_FULL) && iter < 6) {
            w.ensure_contrib(h->hctl->mask_n);
            reset_range(h, &h->ctl->status, sizeof(unsigned), s);
            reset_range(h, &h->ctl->mask_n, sizeof(long long), s);
            continue;
        }
        if (st) throw Err(DSPG_ERR_CUDA, "masked path: computePattern failed, status " + std::to_string(st));
        break;
    }
    const int64_t n = h->hctl->mask_n;
    if (h->has_at && nA > 0) {
        transpose_front(h, s);
        transpose_commit(h, s);
    }
    // C* sorted by (i, j), equal keys merged, in runs of one row; its
    // counts stay on the device (bounded by n for the grids and buffers)
    MaskJob M{};
    auto job = [&]() {
        M.urow = w.urow.p; M.ucol = w.ucol.p; M.ufs = w.ufs.p;
        M.nu_dev = w.ex.p + n;
        M.run_start = w.run_start.p; M.run_row = w.run_row.p;
        M.nruns_dev = w.rex.p + n; M.max_runs = n;
        M.upos = w.upos.p; M.ue = w.ue.p; M.rbits = w.rbits.p;
        M.kept_run = w.kept_run.p; M.kept_a = w.kept_a.p; M.kcap = w.kcap; M.nkept_dev = &h->ctl->mask_kept;
        M.z = (void *)w.z.p; M.h = w.h.p; M.hit = w.hit.p; M.dest = w.dest.p; M.dcap = w.dcap.p;
    };
    auto product_and_merge = [&]() {
        job();
        mask_init_acc(h->sr, M, n, s, h->num_sms);
        CK(cudaMemsetAsync(w.h.p, 0, sizeof(unsigned long long) * n, s));
        CK(cudaMemsetAsync(w.hit.p, 0, n, s));
        mask_product(h->sr, M, h->A.view(), h->Bm().view(), h->ctl, ST_MASK_FULL, s, h->num_sms);
        mask_plan(M, h->C.view(), h->ctl, ST_MASK_FULL, h->opt.slack_min, h->opt.slack_div, s, h->num_sms);
        mask_splice(h->sr, M, h->C.view(), h->C.fb.p, h->ctl, M_C | ST_MASK_FULL, s, h->num_sms);
    };
    if (n > 0) {
        w.ensure_unique(n, h->vsize);
        iota_u32(w.idx.p, n, s, h->num_sms);
        bool alt = false;
        radix_sort_pairs(w.key.p, w.idx.p, w.key_alt.p, w.idx_alt.p, n, rb + cb, w.counts.p, w.scan_tmp.p,
                         w.scan_out.p, s, &alt);
        const uint64_t *K = alt ? w.key_alt.p : w.key.p;
        const uint32_t *I = alt ? w.idx_alt.p : w.idx.p;
        pat_heads(K, n, w.flag.p, s, h->num_sms);
        scan_i32_to_i64(w.flag.p, w.ex.p, n, w.scan_tmp.p, s);
        job();
        CK(cudaMemsetAsync(w.rflag.p, 0, sizeof(int32_t) * n, s));
        pat_unique(K, I, w.bits.p, n, w.ex.p, cb, M, w.rflag.p, s, h->num_sms);
        scan_i32_to_i64(w.rflag.p, w.rex.p, n, w.uscan.p, s);
        CK(cudaMemsetAsync(h->wc.bmR.p, 0, sizeof(uint32_t) * h->wc.bmR.n, s));
        pat_runs(M, w.rflag.p, w.rex.p, n, h->wc.bmR.p, s, h->num_sms);
        // E and R
        CK(cudaMemsetAsync(w.upos.p, 0xff, sizeof(int32_t) * n, s));
        CK(cudaMemsetAsync(w.ue.p, 0, sizeof(unsigned long long) * n, s));
        mask_scan(M, h->C.view(), h->C.fb.p, s, h->num_sms);
        // A^R, the masked product, the merge into C and F
        w.ensure_kept(std::max<int64_t>(int64_t(1) << 16, 4 * n));
        job();
        mask_keep(M, h->A.view(), h->ctl, s, h->num_sms);
        product_and_merge();
    }
    // the rows of C*, for the statistics and dspg_last_affected
    if (n > 0) CK(cudaMemcpyAsync(&h->ctl->mask_u, w.ex.p + n, sizeof(long long), cudaMemcpyDeviceToDevice, s));
    alg_collect(h, h->wc.bmR.p, s);
    CK(cudaGetLastError());
    read_ctl(h, s);
    // what overflowed: the kept list (nothing after it ran), C's arena (the
    // plan wrote places only), the transposed pattern's staging or arena
    for (int iter = 0; iter < 8 && h->hctl->status; iter++) {
        const unsigned st = h->hctl->status;
        if (st & ST_MASK_FULL) {
            w.ensure_kept(h->hctl->mask_kept);
            reset_range(h, &h->ctl->status, sizeof(unsigned), s);
            reset_range(h, &h->ctl->mask_kept, sizeof(long long), s);
            reset_range(h, &h->ctl->c_reloc, sizeof(long long), s);
            job();
            mask_keep(M, h->A.view(), h->ctl, s, h->num_sms);
            product_and_merge();
        } else if (st & ST_C_ARENA) {
            regrow(h, h->C, s);  // the plan wrote nothing but places: plan again in the new arena
            reset_range(h, &h->ctl->status, sizeof(unsigned), s);
            reset_range(h, &h->ctl->c_reloc, sizeof(long long), s);
            job();
            mask_plan(M, h->C.view(), h->ctl, ST_MASK_FULL, h->opt.slack_min, h->opt.slack_div, s, h->num_sms);
            mask_splice(h->sr, M, h->C.view(), h->C.fb.p, h->ctl, M_C | ST_MASK_FULL, s, h->num_sms);
        } else if (st & (ST_AT_STAGE | ST_AT_ARENA)) {
            if ((st & ST_AT_STAGE) && h->wAT.grow_stage(h->hctl->u[2].stage_top + 1024)) h->epoch++;
            if (st & ST_AT_ARENA) regrow(h, h->AT, s);
            reset_range(h, &h->ctl->status, sizeof(unsigned), s);
            reset_range(h, &h->ctl->u[2], sizeof(UpdCtl), s);
            transpose_front(h, s);
            transpose_commit(h, s);
        } else {
            break;
        }
        CK(cudaGetLastError());
        read_ctl(h, s);
    }
    check_debug(h->hctl);
    if (h->hctl->status) throw Err(DSPG_ERR_CUDA, "masked path: update failed, status " + std::to_string(h->hctl->status));
    h->hctl->a_entries = h->hctl->mask_kept;
    h->last_masked = h->hctl->mask_u;
}

// Captures what body() enqueues on cs into an executable graph; the number
// of kernels it launched goes to *nk.  The capture is closed on errors.
template <typename F>
cudaGraphExec_t capture_graph(cudaStream_t cs, unsigned long long *nk, F body) {
    cudaGraph_t graph = nullptr;
    const unsigned long long k0 = launch_counter();
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
        body();
    } catch (...) {
        cudaStreamEndCapture(cs, &graph);
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        throw;
    }
    CK(cudaStreamEndCapture(cs, &graph));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    if (nk) *nk = launch_counter() - k0;
    return exec;
}

void check_tuning(const dspg_tuning &t) {
    if (t.merge_k < 0 || t.merge_k > 8 || t.merge_ub < 0 || t.merge_ub > 64)
        throw Err(DSPG_ERR_INVALID, "tuning: merge_k must be in 0..8 and merge_ub in 0..64");
    if (t.lanes_min != 8 && t.lanes_min != 16 && t.lanes_min != 32)
        throw Err(DSPG_ERR_INVALID, "tuning: lanes_min must be 8, 16 or 32");
    if (t.table_shift < 0 || t.table_shift > 1) throw Err(DSPG_ERR_INVALID, "tuning: table_shift must be 0 or 1");
    if (t.warp_max < 0 || t.warp_max > 1024 || t.cta_max < 0 || t.cta_max > 16384)
        throw Err(DSPG_ERR_INVALID, "tuning: warp_max must be in 0..1024 and cta_max in 0..16384");
    if (t.sort_max < 0 || t.sort_max > 256) throw Err(DSPG_ERR_INVALID, "tuning: sort_max must be in 0..256");
}

// The autotuner's candidates: the defaults first, then one or two changes
// each (group-sort reach, thread-merge reach, lanes per short row, table
// oversizing, the warp/CTA and CTA/global crossovers).
const dspg_tuning kCandidates[] = {
    {8, 64, 8, 0, 1024, 16384, 64},  {8, 64, 8, 0, 1024, 16384, 0},   {8, 64, 8, 0, 1024, 16384, 128},
    {8, 64, 8, 0, 1024, 16384, 256}, {0, 0, 8, 0, 1024, 16384, 0},    {4, 32, 8, 0, 1024, 16384, 0},
    {8, 49, 8, 0, 1024, 16384, 0},   {8, 64, 16, 0, 1024, 16384, 64}, {8, 64, 32, 0, 1024, 16384, 64},
    {8, 64, 8, 1, 1024, 16384, 64},  {8, 64, 8, 0, 512, 16384, 64},   {8, 64, 8, 0, 1024, 4096, 64},
    {8, 64, 8, 0, 1024, 8192, 64},   {8, 64, 8, 1, 1024, 8192, 64},   {8, 64, 32, 0, 1024, 8192, 256},
    {0, 0, 16, 1, 1024, 16384, 0},
};
constexpr int kNumCandidates = (int)(sizeof(kCandidates) / sizeof(kCandidates[0]));

// The recompute of the last batch's affected rows (sizing + numeric), as
// a graph on the handle's stream, under the handle's current tuning.
cudaGraphExec_t capture_recompute(dspg_handle *h) {
    return capture_graph(h->gs, nullptr, [&] {
        reset_c_counters(h, h->gs);
        reset_range(h, &h->ctl->status, sizeof(unsigned), h->gs);
        stage_size(h, h->gs);
        stage_numeric(h, h->gs);
        cudaMemcpyAsync(h->hctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->gs);
    });
}

}  // namespace

// ================================================================ C ABI

extern "C" {

dspg_status dspg_build_form(dspg_handle **out, const dspg_csr *A, const dspg_csr *B, dspg_semiring sr,
                            const dspg_form *form, const dspg_options *opt, void *stream) {
    dspg_handle *h = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    try {
        NvtxRange nvtx_build("dspg/build");
        if (!out) throw Err(DSPG_ERR_INVALID, "out is NULL");
        *out = nullptr;
        if (sr != DSPG_PLUS_TIMES_F64 && sr != DSPG_MIN_PLUS_I32) throw Err(DSPG_ERR_INVALID, "unknown semiring");
        const bool ta = form && form->trans_a, tb = form && form->trans_b;
        check_csr_arg(A, "A");
        const int64_t a_rows = ta ? A->ncols : A->nrows, a_cols = ta ? A->nrows : A->ncols;
        int64_t b_rows, b_cols;
        if (B) {
            check_csr_arg(B, "B");
            b_rows = tb ? B->ncols : B->nrows;
            b_cols = tb ? B->nrows : B->ncols;
        } else {
            b_rows = tb ? A->ncols : A->nrows;
            b_cols = tb ? A->nrows : A->ncols;
        }
        if (a_cols != b_rows) throw Err(DSPG_ERR_INVALID, "the inner dimensions of op(A) op(B) differ");
        if (form && sr == DSPG_MIN_PLUS_I32 &&
            (form->alpha_i <= -MP_LIMIT / 2 || form->alpha_i >= MP_LIMIT / 2 || form->beta_i <= -MP_LIMIT / 2 ||
             form->beta_i >= MP_LIMIT / 2))
            throw Err(DSPG_ERR_INVALID, "(min,+) alpha and beta must be below 2^29 in magnitude");
        if (form && sr == DSPG_PLUS_TIMES_F64 && (!std::isfinite(form->alpha) || !std::isfinite(form->beta)))
            throw Err(DSPG_ERR_INVALID, "alpha and beta must be finite");
        if (form && form->X) {
            check_csr_arg(form->X, "X");
            if (form->X->nrows != a_rows || form->X->ncols != b_cols)
                throw Err(DSPG_ERR_INVALID, "X must have the shape of op(A) op(B)");
        }
        h = new dspg_handle();
        set_defaults(&h->opt);
        if (opt) {
            if (opt->slack_min >= 0) h->opt.slack_min = opt->slack_min;
            if (opt->slack_div > 0) h->opt.slack_div = opt->slack_div;
            if (opt->arena_headroom >= 1.0) h->opt.arena_headroom = opt->arena_headroom;
            h->opt.keep_transpose = opt->keep_transpose;
            h->opt.exact_static = opt->exact_static;
            if (opt->bloom != 0 && opt->bloom != 1) throw Err(DSPG_ERR_INVALID, "options: bloom must be 0 or 1");
            h->opt.bloom = opt->bloom;
        }
        h->bloom = h->opt.bloom == 1;
        h->sr = sr;
        h->vsize = sr == DSPG_PLUS_TIMES_F64 ? 8 : 4;
        h->trans_a = ta;
        h->trans_b = tb;
        if (form) {
            h->fs = FormScalars{form->alpha, form->beta, form->alpha_i, form->beta_i};
            const bool unit = sr == DSPG_PLUS_TIMES_F64 ? form->alpha == 1.0 : form->alpha_i == 0;
            h->form = !unit || form->X != nullptr;
        }
        CK(cudaGetDevice(&h->dev));
        CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev));
        CK(cudaMalloc((void **)&h->ctl, sizeof(Ctl)));
        CK(cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
        if (const char *env = getenv("DSPG_ALL_BINS")) h->gate_bins = env[0] == '0';
        if (const char *env = getenv("DSPG_NO_DIRECT_READ")) h->direct_read = env[0] == '0';
        for (int k = 0; k < NUM_SIDE; k++) {
            CK(cudaStreamCreateWithFlags(&h->nstr[k], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&h->evNum[k], cudaEventDisableTiming));
        }
        for (cudaEvent_t *e : {&h->evIn, &h->evFork, &h->evDetect, &h->evSide, &h->evSize})
            CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        if (const char *env = getenv("DSPG_NO_GRAPHS")) h->use_graphs = env[0] == '0';
        CK(cudaHostAlloc((void **)&h->hctl, sizeof(Ctl), cudaHostAllocMapped));
        CK(cudaHostGetDevicePointer((void **)&h->hctl_dev, h->hctl, 0));
        CK(cudaMalloc((void **)&h->d_args, 3 * sizeof(InArgs)));
        CK(cudaHostAlloc((void **)&h->h_args, 3 * sizeof(InArgs), cudaHostAllocMapped));
        CK(cudaHostGetDevicePointer((void **)&h->h_args_dev, h->h_args, 0));
        std::memset(h->h_args, 0, 3 * sizeof(InArgs));
        std::memset(h->hctl, 0, sizeof(Ctl));
        h->wA.which = 0; h->wA.vsize = h->vsize; h->wA.n_dev = &h->d_args[0].n;
        h->wB.which = 1; h->wB.vsize = h->vsize; h->wB.n_dev = &h->d_args[1].n;
        h->wAT.which = 2; h->wAT.vsize = 0; h->wAT.n_dev = &h->d_args[2].n;
        load_operand(h, h->A, A, ta, s);
        // B is A: one stored operand when both sides are (or neither is)
        // transposed; otherwise a stored copy of A, transposed as its side
        // asks, that every batch of A updates too
        h->b_is_a = (B == nullptr) && ta == tb;
        h->b_alias = (B == nullptr) && ta != tb;
        if (B) load_operand(h, h->B, B, tb, s);
        else if (h->b_alias) load_operand(h, h->B, A, tb, s);
        if (form && form->X) {
            DBuf<int64_t> rp;
            DBuf<int32_t> col;
            DBuf<char> val;
            const int64_t *rp_d;
            const int32_t *col_d;
            const void *val_d;
            load_csr(h, form->X, rp, col, val, &rp_d, &col_d, &val_d, s);
            const int64_t nx = form->X->nnz;
            h->xrp.reserve(form->X->nrows + 1);
            h->xcol.reserve(std::max<int64_t>(nx, 1));
            h->xval.reserve(std::max<int64_t>(nx, 1) * h->vsize);
            CK(cudaMemcpyAsync(h->xrp.p, rp_d, sizeof(int64_t) * (form->X->nrows + 1), cudaMemcpyDeviceToDevice, s));
            if (nx > 0) {
                CK(cudaMemcpyAsync(h->xcol.p, col_d, sizeof(int32_t) * nx, cudaMemcpyDeviceToDevice, s));
                CK(cudaMemcpyAsync(h->xval.p, val_d, (size_t)h->vsize * nx, cudaMemcpyDeviceToDevice, s));
            }
            CK(cudaStreamSynchronize(s));
            h->has_x = true;
        }
        // C = A A (and a stored copy of A as B) needs the transposed pattern
        // for every batch; otherwise it is built on the first B batch
        const bool keep_t = h->b_is_a || h->b_alias || h->opt.keep_transpose > 0 || h->bloom;
        if (keep_t) build_transpose(h, s);
        static_recompute(h, s);
        *out = h;
        return DSPG_OK;
    } catch (const Err &e) {
        g_err = e.what();
        delete h;
        if (out) *out = nullptr;
        return e.st;
    }
}

dspg_status dspg_build(dspg_handle **out, const dspg_csr *A, const dspg_csr *B, dspg_semiring sr,
                       const dspg_options *opt, void *stream) {
    return dspg_build_form(out, A, B, sr, nullptr, opt, stream);
}

dspg_status dspg_apply_batch(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB,
                             dspg_batch_stats *stats, void *stream) {
    if (!h) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    try {
        check_usable(h);
        apply_one(h, dA, dB, stats, (cudaStream_t)stream);
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_apply_batch_async(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB, void *stream) {
    if (!h) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is already in flight"));
    if (h->bloom) return fail(h, Err(DSPG_ERR_STATE, "a handle with the Bloom filter applies batches synchronously"));
    try {
        check_usable(h);
        const cudaStream_t s = (cudaStream_t)stream;
        prepare_batch(h, dA, dB, s);
        h->pending_comp0 = h->compactions;
        run_first(h, s, false);
        h->pending = true;
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_apply_batch_wait(dspg_handle *h, dspg_batch_stats *stats, void *stream) {
    if (!h) return DSPG_ERR_INVALID;
    if (!h->pending) return fail(h, Err(DSPG_ERR_STATE, "no asynchronous batch in flight"));
    try {
        const cudaStream_t s = (cudaStream_t)stream;
        h->pending = false;
        try {
            CK(cudaStreamSynchronize(s));
            if (h->prof) stage_times_from_events(h);
            recover(h, s);
            est_fallback(h, s);
        } catch (const Err &e) {
            if (e.st != DSPG_ERR_INVALID) h->broken = true;
            throw;
        }
        fill_stats(h, stats, h->pending_comp0);
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_apply_batch_algebraic(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB,
                                       dspg_batch_stats *stats, void *stream) {
    if (!h) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    if (h->bloom) return fail(h, Err(DSPG_ERR_STATE, "a handle with the Bloom filter takes dspg_apply_batch"));
    try {
        check_usable(h);
        const cudaStream_t s = (cudaStream_t)stream;
        prepare_batch(h, dA, dB, s);
        const int64_t compactions0 = h->compactions;
        try {
            h->last_alg = apply_algebraic(h, s);
            if (!h->last_alg) {  // general updates: the row path
                run_first(h, s);
                if (h->prof) stage_times_from_events(h);
                recover(h, s);
            }
            est_fallback(h, s);
        } catch (const Err &e) {
            if (e.st != DSPG_ERR_INVALID) h->broken = true;
            throw;
        }
        dspg_batch_stats local;
        if (!stats) stats = &local;
        fill_stats(h, stats, compactions0);
        stats->algebraic = h->last_alg ? 1 : 0;
        trace_batch(h, *stats, h->last_alg ? "delta" : "rows");
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_read_C(dspg_handle *h, int64_t *nnz_out, int64_t *rowptr, int32_t *col, void *val, int on_device,
                        void *stream) {
    if (!h || !nnz_out) return DSPG_ERR_INVALID;
    try {
        check_usable(h);
        *nnz_out = h->form ? read_form(h, nullptr, 0, rowptr, col, val, on_device, (cudaStream_t)stream)
                           : read_mat(h, h->C, nullptr, 0, rowptr, col, val, on_device, (cudaStream_t)stream);
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_read_bloom(dspg_handle *h, int64_t *nnz_out, int64_t *rowptr, int32_t *col, uint64_t *words,
                            int on_device, void *stream) {
    if (!h || !nnz_out) return DSPG_ERR_INVALID;
    if (!h->bloom) return fail(h, Err(DSPG_ERR_STATE, "the handle keeps no Bloom filter (options.bloom = 0)"));
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    try {
        check_usable(h);
        *nnz_out = read_mat(h, h->C, nullptr, 0, rowptr, col, (void *)words, on_device, (cudaStream_t)stream, true);
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_read_A(dspg_handle *h, int64_t *nnz_out, int64_t *rowptr, int32_t *col, void *val, int on_device,
                        void *stream) {
    if (!h || !nnz_out) return DSPG_ERR_INVALID;
    try {
        check_usable(h);
        *nnz_out = read_operand_a(h, rowptr, col, val, on_device, (cudaStream_t)stream);
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_read_rows_C(dspg_handle *h, const int32_t *rows, int64_t nrows, int64_t *nnz_out, int64_t *rowptr,
                             int32_t *col, void *val, int on_device, void *stream) {
    if (!h || !nnz_out || nrows < 0 || (nrows > 0 && !rows)) return DSPG_ERR_INVALID;
    try {
        check_usable(h);
        if (!on_device) {
            for (int64_t i = 0; i < nrows; i++)
                if (rows[i] < 0 || rows[i] >= h->C.nrows) throw Err(DSPG_ERR_INVALID, "row index out of range");
        }
        const int32_t *rr = rows ? rows : (const int32_t *)h->wc.iota.p;
        *nnz_out = h->form ? read_form(h, rr, nrows, rowptr, col, val, on_device, (cudaStream_t)stream)
                           : read_mat(h, h->C, rr, nrows, rowptr, col, val, on_device, (cudaStream_t)stream);
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

int dspg_debug_build(void) { return DSPG_DEBUG ? 1 : 0; }

dspg_status dspg_fault_inject(const char *spec) {
    long long a = 0, v = 0;
    if (!parse_faults(spec, &a, &v)) {
        set_thread_error("fault spec must be NULL, empty, or site@N[,site@N] with site alloc or validate, N >= 1");
        return DSPG_ERR_INVALID;
    }
    arm_faults(a, v);
    return DSPG_OK;
}

// The end of a direct read whose rows over 16384 entries were out of order
// (ro.n_huge of them, listed in the read's scratch): each is sorted in the
// scratch on the device and copied into the caller's col and val (rp: the
// device row pointers, rowptr: the same on the host).
static void read_huge_rows(dspg_handle *h, const ReadOut &ro, const int64_t *rp, const int64_t *rowptr,
                           int32_t *col, void *val, cudaStream_t s) {
    dspg_handle::ReadWs &w = h->rd;
    std::vector<int64_t> lh(ro.n_huge);
    CK(cudaMemcpyAsync(lh.data(), w.huge_l.p, sizeof(int64_t) * ro.n_huge, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::sort(lh.begin(), lh.end());
    sort_listed_host(h, h->C, rp, lh, rowptr, w.c.p, (void *)w.v.p, h->vsize, s);
    for (int64_t x : lh) {
        const int64_t lo = rowptr[x], len = rowptr[x + 1] - rowptr[x];
        CK(cudaMemcpyAsync(col + lo, w.c.p + lo, sizeof(int32_t) * len, cudaMemcpyDeviceToHost, s));
        if (val && h->vsize)
            CK(cudaMemcpyAsync((char *)val + lo * h->vsize, w.v.p + lo * h->vsize, (size_t)h->vsize * len,
                               cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
}

dspg_status dspg_read_affected_C(dspg_handle *h, int64_t rows_cap, int64_t nnz_cap, int64_t *nrows_out,
                                 int64_t *nnz_out, int32_t *rows, int64_t *rowptr, int32_t *col, void *val,
                                 int on_device, void *stream) {
    if (!h || !nrows_out || !nnz_out) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    if (h->form) return fail(h, Err(DSPG_ERR_STATE, "a handle with alpha, beta or X reads its rows by dspg_read_rows_C"));
    cudaStream_t s = (cudaStream_t)stream;
    try {
        check_usable(h);
        NvtxRange r("dspg/read_affected_C");
        const int64_t n = h->last_nR;
        dspg_handle::ReadWs &w = h->rd;
        w.r.reserve(std::max<int64_t>(n, 1));
        DBuf<int64_t> rp_l;
        int64_t *rp = read_scratch(w.rp, rp_l, n + 1);
        // R in row order on the device, from the chunk table of its collection
        const int64_t nch = ((h->A.nrows + 31) / 32 + 255) / 256;
        w.chunk_cnt.reserve(nch + 1);
        w.chunk_ex.reserve(nch + 1);
        DBuf<int32_t> lens_l;
        int32_t *lens = read_scratch(w.lens, lens_l, n);
        // page-locked host buffers: the rows go straight into them, in column
        // order, with one synchronisation (unless R was not collected in
        // order, which the read finds on the device and leaves to the path below)
        int32_t *dcol = rows && !on_device && h->direct_read && rows_cap >= n ? (int32_t *)device_view(col) : nullptr;
        void *dval = (dcol && val && h->vsize) ? device_view(val) : nullptr;
        const bool direct = dcol && (!val || !h->vsize || dval);
        if (direct) w.res.reserve(1);
        // R in row order and its row pointers: two launches (each block scans
        // the chunk table), written into the caller's page-locked rows and
        // rowptr as well on the direct path; with a larger chunk table, the
        // chunk scan, a gather of the lengths and their scan
        const bool two = nch <= read_nch_max();
        int32_t *drows = direct && two ? (int32_t *)device_view(rows) : nullptr;
        int64_t *drp = direct && two ? (int64_t *)device_view(rowptr) : nullptr;
        if (two) {
            read_order_rowptr(h->wc.R.p, h->wc.rchunk.p, nch, n, nullptr, n, nullptr, h->C.len.p, w.r.p, lens,
                              w.chunk_cnt.p, w.chunk_ex.p + nch, rp, drows, drp, direct ? w.res.p : nullptr, s,
                              h->num_sms);
        } else {
            w.chunk_tmp.reserve(scan_tmp_entries(nch + 1) + 1);
            rows_in_order(h->wc.R.p, h->wc.rchunk.p, nch, n, w.chunk_cnt.p, w.chunk_ex.p, w.chunk_tmp.p, w.r.p, s);
            DBuf<int64_t> scan_l;
            int64_t *lens_scan = read_scratch(w.scan, scan_l, scan_tmp_entries(n) + 1);
            lens_of_rows(w.r.p, n, h->C.len.p, lens, s);
            scan_i32_to_i64(lens, rp, n, lens_scan, s);
            if (direct) CK(cudaMemsetAsync(w.res.p, 0, sizeof(ReadOut), s));
        }
        if (direct) {
            w.long_l.reserve(std::max<int64_t>(n, 1));
            w.huge_l.reserve(std::max<int64_t>(n, 1));
            w.c.reserve(std::max<int64_t>(nnz_cap, 1));
            w.v.reserve(std::max<int64_t>(nnz_cap, 1) * std::max(h->vsize, 1));
            read_rows_direct(w.r.p, n, nullptr, h->C.view(), h->vsize, rp, w.chunk_ex.p + nch, nnz_cap, dcol, dval,
                             w.c.p, (void *)w.v.p, w.long_l.p, w.huge_l.p, w.res.p, s, h->num_sms);
            ReadOut ro{};
            CK(cudaMemcpyAsync(&ro, w.res.p, sizeof(ReadOut), cudaMemcpyDeviceToHost, s));
            if (n > 0 && !drows) CK(cudaMemcpyAsync(rows, w.r.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
            if (!drp) CK(cudaMemcpyAsync(rowptr, rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (!(ro.flags & READ_UNORDERED)) {
                *nrows_out = n;
                *nnz_out = ro.nnz;
                if (ro.flags & READ_TOO_SMALL)
                    throw Err(DSPG_ERR_INVALID, "read_affected_C: buffers too small (need " + std::to_string(n) +
                                                    " rows, " + std::to_string(ro.nnz) + " entries)");
                if (ro.n_huge > 0) read_huge_rows(h, ro, rp, rowptr, col, val, s);
                return DSPG_OK;
            }
        }
        int64_t tot[2] = {0, 0};
        CK(cudaMemcpyAsync(&tot[0], w.chunk_ex.p + nch, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&tot[1], rp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (tot[0] != n) {
            // R not from one collection: sort it on the device, size it again
            CK(cudaMemcpyAsync(w.r.p, h->wc.R.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
            w.k0.reserve(n); w.k1.reserve(n); w.i0.reserve(n); w.i1.reserve(n);
            int64_t cnt;
            sort_tmp_sizes(n, &cnt);
            w.counts.reserve(cnt);
            w.so.reserve(cnt + 1);
            w.st.reserve(scan_tmp_entries(cnt) + 1);
            sort_i32_values(w.r.p, n, bits_for(h->A.nrows), w.k0.p, w.k1.p, w.i0.p, w.i1.p, w.counts.p, w.st.p,
                            w.so.p, s);
            tot[1] = mat_rowptr(h, h->C, w.r.p, n, rp, s);
        }
        const int64_t nnz = tot[1];
        *nrows_out = n;
        *nnz_out = nnz;
        if (!rows) return DSPG_OK;
        if (rows_cap < n || nnz_cap < nnz)
            throw Err(DSPG_ERR_INVALID, "read_affected_C: buffers too small (need " + std::to_string(n) + " rows, " +
                                            std::to_string(nnz) + " entries)");
        if (n > 0)
            CK(cudaMemcpyAsync(rows, w.r.p, sizeof(int32_t) * n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               s));
        fill_rows_out(h, h->C, h->C.view(), h->vsize, w.r.p, n, rp, nnz, rowptr, col, val, on_device, s);
        if (on_device) CK(cudaStreamSynchronize(s));
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_apply_read_affected(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB,
                                     int64_t rows_cap, int64_t nnz_cap, int64_t *nrows_out, int64_t *nnz_out,
                                     int32_t *rows, int64_t *rowptr, int32_t *col, void *val,
                                     dspg_batch_stats *stats, void *stream) {
    if (!h || !nrows_out || !nnz_out) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    if (h->form) return fail(h, Err(DSPG_ERR_STATE, "a handle with alpha, beta or X reads its rows by dspg_read_rows_C"));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nch = ((h->A.nrows + 31) / 32 + 255) / 256;
    int32_t *drows = nullptr, *dcol = nullptr;
    int64_t *drp = nullptr;
    void *dval = nullptr;
    bool one = !h->bloom && h->direct_read && rows && rowptr && col && rows_cap >= 0 && nnz_cap >= 0 &&
               nch <= read_nch_max();
    if (one) {
        drows = (int32_t *)device_view(rows);
        drp = (int64_t *)device_view(rowptr);
        dcol = (int32_t *)device_view(col);
        dval = (val && h->vsize) ? device_view(val) : nullptr;
        one = drows && drp && dcol && (!val || !h->vsize || dval);
    }
    if (one) {
        try {
            check_usable(h);
            NvtxRange r("dspg/apply_read_affected");
            // the read's buffers first, so that nothing is allocated while the batch runs
            dspg_handle::ReadWs &w = h->rd;
            const int64_t cap = std::min<int64_t>(rows_cap, h->A.nrows);  // R never has more rows than A
            const int64_t rc = std::max<int64_t>(cap, 1);
            w.r.reserve(rc);
            w.lens.reserve(rc);
            w.rp.reserve(rc + 1);
            w.chunk_cnt.reserve(nch + 1);
            w.chunk_ex.reserve(nch + 1);
            w.res.reserve(1);
            w.long_l.reserve(rc);
            w.huge_l.reserve(rc);
            w.c.reserve(std::max<int64_t>(nnz_cap, 1));
            w.v.reserve(std::max<int64_t>(nnz_cap, 1) * std::max(h->vsize, 1));
            dspg_batch_stats local;
            if (!stats) stats = &local;
            prepare_batch(h, dA, dB, s);
            const int64_t compactions0 = h->compactions;
            bool clean = false;
            ReadOut ro{};
            try {
                run_first(h, s, false);
                // behind the batch: R's size from the device, bounded by cap
                const long long *n_dev = &h->ctl->n_affected;
                read_order_rowptr(h->wc.R.p, h->wc.rchunk.p, nch, rc, n_dev, cap, &h->ctl->status, h->C.len.p, w.r.p,
                                  w.lens.p, w.chunk_cnt.p, w.chunk_ex.p + nch, w.rp.p, drows, drp, w.res.p, s,
                                  h->num_sms);
                read_rows_direct(w.r.p, rc, n_dev, h->C.view(), h->vsize, w.rp.p, w.chunk_ex.p + nch, nnz_cap, dcol,
                                 dval, w.c.p, (void *)w.v.p, w.long_l.p, w.huge_l.p, w.res.p, s, h->num_sms);
                CK(cudaMemcpyAsync(&ro, w.res.p, sizeof(ReadOut), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                // a batch that needs a second pass changes C after the read
                clean = h->hctl->status == 0 && h->hctl->n_ovf <= 0;
                if (h->prof) stage_times_from_events(h);
                recover(h, s);
                est_fallback(h, s);
            } catch (const Err &e) {
                if (e.st != DSPG_ERR_INVALID) h->broken = true;
                throw;
            }
            fill_stats(h, stats, compactions0);
            trace_batch(h, *stats, "rows");
            if (clean && ro.flags == 0 && ro.nr == h->last_nR) {
                *nrows_out = ro.nr;
                *nnz_out = ro.nnz;
                if (ro.n_huge > 0) read_huge_rows(h, ro, w.rp.p, rowptr, col, val, s);
                return DSPG_OK;
            }
        } catch (const Err &e) {
            return fail(h, e);
        }
    } else {
        const dspg_status st = dspg_apply_batch(h, dA, dB, stats, stream);
        if (st != DSPG_OK) return st;
    }
    // the read on its own, after the batch
    return dspg_read_affected_C(h, rows_cap, nnz_cap, nrows_out, nnz_out, rows, rowptr, col, val, 0, stream);
}

dspg_status dspg_last_affected(dspg_handle *h, int64_t *count, int32_t *rows, int on_device, void *stream) {
    if (!h || !count) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    cudaStream_t s = (cudaStream_t)stream;
    try {
        check_usable(h);
        const int64_t n = h->last_nR;
        if (!rows) {
            *count = n;
            return DSPG_OK;
        }
        if (*count < n) throw Err(DSPG_ERR_INVALID, "rows buffer too small");
        *count = n;
        if (n == 0) return DSPG_OK;
        if (!on_device) {
            // R is ascending within each 8192-row chunk of the bitmap it was
            // collected from; the chunk table says where each chunk's rows
            // went, so laying the chunks end to end in chunk order sorts R
            const int64_t nch = (h->A.nrows + 31) / 32 / 256 + 1;
            std::vector<int32_t> &raw = h->rd.h_r;
            std::vector<long long> &ch = h->rd.h_ch;
            if ((int64_t)raw.size() < n) raw.resize(n);
            if ((int64_t)ch.size() < 2 * nch) ch.resize(2 * nch);
            CK(cudaMemcpyAsync(raw.data(), h->wc.R.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(ch.data(), h->wc.rchunk.p, sizeof(long long) * 2 * nch, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const int64_t used = ((h->A.nrows + 31) / 32 + 255) / 256;  // chunks the collection visited
            int64_t o = 0;
            bool ok = true;
            for (int64_t c = 0; c < used && ok; c++) {
                const long long b = ch[2 * c], k = ch[2 * c + 1];
                ok = k >= 0 && b >= 0 && b + k <= n && o + k <= n;
                if (ok && k > 0) {
                    std::memcpy(rows + o, raw.data() + b, sizeof(int32_t) * (size_t)k);
                    o += k;
                }
            }
            for (int64_t x = 1; ok && x < o; x++) ok = rows[x - 1] < rows[x];
            if (ok && o == n) return DSPG_OK;
            // otherwise (R not from one collection): sort it on the device
        }
        // R is at most one entry per row of A: its sort buffers are kept
        dspg_handle::ReadWs &w = h->rd;
        w.r.reserve(n);
        CK(cudaMemcpyAsync(w.r.p, h->wc.R.p, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
        w.k0.reserve(n); w.k1.reserve(n); w.i0.reserve(n); w.i1.reserve(n);
        int64_t cnt;
        sort_tmp_sizes(n, &cnt);
        w.counts.reserve(cnt);
        w.so.reserve(cnt + 1);
        w.st.reserve(scan_tmp_entries(cnt) + 1);
        sort_i32_values(w.r.p, n, bits_for(h->A.nrows), w.k0.p, w.k1.p, w.i0.p, w.i1.p, w.counts.p, w.st.p, w.so.p, s);
        CK(cudaMemcpyAsync(rows, w.r.p, sizeof(int32_t) * n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_recompute_all(dspg_handle *h, void *stream) {
    if (!h) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    try {
        check_usable(h);
        static_recompute(h, (cudaStream_t)stream);
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_info(dspg_handle *h, int64_t *n, int64_t *k, int64_t *m, int64_t *nnz_a, int64_t *nnz_c) {
    if (!h) return DSPG_ERR_INVALID;
    try {
        if (n) *n = h->A.nrows;
        if (k) *k = h->A.ncols;
        if (m) *m = h->Bm().ncols;
        if (nnz_a) *nnz_a = read_mat(h, h->A, nullptr, 0, nullptr, nullptr, nullptr, 0, 0);
        if (nnz_c) *nnz_c = h->form ? read_form(h, nullptr, 0, nullptr, nullptr, nullptr, 0, 0)
                                    : read_mat(h, h->C, nullptr, 0, nullptr, nullptr, nullptr, 0, 0);
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_set_profiling(dspg_handle *h, int on) {
    if (!h) return DSPG_ERR_INVALID;
    try {
        if (on && !h->pev[0])
            for (int k = 0; k < 10; k++) CK(cudaEventCreate(&h->pev[k]));
        h->prof = on != 0;
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_stage_times(dspg_handle *h, float *ms, int n) {
    if (!h || !ms || n < 0) return DSPG_ERR_INVALID;
    for (int k = 0; k < n && k < DSPG_NSTAGES; k++) ms[k] = h->stage_ms[k];
    return DSPG_OK;
}

unsigned long long dspg_kernel_launches(void) { return __atomic_load_n(&launch_counter(), __ATOMIC_RELAXED); }

dspg_status dspg_reserve(dspg_handle *h, int64_t nA, int64_t nB, void *stream) {
    if (!h) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    try {
        if (nA < 0 || nB < 0 || nA > INT32_MAX / 2 || nB > INT32_MAX / 2) throw Err(DSPG_ERR_INVALID, "bad size");
        if ((h->b_is_a || h->b_alias) && nB > 0) throw Err(DSPG_ERR_INVALID, "B is A: reserve through nA");
        h->grp_cap_a = std::max(h->grp_cap_a, batch_bucket(nA));
        h->grp_cap_b = std::max(h->grp_cap_b, batch_bucket(h->b_alias ? nA : nB));
        cudaStream_t s = (cudaStream_t)stream;
        if (h->wA.ensure(h->grp_cap_a, h->A.arena_cap)) h->epoch++;
        if (!h->b_is_a && h->wB.ensure(h->grp_cap_b, h->B.arena_cap)) h->epoch++;
        if (h->has_at && h->wAT.ensure(h->grp_cap_a, h->AT.arena_cap)) h->epoch++;
        CK(cudaStreamSynchronize(s));
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_run_counts(const dspg_handle *h, int64_t *replayed, int64_t *captured, int64_t *eager) {
    if (!h) return DSPG_ERR_INVALID;
    if (replayed) *replayed = h->runs_replayed;
    if (captured) *captured = h->runs_captured;
    if (eager) *eager = h->runs_eager;
    return DSPG_OK;
}

dspg_status dspg_tuning_candidate(int k, dspg_tuning *t) {
    if (k < 0 || k >= kNumCandidates || !t) return DSPG_ERR_INVALID;
    *t = kCandidates[k];
    return DSPG_OK;
}

dspg_status dspg_set_tuning(dspg_handle *h, const dspg_tuning *t) {
    if (!h) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    try {
        const dspg_tuning v = t ? *t : kCandidates[0];
        check_tuning(v);
        h->tune = v;
        reset_bins(h);  // captured pipelines carry the old bins
        return DSPG_OK;
    } catch (const Err &e) {
        return fail(h, e);
    }
}

dspg_status dspg_get_tuning(dspg_handle *h, dspg_tuning *t) {
    if (!h || !t) return DSPG_ERR_INVALID;
    *t = h->tune;
    return DSPG_OK;
}

dspg_status dspg_autotune(dspg_handle *h, const dspg_updates *dA, const dspg_updates *dB, int64_t nbatches,
                          dspg_tuning *best, float *ms, int n_ms, int *n_cand, void *stream) {
    if (!h) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    if (h->bloom) return fail(h, Err(DSPG_ERR_STATE, "the autotuner replays the row path, which a handle with the Bloom filter does not take"));
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<cudaGraphExec_t> execs(kNumCandidates, nullptr);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const dspg_tuning keep = h->tune;
    const bool gate0 = h->gate_bins;
    auto cleanup = [&] {
        for (auto &x : execs)
            if (x) cudaGraphExecDestroy(x);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    try {
        if (nbatches < 0 || (nbatches > 0 && !dA)) throw Err(DSPG_ERR_INVALID, "autotune needs nbatches >= 0 batches");
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        std::vector<double> tot(kNumCandidates, 0.0);
        std::vector<uint64_t> epochs(kNumCandidates, 0);
        reset_bins(h);
        h->gate_bins = false;  // every candidate runs with all its bins
        for (int64_t b = 0; b < nbatches; b++) {
            h->tune = keep;
            apply_one(h, dA + b, dB ? dB + b : nullptr, nullptr, s);
            if (h->last_nR == 0) continue;
            CK(cudaEventRecord(h->evIn, s));
            CK(cudaStreamWaitEvent(h->gs, h->evIn, 0));
            for (int j = 0; j < kNumCandidates; j++) {
                const int c = (int)((b + j) % kNumCandidates);
                h->tune = kCandidates[c];
                if (!execs[c] || epochs[c] != h->epoch) {
                    if (execs[c]) cudaGraphExecDestroy(execs[c]);
                    execs[c] = capture_recompute(h);
                    epochs[c] = h->epoch;
                }
                CK(cudaEventRecord(e0, h->gs));
                CK(cudaGraphLaunch(execs[c], h->gs));
                CK(cudaEventRecord(e1, h->gs));
                CK(cudaStreamSynchronize(h->gs));
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, e0, e1));
                tot[c] += t;
                if (h->hctl->status) recover(h, h->gs);
            }
            CK(cudaEventRecord(h->evIn, h->gs));
            CK(cudaStreamWaitEvent(s, h->evIn, 0));
        }
        int bi = 0;
        for (int c = 1; c < kNumCandidates; c++)
            if (tot[c] < tot[bi]) bi = c;
        h->tune = kCandidates[bi];
        h->gate_bins = gate0;
        reset_bins(h);
        if (best) *best = h->tune;
        for (int c = 0; c < kNumCandidates && ms && c < n_ms; c++) ms[c] = (float)tot[c];
        if (n_cand) *n_cand = kNumCandidates;
        cleanup();
        return DSPG_OK;
    } catch (const Err &e) {
        h->tune = keep;
        h->gate_bins = gate0;
        reset_bins(h);
        cleanup();
        return fail(h, e);
    }
}

dspg_status dspg_set_sizing(dspg_handle *h, int mode, const dspg_estimator *e, int32_t est_min, float margin) {
    if (!h) return DSPG_ERR_INVALID;
    if (h->pending) return fail(h, Err(DSPG_ERR_STATE, "an asynchronous batch is in flight"));
    try {
        if (mode != DSPG_SIZE_BOUND && mode != DSPG_SIZE_EXACT && mode != DSPG_SIZE_LEARNED)
            throw Err(DSPG_ERR_INVALID, "unknown sizing mode");
        if (mode == DSPG_SIZE_LEARNED) {
            if (!e) throw Err(DSPG_ERR_INVALID, "learned sizing needs an estimator");
            if (est_min < 0 || !(margin >= 0.0f) || margin > 1e6f) throw Err(DSPG_ERR_INVALID, "est_min and margin must be >= 0");
            h->est_w.reserve(EST_PARAMS);
            CK(cudaMemcpy(h->est_w.p, e->w, sizeof(uint16_t) * EST_PARAMS, cudaMemcpyDeviceToDevice));
            h->est_min = est_min;
            h->est_margin = margin;
        }
        h->sizing = mode;
        reset_bins(h);  // captured pipelines carry the old sizing
        return DSPG_OK;
    } catch (const Err &x) {
        return fail(h, x);
    }
}

dspg_status dspg_row_features(dspg_handle *h, const int32_t *rows, int64_t n, float *X, float *y, void *stream) {
    if (!h) return DSPG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    try {
        if (!X || n < 0) throw Err(DSPG_ERR_INVALID, "X is NULL or n < 0");
        if (!rows && n != h->A.nrows) throw Err(DSPG_ERR_INVALID, "rows == NULL needs n = nrows");
        DBuf<unsigned> bad;
        bad.reserve(1);
        CK(cudaMemsetAsync(bad.p, 0, sizeof(unsigned), s));
        row_features(h->A.view(), h->Bm().view(), h->C.view(), rows, n, X, y, bad.p, s);
        CK(cudaGetLastError());
        unsigned hb = 0;
        CK(cudaMemcpyAsync(&hb, bad.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hb) throw Err(DSPG_ERR_INVALID, "row index out of range");
        return DSPG_OK;
    } catch (const Err &x) {
        return fail(h, x);
    }
}

dspg_status dspg_footprint(dspg_handle *h, const dspg_updates *dA, uint32_t *f, uint32_t *u, int or_anyway,
                           int *admitted, int64_t *rows, void *stream) {
    if (!h) return DSPG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    try {
        if (h->pending) throw Err(DSPG_ERR_STATE, "an asynchronous batch is in flight");
        if (!dA || !f) throw Err(DSPG_ERR_INVALID, "dA and f must not be NULL");
        if (h->trans_a || h->trans_b || h->b_alias)
            throw Err(DSPG_ERR_INVALID, "footprints are not available for a product with transposed operands");
        if (u && !admitted) throw Err(DSPG_ERR_INVALID, "admitted must not be NULL when u is given");
        const int64_t n = dA->n;
        if (n < 0 || (n > 0 && (!dA->row || !dA->col))) throw Err(DSPG_ERR_INVALID, "bad batch");
        const int64_t words = (h->A.nrows + 31) / 32;
        FpWs &w = h->fp;
        w.cnt.reserve(4);  // out-of-range flag, overlapping words, rows of f
        w.hcnt.reserve_host(4);
        CK(cudaMemsetAsync(f, 0, sizeof(uint32_t) * words, s));
        CK(cudaMemsetAsync(w.cnt.p, 0, 4 * sizeof(unsigned long long), s));
        const int32_t *rp = dA->row, *cp = dA->col;
        if (n > 0 && !dA->on_device) {
            w.row.reserve(n);
            w.col.reserve(n);
            CK(cudaMemcpyAsync(w.row.p, dA->row, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(w.col.p, dA->col, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
            rp = w.row.p;
            cp = w.col.p;
        }
        if (n > 0)
            run_footprint(rp, cp, n, h->A.nrows, h->A.ncols, h->b_is_a, h->AT.view(), f, (unsigned *)w.cnt.p, s,
                          h->num_sms);
        run_bitmap_overlap(f, u, words, w.cnt.p + 1, s, h->num_sms);
        if (u) run_bitmap_or(f, u, words, w.cnt.p + 1, or_anyway, s, h->num_sms);
        CK(cudaMemcpyAsync(w.hcnt.p, w.cnt.p, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if ((unsigned)w.hcnt.p[0]) throw Err(DSPG_ERR_INVALID, "batch entry out of range");
        if (u) *admitted = w.hcnt.p[1] == 0 ? 1 : 0;
        if (rows) *rows = (int64_t)w.hcnt.p[2];
        return DSPG_OK;
    } catch (const Err &x) {
        return fail(h, x);
    }
}

dspg_status dspg_footprint_batch(dspg_handle *h, const dspg_updates *batches, int64_t k, uint32_t *f, uint32_t *u,
                                 int or_anyway, int *admitted, int64_t *rows, void *stream) {
    if (!h) return DSPG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    try {
        if (h->pending) throw Err(DSPG_ERR_STATE, "an asynchronous batch is in flight");
        if (k < 0 || (k > 0 && (!batches || !f || !u || !admitted))) throw Err(DSPG_ERR_INVALID, "NULL argument");
        if (h->trans_a || h->trans_b || h->b_alias)
            throw Err(DSPG_ERR_INVALID, "footprints are not available for a product with transposed operands");
        if (k == 0) return DSPG_OK;
        const int64_t words = (h->A.nrows + 31) / 32;
        int64_t host_entries = 0;
        for (int64_t j = 0; j < k; j++) {
            const int64_t n = batches[j].n;
            if (n < 0 || (n > 0 && (!batches[j].row || !batches[j].col))) throw Err(DSPG_ERR_INVALID, "bad batch");
            if (!batches[j].on_device) host_entries += n;
        }
        FpWs &w = h->fp;
        // [0] an entry out of range, [1] the stop flag, then per footprint:
        // overlapping words and bits set
        w.cnt.reserve(2 + 2 * k);
        w.hcnt.reserve_host(2 + 2 * k);
        w.row.reserve(std::max<int64_t>(host_entries, 1));
        w.col.reserve(std::max<int64_t>(host_entries, 1));
        CK(cudaMemsetAsync(f, 0, sizeof(uint32_t) * words * k, s));
        CK(cudaMemsetAsync(w.cnt.p, 0, (2 + 2 * k) * sizeof(unsigned long long), s));
        int64_t at = 0;
        for (int64_t j = 0; j < k; j++) {
            const dspg_updates &b = batches[j];
            const int32_t *rp = b.row, *cp = b.col;
            if (b.n > 0 && !b.on_device) {
                CK(cudaMemcpyAsync(w.row.p + at, b.row, sizeof(int32_t) * b.n, cudaMemcpyHostToDevice, s));
                CK(cudaMemcpyAsync(w.col.p + at, b.col, sizeof(int32_t) * b.n, cudaMemcpyHostToDevice, s));
                rp = w.row.p + at;
                cp = w.col.p + at;
                at += b.n;
            }
            uint32_t *fj = f + words * j;
            unsigned long long *cj = w.cnt.p + 2 + 2 * j;
            if (b.n > 0)
                run_footprint(rp, cp, b.n, h->A.nrows, h->A.ncols, h->b_is_a, h->AT.view(), fj, (unsigned *)w.cnt.p, s,
                              h->num_sms);
            run_bitmap_overlap(fj, u, words, cj, s, h->num_sms);
            run_bitmap_or(fj, u, words, cj, or_anyway, s, h->num_sms, (unsigned *)(w.cnt.p + 1));
        }
        CK(cudaMemcpyAsync(w.hcnt.p, w.cnt.p, (2 + 2 * k) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if ((unsigned)w.hcnt.p[0]) throw Err(DSPG_ERR_INVALID, "batch entry out of range");
        bool stop = false;
        for (int64_t j = 0; j < k; j++) {
            const bool hit = w.hcnt.p[2 + 2 * j] != 0;
            admitted[j] = (!stop && !hit) ? 1 : 0;
            if (hit && !or_anyway) stop = true;
            if (rows) rows[j] = (int64_t)w.hcnt.p[3 + 2 * j];
        }
        return DSPG_OK;
    } catch (const Err &x) {
        return fail(h, x);
    }
}

dspg_status dspg_group_create(dspg_group **out, dspg_handle *const *handles, int64_t n) {
    dspg_group *g = nullptr;
    try {
        if (!out) throw Err(DSPG_ERR_INVALID, "out is NULL");
        *out = nullptr;
        if (n < 0 || (n > 0 && !handles)) throw Err(DSPG_ERR_INVALID, "group needs n >= 0 handles");
        std::vector<dspg_handle *> hs(handles, handles + n);
        for (int64_t t = 0; t < n; t++) {
            if (!hs[t]) throw Err(DSPG_ERR_INVALID, "group member " + std::to_string(t) + " is NULL");
            if (hs[t]->bloom) throw Err(DSPG_ERR_STATE, "group member " + std::to_string(t) + " keeps a Bloom filter");
            for (int64_t u = 0; u < t; u++)
                if (hs[u] == hs[t]) throw Err(DSPG_ERR_INVALID, "group member " + std::to_string(t) + " repeats member " + std::to_string(u));
        }
        g = new dspg_group();
        g->hs = std::move(hs);
        CK(cudaStreamCreateWithFlags(&g->gs, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&g->evIn, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&g->evFork, cudaEventDisableTiming));
        *out = g;
        return DSPG_OK;
    } catch (const Err &e) {
        g_err = e.what();
        dspg_group_destroy(g);
        return e.st;
    }
}

dspg_status dspg_group_apply(dspg_group *g, const dspg_updates *dA, const dspg_updates *dB,
                             dspg_batch_stats *stats, dspg_status *status, void *stream) {
    if (!g) return DSPG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = g->hs.size();
    try {
        if (n > 0 && !dA) throw Err(DSPG_ERR_INVALID, "dA is NULL");
        // host-side checks and uploads for every member before anything runs
        std::vector<int64_t> key;
        std::vector<int64_t> comp0(n);
        key.reserve(3 * n);
        for (size_t t = 0; t < n; t++) {
            dspg_handle *h = g->hs[t];
            try {
                if (h->pending) throw Err(DSPG_ERR_STATE, "an asynchronous batch is in flight");
                prepare_batch(h, dA + t, dB ? dB + t : nullptr, s);
                // a member launches at the largest size it has seen (an
                // empty batch runs as a zero-length one), so that one
                // captured group pipeline serves every later combination of
                // batch sizes up to those
                h->grp_cap_a = std::max(h->grp_cap_a, h->inA.cap);
                h->grp_cap_b = std::max(h->grp_cap_b, h->inB.cap);
                h->inA.cap = h->grp_cap_a;
                h->inB.cap = h->b_is_a ? 0 : h->grp_cap_b;
                if (h->wA.ensure(h->inA.cap, h->A.arena_cap)) h->epoch++;
                if (!h->b_is_a && h->wB.ensure(h->inB.cap, h->B.arena_cap)) h->epoch++;
                if (h->has_at && h->wAT.ensure(h->inA.cap, h->AT.arena_cap)) h->epoch++;
            } catch (const Err &e) {
                h->err = e.what();
                throw Err(e.st, "member " + std::to_string(t) + ": " + e.what());
            }
            comp0[t] = h->compactions;
            key.push_back(h->inA.cap);
            key.push_back(h->inB.cap);
            key.push_back((int64_t)h->epoch);
        }
        const bool use_graphs = n > 0 && g->hs[0]->use_graphs;
        dspg_group::Graph *hit = nullptr;
        for (auto &x : g->graphs)
            if (x.key == key) hit = &x;
        bool seen = false;
        for (auto &k : g->seen) seen |= (k == key);
        if (use_graphs && !hit && seen) {
            unsigned long long nk = 0;
            cudaGraphExec_t exec = capture_graph(g->gs, &nk, [&] {
                CK(cudaEventRecord(g->evFork, g->gs));
                for (dspg_handle *h : g->hs) {
                    CK(cudaStreamWaitEvent(h->gs, g->evFork, 0));
                    begin_batch(h->h_args_dev, h->d_args, h->ctl, h->gs);
                    pipeline(h, h->gs, false, true);
                    end_batch(h->ctl, h->hctl_dev, h->gs);
                    CK(cudaEventRecord(h->evIn, h->gs));
                    CK(cudaStreamWaitEvent(g->gs, h->evIn, 0));
                }
            });
            if (g->graphs.size() >= 4) {
                cudaGraphExecDestroy(g->graphs.front().exec);
                g->graphs.erase(g->graphs.begin());
            }
            // the capture counted the kernels once: that is this first replay
            __atomic_fetch_sub(&launch_counter(), nk, __ATOMIC_RELAXED);
            g->graphs.push_back(dspg_group::Graph{key, exec, nk});
            hit = &g->graphs.back();
        }
        if (hit) {
            for (dspg_handle *h : g->hs) h->runs_replayed++;
            CK(cudaEventRecord(g->evIn, s));
            CK(cudaStreamWaitEvent(g->gs, g->evIn, 0));
            CK(cudaGraphLaunch(hit->exec, g->gs));
            __atomic_fetch_add(&launch_counter(), hit->kernels, __ATOMIC_RELAXED);
            CK(cudaEventRecord(g->evIn, g->gs));
            CK(cudaStreamWaitEvent(s, g->evIn, 0));
            CK(cudaStreamSynchronize(g->gs));
        } else {
            if (use_graphs) {
                if (g->seen.size() >= 8) g->seen.erase(g->seen.begin());
                g->seen.push_back(key);
            }
            CK(cudaEventRecord(g->evFork, s));
            for (dspg_handle *h : g->hs) {
                h->runs_eager++;
                CK(cudaStreamWaitEvent(h->gs, g->evFork, 0));
                begin_batch(h->h_args_dev, h->d_args, h->ctl, h->gs);
                pipeline(h, h->gs, false, false);
                CK(cudaMemcpyAsync(h->hctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->gs));
                CK(cudaEventRecord(h->evIn, h->gs));
                CK(cudaStreamWaitEvent(s, h->evIn, 0));
            }
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(s));
        }
        // members that overflowed a buffer are grown and re-run one by one
        dspg_status first = DSPG_OK;
        g->err.clear();
        for (size_t t = 0; t < n; t++) {
            dspg_handle *h = g->hs[t];
            dspg_status st = DSPG_OK;
            try {
                recover(h, s);
                est_fallback(h, s);
                fill_stats(h, stats ? stats + t : nullptr, comp0[t]);
            } catch (const Err &e) {
                h->err = e.what();
                st = e.st;
                if (first == DSPG_OK) {
                    first = st;
                    g->err = "member " + std::to_string(t) + ": " + e.what();
                }
                if (st == DSPG_ERR_CUDA) throw;
            }
            if (status) status[t] = st;
        }
        return first;
    } catch (const Err &e) {
        g->err = e.what();
        if (status)
            for (size_t t = 0; t < n; t++) status[t] = e.st;
        return e.st;
    }
}

void dspg_group_destroy(dspg_group *g) {
    if (!g) return;
    if (g->gs) cudaStreamSynchronize(g->gs);
    for (auto &x : g->graphs) cudaGraphExecDestroy(x.exec);
    if (g->evIn) cudaEventDestroy(g->evIn);
    if (g->evFork) cudaEventDestroy(g->evFork);
    if (g->gs) cudaStreamDestroy(g->gs);
    delete g;
}

const char *dspg_group_last_error(const dspg_group *g) { return g ? g->err.c_str() : g_err.c_str(); }

void dspg_destroy(dspg_handle *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    for (int k = 0; k < 10; k++)
        if (h->pev[k]) cudaEventDestroy(h->pev[k]);
    for (cudaEvent_t e : {h->evIn, h->evFork, h->evDetect, h->evSide, h->evSize})
        if (e) cudaEventDestroy(e);
    for (int k = 0; k < NUM_SIDE; k++) {
        if (h->evNum[k]) cudaEventDestroy(h->evNum[k]);
        if (h->nstr[k]) cudaStreamDestroy(h->nstr[k]);
    }
    for (cudaStream_t st : {h->gs, h->side})
        if (st) cudaStreamDestroy(st);
    if (h->ctl) cudaFree(h->ctl);
    if (h->hctl) cudaFreeHost(h->hctl);
    if (h->d_args) cudaFree(h->d_args);
    if (h->h_args) cudaFreeHost(h->h_args);
    delete h;
}

const char *dspg_last_error(const dspg_handle *h) { return h ? h->err.c_str() : g_err.c_str(); }

}  // extern "C"
