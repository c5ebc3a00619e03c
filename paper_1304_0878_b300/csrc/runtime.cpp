// Host side of the b3t C ABI: handles, codelets, dependency derivation,
// task-table build, launch, wait and graph capture.
//
// The model (Section 2 of the paper): tasks with declared implementations and
// per-buffer access modes; registered buffers; asynchronous invocation; the
// dependency graph follows from the access modes and the invocation order;
// a wait joins everything.  Submissions accumulate in a pending batch; a
// flush turns the batch into one task table + CSR successor graph and runs
// it in one persistent-kernel launch on the context's stream.
#include "b3t.h"
#include "b3t_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cerrno>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace b3t;

namespace {

struct Handle {
    void *ptr = nullptr;
    size_t nelems = 0, elemsize = 0;
    int64_t ld = 0;
    bool alive = false;
    int32_t parent = -1;
    std::vector<int32_t> parts;
    // dependency state of a leaf within the pending batch
    int32_t last_writer = -1;
    std::vector<int32_t> readers;
    bool touched = false;
};

struct Codelet {
    std::string name;
    int kind = 0;
    int nbuf = 0;
    uint8_t modes[kMaxBuffers] = {0, 0, 0, 0};
    size_t scalar_bytes = 0;
};

struct Pending {
    TaskRec rec;
    float cost;
};

// Device arena of one launch (task table, graph, counters, rings, status).
struct Arena {
    TaskRec *tasks = nullptr;  size_t cap_tasks = 0;
    int32_t *succ = nullptr;   size_t cap_succ = 0;
    int32_t *indeg = nullptr;  int32_t *counters = nullptr; int32_t *done = nullptr;
    int32_t *next = nullptr;
    size_t cap_cnt = 0;
    unsigned long long *slots = nullptr; size_t cap_slots = 0;
    unsigned long long *roots = nullptr; size_t cap_roots = 0;
    Ctl *ctl = nullptr;

    void release() {
        cudaFree(tasks); cudaFree(succ); cudaFree(indeg); cudaFree(counters);
        cudaFree(done); cudaFree(next); cudaFree(slots); cudaFree(roots); cudaFree(ctl);
        *this = Arena();
    }
};

template <class T>
int grow(T *&p, size_t &cap, size_t need) {
    if (need <= cap && p) return 0;
    size_t n = std::max<size_t>(need, std::max<size_t>(cap * 2, 64));
    if (p) { cudaFree(p); p = nullptr; cap = 0; }
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) { p = nullptr; return -ENOMEM; }
    cap = n;
    return 0;
}

struct GraphRec {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Arena arena;
    int64_t ntasks = 0, nitems = 0;
    int nctas = 0;
    bool alive = false;
};

// Signature of each kind: buffers, modes, element sizes, scalar blob size.
struct KindSig {
    int nbuf;
    uint8_t modes[kMaxBuffers];
    int elem[kMaxBuffers];     // element size in bytes; 1 = quantised tile
    size_t scalar_bytes;
    bool tile;
};

const KindSig kSigs[kNumKinds] = {
    /* NOOP     */ {-1, {0, 0, 0, 0}, {0, 0, 0, 0}, 0, false},
    /* SCAL_F32 */ {1, {B3T_RW}, {4}, 4, false},
    /* POTRF    */ {1, {B3T_RW}, {8}, 4, true},
    /* TRSM     */ {2, {B3T_R, B3T_RW}, {8, 8}, 0, true},
    /* SYRK     */ {2, {B3T_R, B3T_RW}, {8, 8}, 0, true},
    /* GEMM     */ {3, {B3T_R, B3T_R, B3T_RW}, {8, 8, 8}, 0, true},
    /* POTRF_MX */ {2, {B3T_R, B3T_W}, {4, 8}, 4, true},
    /* TRSM_MX  */ {3, {B3T_R, B3T_R, B3T_W}, {8, 4, 8}, 0, true},
    /* SYRK_MX  */ {2, {B3T_R, B3T_RW}, {1, 4}, 4, true},
    /* GEMM_MX  */ {3, {B3T_R, B3T_R, B3T_RW}, {1, 1, 4}, 4, true},
    /* QUANT    */ {2, {B3T_R, B3T_W}, {8, 1}, 4, true},
    /* TRSV_L   */ {2, {B3T_R, B3T_RW}, {8, 8}, sizeof(VecArgs), false},
    /* GEMV_L   */ {3, {B3T_R, B3T_R, B3T_RW}, {8, 8, 8}, sizeof(VecArgs), false},
    /* TRSV_LT  */ {2, {B3T_R, B3T_RW}, {8, 8}, sizeof(VecArgs), false},
    /* GEMV_LT  */ {3, {B3T_R, B3T_R, B3T_RW}, {8, 8, 8}, sizeof(VecArgs), false},
    /* AXPY     */ {2, {B3T_RW, B3T_R}, {8, 8}, sizeof(VecArgs), false},
    /* RESID    */ {4, {B3T_R, B3T_R, B3T_R, B3T_W}, {8, 8, 8, 8}, sizeof(VecArgs), false},
    /* NRM      */ {3, {B3T_R, B3T_R, B3T_W}, {8, 8, 8}, sizeof(VecArgs), false},
    /* POTRF_D  */ {1, {B3T_RW}, {8}, sizeof(PanelArgs), false},
    /* PANEL_TR */ {1, {B3T_RW}, {8}, sizeof(PanelArgs), false},
    /* PANEL_UP */ {2, {B3T_R, B3T_RW}, {8, 8}, sizeof(PanelArgs), false},
    /* CVT      */ {2, {B3T_R, B3T_W}, {4, 8}, 0, true},
    /* TRTRI    */ {2, {B3T_R, B3T_W}, {8, 8}, 0, true},
    /* TRMM_MX  */ {3, {B3T_R, B3T_R, B3T_W}, {8, 4, 8}, 0, true},
    /* SLICE_A  */ {3, {B3T_R, B3T_W, B3T_W}, {8, 1, 1}, sizeof(SliceArgs), false},
    /* SLICE_X  */ {2, {B3T_R, B3T_W}, {8, 1}, sizeof(SliceArgs), false},
    /* RESID_SL */ {4, {B3T_R, B3T_R, B3T_R, B3T_W}, {1, 1, 8, 8}, sizeof(SliceArgs), false},
    /* SLICE_W  */ {2, {B3T_R, B3T_W}, {4, 1}, 0, false},
    /* SLICE_U  */ {2, {B3T_R, B3T_W}, {8, 1}, 0, false},
    /* TRMM_SL  */ {3, {B3T_R, B3T_R, B3T_W}, {1, 1, 8}, 0, false},
    /* TRTRI_CO */ {3, {B3T_R, B3T_R, B3T_W}, {8, 8, 8}, sizeof(PanelArgs), false},
};

const char *kKindNames[kNumKinds] = {"noop", "scal_f32", "potrf", "trsm", "syrk", "gemm",
                                     "potrf_mx", "trsm_mx", "syrk_mx", "gemm_mx", "quant",
                                     "trsv_l", "gemv_l", "trsv_lt", "gemv_lt", "axpy", "resid", "nrm",
                                     "potrf_d", "panel_trsm", "panel_upd", "cvt", "trtri", "trmm_mx",
                                     "slice_a", "slice_x", "resid_sl", "slice_w", "slice_u", "trmm_sl",
                                     "trtri_col"};
bool is_panel(int kind) { return (kind >= kPotrfD && kind <= kPanelUpd) || kind == kTrtriCol; }
bool is_vec(int kind) { return kind >= kTrsvL && kind <= kNrm; }

bool is_mx(int kind) { return kind == kSyrkMx || kind == kGemmMx || kind == kResidSl || kind == kTrmmSl; }
bool is_slice(int kind) { return kind >= kSliceA && kind <= kResidSl; }
bool has_fmt(int kind) { return kind == kSyrkMx || kind == kGemmMx || kind == kQuant; }

// fine: the split of a small launch (build_launch decides) for tiles of at
// most kSmallTile rows; the device tells the two splits apart by the item
// count
int64_t items_of(int kind, int64_t n, bool fine = false) {
    fine = fine && n <= kSmallTile;
    switch (kind) {
    case kScalF32: return std::max<int64_t>(1, (n + kScalChunk - 1) / kScalChunk);
    case kPotrf: case kPotrfMx: case kNoop: return 1;
    case kCvt: return n / kCvtCols;
    case kQuant: return 1;   // set from the format at submit (one item per 16 KiB chunk)
    case kTrsm: return fine ? n / kSmallTrsmRows : n / kTrsmRows;
    case kTrsmMx: return n / kTrsmRows;
    case kTrtri: return n / kTrtriRows;
    case kSyrk: {
        int64_t m = n / kGemmBlk;
        return fine ? (n / kSmallGemmRows) * m : m * (m + 1) / 2;
    }
    case kGemm: {
        int64_t m = n / kGemmBlk;
        return fine ? (n / kSmallGemmRows) * m : m * m;
    }
    case kTrmmMx: return (n / kTrmmRows) * (n / kGemmBlk);
    case kSyrkMx: { int64_t m = n / kMxBlk; return m * (m + 1) / 2; }
    case kGemmMx: { int64_t m = n % kMxWideBlk == 0 ? n / kMxWideBlk : n / kMxBlk; return m * m; }
    case kGemvL: case kGemvLT: return n / kGemvRows;
    case kResid: return n / kResidRows;
    case kAxpy: case kNrm: return 1;
    case kSliceA: case kSliceX: return 1;
    case kResidSl: return n / kSlRows;
    case kSliceW: return n / 128;
    case kSliceU: return n / kTsCols;
    case kTrmmSl: return (n / 128) * (n / kTsCols);
    }
    return 1;
}

// Rough device time of a task in ns on one CTA, only used to rank tasks by
// their distance to the end of the graph (upward rank, the scheduling hint
// Section 5.3 of the paper proposes).
float cost_of(int kind, int64_t n, int nrhs = 1, int T = 1, bool f32 = false) {
    double b = (double)n;
    const double vec = f32 ? 60.0 : 3.7;
    const double fp64 = 3.7;   // flop / ns per CTA (FP64 DFMA, 2 CTAs / SM)
    const double mx = 2000.0;  // flop / ns per CTA (tensor cores)
    switch (kind) {
    case kScalF32: return (float)(8.0 * b / 20.0);
    case kPotrf: case kPotrfMx: return (float)(b * b * b / 3.0 / fp64);
    case kTrsm: case kTrsmMx: case kTrmmMx: return (float)(b * b * b / fp64);
    case kSyrk: return (float)(b * b * b / fp64);
    case kGemm: return (float)(2.0 * b * b * b / fp64);
    case kSyrkMx: return (float)(b * b * b / mx + 4.0 * b * b / 20.0);
    case kGemmMx: return (float)(2.0 * b * b * b / mx + 8.0 * b * b / 20.0);
    case kQuant: return (float)(10.0 * b * b / 20.0);
    case kTrsvL: case kTrsvLT: return (float)(b * b / vec + 32.0 * b / 32.0 * 20.0);
    case kGemvL: case kGemvLT: return (float)(2.0 * b * b * nrhs / vec + 8.0 * b * b / 20.0);
    case kAxpy: return (float)(b * nrhs / 10.0 + 1000.0);
    case kResid: return (float)(2.0 * b * b * T * nrhs / 3.7);
    case kNrm: return 5000.0f;
    case kCvt: return (float)(12.0 * b * b / 20.0);
    case kTrtri: return (float)(b * b * b / fp64);    // the first item's share dominates
    case kSliceA: return (float)(2.0 * b * b / 4.0 + b * b / fp64);
    case kSliceX: return (float)(16.0 * b / 4.0 + 2000.0);
    case kResidSl: return (float)(T * b * 50.0);
    case kSliceW: case kSliceU: return (float)(b * b / 20.0 + 5000.0);
    case kTrmmSl: return (float)(b * 60.0 + 5000.0);
    }
    return 1000.0f;
}

size_t q_bytes(int b, int fmt) {
    size_t elems = (size_t)b * b;
    return (fmt == B3T_FMT_BF16 ? elems * 2 : elems) + 16;
}

}  // namespace

struct b3t_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    b3t_config cfg{};
    std::vector<Handle> handles;
    std::unordered_map<uintptr_t, int32_t> by_ptr;
    std::vector<Codelet> codelets;
    std::vector<Pending> tasks;
    std::vector<std::pair<int32_t, int32_t>> edges;
    std::vector<int32_t> extra_deps;        // phantom predecessors (tests)
    std::vector<int32_t> touched;
    bool capturing = false;
    Arena arena;
    // pinned staging for uploads, reused once the previous copy completed
    void *staging = nullptr; size_t staging_cap = 0;
    cudaEvent_t staging_done = nullptr;
    // pinned mirrors of the status blocks of launches since the last wait
    std::vector<Ctl *> mirrors;
    std::vector<std::pair<Ctl *, Ctl *>> inflight;   // (device ctl, mirror)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int64_t last_ntasks = 0, last_nitems = 0;
    int last_nctas = 0;
    bool last_timed = false;
    int32_t err_task = -1, err_info = -1;
    std::vector<GraphRec> graphs;
    b3t_codelet kind_cl[kNumKinds];
    // tracing: one record per finished work item of the launches built
    // while it is on (device buffer; the count is the first 8 bytes)
    TraceRec *trace = nullptr;
    unsigned long long *trace_n = nullptr;
    int64_t trace_cap = 0;
    bool trace_on = false;
    // stream mode: one resident kernel fed with task graphs while it runs
    struct Stream {
        bool open = false;
        cudaStream_t feed = nullptr;
        cudaEvent_t staged = nullptr;
        int64_t max_tasks = 0, max_edges = 0;
        int32_t max_batches = 0;
        TaskRec *tasks = nullptr;
        int32_t *succ = nullptr, *level = nullptr, *counters = nullptr, *done = nullptr, *next = nullptr;
        int32_t *task_batch = nullptr, *batch_left = nullptr, *batch_info = nullptr;
        unsigned long long *slots = nullptr, *sroots = nullptr;
        SubDesc *subs = nullptr;
        StreamCtl *sctl = nullptr;
        Ctl *ctl = nullptr;
        int32_t *done_h = nullptr;            // host-mapped batch status
        int32_t *done_d = nullptr;
        void *staging = nullptr;
        size_t staging_cap = 0;
        int64_t ntasks = 0, nedges = 0, nroots = 0;
        int32_t nbatches = 0;
        std::vector<int32_t> handle_batch;    // last batch that used each handle
    } st;
};

namespace {

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return 0;
    if (e == cudaErrorMemoryAllocation) return -ENOMEM;
    return -EIO;
}

void reset_dep_state(b3t_ctx *c) {
    for (int32_t h : c->touched) {
        Handle &H = c->handles[h];
        H.last_writer = -1;
        H.readers.clear();
        H.touched = false;
    }
    c->touched.clear();
}

// Section 2: access modes + invocation order -> RAW / WAR / WAW edges.
void derive(b3t_ctx *c, int32_t t, const int32_t *leaves, const uint8_t *modes, int n,
            std::vector<int32_t> &preds) {
    preds.clear();
    for (int i = 0; i < n; ++i) {
        Handle &H = c->handles[leaves[i]];
        if (!H.touched) { H.touched = true; c->touched.push_back(leaves[i]); }
        if (modes[i] & B3T_W) {
            if (!H.readers.empty()) {
                for (int32_t r : H.readers) if (r != t) preds.push_back(r);
            } else if (H.last_writer >= 0 && H.last_writer != t) {
                preds.push_back(H.last_writer);
            }
            H.last_writer = t;
            H.readers.clear();
        } else {
            if (H.last_writer >= 0 && H.last_writer != t) preds.push_back(H.last_writer);
            H.readers.push_back(t);
        }
    }
    std::sort(preds.begin(), preds.end());
    preds.erase(std::unique(preds.begin(), preds.end()), preds.end());
}

// Priority of every task of the pending batch (higher level = claimed first):
//   critical path first (default): the tasks whose downward plus upward rank
//   is the graph's longest path on the top level, the others bucketed by
//   upward rank below it (Section 5.3's scheduling hints);
//   upward rank: the longest cost-weighted path from the task to the end of
//   the graph, the task's own cost included, bucketed linearly into L levels;
//   depth: the longest path from a source, in tasks (successor first).
// off/succ: CSR successor lists of the batch (successors are later tasks).
void compute_levels(const b3t_ctx *c, const std::vector<int32_t> &off, const int32_t *succ,
                    std::vector<float> &rank, std::vector<int32_t> &level);

// Rings per priority level of a launch: as many as the claiming warp reads in
// one round trip (64 rings: 8 per level with 8 levels, 64 with one);
// B3T_SUB_RINGS overrides it (1 .. that number), for measurements.
int sub_rings(const b3t_ctx *c) {
    const int most = kMaxRings / std::max(1, c->cfg.prio_levels);
    int n = most;
    if (const char *e = std::getenv("B3T_SUB_RINGS")) {
        const int v = std::atoi(e);
        if (v >= 1 && v <= most) n = v;
    }
    return n;
}

// Item chains (config item_chains; Section 2's scheduler that sees only part
// of the graph, applied at item granularity): a SCAL task t whose only
// successor s is a SCAL task on the same buffer and length, s having no
// other predecessor, is linked to s; item i of s reads exactly what item i of
// t wrote.  A maximal run of links becomes one chain of up to kMaxChain
// absorbed members after its head: the CTA that runs item i of the head
// applies every member's factor to the chunk, in order, before storing it.
// Members are never queued (their one predecessor's retirement releases
// nothing); each retires when its last item is done, and the last member
// releases the chain's outgoing edges.  chain_aux[t]: k members (head), -1
// (member), 0; chain_at[head]: offset in succ_lv of the members' ids, then
// of their factor bits (appended to succ_lv).
static void find_item_chains(const b3t_ctx *c, const std::vector<int32_t> &off, const int32_t *succ,
                             const std::vector<int32_t> &indeg, std::vector<int32_t> &chain_aux,
                             std::vector<int32_t> &chain_at, std::vector<int32_t> &succ_lv) {
    const int64_t nt = (int64_t)c->tasks.size();
    std::vector<int32_t> nxt(nt, -1);
    std::vector<char> linked(nt, 0);
    bool any = false;
    for (int64_t t = 0; t < nt; ++t) {
        const TaskRec &r = c->tasks[t].rec;
        if (r.kind != kScalF32 || off[t + 1] - off[t] != 1) continue;
        const int32_t sx = succ[off[t]];
        const TaskRec &q = c->tasks[sx].rec;
        if (q.kind != kScalF32 || indeg[sx] != 1 || q.buf[0] != r.buf[0] || q.n != r.n || q.nitems != r.nitems)
            continue;
        nxt[t] = sx;
        linked[sx] = 1;
        any = true;
    }
    if (!any) return;
    chain_aux.assign(nt, 0);
    chain_at.assign(nt, 0);
    std::vector<int32_t> mem;
    for (int64_t t = 0; t < nt; ++t) {
        if (nxt[t] < 0 || linked[t]) continue;
        // t heads a run of links; cut it into chains of at most kMaxChain members
        int32_t h = (int32_t)t;
        while (h >= 0 && nxt[h] >= 0) {
            mem.clear();
            int32_t m = nxt[h];
            while (m >= 0 && (int)mem.size() < kMaxChain) {
                mem.push_back(m);
                m = nxt[m];
            }
            chain_aux[h] = (int32_t)mem.size();
            chain_at[h] = (int32_t)succ_lv.size();
            for (int32_t x : mem) {
                chain_aux[x] = -1;
                succ_lv.push_back(x);
            }
            for (int32_t x : mem) succ_lv.push_back((int32_t)c->tasks[x].rec.scal);
            // a cut run continues with the next task as a new head, released
            // by the last member like any successor
            h = m;
        }
    }
}

// Build the task table, CSR graph, ready rings and root lists of the pending
// batch into arena `a` (uploaded through the pinned staging buffer on the
// context's stream) and fill the launch parameters.
int build_launch(b3t_ctx *c, Arena &a, InitParams &ip, LaunchParams &lp, int64_t &nitems_out,
                 bool &has_mx) {
    const int64_t nt = (int64_t)c->tasks.size();
    // a small launch (one factorisation of a few thousand rows, bound by its
    // critical path) splits FP64 TRSM / SYRK / GEMM tasks on tiles of at
    // most kSmallTile rows finer, so that one task spreads over more SMs;
    // large launches (many factorisations, big T) keep the coarse split
    const bool fine = nt <= kFineLaunchTasks;
    for (auto &tk : c->tasks) {
        TaskRec &r = tk.rec;
        if ((r.kind == kTrsm || r.kind == kSyrk || r.kind == kGemm) && r.n <= kSmallTile)
            r.nitems = (int32_t)items_of(r.kind, r.n, fine);
    }
    const int64_t ne = (int64_t)c->edges.size();
    const int L = c->cfg.prio_levels;
    std::vector<int32_t> off(nt + 1, 0), indeg(nt, 0);
    for (auto &e : c->edges) { off[e.first + 1]++; indeg[e.second]++; }
    for (int64_t t = 0; t < nt; ++t) off[t + 1] += off[t];
    const int64_t ne_pad = std::max<int64_t>(ne, 1);
    // device layout of the succ buffer: [successors (ne_pad)] [level (nt)]
    // [item chains: per head, its members' ids then their factor bits]
    std::vector<int32_t> succ_lv(ne_pad + nt, 0);
    {
        std::vector<int32_t> pos(off.begin(), off.end() - 1);
        for (auto &e : c->edges) succ_lv[pos[e.first]++] = e.second;
    }
    for (int64_t t = 0; t < nt && t < (int64_t)c->extra_deps.size(); ++t) indeg[t] += c->extra_deps[t];
    uint32_t fams0 = 0;
    for (int64_t t = 0; t < nt; ++t) fams0 |= family_of(c->tasks[t].rec.kind);
    std::vector<int32_t> chain_aux, chain_at;
    if (c->cfg.item_chains && !(variant_of(fams0) & kFamMx))
        find_item_chains(c, off, succ_lv.data(), indeg, chain_aux, chain_at, succ_lv);
    std::vector<float> rank;
    std::vector<int32_t> level;
    compute_levels(c, off, succ_lv.data(), rank, level);
    // ring of task t: level * nsub + t % nsub (the device pushes successors
    // by the same rule); capacities and roots are counted per ring
    const int nsub = sub_rings(c);
    const int NR = L * nsub;
    unsigned long long cap[kMaxRings] = {0}, rootcnt[kMaxRings] = {0};
    int64_t nitems = 0;
    has_mx = false;
    uint32_t fams = 0;
    for (int64_t t = 0; t < nt; ++t) {
        TaskRec &r = c->tasks[t].rec;
        r.succ_off = off[t];
        r.nsucc = off[t + 1] - off[t];
        const int lv = level[t];
        succ_lv[ne_pad + t] = lv;
        const int ring = lv * nsub + (int)(t % nsub);
        cap[ring] += 1;
        if (indeg[t] == 0) rootcnt[ring] += 1;
        nitems += r.nitems;
        if (is_mx(r.kind)) has_mx = true;
        fams |= family_of(r.kind);
    }
    unsigned long long ringoff[kMaxRings] = {0}, rootoff[kMaxRings] = {0};
    unsigned long long nslots = 0, nroots = 0;
    for (int l = 0; l < NR; ++l) {
        ringoff[l] = nslots; nslots += cap[l];
        rootoff[l] = nroots; nroots += rootcnt[l];
    }
    std::vector<unsigned long long> roots(std::max<unsigned long long>(nroots, 1), kEmpty);
    {
        unsigned long long fill[kMaxRings];
        for (int l = 0; l < NR; ++l) fill[l] = rootoff[l];
        for (int64_t t = 0; t < nt; ++t)
            if (indeg[t] == 0) roots[fill[succ_lv[ne_pad + t] * nsub + (int)(t % nsub)]++] =
                                   pack_slot(t, c->tasks[t].rec.nitems);
    }
    int rc;
    if ((rc = grow(a.tasks, a.cap_tasks, nt))) return rc;
    if ((rc = grow(a.succ, a.cap_succ, succ_lv.size()))) return rc;
    if ((size_t)nt > a.cap_cnt || !a.indeg) {
        size_t n = std::max<size_t>(nt, std::max<size_t>(a.cap_cnt * 2, 64));
        cudaFree(a.indeg); cudaFree(a.counters); cudaFree(a.done); cudaFree(a.next);
        a.indeg = a.counters = a.done = a.next = nullptr; a.cap_cnt = 0;
        if (cudaMalloc(&a.indeg, n * 4) != cudaSuccess || cudaMalloc(&a.counters, n * 4) != cudaSuccess ||
            cudaMalloc(&a.done, n * 4) != cudaSuccess || cudaMalloc(&a.next, n * 4) != cudaSuccess)
            return -ENOMEM;
        a.cap_cnt = n;
    }
    if ((rc = grow(a.slots, a.cap_slots, std::max<unsigned long long>(nslots, 1)))) return rc;
    if ((rc = grow(a.roots, a.cap_roots, roots.size()))) return rc;
    if (!a.ctl) {
        if (cudaMalloc(&a.ctl, sizeof(Ctl)) != cudaSuccess) return -ENOMEM;
        if ((rc = cuda_err(cudaMemsetAsync(a.ctl, 0, sizeof(Ctl), c->stream)))) return rc;
    }
    // staging: tasks | succ_lv | indeg | roots
    const size_t o_t = 0, o_s = o_t + nt * sizeof(TaskRec), o_i = o_s + succ_lv.size() * 4,
                 o_r = (o_i + nt * 4 + 15) / 16 * 16, bytes = o_r + roots.size() * 8;
    if (c->staging) cudaEventSynchronize(c->staging_done);
    if (bytes > c->staging_cap) {
        if (c->staging) cudaFreeHost(c->staging);
        c->staging = nullptr;
        const size_t cap2 = std::max(bytes, c->staging_cap * 2);
        if (cudaMallocHost(&c->staging, cap2) != cudaSuccess) { c->staging_cap = 0; return -ENOMEM; }
        c->staging_cap = cap2;
    }
    char *s = (char *)c->staging;
    for (int64_t t = 0; t < nt; ++t) std::memcpy(s + o_t + t * sizeof(TaskRec), &c->tasks[t].rec, sizeof(TaskRec));
    // item chains: the head's aux counts its members, buf[1] points at their
    // ids (then their factor bits) in the uploaded succ buffer; members get -1
    for (int64_t t = 0; t < (int64_t)chain_aux.size(); ++t) {
        if (!chain_aux[t]) continue;
        TaskRec *r = reinterpret_cast<TaskRec *>(s + o_t + t * sizeof(TaskRec));
        r->aux = chain_aux[t];
        if (chain_aux[t] > 0) r->buf[1] = (uint64_t)(uintptr_t)(a.succ + chain_at[t]);
    }
    std::memcpy(s + o_s, succ_lv.data(), succ_lv.size() * 4);
    std::memcpy(s + o_i, indeg.data(), nt * 4);
    std::memcpy(s + o_r, roots.data(), roots.size() * 8);
    cudaMemcpyAsync(a.tasks, s + o_t, nt * sizeof(TaskRec), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(a.succ, s + o_s, succ_lv.size() * 4, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(a.indeg, s + o_i, nt * 4, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(a.roots, s + o_r, roots.size() * 8, cudaMemcpyHostToDevice, c->stream);
    if ((rc = cuda_err(cudaEventRecord(c->staging_done, c->stream)))) return rc;

    ip = InitParams{};
    ip.indeg = a.indeg; ip.counters = a.counters; ip.done_items = a.done; ip.next_item = a.next;
    ip.slots = a.slots; ip.nslots = nslots; ip.roots = a.roots; ip.ctl = a.ctl;
    ip.ntasks = nt; ip.nlevels = L; ip.nrings = NR;
    lp = LaunchParams{};
    lp.tasks = a.tasks; lp.succ = a.succ; lp.level = a.succ + ne_pad;
    lp.counters = a.counters; lp.done_items = a.done; lp.next_item = a.next;
    lp.slots = a.slots; lp.ctl = a.ctl; lp.ntasks = nt; lp.nlevels = L; lp.nsub = nsub;
    lp.has_mx = has_mx ? 1 : 0;
    lp.variant = variant_of(fams);
    lp.fams = fams;
    lp.timeout_ns = c->cfg.timeout_ns;
    lp.debug = c->cfg.debug_checks;
    if (c->trace_on) { lp.trace = c->trace; lp.trace_n = c->trace_n; lp.trace_cap = c->trace_cap; }
    for (int l = 0; l < NR; ++l) {
        ip.root_off[l] = rootoff[l]; ip.root_cnt[l] = rootcnt[l];
        lp.ring_off[l] = ringoff[l]; lp.ring_cap[l] = cap[l];
    }
    nitems_out = nitems;
    return 0;
}

void compute_levels(const b3t_ctx *c, const std::vector<int32_t> &off, const int32_t *succ,
                    std::vector<float> &rank, std::vector<int32_t> &level) {
    const int64_t nt = (int64_t)c->tasks.size();
    const int L = c->cfg.prio_levels;
    rank.assign(nt, 0.f);
    level.assign(nt, 0);
    float maxr = 0.f;
    std::vector<char> crit;
    if (c->cfg.prio_policy == B3T_PRIO_DEPTH) {
        for (int64_t t = 0; t < nt; ++t) {
            for (int32_t k = off[t]; k < off[t + 1]; ++k) rank[succ[k]] = std::max(rank[succ[k]], rank[t] + 1.f);
            maxr = std::max(maxr, rank[t]);
        }
    } else if (c->cfg.prio_policy == B3T_PRIO_CRITICAL) {
        // upward rank (longest path from t to the end, t's cost included)
        // and downward rank (longest path from a source to t, t's cost
        // excluded) in double; their sum is the longest path through t, and
        // the tasks whose sum is the graph's longest path (no slack) go on
        // the top level
        std::vector<double> up(nt, 0.0), down(nt, 0.0);
        double longest = 0.0;
        for (int64_t t = nt - 1; t >= 0; --t) {
            double m = 0.0;
            for (int32_t k = off[t]; k < off[t + 1]; ++k) m = std::max(m, up[succ[k]]);
            up[t] = (double)c->tasks[t].cost + m;
            rank[t] = (float)up[t];
            maxr = std::max(maxr, rank[t]);
            longest = std::max(longest, up[t]);
        }
        for (int64_t t = 0; t < nt; ++t)
            for (int32_t k = off[t]; k < off[t + 1]; ++k)
                down[succ[k]] = std::max(down[succ[k]], down[t] + (double)c->tasks[t].cost);
        crit.assign(nt, 0);
        for (int64_t t = 0; t < nt; ++t) crit[t] = down[t] + up[t] >= longest * (1.0 - 1e-9);
    } else {
        for (int64_t t = nt - 1; t >= 0; --t) {
            float m = 0.f;
            for (int32_t k = off[t]; k < off[t + 1]; ++k) m = std::max(m, rank[succ[k]]);
            rank[t] = c->tasks[t].cost + m;
            maxr = std::max(maxr, rank[t]);
        }
    }
    if (L <= 1 || !(maxr > 0.f)) return;
    for (int64_t t = 0; t < nt; ++t)
        level[t] = c->cfg.prio_policy == B3T_PRIO_DEPTH
                       ? std::min(L - 1, (int)rank[t])
                   : !crit.empty()
                       ? (crit[t] ? L - 1 : std::min(L - 2, (int)((double)(L - 1) * rank[t] / (maxr * 1.000001))))
                       : std::min(L - 1, (int)((double)L * rank[t] / (maxr * 1.000001)));
}

int grid_for(b3t_ctx *c, uint32_t variant, int *nctas, size_t *smem, int free_sms = 0, uint32_t fams = ~0u) {
    // the vector variant's SCAL ring: 12 stages (one CTA per SM) for the
    // successor-first order or an explicit one-CTA grid, where a block's
    // chain stays in L2 and each CTA must keep many bytes in flight; 4
    // stages (three CTAs per SM) for breadth-first streaming from HBM
    int32_t stages = 4;
    if (variant == kVarScal) {
        int one = c->cfg.ctas_per_sm == 1 || (c->cfg.ctas_per_sm == 0 && c->cfg.prio_policy == B3T_PRIO_DEPTH);
        if (const char *e = std::getenv("B3T_CTAS_PER_SM")) one = std::atoi(e) == 1;
        stages = one ? 12 : 4;
    }
    *smem = b3t_internal_smem_bytes(variant, stages);
    int per_sm = 0, sms = 0;
    int rc = b3t_internal_occupancy(&per_sm, *smem, &sms, variant);
    if (rc) return rc;
    // a DAG of empty tasks only is claim-bound: more CTAs than two per SM
    // polling the queue measured slower (1.43 M against 1.76 M tasks/s)
    if (fams == 0) per_sm = std::min(per_sm, 2);
    if (c->cfg.ctas_per_sm > 0) per_sm = std::min(per_sm, c->cfg.ctas_per_sm);
    // B3T_CTAS_PER_SM overrides the occupancy query (1..4).  Claims never
    // wait on other work items, so a grid larger than what is resident is
    // still correct: the extra CTAs start as others finish.
    if (const char *e = std::getenv("B3T_CTAS_PER_SM")) {
        const int v = std::atoi(e);
        if (v >= 1 && v <= 4) per_sm = v;
    }
    if (per_sm < 1) return -EINVAL;
    *nctas = per_sm * std::max(1, sms - free_sms);
    return 0;
}

void clear_batch(b3t_ctx *c) {
    c->tasks.clear();
    c->edges.clear();
    c->extra_deps.clear();
    reset_dep_state(c);
}

// Queue a device->host copy of a launch's status block into a pinned mirror.
int track(b3t_ctx *c, Ctl *dev) {
    if (c->inflight.size() == c->mirrors.size()) {
        Ctl *m = nullptr;
        if (cudaMallocHost(&m, sizeof(Ctl)) != cudaSuccess) return -ENOMEM;
        std::memset(m, 0, sizeof(Ctl));
        c->mirrors.push_back(m);
    }
    Ctl *m = c->mirrors[c->inflight.size()];
    c->inflight.emplace_back(dev, m);
    return cuda_err(cudaMemcpyAsync(m, dev, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
}

int flush_impl(b3t_ctx *c) {
    if (c->tasks.empty()) return 0;
    if (c->st.open) return -EBUSY;
    if (c->cfg.host_only) { clear_batch(c); return -ENODEV; }
    InitParams ip; LaunchParams lp; int64_t nitems; bool has_mx;
    int rc = build_launch(c, c->arena, ip, lp, nitems, has_mx);
    if (rc) { clear_batch(c); return rc; }
    int nctas; size_t smem;
    if ((rc = grid_for(c, lp.variant, &nctas, &smem, 0, lp.fams))) { clear_batch(c); return rc; }
    lp.scal_stages = b3t_internal_scal_stages(lp.variant, smem);
    rc = b3t_internal_launch(&ip, &lp, nctas, smem, c->stream, c->ev0, c->ev1);
    c->last_ntasks = (int64_t)c->tasks.size();
    c->last_nitems = nitems;
    c->last_nctas = nctas;
    c->last_timed = true;
    const int r2 = track(c, c->arena.ctl);
    clear_batch(c);
    return rc ? rc : r2;
}

int sync_stream(b3t_ctx *c, int64_t timeout_ns) {
    if (timeout_ns <= 0) return cuda_err(cudaStreamSynchronize(c->stream));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(c->stream);
        if (e == cudaSuccess) return 0;
        if (e != cudaErrorNotReady) return cuda_err(e);
        const auto dt = std::chrono::duration_cast<std::chrono::nanoseconds>(
                            std::chrono::steady_clock::now() - t0).count();
        if (dt > timeout_ns) return -ETIMEDOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// After a stream sync: the first error reported by any launch since the last
// wait; sticky device errors are cleared for the launches that follow.
int read_status(b3t_ctx *c) {
    int first = 0;
    static const int32_t zero[4] = {0, -1, -1, 0};
    for (auto &f : c->inflight) {
        Ctl &s = *f.second;
        if (s.error) {
            if (!first) {
                first = -s.error;
                c->err_task = s.err_task;
                c->err_info = s.err_info;
            }
            cudaMemcpy(f.first, zero, sizeof(zero), cudaMemcpyHostToDevice);
            s.error = 0;
        }
    }
    c->inflight.clear();
    return first;
}

int wait_impl(b3t_ctx *c, int64_t timeout_ns) {
    if (c->st.open) return -EBUSY;
    int rc = flush_impl(c);
    if (c->cfg.host_only) return rc;
    const int rs = sync_stream(c, timeout_ns);
    if (rs) return rs;
    const int st = read_status(c);
    return rc ? rc : st;
}

int check_handle(b3t_ctx *c, b3t_handle h) {
    if (h < 0 || h >= (int32_t)c->handles.size() || !c->handles[h].alive) return -ENOENT;
    return 0;
}

int submit_impl(b3t_ctx *c, b3t_codelet cl, const b3t_handle *handles, const uint8_t *modes,
                int nbuffers, const void *scalars, size_t scalar_bytes) {
    if (!c || cl < 0 || cl >= (int32_t)c->codelets.size()) return -EINVAL;
    const Codelet &C = c->codelets[cl];
    if (nbuffers != C.nbuf || scalar_bytes != C.scalar_bytes) return -EINVAL;
    if (scalar_bytes && !scalars) return -EINVAL;
    if (nbuffers && !handles) return -EINVAL;
    for (int i = 0; i < nbuffers; ++i) {
        const int rc = check_handle(c, handles[i]);
        if (rc) return rc;
        if (modes && modes[i] != C.modes[i]) return -EINVAL;
    }
    const KindSig &S = kSigs[C.kind];
    TaskRec r;
    std::memset(&r, 0, sizeof(r));
    r.kind = C.kind;
    for (int i = 0; i < nbuffers; ++i) r.buf[i] = (uint64_t)(uintptr_t)c->handles[handles[i]].ptr;
    if (C.kind == kScalF32) {
        const Handle &H = c->handles[handles[0]];
        if (H.elemsize != 4 || r.buf[0] % 16) return -EINVAL;   // 128-bit accesses
        r.n = (int64_t)H.nelems;
        std::memcpy(&r.scal, scalars, 4);
    } else if (S.tile) {
        const int64_t b = c->handles[handles[0]].ld;
        if (scalar_bytes == 4) std::memcpy(&r.aux, scalars, 4);
        const int fmt = has_fmt(C.kind) ? r.aux : 0;
        if (fmt != B3T_FMT_BF16 && fmt != B3T_FMT_E4M3) return -EINVAL;
        if (b <= 0 || b % kGemmBlk || b > 4096) return -EINVAL;
        if (((C.kind >= kPotrfMx && C.kind <= kQuant) || C.kind == kCvt || C.kind == kTrmmMx) && b % kMxBlk)
            return -EINVAL;
        for (int i = 0; i < nbuffers; ++i) {
            const Handle &H = c->handles[handles[i]];
            if (H.ld != b || r.buf[i] % 16) return -EINVAL;
            if (S.elem[i] == 1) {
                if (H.elemsize != 1 || H.nelems != q_bytes((int)b, fmt)) return -EINVAL;
            } else if (H.elemsize != (size_t)S.elem[i] || H.nelems < (size_t)(b * b)) {
                return -EINVAL;
            }
        }
        r.n = b;
    }
    if (C.kind == kSliceW || C.kind == kSliceU || C.kind == kTrmmSl) {
        // b from the FP32 / FP64 tile operand's leading dimension
        const Handle &Ht = c->handles[handles[C.kind == kTrmmSl ? 2 : 0]];
        const int64_t b = Ht.ld;
        bool ok = b >= 128 && b <= 4096 && b % 128 == 0;
        for (int i = 0; ok && i < nbuffers; ++i) ok = r.buf[i] % 16 == 0;
        if (ok) {
            const size_t tb = (size_t)b * b;
            const Handle &H0 = c->handles[handles[0]], &H1 = c->handles[handles[1]];
            if (C.kind == kSliceW)
                ok = H0.elemsize == 4 && H0.nelems >= tb && H1.elemsize == 1 && H1.nelems >= (size_t)sl_w_bytes((int)b);
            else if (C.kind == kSliceU)
                ok = H0.elemsize == 8 && H0.nelems >= tb && H1.elemsize == 1 && H1.nelems >= (size_t)sl_u_bytes((int)b);
            else
                ok = H0.elemsize == 1 && H0.nelems >= (size_t)sl_u_bytes((int)b) && H1.elemsize == 1 &&
                     H1.nelems >= (size_t)sl_w_bytes((int)b) && Ht.elemsize == 8 && Ht.nelems >= tb;
        }
        if (!ok) return -EINVAL;
        r.n = b;
    }
    float pcost = -1.f;
    if (is_panel(C.kind)) {
        PanelArgs a;
        std::memcpy(&a, scalars, sizeof(a));
        const int np = a.pw > 0 ? a.b / a.pw : 0;
        bool ok = (a.pw == 64 || a.pw == 128) && a.b >= a.pw && a.b <= 4096 && a.b % a.pw == 0 &&
                  a.kk >= 0 && a.kk < np && a.col0 >= 0;
        if (C.kind == kPanelTrsm) ok = ok && a.kk < np - 1;
        if (C.kind == kTrtriCol) ok = ok && a.pw == 64;
        if (C.kind == kPanelUpd) ok = ok && a.jj > a.kk && a.jj < np;
        for (int i = 0; ok && i < nbuffers; ++i) {
            const Handle &H = c->handles[handles[i]];
            ok = H.elemsize == 8 && H.nelems >= (size_t)a.b * a.pw && r.buf[i] % 16 == 0;
        }
        if (!ok) return -EINVAL;
        r.n = a.b;
        r.aux = a.col0;
        r.scal = (uint32_t)a.kk | ((uint32_t)a.jj << 8) | ((uint32_t)a.pw << 16);
        const double bb = a.b, pw = a.pw;
        if (C.kind == kPotrfD) { r.nitems = 1; pcost = (float)(pw * pw * pw / 3.0 / 3.7 + 20000.0); }
        if (C.kind == kPanelTrsm) {
            r.nitems = (a.b - (a.kk + 1) * a.pw) / kPanelTrsmRows;
            pcost = (float)(kPanelTrsmRows * pw * pw / 3.7 + 5000.0);
        }
        if (C.kind == kPanelUpd) {
            r.nitems = ((a.b - a.jj * a.pw) / kPanelUpdRows) * (a.pw / 64);
            pcost = (float)(2.0 * kPanelUpdRows * 64 * pw / 3.7 + 5000.0);
        }
        if (C.kind == kTrtriCol) {
            r.nitems = a.b / kTrtriRows;
            pcost = (float)(kTrtriRows * 64.0 * (a.kk + 1) * 64.0 / 3.7 + 5000.0);
        }
        (void)bb;
    }
    int vnrhs = 1, vT = 1;
    bool vf32 = false;
    if (is_slice(C.kind)) {
        SliceArgs a;
        std::memcpy(&a, scalars, sizeof(a));
        const Handle *Hs[kMaxBuffers];
        for (int i = 0; i < nbuffers; ++i) Hs[i] = &c->handles[handles[i]];
        auto bytes = [&](int i) { return Hs[i]->nelems * Hs[i]->elemsize; };
        bool ok = a.T >= 1 && a.T <= 4096 && a.b >= 128 && a.b <= 4096 && a.b % 128 == 0 && a.i >= 0 &&
                  a.i < a.T && a.j >= 0 && a.j < a.T;
        for (int i = 0; ok && i < nbuffers; ++i) ok = r.buf[i] % 16 == 0;
        const size_t T = ok ? (size_t)a.T : 0, b = ok ? (size_t)a.b : 0;
        const size_t PB = ok ? (size_t)sl_a_part_bytes(a.b) : 0, XB = ok ? (size_t)sl_x_part_bytes(a.b) : 0;
        if (ok && C.kind == kSliceA)
            ok = a.j <= a.i && Hs[0]->elemsize == 8 && Hs[0]->nelems >= T * (T + 1) / 2 * b * b &&
                 bytes(1) >= PB && bytes(2) >= PB && (a.i == a.j) == (handles[1] == handles[2]);
        if (ok && C.kind == kSliceX)
            ok = a.nrhs >= 1 && a.nrhs <= kSlNp && Hs[0]->elemsize == 8 && Hs[0]->nelems >= b * a.nrhs &&
                 bytes(1) >= XB;
        if (ok && C.kind == kResidSl)
            ok = a.nrhs >= 1 && a.nrhs <= kSlNp && bytes(0) >= T * T * PB && bytes(1) >= T * XB &&
                 Hs[2]->elemsize == 8 && Hs[2]->nelems >= T * b * a.nrhs && Hs[3]->elemsize == 8 &&
                 Hs[3]->nelems >= (size_t)resid_part_elems(a.b, a.nrhs);
        if (!ok) return -EINVAL;
        r.n = a.b;
        r.aux = a.i | (a.j << 16);
        r.scal = (uint32_t)a.T | ((uint32_t)(C.kind == kSliceA ? 0 : a.nrhs) << 16);
        vT = a.T;
    }
    if (is_vec(C.kind)) {
        VecArgs v;
        std::memcpy(&v, scalars, sizeof(v));
        if (v.nrhs < 1 || v.nrhs > kMaxRhs || v.flags < 0 || v.flags > 31 || v.T < 1 || v.T > 65535 ||
            v.i < 0 || v.i >= v.T || v.b < 64 || v.b > 4096 || v.b % 64)
            return -EINVAL;
        const size_t b = (size_t)v.b, blk = b * v.nrhs, T = (size_t)v.T;
        auto need = [&](int i, size_t elems) {
            const Handle &H = c->handles[handles[i]];
            return H.elemsize == 8 && H.nelems >= elems && r.buf[i] % 8 == 0;
        };
        bool ok = true;
        switch (C.kind) {
        case kTrsvL: case kTrsvLT:
            ok = c->handles[handles[0]].ld == (int64_t)b && need(0, b * b) && need(1, blk);
            break;
        case kGemvL: case kGemvLT:
            ok = c->handles[handles[0]].ld == (int64_t)b && need(0, b * b) && need(1, blk) && need(2, blk);
            break;
        case kAxpy: ok = need(0, blk) && need(1, blk); break;
        case kResid:
            ok = need(0, T * (T + 1) / 2 * b * b) && need(1, T * blk) && need(2, T * blk) &&
                 need(3, (size_t)resid_part_elems(v.b, v.nrhs));
            break;
        case kNrm:
            ok = need(0, T * (size_t)resid_part_elems(v.b, v.nrhs)) && need(1, T * blk) &&
                 need(2, (size_t)v.nrhs + 1);
            break;
        }
        if (!ok) return -EINVAL;
        r.n = v.b;
        r.aux = v.i | (v.flags << 24);
        r.scal = (uint32_t)v.T | ((uint32_t)v.nrhs << 16);
        vnrhs = v.nrhs; vT = v.T; vf32 = v.flags & kVecF32;
    }
    if (!is_panel(C.kind))
        r.nitems = (int32_t)(C.kind == kTrsvL || C.kind == kTrsvLT ? vnrhs : items_of(C.kind, r.n));
    if (C.kind == kQuant)   // chunks of 128 rows x 128 bytes of K: (b/128) x (b*esize/128)
        r.nitems = (int32_t)((r.n / 128) * (r.n * (r.aux == B3T_FMT_BF16 ? 2 : 1) / 128));
    const int32_t t = (int32_t)c->tasks.size();
    // expand partitioned parents to their parts; OR the modes of repeats
    std::vector<int32_t> leaves;
    std::vector<uint8_t> lmodes;
    size_t nleaves = 0;
    for (int i = 0; i < nbuffers; ++i) {
        const Handle &H = c->handles[handles[i]];
        nleaves += H.parts.empty() ? 1 : H.parts.size();
    }
    // repeats are found by a scan for a few leaves, by a hash map for a
    // partitioned parent's many parts (the first occurrence keeps its place)
    std::unordered_map<int32_t, size_t> seen;
    const bool many = nleaves > 32;
    for (int i = 0; i < nbuffers; ++i) {
        const Handle &H = c->handles[handles[i]];
        const uint8_t m = C.modes[i];
        auto add = [&](int32_t leaf) {
            if (many) {
                auto it = seen.find(leaf);
                if (it != seen.end()) { lmodes[it->second] |= m; return; }
                seen.emplace(leaf, leaves.size());
            } else {
                for (size_t k = 0; k < leaves.size(); ++k)
                    if (leaves[k] == leaf) { lmodes[k] |= m; return; }
            }
            leaves.push_back(leaf);
            lmodes.push_back(m);
        };
        if (H.parts.empty()) add(handles[i]);
        else for (int32_t k : H.parts) add(k);
    }
    std::vector<int32_t> preds;
    derive(c, t, leaves.data(), lmodes.data(), (int)leaves.size(), preds);
    for (int32_t p : preds) c->edges.emplace_back(p, t);
    Pending P;
    P.rec = r;
    P.cost = pcost >= 0.f ? pcost : cost_of(C.kind, r.n, vnrhs, vT, vf32);
    c->tasks.push_back(P);
    return 0;
}

}  // namespace

extern "C" {

size_t b3t_q_bytes(int b, int fmt) {
    if (b <= 0 || b % kMxBlk || (fmt != B3T_FMT_BF16 && fmt != B3T_FMT_E4M3)) return 0;
    return q_bytes(b, fmt);
}

int b3t_init(b3t_ctx **out, const b3t_config *cfg, void *cuda_stream) {
    if (!out) return -EINVAL;
    *out = nullptr;
    const bool host_only = cfg && cfg->host_only;
    int ndev = 0;
    if (!host_only && (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)) {
        cudaGetLastError();
        return -ENODEV;
    }
    b3t_ctx *c = new (std::nothrow) b3t_ctx();
    if (!c) return -ENOMEM;
    if (cfg) c->cfg = *cfg;
    if (c->cfg.timeout_ns <= 0) c->cfg.timeout_ns = 10'000'000'000LL;
    if (c->cfg.prio_levels <= 0) c->cfg.prio_levels = kMaxLevels;
    if (c->cfg.prio_policy != B3T_PRIO_DEPTH && c->cfg.prio_policy != B3T_PRIO_UPWARD)
        c->cfg.prio_policy = B3T_PRIO_CRITICAL;
    c->cfg.prio_levels = std::min(c->cfg.prio_levels, kMaxLevels);
    for (int k = 0; k < kNumKinds; ++k) c->kind_cl[k] = -1;
    if (host_only) { *out = c; return 0; }
    cudaGetDevice(&c->device);
    c->stream = (cudaStream_t)cuda_stream;
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->staging_done, cudaEventDisableTiming) != cudaSuccess) {
        delete c;
        return -EIO;
    }
    *out = c;
    return 0;
}

int b3t_shutdown(b3t_ctx *c) {
    if (!c) return -EINVAL;
    if (c->cfg.host_only) { delete c; return 0; }
    if (c->st.open) b3t_stream_close(c);
    const int rc = wait_impl(c, 0);
    for (auto &g : c->graphs) {
        if (!g.alive) continue;        // destroyed already (its arena released)
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        g.arena.release();
    }
    c->arena.release();
    if (c->trace_n) cudaFree(c->trace_n);
    if (c->staging) cudaFreeHost(c->staging);
    for (Ctl *m : c->mirrors) cudaFreeHost(m);
    cudaEventDestroy(c->ev0);
    cudaEventDestroy(c->ev1);
    cudaEventDestroy(c->staging_done);
    delete c;
    return rc;
}

int b3t_task_decl(b3t_ctx *c, const char *name, int kind, int nbuffers, const uint8_t *modes,
                  size_t scalar_bytes, b3t_codelet *out) {
    if (!c || !out || kind < 0 || kind >= kNumKinds) return -EINVAL;
    if (nbuffers < 0 || nbuffers > kMaxBuffers || (nbuffers && !modes)) return -EINVAL;
    const KindSig &s = kSigs[kind];
    if (kind == kNoop) {
        if (scalar_bytes != 0) return -EINVAL;
        for (int i = 0; i < nbuffers; ++i) if (modes[i] < 1 || modes[i] > 3) return -EINVAL;
    } else {
        if (nbuffers != s.nbuf || scalar_bytes != s.scalar_bytes) return -EINVAL;
        for (int i = 0; i < nbuffers; ++i) if (modes[i] != s.modes[i]) return -EINVAL;
    }
    Codelet cl;
    cl.name = name ? name : "";
    cl.kind = kind;
    cl.nbuf = nbuffers;
    for (int i = 0; i < nbuffers; ++i) cl.modes[i] = modes[i];
    cl.scalar_bytes = scalar_bytes;
    c->codelets.push_back(cl);
    *out = (b3t_codelet)(c->codelets.size() - 1);
    return 0;
}

int b3t_data_register(b3t_ctx *c, void *p, size_t nelems, size_t elemsize, int64_t ld,
                      b3t_handle *out) {
    if (!c || !out || !p || nelems == 0 || elemsize == 0 || ld < 0) return -EINVAL;
    if (c->by_ptr.count((uintptr_t)p)) return -EEXIST;
    Handle H;
    H.ptr = p; H.nelems = nelems; H.elemsize = elemsize; H.ld = ld; H.alive = true;
    c->handles.push_back(std::move(H));
    const int32_t h = (int32_t)(c->handles.size() - 1);
    c->by_ptr[(uintptr_t)p] = h;
    *out = h;
    return 0;
}

int b3t_data_lookup(b3t_ctx *c, const void *p, b3t_handle *out) {
    if (!c || !out) return -EINVAL;
    auto it = c->by_ptr.find((uintptr_t)p);
    if (it == c->by_ptr.end()) return -ENOENT;
    *out = it->second;
    return 0;
}

int b3t_data_partition(b3t_ctx *c, b3t_handle parent, int32_t nparts, size_t part_nelems,
                       b3t_handle *parts_out) {
    if (!c || !parts_out || nparts <= 0 || part_nelems == 0) return -EINVAL;
    int rc = check_handle(c, parent);
    if (rc) return rc;
    if (!c->handles[parent].parts.empty() || c->handles[parent].parent >= 0) return -EEXIST;
    if ((size_t)nparts * part_nelems > c->handles[parent].nelems) return -EINVAL;
    if (c->handles[parent].touched) return -EBUSY;
    const size_t es = c->handles[parent].elemsize;
    std::vector<int32_t> kids;
    for (int32_t i = 0; i < nparts; ++i) {
        Handle H;
        H.ptr = (char *)c->handles[parent].ptr + (size_t)i * part_nelems * es;
        H.nelems = part_nelems; H.elemsize = es; H.ld = 0; H.alive = true; H.parent = parent;
        c->handles.push_back(std::move(H));
        const int32_t h = (int32_t)(c->handles.size() - 1);
        if (i > 0) c->by_ptr[(uintptr_t)c->handles[h].ptr] = h;   // part 0 shares the parent's address
        kids.push_back(h);
        parts_out[i] = h;
    }
    c->handles[parent].parts = kids;
    return 0;
}

int b3t_task_submit(b3t_ctx *c, b3t_codelet cl, const b3t_handle *handles, const uint8_t *modes,
                    int nbuffers, const void *scalars, size_t scalar_bytes) {
    return submit_impl(c, cl, handles, modes, nbuffers, scalars, scalar_bytes);
}

int b3t_task_submit_ptrs(b3t_ctx *c, b3t_codelet cl, void *const *ptrs, int nbuffers,
                         const void *scalars, size_t scalar_bytes) {
    if (!c || nbuffers < 0 || nbuffers > kMaxBuffers || (nbuffers && !ptrs)) return -EINVAL;
    b3t_handle hs[kMaxBuffers];
    for (int i = 0; i < nbuffers; ++i) {
        const int rc = b3t_data_lookup(c, ptrs[i], &hs[i]);
        if (rc) return rc;
    }
    return submit_impl(c, cl, hs, nullptr, nbuffers, scalars, scalar_bytes);
}

int b3t_task_flush(b3t_ctx *c) {
    if (!c) return -EINVAL;
    if (c->capturing) return 0;
    return flush_impl(c);
}

int b3t_task_wait(b3t_ctx *c, int64_t timeout_ns) {
    if (!c) return -EINVAL;
    if (c->capturing) return -EBUSY;
    return wait_impl(c, timeout_ns);
}

int b3t_data_acquire(b3t_ctx *c, b3t_handle h, uint8_t mode) {
    if (!c || mode < 1 || mode > 3) return -EINVAL;
    const int rc = check_handle(c, h);
    if (rc) return rc;
    if (c->capturing) return -EBUSY;
    // joins every pending and in-flight task: a superset of the writers (and
    // readers) of h, which is what acquire has to wait for
    return wait_impl(c, 0);
}

static bool stream_handle_busy(b3t_ctx *c, b3t_handle h) {
    auto &S = c->st;
    if (!S.open || h >= (int32_t)S.handle_batch.size()) return false;
    std::vector<int32_t> hs{h};
    for (int32_t k : c->handles[h].parts) hs.push_back(k);
    for (int32_t x : hs) {
        if (x < (int32_t)S.handle_batch.size()) {
            const int32_t b = S.handle_batch[x];
            if (b >= 0 && ((volatile int32_t *)S.done_h)[b] == 0) return true;
        }
        if (c->handles[x].touched) return true;    // named by a pending task
    }
    return false;
}

// Forget a handle and its partition parts (parts 1.. are looked up by their
// own addresses, so they leave the address map too).
static void drop_handle(b3t_ctx *c, b3t_handle h) {
    Handle &H = c->handles[h];
    for (int32_t k : H.parts) {
        auto it = c->by_ptr.find((uintptr_t)c->handles[k].ptr);
        if (it != c->by_ptr.end() && it->second == k) c->by_ptr.erase(it);
        c->handles[k].alive = false;
    }
    auto it = c->by_ptr.find((uintptr_t)H.ptr);
    if (it != c->by_ptr.end() && it->second == h) c->by_ptr.erase(it);
    H.alive = false;
    H.parts.clear();
}

int b3t_data_unregister(b3t_ctx *c, b3t_handle h) {
    if (!c) return -EINVAL;
    int rc = check_handle(c, h);
    if (rc) return rc;
    if (c->st.open) {
        // stream mode: no wait; the buffer must not be in use
        if (stream_handle_busy(c, h)) return -EBUSY;
    } else {
        rc = c->capturing ? 0 : wait_impl(c, 0);
    }
    drop_handle(c, h);
    return rc;
}

int b3t_last_error(b3t_ctx *c, int32_t *task_id, int32_t *info) {
    if (!c) return -EINVAL;
    if (task_id) *task_id = c->err_task;
    if (info) *info = c->err_info;
    return 0;
}

const char *b3t_strerror(int err) {
    switch (-err) {
    case 0: return "success";
    case EINVAL: return "invalid argument or task/implementation signature mismatch";
    case ENOENT: return "attempt to use unregistered pointer or handle";
    case ENOMEM: return "out of memory";
    case ETIMEDOUT: return "timed out waiting for tasks";
    case EDOM: return "matrix is not positive definite (see b3t_last_error)";
    case EIO: return "CUDA error";
    case EBUSY: return "operation not allowed while capturing or with pending tasks";
    case EEXIST: return "already registered or partitioned";
    case ENODEV: return "no CUDA device";
    case EPROTO: return "internal consistency check failed on the device";
    case ERANGE: return "iterative refinement did not converge";
    }
    return "unknown error";
}

int b3t_graph_capture_begin(b3t_ctx *c) {
    if (!c) return -EINVAL;
    if (c->capturing || !c->tasks.empty()) return -EBUSY;
    c->capturing = true;
    return 0;
}

int b3t_graph_capture_end(b3t_ctx *c, b3t_graph *out) {
    if (!c || !out || !c->capturing) return -EINVAL;
    c->capturing = false;
    if (c->tasks.empty()) return -EINVAL;
    if (c->cfg.host_only) { clear_batch(c); return -ENODEV; }
    GraphRec g;
    InitParams ip; LaunchParams lp; int64_t nitems; bool has_mx;
    int rc = build_launch(c, g.arena, ip, lp, nitems, has_mx);
    if (!rc) rc = cuda_err(cudaStreamSynchronize(c->stream));
    int nctas = 0; size_t smem = 0;
    if (!rc) rc = grid_for(c, lp.variant, &nctas, &smem, 0, lp.fams);
    lp.scal_stages = b3t_internal_scal_stages(lp.variant, smem);
    if (rc) { clear_batch(c); g.arena.release(); return rc; }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        clear_batch(c); g.arena.release(); return -EIO;
    }
    cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    rc = b3t_internal_launch(&ip, &lp, nctas, smem, cs, nullptr, nullptr);
    const cudaError_t ec = cudaStreamEndCapture(cs, &g.graph);
    cudaStreamDestroy(cs);
    if (rc || ec != cudaSuccess || !g.graph) { clear_batch(c); g.arena.release(); return rc ? rc : -EIO; }
    if (cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess) {
        cudaGraphDestroy(g.graph); clear_batch(c); g.arena.release(); return -EIO;
    }
    g.ntasks = (int64_t)c->tasks.size();
    g.nitems = nitems;
    g.nctas = nctas;
    g.alive = true;
    clear_batch(c);
    c->graphs.push_back(g);
    *out = (b3t_graph)(c->graphs.size() - 1);
    return 0;
}

int b3t_graph_replay(b3t_ctx *c, b3t_graph gi) {
    if (!c || gi < 0 || gi >= (int32_t)c->graphs.size() || !c->graphs[gi].alive) return -EINVAL;
    if (c->capturing) return -EBUSY;
    const int rc = flush_impl(c);
    if (rc) return rc;
    GraphRec &g = c->graphs[gi];
    cudaEventRecord(c->ev0, c->stream);
    const int rl = cuda_err(cudaGraphLaunch(g.exec, c->stream));
    cudaEventRecord(c->ev1, c->stream);
    const int r2 = track(c, g.arena.ctl);
    c->last_ntasks = g.ntasks; c->last_nitems = g.nitems; c->last_nctas = g.nctas;
    c->last_timed = true;
    return rl ? rl : r2;
}

int b3t_graph_destroy(b3t_ctx *c, b3t_graph gi) {
    if (!c || gi < 0 || gi >= (int32_t)c->graphs.size() || !c->graphs[gi].alive) return -EINVAL;
    const int rc = wait_impl(c, 0);
    GraphRec &g = c->graphs[gi];
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g.exec = nullptr;                  // b3t_shutdown must not destroy them again
    g.graph = nullptr;
    g.arena.release();
    g.alive = false;
    return rc;
}

int b3t_dag_stats(b3t_ctx *c, int64_t *ntasks, int64_t *nedges) {
    if (!c) return -EINVAL;
    if (ntasks) *ntasks = (int64_t)c->tasks.size();
    if (nedges) *nedges = (int64_t)c->edges.size();
    return 0;
}

int b3t_dag_edges(b3t_ctx *c, int32_t *pred, int32_t *succ, int64_t cap, int64_t *count) {
    if (!c) return -EINVAL;
    const int64_t n = (int64_t)c->edges.size();
    if (count) *count = n;
    for (int64_t i = 0; i < n && i < cap; ++i) {
        if (pred) pred[i] = c->edges[i].first;
        if (succ) succ[i] = c->edges[i].second;
    }
    return 0;
}

int b3t_dag_levels(b3t_ctx *c, float *rank, int32_t *level, int64_t cap, int64_t *count) {
    if (!c) return -EINVAL;
    const int64_t nt = (int64_t)c->tasks.size();
    if (count) *count = nt;
    std::vector<int32_t> off(nt + 1, 0);
    for (auto &e : c->edges) off[e.first + 1]++;
    for (int64_t t = 0; t < nt; ++t) off[t + 1] += off[t];
    std::vector<int32_t> succ(std::max<size_t>(c->edges.size(), 1));
    {
        std::vector<int32_t> pos(off.begin(), off.end() - 1);
        for (auto &e : c->edges) succ[pos[e.first]++] = e.second;
    }
    std::vector<float> rk;
    std::vector<int32_t> lv;
    compute_levels(c, off, succ.data(), rk, lv);
    for (int64_t t = 0; t < nt && t < cap; ++t) {
        if (rank) rank[t] = rk[t];
        if (level) level[t] = lv[t];
    }
    return 0;
}

int b3t_dag_item_chains(b3t_ctx *c, int32_t *aux, int64_t cap, int64_t *count) {
    if (!c) return -EINVAL;
    const int64_t nt = (int64_t)c->tasks.size();
    if (count) *count = nt;
    std::vector<int32_t> off(nt + 1, 0), indeg(nt, 0);
    for (auto &e : c->edges) { off[e.first + 1]++; indeg[e.second]++; }
    for (int64_t t = 0; t < nt; ++t) off[t + 1] += off[t];
    for (int64_t t = 0; t < nt && t < (int64_t)c->extra_deps.size(); ++t) indeg[t] += c->extra_deps[t];
    std::vector<int32_t> succ(std::max<size_t>(c->edges.size(), 1));
    {
        std::vector<int32_t> pos(off.begin(), off.end() - 1);
        for (auto &e : c->edges) succ[pos[e.first]++] = e.second;
    }
    uint32_t fams = 0;
    for (int64_t t = 0; t < nt; ++t) fams |= family_of(c->tasks[t].rec.kind);
    std::vector<int32_t> ch_aux, ch_at, data = succ;
    if (c->cfg.item_chains && !(variant_of(fams) & kFamMx)) find_item_chains(c, off, succ.data(), indeg, ch_aux, ch_at, data);
    for (int64_t t = 0; t < nt && t < cap; ++t) aux[t] = ch_aux.empty() ? 0 : ch_aux[t];
    return 0;
}

int b3t_last_launch(b3t_ctx *c, int64_t *ntasks, int64_t *nitems, int32_t *nctas, int64_t *kernel_ns) {
    if (!c) return -EINVAL;
    if (ntasks) *ntasks = c->last_ntasks;
    if (nitems) *nitems = c->last_nitems;
    if (nctas) *nctas = c->last_nctas;
    if (kernel_ns) {
        *kernel_ns = -1;
        float ms = 0.f;
        if (c->last_timed && cudaEventQuery(c->ev1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess)
            *kernel_ns = (int64_t)((double)ms * 1e6);
        cudaGetLastError();
    }
    return 0;
}

int b3t_debug_block_task(b3t_ctx *c, int64_t t) {
    if (!c || t < 0 || t >= (int64_t)c->tasks.size()) return -EINVAL;
    if (c->extra_deps.size() < c->tasks.size()) c->extra_deps.resize(c->tasks.size(), 0);
    c->extra_deps[t] += 1;
    return 0;
}

// ------------------------------------------------------------- stream mode

constexpr size_t kStreamStaging = (size_t)64 << 20;   // pinned upload buffer of a stream
constexpr int kStreamFreeSms = 8;                      // SMs a resident stream kernel leaves free

static void stream_free(b3t_ctx *c) {
    auto &S = c->st;
    cudaFree(S.tasks); cudaFree(S.succ); cudaFree(S.level); cudaFree(S.counters); cudaFree(S.done);
    cudaFree(S.next); cudaFree(S.task_batch); cudaFree(S.batch_left); cudaFree(S.batch_info);
    cudaFree(S.slots); cudaFree(S.sroots); cudaFree(S.subs); cudaFree(S.sctl); cudaFree(S.ctl);
    if (S.done_h) cudaFreeHost(S.done_h);
    if (S.staging) cudaFreeHost(S.staging);
    if (S.staged) cudaEventDestroy(S.staged);
    if (S.feed) cudaStreamDestroy(S.feed);
    c->st = b3t_ctx::Stream();
}

int b3t_stream_open(b3t_ctx *c, int64_t max_tasks, int64_t max_edges, int32_t max_batches,
                    int64_t deadline_ns) {
    if (!c || max_tasks <= 0 || max_edges < 0 || max_batches <= 0 || deadline_ns <= 0) return -EINVAL;
    if (c->cfg.host_only) return -ENODEV;
    if (c->st.open || c->capturing || !c->tasks.empty()) return -EBUSY;
    int rc = wait_impl(c, 0);
    if (rc) return rc;
    auto &S = c->st;
    const int L = c->cfg.prio_levels;
    const size_t nt = (size_t)max_tasks, ne = (size_t)std::max<int64_t>(max_edges, 1);
    bool ok = cudaMalloc(&S.tasks, nt * sizeof(TaskRec)) == cudaSuccess &&
              cudaMalloc(&S.succ, ne * 4) == cudaSuccess && cudaMalloc(&S.level, nt * 4) == cudaSuccess &&
              cudaMalloc(&S.counters, nt * 4) == cudaSuccess && cudaMalloc(&S.done, nt * 4) == cudaSuccess &&
              cudaMalloc(&S.next, nt * 4) == cudaSuccess && cudaMalloc(&S.task_batch, nt * 4) == cudaSuccess &&
              cudaMalloc(&S.batch_left, (size_t)max_batches * 4) == cudaSuccess &&
              cudaMalloc(&S.batch_info, (size_t)max_batches * 4) == cudaSuccess &&
              cudaMalloc(&S.slots, (size_t)L * nt * 8) == cudaSuccess &&
              cudaMalloc(&S.sroots, nt * 8) == cudaSuccess &&
              cudaMalloc(&S.subs, (size_t)max_batches * sizeof(SubDesc)) == cudaSuccess &&
              cudaMalloc(&S.sctl, sizeof(StreamCtl)) == cudaSuccess && cudaMalloc(&S.ctl, sizeof(Ctl)) == cudaSuccess &&
              cudaHostAlloc((void **)&S.done_h, (size_t)max_batches * 4, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&S.done_d, S.done_h, 0) == cudaSuccess &&
              cudaStreamCreateWithFlags(&S.feed, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&S.staged, cudaEventDisableTiming) == cudaSuccess &&
              cudaMallocHost(&S.staging, kStreamStaging) == cudaSuccess;
    if (!ok) { cudaGetLastError(); stream_free(c); return -ENOMEM; }
    S.staging_cap = kStreamStaging;
    S.max_tasks = max_tasks; S.max_edges = (int64_t)ne; S.max_batches = max_batches;
    std::memset(S.done_h, 0, (size_t)max_batches * 4);
    cudaMemsetAsync(S.slots, 0xff, (size_t)L * nt * 8, c->stream);
    cudaMemsetAsync(S.ctl, 0, sizeof(Ctl), c->stream);
    cudaMemsetAsync(S.sctl, 0, sizeof(StreamCtl), c->stream);
    cudaMemsetAsync(S.batch_info, 0, (size_t)max_batches * 4, c->stream);
    if ((rc = cuda_err(cudaStreamSynchronize(c->stream)))) { stream_free(c); return rc; }
    S.handle_batch.assign(c->handles.size(), -1);
    LaunchParams lp{};
    lp.tasks = S.tasks; lp.succ = S.succ; lp.level = S.level; lp.counters = S.counters;
    lp.done_items = S.done; lp.next_item = S.next; lp.slots = S.slots; lp.ctl = S.ctl;
    // one ring per level: a stream's rings are sized before its tasks are known
    for (int l = 0; l < L; ++l) { lp.ring_off[l] = (unsigned long long)l * nt; lp.ring_cap[l] = nt; }
    lp.nsub = 1;
    const uint32_t svar = c->cfg.stream_no_mx ? kVarNoMx : kVarAll;
    lp.ntasks = max_tasks; lp.nlevels = L; lp.has_mx = c->cfg.stream_no_mx ? 0 : 1;
    lp.variant = svar; lp.fams = svar;
    lp.timeout_ns = c->cfg.timeout_ns;
    lp.debug = c->cfg.debug_checks; lp.stream_mode = 1;
    if (c->trace_on) { lp.trace = c->trace; lp.trace_n = c->trace_n; lp.trace_cap = c->trace_cap; }
    lp.sctl = S.sctl; lp.subs = S.subs; lp.sroots = S.sroots; lp.task_batch = S.task_batch;
    lp.batch_left = S.batch_left; lp.batch_info = S.batch_info; lp.batch_done = S.done_d;
    lp.deadline_ns = deadline_ns;
    // leave SMs free for work issued while the kernel is resident (input
    // generation, copies): a kernel that needs a whole SM's shared memory
    // could not start otherwise, and whoever waits for it would stall
    const int free_sms = c->cfg.stream_free_sms > 0 ? c->cfg.stream_free_sms : kStreamFreeSms;
    int nctas; size_t smem;
    if ((rc = grid_for(c, svar, &nctas, &smem, free_sms))) { stream_free(c); return rc; }
    lp.scal_stages = b3t_internal_scal_stages(lp.variant, smem);
    if ((rc = b3t_internal_launch_exec(&lp, nctas, smem, c->stream, c->ev0))) { stream_free(c); return rc; }
    S.open = true;
    c->last_nctas = nctas;
    return 0;
}

int b3t_stream_submit(b3t_ctx *c, int32_t *batch_id) {
    if (!c || !batch_id) return -EINVAL;
    auto &S = c->st;
    if (!S.open) return -EINVAL;
    const int64_t nt = (int64_t)c->tasks.size(), ne = (int64_t)c->edges.size();
    if (nt == 0) return -EINVAL;
    if (c->cfg.stream_no_mx)   // the resident kernel was compiled without these kinds
        for (const auto &tk : c->tasks)
            if (family_of(tk.rec.kind) & kFamMx) return -EINVAL;
    if (S.ntasks + nt > S.max_tasks || S.nedges + ne > S.max_edges || S.nroots + nt > S.max_tasks ||
        S.nbatches >= S.max_batches)
        return -ENOMEM;
    // a buffer still used by an unfinished batch may not be named again
    if (S.handle_batch.size() < c->handles.size()) S.handle_batch.resize(c->handles.size(), -1);
    for (int32_t h : c->touched) {
        const int32_t b = S.handle_batch[h];
        if (b >= 0 && ((volatile int32_t *)S.done_h)[b] == 0) return -EBUSY;
    }
    const int32_t batch = S.nbatches;
    const int64_t base = S.ntasks, eoff = S.nedges;
    const int L = c->cfg.prio_levels;
    std::vector<int32_t> off(nt + 1, 0), indeg(nt, 0), succ(std::max<int64_t>(ne, 1));
    for (auto &e : c->edges) { off[e.first + 1]++; indeg[e.second]++; }
    for (int64_t t = 0; t < nt; ++t) off[t + 1] += off[t];
    {
        std::vector<int32_t> pos(off.begin(), off.end() - 1);
        for (auto &e : c->edges) succ[pos[e.first]++] = (int32_t)(base + e.second);
    }
    for (int64_t t = 0; t < nt && t < (int64_t)c->extra_deps.size(); ++t) indeg[t] += c->extra_deps[t];
    std::vector<float> rank(nt, 0.f);
    float maxr = 0.f;
    for (int64_t t = nt - 1; t >= 0; --t) {
        float m = 0.f;
        for (int32_t k = off[t]; k < off[t + 1]; ++k) m = std::max(m, rank[succ[k] - base]);
        rank[t] = c->tasks[t].cost + m;
        maxr = std::max(maxr, rank[t]);
    }
    std::vector<int32_t> level(nt), tb(nt, batch), zeros(nt, 0);
    std::vector<unsigned long long> roots;
    for (int64_t t = 0; t < nt; ++t) {
        TaskRec &r = c->tasks[t].rec;
        r.succ_off = (int32_t)(eoff + off[t]);
        r.nsucc = off[t + 1] - off[t];
        level[t] = (L > 1 && maxr > 0.f) ? std::min(L - 1, (int)((double)L * rank[t] / (maxr * 1.000001))) : 0;
        if (indeg[t] == 0) roots.push_back(pack_slot(base + t, r.nitems));
    }
    const int64_t nr = (int64_t)roots.size();
    // staging layout
    const size_t o_t = 0, o_s = o_t + nt * sizeof(TaskRec), o_l = o_s + ne * 4, o_i = o_l + nt * 4,
                 o_z = o_i + nt * 4, o_b = o_z + nt * 4, o_r = (o_b + nt * 4 + 15) / 16 * 16,
                 o_m = o_r + nr * 8, bytes = o_m + 64;
    // the staging buffer is fixed for the life of the stream: freeing pinned
    // memory implies a device-wide synchronisation, which would wait for the
    // resident kernel itself
    if (bytes > S.staging_cap) return -E2BIG;
    cudaEventSynchronize(S.staged);
    char *sp = (char *)S.staging;
    for (int64_t t = 0; t < nt; ++t) std::memcpy(sp + o_t + t * sizeof(TaskRec), &c->tasks[t].rec, sizeof(TaskRec));
    if (ne) std::memcpy(sp + o_s, succ.data(), ne * 4);
    std::memcpy(sp + o_l, level.data(), nt * 4);
    std::memcpy(sp + o_i, indeg.data(), nt * 4);
    std::memcpy(sp + o_z, zeros.data(), nt * 4);
    std::memcpy(sp + o_b, tb.data(), nt * 4);
    std::memcpy(sp + o_r, roots.data(), nr * 8);
    int32_t *misc = (int32_t *)(sp + o_m);
    misc[0] = (int32_t)nt;   // batch_left
    misc[1] = 0;             // batch_info
    SubDesc sd{(unsigned long long)S.nroots, (uint32_t)nr, (uint32_t)batch};
    std::memcpy(sp + o_m + 16, &sd, sizeof(sd));
    unsigned long long pub[2] = {(unsigned long long)batch + 1, (unsigned long long)(base + nt)};
    std::memcpy(sp + o_m + 32, pub, sizeof(pub));
    ((volatile int32_t *)S.done_h)[batch] = 0;
    cudaStream_t f = S.feed;
    cudaMemcpyAsync(S.tasks + base, sp + o_t, nt * sizeof(TaskRec), cudaMemcpyHostToDevice, f);
    if (ne) cudaMemcpyAsync(S.succ + eoff, sp + o_s, ne * 4, cudaMemcpyHostToDevice, f);
    cudaMemcpyAsync(S.level + base, sp + o_l, nt * 4, cudaMemcpyHostToDevice, f);
    cudaMemcpyAsync(S.counters + base, sp + o_i, nt * 4, cudaMemcpyHostToDevice, f);
    cudaMemcpyAsync(S.done + base, sp + o_z, nt * 4, cudaMemcpyHostToDevice, f);
    cudaMemcpyAsync(S.next + base, sp + o_z, nt * 4, cudaMemcpyHostToDevice, f);
    cudaMemcpyAsync(S.task_batch + base, sp + o_b, nt * 4, cudaMemcpyHostToDevice, f);
    cudaMemcpyAsync(S.sroots + S.nroots, sp + o_r, nr * 8, cudaMemcpyHostToDevice, f);
    cudaMemcpyAsync(S.batch_left + batch, sp + o_m, 4, cudaMemcpyHostToDevice, f);
    cudaMemcpyAsync(S.batch_info + batch, sp + o_m + 4, 4, cudaMemcpyHostToDevice, f);
    cudaMemcpyAsync(S.subs + batch, sp + o_m + 16, sizeof(SubDesc), cudaMemcpyHostToDevice, f);
    // publish last: the kernel reads the data only after it sees the counters
    cudaMemcpyAsync(S.sctl, sp + o_m + 32, 16, cudaMemcpyHostToDevice, f);
    const int rc = cuda_err(cudaEventRecord(S.staged, f));
    if (rc) return rc;
    for (int32_t h : c->touched) S.handle_batch[h] = batch;
    S.ntasks += nt;
    S.nedges += ne;
    S.nroots += nr;
    S.nbatches += 1;
    clear_batch(c);
    *batch_id = batch;
    return 0;
}

int b3t_stream_query(b3t_ctx *c, int32_t batch, int32_t *info) {
    if (!c || !c->st.open || batch < 0 || batch >= c->st.nbatches) return -EINVAL;
    const int32_t v = ((volatile int32_t *)c->st.done_h)[batch];
    if (v) {
        if (info) *info = v >= 2 ? v - 2 : 0;
        return 1;
    }
    const cudaError_t e = cudaStreamQuery(c->stream);
    if (e == cudaErrorNotReady) return 0;
    // the resident kernel has stopped with this batch unfinished
    Ctl h;
    if (e != cudaSuccess || cudaMemcpy(&h, c->st.ctl, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return -EIO;
    }
    if (h.error) { c->err_task = h.err_task; c->err_info = h.err_info; return -h.error; }
    return -EIO;
}

int b3t_stream_close(b3t_ctx *c) {
    if (!c || !c->st.open) return -EINVAL;
    auto &S = c->st;
    int rc = 0;
    cudaEventSynchronize(S.staged);
    unsigned long long *stopflag = (unsigned long long *)S.staging;
    *stopflag = 1;
    cudaMemcpyAsync(&S.sctl->stop, stopflag, 8, cudaMemcpyHostToDevice, S.feed);
    cudaStreamSynchronize(S.feed);
    const int rs = cuda_err(cudaStreamSynchronize(c->stream));
    Ctl h;
    std::memset(&h, 0, sizeof(h));
    if (!rs && cudaMemcpy(&h, S.ctl, sizeof(h), cudaMemcpyDeviceToHost) == cudaSuccess && h.error) {
        c->err_task = h.err_task;
        c->err_info = h.err_info;
        if (!rc) rc = -h.error;
    }
    stream_free(c);
    return rc ? rc : rs;
}

// ------------------------------------------------------------- Cholesky

static int kind_codelet(b3t_ctx *c, int kind, b3t_codelet *cl) {
    if (c->kind_cl[kind] >= 0) { *cl = c->kind_cl[kind]; return 0; }
    const KindSig &s = kSigs[kind];
    const int rc = b3t_task_decl(c, kKindNames[kind], kind, s.nbuf, s.modes, s.scalar_bytes, cl);
    if (!rc) c->kind_cl[kind] = *cl;
    return rc;
}

static int64_t tidx(int32_t i, int32_t j, int32_t T) {
    return (int64_t)j * T - (int64_t)j * (j - 1) / 2 + (i - j);
}

static int reg_tiles(b3t_ctx *c, void *const *tiles, int64_t nt, size_t nelems, size_t es, int64_t ld,
                     std::vector<b3t_handle> &h) {
    h.resize(nt);
    for (int64_t t = 0; t < nt; ++t) {
        int rc = b3t_data_lookup(c, tiles[t], &h[t]);
        if (rc == -ENOENT) rc = b3t_data_register(c, tiles[t], nelems, es, ld, &h[t]);
        if (rc) return rc;
        const Handle &H = c->handles[h[t]];
        if (H.ld != ld || H.elemsize != es || H.nelems != nelems) return -EINVAL;
    }
    return 0;
}

// Partition a diagonal tile handle into b / pw column panels (reuse an
// existing partition of the same shape).
static int panel_parts(b3t_ctx *c, b3t_handle h, int32_t b, int32_t pw, std::vector<b3t_handle> &parts) {
    Handle &H = c->handles[h];
    const int32_t np = b / pw;
    if (!H.parts.empty()) {
        if ((int32_t)H.parts.size() != np || c->handles[H.parts[0]].nelems != (size_t)b * pw) return -EINVAL;
        parts = H.parts;
        return 0;
    }
    parts.resize(np);
    return b3t_data_partition(c, h, np, (size_t)b * pw, parts.data());
}

// POTRF of one diagonal tile as the panel DAG on its partition parts.
static int submit_panel_potrf(b3t_ctx *c, const std::vector<b3t_handle> &P, int32_t b, int32_t pw,
                              int32_t col0) {
    b3t_codelet cd, ct, cu;
    int rc;
    if ((rc = kind_codelet(c, kPotrfD, &cd)) || (rc = kind_codelet(c, kPanelTrsm, &ct)) ||
        (rc = kind_codelet(c, kPanelUpd, &cu)))
        return rc;
    const int32_t np = b / pw;
    for (int32_t kk = 0; kk < np; ++kk) {
        PanelArgs a{b, pw, kk, 0, col0};
        if ((rc = submit_impl(c, cd, &P[kk], nullptr, 1, &a, sizeof(a)))) return rc;
        if (kk < np - 1 && (rc = submit_impl(c, ct, &P[kk], nullptr, 1, &a, sizeof(a)))) return rc;
        for (int32_t jj = kk + 1; jj < np; ++jj) {
            PanelArgs u{b, pw, kk, jj, col0};
            const b3t_handle h2[2] = {P[kk], P[jj]};
            if ((rc = submit_impl(c, cu, h2, nullptr, 2, &u, sizeof(u)))) return rc;
        }
    }
    return 0;
}

// Panel width of the diagonal-tile DAG for tile size b, 0 for one POTRF task
// per diagonal tile.  B3T_PANEL_WIDTH (64 or 128; 0 for none) overrides the
// default, for measurements.
static int32_t panel_width(int32_t b, int32_t preferred = kPanelWidth) {
    int32_t pw = (b >= 2 * preferred && b % preferred == 0) ? preferred : 0;
    if (const char *e = std::getenv("B3T_PANEL_WIDTH")) {
        const int v = std::atoi(e);
        if (v == 0) pw = 0;
        else if ((v == 64 || v == 128) && b >= 2 * v && b % v == 0) pw = v;
    }
    return pw;
}

int b3t_cholesky_submit(b3t_ctx *c, double *const *tiles, int32_t T, int32_t b, int32_t col0) {
    if (!c || !tiles || T <= 0 || b <= 0 || b % kGemmBlk) return -EINVAL;
    const int64_t nt = (int64_t)T * (T + 1) / 2;
    std::vector<b3t_handle> h;
    int rc = reg_tiles(c, (void *const *)tiles, nt, (size_t)b * b, 8, b, h);
    if (rc) return rc;
    b3t_codelet cp, ct, cs, cg;
    if ((rc = kind_codelet(c, kPotrf, &cp)) || (rc = kind_codelet(c, kTrsm, &ct)) ||
        (rc = kind_codelet(c, kSyrk, &cs)) || (rc = kind_codelet(c, kGemm, &cg)))
        return rc;
    // in a small factorisation (T <= 16) tiles below two 128-wide panels take
    // 64-wide ones (a pipelined 64 x 64 POTRF, its panel solve and update
    // instead of one CTA's whole tile); larger ones keep one POTRF task per
    // tile.  The choice depends on the factorisation alone, so that a
    // request's result is the same alone and in a stream of others
    const int32_t pw = (b < 2 * kPanelWidth && T <= 16) ? panel_width(b, 64) : panel_width(b);
    const bool panels = pw > 0;
    std::vector<std::vector<b3t_handle>> dparts(panels ? T : 0);
    for (int32_t k = 0; panels && k < T; ++k)
        if ((rc = panel_parts(c, h[tidx(k, k, T)], b, pw, dparts[k]))) return rc;
    for (int32_t k = 0; k < T; ++k) {
        const int32_t c0 = col0 + k * b;
        const b3t_handle hp[1] = {h[tidx(k, k, T)]};
        if (panels) {
            if ((rc = submit_panel_potrf(c, dparts[k], b, pw, c0))) return rc;
        } else if ((rc = submit_impl(c, cp, hp, nullptr, 1, &c0, 4))) {
            return rc;
        }
        for (int32_t i = k + 1; i < T; ++i) {
            const b3t_handle ht[2] = {h[tidx(k, k, T)], h[tidx(i, k, T)]};
            if ((rc = submit_impl(c, ct, ht, nullptr, 2, nullptr, 0))) return rc;
        }
        for (int32_t i = k + 1; i < T; ++i) {
            const b3t_handle hs[2] = {h[tidx(i, k, T)], h[tidx(i, i, T)]};
            if ((rc = submit_impl(c, cs, hs, nullptr, 2, nullptr, 0))) return rc;
            for (int32_t j = k + 1; j < i; ++j) {
                const b3t_handle hg[3] = {h[tidx(i, k, T)], h[tidx(j, k, T)], h[tidx(i, j, T)]};
                if ((rc = submit_impl(c, cg, hg, nullptr, 3, nullptr, 0))) return rc;
            }
        }
    }
    return 0;
}

int b3t_cholesky_mx_submit(b3t_ctx *c, float *const *W, double *const *L, void *const *Q,
                           int32_t T, int32_t b, int32_t fmt, int32_t col0) {
    if (!c || !W || !L || !Q || T <= 0 || b <= 0 || b % kMxBlk) return -EINVAL;
    if (fmt != B3T_FMT_BF16 && fmt != B3T_FMT_E4M3) return -EINVAL;
    const int64_t nt = (int64_t)T * (T + 1) / 2;
    std::vector<b3t_handle> hw, hl, hq;
    int rc = reg_tiles(c, (void *const *)W, nt, (size_t)b * b, 4, b, hw);
    if (!rc) rc = reg_tiles(c, (void *const *)L, nt, (size_t)b * b, 8, b, hl);
    if (rc) return rc;
    hq.assign(nt, -1);
    for (int32_t j = 0; j < T; ++j)
        for (int32_t i = j + 1; i < T; ++i) {
            const int64_t t = tidx(i, j, T);
            rc = b3t_data_lookup(c, Q[t], &hq[t]);
            if (rc == -ENOENT) rc = b3t_data_register(c, Q[t], q_bytes(b, fmt), 1, b, &hq[t]);
            if (rc) return rc;
        }
    b3t_codelet cp, ct, cq, cs, cg, cc;
    if ((rc = kind_codelet(c, kPotrfMx, &cp)) || (rc = kind_codelet(c, kTrsmMx, &ct)) ||
        (rc = kind_codelet(c, kQuant, &cq)) || (rc = kind_codelet(c, kSyrkMx, &cs)) ||
        (rc = kind_codelet(c, kGemmMx, &cg)) || (rc = kind_codelet(c, kCvt, &cc)))
        return rc;
    const int32_t pw = panel_width(b);
    const bool panels = pw > 0;
    std::vector<std::vector<b3t_handle>> dparts(panels ? T : 0);
    for (int32_t k = 0; panels && k < T; ++k)
        if ((rc = panel_parts(c, hl[tidx(k, k, T)], b, pw, dparts[k]))) return rc;
    for (int32_t k = 0; k < T; ++k) {
        const int32_t c0 = col0 + k * b;
        const b3t_handle hp[2] = {hw[tidx(k, k, T)], hl[tidx(k, k, T)]};
        if (panels) {
            if ((rc = submit_impl(c, cc, hp, nullptr, 2, nullptr, 0))) return rc;
            if ((rc = submit_panel_potrf(c, dparts[k], b, pw, c0))) return rc;
        } else if ((rc = submit_impl(c, cp, hp, nullptr, 2, &c0, 4))) {
            return rc;
        }
        for (int32_t i = k + 1; i < T; ++i) {
            const b3t_handle ht[3] = {hl[tidx(k, k, T)], hw[tidx(i, k, T)], hl[tidx(i, k, T)]};
            if ((rc = submit_impl(c, ct, ht, nullptr, 3, nullptr, 0))) return rc;
            const b3t_handle hqq[2] = {hl[tidx(i, k, T)], hq[tidx(i, k, T)]};
            if ((rc = submit_impl(c, cq, hqq, nullptr, 2, &fmt, 4))) return rc;
        }
        for (int32_t i = k + 1; i < T; ++i) {
            const b3t_handle hs[2] = {hq[tidx(i, k, T)], hw[tidx(i, i, T)]};
            if ((rc = submit_impl(c, cs, hs, nullptr, 2, &fmt, 4))) return rc;
            for (int32_t j = k + 1; j < i; ++j) {
                const b3t_handle hg[3] = {hq[tidx(i, k, T)], hq[tidx(j, k, T)], hw[tidx(i, j, T)]};
                if ((rc = submit_impl(c, cg, hg, nullptr, 3, &fmt, 4))) return rc;
            }
        }
    }
    return 0;
}

// Mixed precision with the panel solve as a product: per step k, after the
// diagonal factor, TRTRI(L_kk -> U_k) and, for every i > k,
// TRMM_MX(U_k, W_ik -> L_ik) and QUANT(L_ik -> Q_ik); the updates as in
// b3t_cholesky_mx_submit.
int b3t_cholesky_mx_inv_submit(b3t_ctx *c, float *const *W, double *const *L, void *const *Q,
                               double *const *U, int32_t T, int32_t b, int32_t fmt, int32_t col0) {
    if (!c || !W || !L || !Q || !U || T <= 0 || b <= 0 || b % kMxBlk) return -EINVAL;
    if (fmt != B3T_FMT_BF16 && fmt != B3T_FMT_E4M3) return -EINVAL;
    const int64_t nt = (int64_t)T * (T + 1) / 2;
    std::vector<b3t_handle> hw, hl, hq, hu;
    int rc = reg_tiles(c, (void *const *)W, nt, (size_t)b * b, 4, b, hw);
    if (!rc) rc = reg_tiles(c, (void *const *)L, nt, (size_t)b * b, 8, b, hl);
    if (!rc) rc = reg_tiles(c, (void *const *)U, T, (size_t)b * b, 8, b, hu);
    if (rc) return rc;
    hq.assign(nt, -1);
    for (int32_t j = 0; j < T; ++j)
        for (int32_t i = j + 1; i < T; ++i) {
            const int64_t t = tidx(i, j, T);
            rc = b3t_data_lookup(c, Q[t], &hq[t]);
            if (rc == -ENOENT) rc = b3t_data_register(c, Q[t], q_bytes(b, fmt), 1, b, &hq[t]);
            if (rc) return rc;
        }
    b3t_codelet cp, ci, cm, cq, cs, cg, cc;
    if ((rc = kind_codelet(c, kPotrfMx, &cp)) || (rc = kind_codelet(c, kTrtri, &ci)) ||
        (rc = kind_codelet(c, kTrmmMx, &cm)) || (rc = kind_codelet(c, kQuant, &cq)) ||
        (rc = kind_codelet(c, kSyrkMx, &cs)) || (rc = kind_codelet(c, kGemmMx, &cg)) ||
        (rc = kind_codelet(c, kCvt, &cc)))
        return rc;
    const int32_t pw = panel_width(b);
    const bool panels = pw > 0;
    std::vector<std::vector<b3t_handle>> dparts(panels ? T : 0);
    for (int32_t k = 0; panels && k < T; ++k)
        if ((rc = panel_parts(c, hl[tidx(k, k, T)], b, pw, dparts[k]))) return rc;
    for (int32_t k = 0; k < T; ++k) {
        const int32_t c0 = col0 + k * b;
        const b3t_handle hp[2] = {hw[tidx(k, k, T)], hl[tidx(k, k, T)]};
        if (panels) {
            if ((rc = submit_impl(c, cc, hp, nullptr, 2, nullptr, 0))) return rc;
            if ((rc = submit_panel_potrf(c, dparts[k], b, pw, c0))) return rc;
        } else if ((rc = submit_impl(c, cp, hp, nullptr, 2, &c0, 4))) {
            return rc;
        }
        if (k + 1 < T) {
            const b3t_handle hi[2] = {hl[tidx(k, k, T)], hu[k]};
            if ((rc = submit_impl(c, ci, hi, nullptr, 2, nullptr, 0))) return rc;
        }
        for (int32_t i = k + 1; i < T; ++i) {
            const b3t_handle ht[3] = {hu[k], hw[tidx(i, k, T)], hl[tidx(i, k, T)]};
            if ((rc = submit_impl(c, cm, ht, nullptr, 3, nullptr, 0))) return rc;
            const b3t_handle hqq[2] = {hl[tidx(i, k, T)], hq[tidx(i, k, T)]};
            if ((rc = submit_impl(c, cq, hqq, nullptr, 2, &fmt, 4))) return rc;
        }
        for (int32_t i = k + 1; i < T; ++i) {
            const b3t_handle hs[2] = {hq[tidx(i, k, T)], hw[tidx(i, i, T)]};
            if ((rc = submit_impl(c, cs, hs, nullptr, 2, &fmt, 4))) return rc;
            for (int32_t j = k + 1; j < i; ++j) {
                const b3t_handle hg[3] = {hq[tidx(i, k, T)], hq[tidx(j, k, T)], hw[tidx(i, j, T)]};
                if ((rc = submit_impl(c, cg, hg, nullptr, 3, &fmt, 4))) return rc;
            }
        }
    }
    return 0;
}

// Mixed precision with the panel product on the tensor cores: per step k,
// after the diagonal factor, TRTRI(L_kk -> U_k) and SLICE_U(U_k -> US_k); for
// every i > k SLICE_W(W_ik -> WS_ik) (W_ik is final once step k - 1 has
// updated it), TRMM_SL(US_k, WS_ik -> L_ik) and QUANT(L_ik -> Q_ik); the
// updates as in b3t_cholesky_mx_submit.
static int reg_bytes(b3t_ctx *c, void *p, size_t bytes, b3t_handle *h) {
    int rc = b3t_data_lookup(c, p, h);
    if (rc == -ENOENT) rc = b3t_data_register(c, p, bytes, 1, 0, h);
    if (rc) return rc;
    return c->handles[*h].elemsize == 1 && c->handles[*h].nelems >= bytes ? 0 : -EINVAL;
}

int b3t_cholesky_mx_sliced_submit(b3t_ctx *c, float *const *W, double *const *L, void *const *Q,
                                  double *const *U, void *const *WS, void *const *US, int32_t T, int32_t b,
                                  int32_t fmt, int32_t col0) {
    if (!c || !W || !L || !Q || !U || !WS || !US || T <= 0 || b < 128 || b > 4096 || b % kMxBlk) return -EINVAL;
    if (fmt != B3T_FMT_BF16 && fmt != B3T_FMT_E4M3) return -EINVAL;
    const int64_t nt = (int64_t)T * (T + 1) / 2;
    std::vector<b3t_handle> hw, hl, hq, hu, hws(nt, -1), hus(T, -1);
    int rc = reg_tiles(c, (void *const *)W, nt, (size_t)b * b, 4, b, hw);
    if (!rc) rc = reg_tiles(c, (void *const *)L, nt, (size_t)b * b, 8, b, hl);
    if (!rc) rc = reg_tiles(c, (void *const *)U, T, (size_t)b * b, 8, b, hu);
    if (rc) return rc;
    hq.assign(nt, -1);
    for (int32_t j = 0; j < T; ++j)
        for (int32_t i = j + 1; i < T; ++i) {
            const int64_t t = tidx(i, j, T);
            rc = b3t_data_lookup(c, Q[t], &hq[t]);
            if (rc == -ENOENT) rc = b3t_data_register(c, Q[t], q_bytes(b, fmt), 1, b, &hq[t]);
            if (!rc) rc = reg_bytes(c, WS[t], (size_t)sl_w_bytes(b), &hws[t]);
            if (rc) return rc;
        }
    for (int32_t k = 0; k + 1 < T; ++k)
        if ((rc = reg_bytes(c, US[k], (size_t)sl_u_bytes(b), &hus[k]))) return rc;
    b3t_codelet cp, ci, ctc, csu, csw, cm, cq, cs, cg, cc;
    if ((rc = kind_codelet(c, kPotrfMx, &cp)) || (rc = kind_codelet(c, kTrtri, &ci)) ||
        (rc = kind_codelet(c, kTrtriCol, &ctc)) ||
        (rc = kind_codelet(c, kSliceU, &csu)) || (rc = kind_codelet(c, kSliceW, &csw)) ||
        (rc = kind_codelet(c, kTrmmSl, &cm)) || (rc = kind_codelet(c, kQuant, &cq)) ||
        (rc = kind_codelet(c, kSyrkMx, &cs)) || (rc = kind_codelet(c, kGemmMx, &cg)) ||
        (rc = kind_codelet(c, kCvt, &cc)))
        return rc;
    // the panel product is off the FP64 pipe, so the diagonal chain bounds the
    // factorisation: 64-wide diagonal panels (8 POTRF_D of ~0.13 ms per tile
    // instead of 4 of ~0.37 ms) shorten it (makespan 214 -> 194 ms at N = 32768)
    const int32_t pw = panel_width(b, 64);
    const bool panels = pw > 0;
    std::vector<std::vector<b3t_handle>> dparts(panels ? T : 0);
    for (int32_t k = 0; panels && k < T; ++k)
        if ((rc = panel_parts(c, hl[tidx(k, k, T)], b, pw, dparts[k]))) return rc;
    for (int32_t k = 0; k < T; ++k) {
        const int32_t c0 = col0 + k * b;
        const b3t_handle hp[2] = {hw[tidx(k, k, T)], hl[tidx(k, k, T)]};
        if (panels) {
            if ((rc = submit_impl(c, cc, hp, nullptr, 2, nullptr, 0))) return rc;
            if ((rc = submit_panel_potrf(c, dparts[k], b, pw, c0))) return rc;
        } else if ((rc = submit_impl(c, cp, hp, nullptr, 2, &c0, 4))) {
            return rc;
        }
        if (k + 1 < T) {
            if (pw == 64) {
                // U_k column block by column block, each as soon as its rows of
                // L_kk are final (after panel cb of the diagonal DAG), so that
                // only the last block follows the diagonal factor
                std::vector<b3t_handle> up;
                if ((rc = panel_parts(c, hu[k], b, pw, up))) return rc;
                for (int32_t cb = 0; cb < b / pw; ++cb) {
                    PanelArgs a{b, pw, cb, 0, 0};
                    const b3t_handle h3[3] = {dparts[k][cb], up[cb > 0 ? cb - 1 : 0], up[cb]};
                    if ((rc = submit_impl(c, ctc, h3, nullptr, 3, &a, sizeof(a)))) return rc;
                }
            } else {
                const b3t_handle hi[2] = {hl[tidx(k, k, T)], hu[k]};
                if ((rc = submit_impl(c, ci, hi, nullptr, 2, nullptr, 0))) return rc;
            }
            const b3t_handle hsu[2] = {hu[k], hus[k]};
            if ((rc = submit_impl(c, csu, hsu, nullptr, 2, nullptr, 0))) return rc;
        }
        for (int32_t i = k + 1; i < T; ++i) {
            const int64_t t = tidx(i, k, T);
            const b3t_handle hsw[2] = {hw[t], hws[t]};
            if ((rc = submit_impl(c, csw, hsw, nullptr, 2, nullptr, 0))) return rc;
            const b3t_handle ht[3] = {hus[k], hws[t], hl[t]};
            if ((rc = submit_impl(c, cm, ht, nullptr, 3, nullptr, 0))) return rc;
            const b3t_handle hqq[2] = {hl[t], hq[t]};
            if ((rc = submit_impl(c, cq, hqq, nullptr, 2, &fmt, 4))) return rc;
        }
        for (int32_t i = k + 1; i < T; ++i) {
            const b3t_handle hs2[2] = {hq[tidx(i, k, T)], hw[tidx(i, i, T)]};
            if ((rc = submit_impl(c, cs, hs2, nullptr, 2, &fmt, 4))) return rc;
            for (int32_t j = k + 1; j < i; ++j) {
                const b3t_handle hg[3] = {hq[tidx(i, k, T)], hq[tidx(j, k, T)], hw[tidx(i, j, T)]};
                if ((rc = submit_impl(c, cg, hg, nullptr, 3, &fmt, 4))) return rc;
            }
        }
    }
    return 0;
}

size_t b3t_slice_w_bytes(int32_t b) {
    return (b < 128 || b > 4096 || b % 128) ? 0 : (size_t)sl_w_bytes(b);
}

size_t b3t_slice_u_bytes(int32_t b) {
    return (b < 128 || b > 4096 || b % 128) ? 0 : (size_t)sl_u_bytes(b);
}

// Register ptr as a vector of nparts parts of part_elems f64 (reusing an
// existing registration of the same shape).
static int reg_parted(b3t_ctx *c, void *ptr, int32_t nparts, size_t part_elems, b3t_handle *parent,
                      std::vector<b3t_handle> &parts) {
    int rc = b3t_data_lookup(c, ptr, parent);
    if (rc == -ENOENT) rc = b3t_data_register(c, ptr, (size_t)nparts * part_elems, 8, 0, parent);
    if (rc) return rc;
    Handle &H = c->handles[*parent];
    if (H.elemsize != 8) return -EINVAL;
    if (H.parts.empty()) {
        if (H.nelems < (size_t)nparts * part_elems) return -EINVAL;
        parts.resize(nparts);
        return b3t_data_partition(c, *parent, nparts, part_elems, parts.data());
    }
    if ((int32_t)H.parts.size() != nparts || c->handles[H.parts[0]].nelems != part_elems) return -EINVAL;
    parts = H.parts;
    return 0;
}

static int reg_vec(b3t_ctx *c, const void *ptr, size_t elems, b3t_handle *h) {
    int rc = b3t_data_lookup(c, ptr, h);
    if (rc == -ENOENT) rc = b3t_data_register(c, (void *)ptr, elems, 8, 0, h);
    if (rc) return rc;
    return c->handles[*h].nelems >= elems && c->handles[*h].elemsize == 8 ? 0 : -EINVAL;
}

static int submit_solve(b3t_ctx *c, const std::vector<b3t_handle> &hl, const std::vector<b3t_handle> &hy,
                        int32_t T, int32_t b, int32_t nrhs, int32_t flags) {
    b3t_codelet tl, gl, tlt, glt;
    int rc;
    if ((rc = kind_codelet(c, kTrsvL, &tl)) || (rc = kind_codelet(c, kGemvL, &gl)) ||
        (rc = kind_codelet(c, kTrsvLT, &tlt)) || (rc = kind_codelet(c, kGemvLT, &glt)))
        return rc;
    VecArgs v{nrhs, flags & kVecF32, 0, T, b};
    for (int32_t k = 0; k < T; ++k) {
        const b3t_handle h2[2] = {hl[tidx(k, k, T)], hy[k]};
        if ((rc = submit_impl(c, tl, h2, nullptr, 2, &v, sizeof(v)))) return rc;
        for (int32_t i = k + 1; i < T; ++i) {
            const b3t_handle h3[3] = {hl[tidx(i, k, T)], hy[k], hy[i]};
            if ((rc = submit_impl(c, gl, h3, nullptr, 3, &v, sizeof(v)))) return rc;
        }
    }
    for (int32_t k = T - 1; k >= 0; --k) {
        const b3t_handle h2[2] = {hl[tidx(k, k, T)], hy[k]};
        if ((rc = submit_impl(c, tlt, h2, nullptr, 2, &v, sizeof(v)))) return rc;
        for (int32_t i = 0; i < k; ++i) {
            const b3t_handle h3[3] = {hl[tidx(k, i, T)], hy[k], hy[i]};
            if ((rc = submit_impl(c, glt, h3, nullptr, 3, &v, sizeof(v)))) return rc;
        }
    }
    return 0;
}

int b3t_chol_solve_submit(b3t_ctx *c, double *const *L, double *Y, int32_t T, int32_t b, int32_t nrhs,
                          int64_t part_stride, int32_t flags) {
    if (!c || !L || !Y || T <= 0 || b <= 0 || b % 64 || nrhs < 1 || nrhs > kMaxRhs ||
        part_stride < (int64_t)b * nrhs)
        return -EINVAL;
    std::vector<b3t_handle> hl, hy;
    b3t_handle hp;
    int rc = reg_tiles(c, (void *const *)L, (int64_t)T * (T + 1) / 2, (size_t)b * b, 8, b, hl);
    if (!rc) rc = reg_parted(c, Y, T, (size_t)part_stride, &hp, hy);
    if (!rc) rc = submit_solve(c, hl, hy, T, b, nrhs, flags);
    return rc;
}

// U_k <- L_kk^{-T} for every diagonal tile (TRTRI tasks).
static int submit_inv(b3t_ctx *c, const std::vector<b3t_handle> &hl, const std::vector<b3t_handle> &hu,
                      int32_t T) {
    b3t_codelet ci;
    int rc = kind_codelet(c, kTrtri, &ci);
    if (rc) return rc;
    for (int32_t k = 0; k < T; ++k) {
        const b3t_handle h2[2] = {hl[tidx(k, k, T)], hu[k]};
        if ((rc = submit_impl(c, ci, h2, nullptr, 2, nullptr, 0))) return rc;
    }
    return 0;
}

// Solve with inverted diagonal tiles (U_k = L_kk^{-T}).  Forward, k
// ascending: Z_k = L_kk^{-1} Y_k, then Y_i -= L_ik Z_k below; backward, k
// descending: Y_k = L_kk^{-T} Z_k, then Z_i -= L_ki^T Y_k above.  The
// solution ends in Y.  Each diagonal step is a triangular multiply split
// into 64-row items instead of a substitution that runs row after row.
static int submit_solve_inv(b3t_ctx *c, const std::vector<b3t_handle> &hl, const std::vector<b3t_handle> &hu,
                            const std::vector<b3t_handle> &hy, const std::vector<b3t_handle> &hz, int32_t T,
                            int32_t b, int32_t nrhs, int32_t flags) {
    b3t_codelet gl, glt;
    int rc;
    if ((rc = kind_codelet(c, kGemvL, &gl)) || (rc = kind_codelet(c, kGemvLT, &glt))) return rc;
    const int32_t f32 = flags & kVecF32;
    const VecArgs v{nrhs, f32, 0, T, b};
    const VecArgs vf{nrhs, f32 | kVecAssign | kVecLowerM, 0, T, b};   // M = U_k^T = L_kk^{-1}
    const VecArgs vb{nrhs, f32 | kVecAssign | kVecUpperM, 0, T, b};   // M = U_k = L_kk^{-T}
    for (int32_t k = 0; k < T; ++k) {
        const b3t_handle h3[3] = {hu[k], hy[k], hz[k]};
        if ((rc = submit_impl(c, glt, h3, nullptr, 3, &vf, sizeof(vf)))) return rc;
        for (int32_t i = k + 1; i < T; ++i) {
            const b3t_handle g3[3] = {hl[tidx(i, k, T)], hz[k], hy[i]};
            if ((rc = submit_impl(c, gl, g3, nullptr, 3, &v, sizeof(v)))) return rc;
        }
    }
    for (int32_t k = T - 1; k >= 0; --k) {
        const b3t_handle h3[3] = {hu[k], hz[k], hy[k]};
        if ((rc = submit_impl(c, gl, h3, nullptr, 3, &vb, sizeof(vb)))) return rc;
        for (int32_t i = 0; i < k; ++i) {
            const b3t_handle g3[3] = {hl[tidx(k, i, T)], hy[k], hz[i]};
            if ((rc = submit_impl(c, glt, g3, nullptr, 3, &v, sizeof(v)))) return rc;
        }
    }
    return 0;
}

int b3t_chol_inv_submit(b3t_ctx *c, double *const *L, double *const *U, int32_t T, int32_t b) {
    if (!c || !L || !U || T <= 0 || b <= 0 || b % 64) return -EINVAL;
    std::vector<b3t_handle> hl, hu;
    int rc = reg_tiles(c, (void *const *)L, (int64_t)T * (T + 1) / 2, (size_t)b * b, 8, b, hl);
    if (!rc) rc = reg_tiles(c, (void *const *)U, T, (size_t)b * b, 8, b, hu);
    if (!rc) rc = submit_inv(c, hl, hu, T);
    return rc;
}

int b3t_chol_solve_inv_submit(b3t_ctx *c, double *const *L, double *const *U, double *Y, double *Z, int32_t T,
                              int32_t b, int32_t nrhs, int64_t part_stride, int32_t flags) {
    if (!c || !L || !U || !Y || !Z || T <= 0 || b <= 0 || b % 64 || nrhs < 1 || nrhs > kMaxRhs ||
        part_stride < (int64_t)b * nrhs)
        return -EINVAL;
    std::vector<b3t_handle> hl, hu, hy, hz;
    b3t_handle hyp, hzp;
    int rc = reg_tiles(c, (void *const *)L, (int64_t)T * (T + 1) / 2, (size_t)b * b, 8, b, hl);
    if (!rc) rc = reg_tiles(c, (void *const *)U, T, (size_t)b * b, 8, b, hu);
    if (!rc) rc = reg_parted(c, Y, T, (size_t)part_stride, &hyp, hy);
    if (!rc) rc = reg_parted(c, Z, T, (size_t)part_stride, &hzp, hz);
    if (!rc) rc = submit_solve_inv(c, hl, hu, hy, hz, T, b, nrhs, flags);
    return rc;
}

// Refinement workspace: [T residual parts] [Z: T parts of b x nrhs]
// [U: T tiles of b x b], each region starting on a 256-byte boundary.
static size_t round32(size_t n) { return (n + 31) / 32 * 32; }
static size_t ir_z_off(int32_t T, int32_t b, int32_t nrhs) {
    return round32((size_t)T * (size_t)resid_part_elems(b, nrhs));
}
static size_t ir_u_off(int32_t T, int32_t b, int32_t nrhs) {
    return ir_z_off(T, b, nrhs) + round32((size_t)T * b * nrhs);
}

size_t b3t_resid_part_elems(int32_t b, int32_t nrhs) {
    if (b <= 0 || b % 64 || nrhs < 1 || nrhs > kMaxRhs) return 0;
    return (size_t)resid_part_elems(b, nrhs);
}

size_t b3t_ir_work_elems(int32_t T, int32_t b, int32_t nrhs) {
    if (T <= 0 || b <= 0 || b % 64 || nrhs < 1 || nrhs > kMaxRhs) return 0;
    return ir_u_off(T, b, nrhs) + (size_t)T * b * b;
}

// Registration shared by the refinement helpers.
struct IrHandles {
    std::vector<b3t_handle> hl, hx, hr, hz, hu;
    b3t_handle ha, hxp, hrp, hbp, he, hzp;
    // sliced residual: the A slice area (one buffer) and the T X slice parts
    std::vector<b3t_handle> hxs;
    b3t_handle hasp = -1, hxsp = -1;
};

// Slice area of the sliced refinement: [T*T A slice parts][T X slice parts],
// the second region 256-byte aligned.
static size_t sl_x_off(int32_t T, int32_t b) {
    const size_t n = (size_t)T * T * (size_t)sl_a_part_bytes(b);
    return (n + 255) / 256 * 256;
}

size_t b3t_ir_slice_bytes(int32_t T, int32_t b) {
    if (T <= 0 || T > 4096 || b < 128 || b > 4096 || b % 128) return 0;
    return sl_x_off(T, b) + (size_t)T * (size_t)sl_x_part_bytes(b);
}

size_t b3t_slice_a_part_bytes(int32_t b) {
    return (b < 128 || b > 4096 || b % 128) ? 0 : (size_t)sl_a_part_bytes(b);
}

size_t b3t_slice_x_part_bytes(int32_t b) {
    return (b < 128 || b > 4096 || b % 128) ? 0 : (size_t)sl_x_part_bytes(b);
}

// Register ptr as nparts byte parts of part_bytes (reusing an existing
// registration of the same shape).
static int reg_byte_parts(b3t_ctx *c, void *ptr, int32_t nparts, size_t part_bytes, b3t_handle *parent,
                          std::vector<b3t_handle> &parts) {
    int rc = b3t_data_lookup(c, ptr, parent);
    if (rc == -ENOENT) rc = b3t_data_register(c, ptr, (size_t)nparts * part_bytes, 1, 0, parent);
    if (rc) return rc;
    Handle &H = c->handles[*parent];
    if (H.elemsize != 1) return -EINVAL;
    if (H.parts.empty()) {
        if (H.nelems < (size_t)nparts * part_bytes) return -EINVAL;
        parts.resize(nparts);
        return b3t_data_partition(c, *parent, nparts, part_bytes, parts.data());
    }
    if ((int32_t)H.parts.size() != nparts || c->handles[H.parts[0]].nelems != part_bytes) return -EINVAL;
    parts = H.parts;
    return 0;
}

// Slices of A, once per solve, in a launch of their own: SLICE_A per stored
// tile into the T x T use parts.  The finished slice area is then
// registered again as one plain buffer, so that the residual tasks of every
// step name one buffer instead of T x T parts (nothing writes it during the
// refinement); the X slices keep their T parts.
static int ir_register_slices(b3t_ctx *c, unsigned char *S, int32_t T, int32_t b, IrHandles &H) {
    b3t_handle hp = -1;
    std::vector<b3t_handle> parts;
    int rc = reg_byte_parts(c, S, T * T, (size_t)sl_a_part_bytes(b), &hp, parts);
    b3t_codelet csa;
    if (!rc) rc = kind_codelet(c, kSliceA, &csa);
    for (int32_t j = 0; !rc && j < T; ++j)
        for (int32_t i = j; !rc && i < T; ++i) {
            const SliceArgs a{i, j, T, b, 0};
            const b3t_handle h3[3] = {H.ha, parts[(size_t)i * T + j], parts[(size_t)j * T + i]};
            rc = submit_impl(c, csa, h3, nullptr, 3, &a, sizeof(a));
        }
    const int rw = rc ? 0 : wait_impl(c, 0);
    if (rc) wait_impl(c, 0);
    if (hp >= 0 && c->handles[hp].alive) drop_handle(c, hp);
    if (rc || rw) return rc ? rc : rw;
    rc = b3t_data_register(c, S, (size_t)T * T * (size_t)sl_a_part_bytes(b), 1, 0, &H.hasp);
    if (!rc) rc = reg_byte_parts(c, S + sl_x_off(T, b), T, (size_t)sl_x_part_bytes(b), &H.hxsp, H.hxs);
    return rc;
}

static std::vector<double *> ir_u_tiles(double *R, int32_t T, int32_t b, int32_t nrhs) {
    std::vector<double *> u(T);
    for (int32_t k = 0; k < T; ++k) u[k] = R + ir_u_off(T, b, nrhs) + (size_t)k * b * b;
    return u;
}

static int ir_register(b3t_ctx *c, const double *A, double *const *L, const double *B, double *X, double *R,
                       double *eta, int32_t T, int32_t b, int32_t nrhs, IrHandles &H) {
    const int64_t nt = (int64_t)T * (T + 1) / 2;
    const size_t blk = (size_t)b * nrhs, PR = (size_t)resid_part_elems(b, nrhs);
    const std::vector<double *> u = ir_u_tiles(R, T, b, nrhs);
    int rc = reg_tiles(c, (void *const *)L, nt, (size_t)b * b, 8, b, H.hl);
    if (!rc) rc = reg_vec(c, A, (size_t)nt * b * b, &H.ha);
    if (!rc) rc = reg_parted(c, X, T, blk, &H.hxp, H.hx);
    if (!rc) rc = reg_vec(c, B, (size_t)T * blk, &H.hbp);
    if (!rc) rc = reg_parted(c, R, T, PR, &H.hrp, H.hr);
    if (!rc) rc = reg_parted(c, R + ir_z_off(T, b, nrhs), T, blk, &H.hzp, H.hz);
    if (!rc) rc = reg_tiles(c, (void *const *)u.data(), T, (size_t)b * b, 8, b, H.hu);
    if (!rc) rc = reg_vec(c, eta, (size_t)nrhs + 1, &H.he);
    return rc;
}

int b3t_ir_release(b3t_ctx *c, double *R, int32_t T, int32_t b, int32_t nrhs) {
    if (!c || !R || T <= 0 || b <= 0 || b % 64 || nrhs < 1 || nrhs > kMaxRhs) return -EINVAL;
    const std::vector<double *> u = ir_u_tiles(R, T, b, nrhs);
    void *const regions[2] = {R, R + ir_z_off(T, b, nrhs)};
    if (c->st.open) {
        b3t_handle h;
        for (void *p : regions)
            if (b3t_data_lookup(c, p, &h) == 0 && stream_handle_busy(c, h)) return -EBUSY;
        for (double *p : u)
            if (b3t_data_lookup(c, p, &h) == 0 && stream_handle_busy(c, h)) return -EBUSY;
    } else if (!c->capturing) {
        const int rc = wait_impl(c, 0);
        if (rc) return rc;
    }
    b3t_handle h;
    for (void *p : regions)
        if (b3t_data_lookup(c, p, &h) == 0) drop_handle(c, h);
    for (double *p : u)
        if (b3t_data_lookup(c, p, &h) == 0) drop_handle(c, h);
    return 0;
}

// One refinement step: [first: r = b, U_k = L_kk^{-T}]; d = (L L^T)^{-1} r
// (with the inverted diagonal tiles); x (+)= d; r = b - A x; eta.
// With slices (H.hasp >= 0, A sliced beforehand) the residual r = b - A x is
// RESID_SL: every step slices x (SLICE_X) and forms r on the tensor cores.
static int ir_step_resid(b3t_ctx *c, IrHandles &H, int32_t T, int32_t b, int32_t nrhs, bool first);

// part 0: the whole step; 1: only its first half (the solves and AXPY).
static int ir_step(b3t_ctx *c, IrHandles &H, int32_t T, int32_t b, int32_t nrhs, int32_t flags, bool first,
                   int part = 0) {
    b3t_codelet cres, cax;
    int rc;
    if ((rc = kind_codelet(c, kResid, &cres)) || (rc = kind_codelet(c, kAxpy, &cax))) return rc;
    const bool sliced = H.hasp >= 0;
    auto resid = [&](int32_t fl) -> int {
        for (int32_t i = 0; i < T; ++i) {
            VecArgs v{nrhs, fl, i, T, b};
            const b3t_handle h4[4] = {H.ha, H.hxp, H.hbp, H.hr[i]};
            const int r2 = submit_impl(c, cres, h4, nullptr, 4, &v, sizeof(v));
            if (r2) return r2;
        }
        return 0;
    };
    if (first && (rc = resid(kVecAssign))) return rc;          // r_0 = b (x_0 = 0)
    if (first && (rc = submit_inv(c, H.hl, H.hu, T))) return rc;   // U_k = L_kk^{-T}, kept for later steps

    if ((rc = submit_solve_inv(c, H.hl, H.hu, H.hr, H.hz, T, b, nrhs, flags))) return rc;
    for (int32_t i = 0; i < T; ++i) {
        VecArgs v{nrhs, first ? kVecAssign : 0, i, T, b};
        const b3t_handle h2[2] = {H.hx[i], H.hr[i]};
        if ((rc = submit_impl(c, cax, h2, nullptr, 2, &v, sizeof(v)))) return rc;
    }
    if (part == 1) return 0;
    if (sliced && part == 0) {
        // the solves in a launch of their own (the vector variant, more CTAs
        // per SM), then the slicing and the tensor-core residual
        if (!c->capturing && (rc = flush_impl(c))) return rc;
    }
    return ir_step_resid(c, H, T, b, nrhs, first);
}

// The second half of a refinement step: r = b - A x (RESID, or SLICE_X and
// RESID_SL with slices) and eta (NRM).
static int ir_step_resid(b3t_ctx *c, IrHandles &H, int32_t T, int32_t b, int32_t nrhs, bool first) {
    b3t_codelet cres, cnrm;
    int rc;
    if ((rc = kind_codelet(c, kResid, &cres)) || (rc = kind_codelet(c, kNrm, &cnrm))) return rc;
    const bool sliced = H.hasp >= 0;
    if (sliced) {
        b3t_codelet csx, crs;
        if ((rc = kind_codelet(c, kSliceX, &csx)) || (rc = kind_codelet(c, kResidSl, &crs))) return rc;
        for (int32_t j = 0; j < T; ++j) {
            const SliceArgs a{j, 0, T, b, nrhs};
            const b3t_handle h2[2] = {H.hx[j], H.hxs[j]};
            if ((rc = submit_impl(c, csx, h2, nullptr, 2, &a, sizeof(a)))) return rc;
        }
        for (int32_t i = 0; i < T; ++i) {
            const SliceArgs a{i, 0, T, b, nrhs};
            const b3t_handle h4[4] = {H.hasp, H.hxsp, H.hbp, H.hr[i]};
            if ((rc = submit_impl(c, crs, h4, nullptr, 4, &a, sizeof(a)))) return rc;
        }
    } else {
        // the |A| row sums are formed by the first step's residual and kept
        for (int32_t i = 0; i < T; ++i) {
            VecArgs v{nrhs, first ? 0 : kVecKeepNorm, i, T, b};
            const b3t_handle h4[4] = {H.ha, H.hxp, H.hbp, H.hr[i]};
            if ((rc = submit_impl(c, cres, h4, nullptr, 4, &v, sizeof(v)))) return rc;
        }
    }
    VecArgs v{nrhs, 0, 0, T, b};
    const b3t_handle h3[3] = {H.hrp, H.hbp, H.he};
    return submit_impl(c, cnrm, h3, nullptr, 3, &v, sizeof(v));
}

int b3t_ir_step_submit(b3t_ctx *c, const double *A, double *const *L, const double *B, double *X, double *R,
                       double *eta, int32_t T, int32_t b, int32_t nrhs, int32_t flags, int32_t first) {
    if (!c || !A || !L || !B || !X || !R || !eta || T <= 0 || b <= 0 || b % 64 || nrhs < 1 || nrhs > kMaxRhs)
        return -EINVAL;
    IrHandles H;
    int rc = ir_register(c, A, L, B, X, R, eta, T, b, nrhs, H);
    return rc ? rc : ir_step(c, H, T, b, nrhs, flags, first != 0);
}

static int ir_loop(b3t_ctx *c, IrHandles &H, double *eta, int32_t T, int32_t b, int32_t nrhs, int32_t flags,
                   double tol, int32_t max_iter, int32_t *iters, double *eta_out);

int b3t_ir_solve(b3t_ctx *c, const double *A, double *const *L, const double *B, double *X, double *R,
                 double *eta, int32_t T, int32_t b, int32_t nrhs, int32_t flags, double tol, int32_t max_iter,
                 int32_t *iters, double *eta_out) {
    if (!c || !A || !L || !B || !X || !R || !eta || T <= 0 || b <= 0 || b % 64 || nrhs < 1 ||
        nrhs > kMaxRhs || max_iter < 1 || c->capturing)
        return -EINVAL;
    if (c->cfg.host_only) return -ENODEV;
    if (c->st.open) return -EBUSY;
    IrHandles H;
    int rc = ir_register(c, A, L, B, X, R, eta, T, b, nrhs, H);
    if (rc) return rc;
    return ir_loop(c, H, eta, T, b, nrhs, flags, tol, max_iter, iters, eta_out);
}

int b3t_ir_solve_sliced(b3t_ctx *c, const double *A, double *const *L, const double *B, double *X, double *R,
                        void *S, double *eta, int32_t T, int32_t b, int32_t nrhs, int32_t flags, double tol,
                        int32_t max_iter, int32_t *iters, double *eta_out) {
    if (!c || !A || !L || !B || !X || !R || !S || !eta || T <= 0 || T > 4096 || b < 128 || b > 4096 ||
        b % 128 || nrhs < 1 || nrhs > kSlNp || max_iter < 1 || c->capturing || (uintptr_t)S % 256)
        return -EINVAL;
    if (c->cfg.host_only) return -ENODEV;
    if (c->st.open) return -EBUSY;
    IrHandles H;
    int rc = ir_register(c, A, L, B, X, R, eta, T, b, nrhs, H);
    if (!rc) rc = ir_register_slices(c, (unsigned char *)S, T, b, H);
    if (!rc) rc = ir_loop(c, H, eta, T, b, nrhs, flags, tol, max_iter, iters, eta_out);
    // the slices are the call's own: forget them once every task is done
    const int rw = wait_impl(c, 0);
    if (H.hasp >= 0) drop_handle(c, H.hasp);
    if (H.hxsp >= 0) drop_handle(c, H.hxsp);
    return rc ? rc : rw;
}

// Steps after the first are the same task graph every time: they are
// captured once (two graphs with slices, whose halves run in launches of
// their own, else one) and replayed, so the host derives and uploads their
// dependencies once per solve instead of once per step.
struct IrGraphs {
    b3t_ctx *c;
    b3t_graph g[2] = {-1, -1};
    ~IrGraphs() {
        for (b3t_graph x : g)
            if (x >= 0) b3t_graph_destroy(c, x);
    }
};

static int ir_loop(b3t_ctx *c, IrHandles &H, double *eta, int32_t T, int32_t b, int32_t nrhs, int32_t flags,
                   double tol, int32_t max_iter, int32_t *iters, double *eta_out) {
    int rc;
    std::vector<double> host(nrhs + 1, 0.0);
    double prev = 0.0;
    IrGraphs G{c};
    const bool sliced = H.hasp >= 0;
    for (int32_t it = 1; it <= max_iter; ++it) {
        if (it == 1) {
            if ((rc = ir_step(c, H, T, b, nrhs, flags, true))) return rc;
        } else {
            if (G.g[0] < 0) {
                if ((rc = b3t_graph_capture_begin(c))) return rc;
                rc = ir_step(c, H, T, b, nrhs, flags, false, sliced ? 1 : 0);
                const int re = b3t_graph_capture_end(c, &G.g[0]);
                if (rc || re) return rc ? rc : re;
                if (sliced) {
                    if ((rc = b3t_graph_capture_begin(c))) return rc;
                    rc = ir_step_resid(c, H, T, b, nrhs, false);
                    const int re2 = b3t_graph_capture_end(c, &G.g[1]);
                    if (rc || re2) return rc ? rc : re2;
                }
            }
            for (b3t_graph x : G.g)
                if (x >= 0 && (rc = b3t_graph_replay(c, x))) return rc;
        }
        if ((rc = wait_impl(c, 0))) return rc;
        if ((rc = cuda_err(cudaMemcpyAsync(host.data(), eta, (nrhs + 1) * sizeof(double),
                                           cudaMemcpyDeviceToHost, c->stream))) ||
            (rc = cuda_err(cudaStreamSynchronize(c->stream))))
            return rc;
        if (iters) *iters = it;
        if (eta_out) std::memcpy(eta_out, host.data(), (nrhs + 1) * sizeof(double));
        const double e = host[nrhs];
        if (e <= tol) return 0;
        if (it >= 2 && !(e < 0.9 * prev)) return -ERANGE;
        prev = e;
    }
    return -ERANGE;
}

int b3t_trace_start(b3t_ctx *c, int64_t capacity) {
    if (!c || capacity < 1) return -EINVAL;
    if (c->cfg.host_only) return -ENODEV;
    if (c->st.open) return -EBUSY;
    int rc = wait_impl(c, 0);
    if (rc) return rc;
    if (capacity > c->trace_cap) {
        if (c->trace_n) cudaFree(c->trace_n);
        c->trace_n = nullptr; c->trace = nullptr; c->trace_cap = 0;
        void *m = nullptr;
        // the count and the records in one allocation (records 256-byte aligned)
        if ((rc = cuda_err(cudaMalloc(&m, 256 + (size_t)capacity * sizeof(TraceRec))))) return rc;
        c->trace_n = (unsigned long long *)m;
        c->trace = (TraceRec *)((char *)m + 256);
        c->trace_cap = capacity;
    }
    if ((rc = cuda_err(cudaMemsetAsync(c->trace_n, 0, sizeof(unsigned long long), c->stream)))) return rc;
    c->trace_on = true;
    return 0;
}

int b3t_trace_read(b3t_ctx *c, void *records, int64_t capacity, int64_t *count) {
    if (!c || !count || capacity < 0 || (capacity && !records)) return -EINVAL;
    if (c->cfg.host_only) return -ENODEV;
    if (!c->trace_n) return -ENOENT;
    if (c->st.open) return -EBUSY;
    int rc = wait_impl(c, 0);
    if (rc) return rc;
    unsigned long long n = 0;
    if ((rc = cuda_err(cudaMemcpy(&n, c->trace_n, sizeof(n), cudaMemcpyDeviceToHost)))) return rc;
    *count = (int64_t)n;
    const int64_t k = std::min<int64_t>({(int64_t)n, capacity, c->trace_cap});
    if (k > 0) rc = cuda_err(cudaMemcpy(records, c->trace, (size_t)k * sizeof(TraceRec), cudaMemcpyDeviceToHost));
    return rc;
}

int b3t_trace_stop(b3t_ctx *c) {
    if (!c) return -EINVAL;
    c->trace_on = false;
    return 0;
}

int b3t_tiles_unregister(b3t_ctx *c, void *const *tiles, int32_t T) {
    if (!c || !tiles || T <= 0) return -EINVAL;
    const int64_t nt = (int64_t)T * (T + 1) / 2;
    int rc = 0;
    if (c->st.open) {
        for (int64_t t = 0; t < nt; ++t) {
            b3t_handle h;
            if (tiles[t] && b3t_data_lookup(c, tiles[t], &h) == 0 && stream_handle_busy(c, h)) return -EBUSY;
        }
    } else {
        rc = c->capturing ? -EBUSY : wait_impl(c, 0);
    }
    for (int64_t t = 0; t < nt; ++t) {
        b3t_handle h;
        if (tiles[t] && b3t_data_lookup(c, tiles[t], &h) == 0) drop_handle(c, h);
    }
    return rc;
}

}  // extern "C"
