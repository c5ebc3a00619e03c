// Internal layout shared by the host runtime (runtime.cpp) and the device
// executor (executor.cu).  Not part of the public ABI.
#pragma once
#include <stdint.h>
#include <stddef.h>

#ifdef __CUDACC__
#define B3T_HD __host__ __device__
#else
#define B3T_HD
#endif

namespace b3t {

constexpr int kMaxBuffers = 4;
constexpr int kMaxLevels = 8;
// Each priority level's ready queue is split into nsub rings (task id mod
// nsub), each with its own head and tail, so that claims contend on several
// heads instead of one; a claiming warp reads every ring's head and tail in
// one round trip (two rings per lane), so levels x nsub <= 64.
constexpr int kMaxRings = 64;
constexpr int kThreads = 256;            // threads per persistent CTA

// Work-item decomposition of each kind (the host computes nitems, the
// device maps item -> sub-block with the same constants).
constexpr int64_t kScalChunk = 1 << 16;  // f32 elements per SCAL item
constexpr int kMaxChain = 32;            // SCAL tasks absorbed by one item-chain head
constexpr int kGemmBlk = 64;             // f64 GEMM / SYRK item: 64 x 64 of C
constexpr int kTrsmRows = 32;            // f64 TRSM item: 32 rows of A_ik
// In launches of at most kFineLaunchTasks tasks (a factorisation of a few
// thousand rows, bound by its critical path), tiles of at most kSmallTile
// rows split finer: TRSM items of kSmallTrsmRows rows, SYRK / GEMM items of
// kSmallGemmRows x 64, so that one task's work spreads over more SMs (one SM
// does ~8 GFLOP/s of FP64).  The device tells the splits apart by the
// task's item count.
constexpr int kSmallTile = 128;
constexpr int64_t kFineLaunchTasks = 2048;
constexpr int kSmallTrsmRows = 8;
constexpr int kSmallGemmRows = 16;
#ifndef B3T_TRTRI_ROWS
#define B3T_TRTRI_ROWS 8
#endif
#ifndef B3T_TRMM_ROWS
#define B3T_TRMM_ROWS 32
#endif
constexpr int kTrtriRows = B3T_TRTRI_ROWS;   // TRTRI item: rows of U_k (8, 16 or 32)
constexpr int kTrmmRows = B3T_TRMM_ROWS;     // TRMM_MX item: rows x 64 columns of L_ik (32 or 64)
static_assert(kTrmmRows == 32 || kTrmmRows == 64, "TRMM_MX rows per item");
constexpr int kMxBlk = 128;              // MX GEMM / SYRK item: 128 x 128 of C
constexpr int kMxWideBlk = 256;          // GEMM_MX item when b is a multiple of 256: 256 x 256
constexpr int kCvtCols = 16;             // CVT item: 16 columns of the tile
constexpr int kGemvRows = 16;            // GEMV item: 16 rows of the updated part
constexpr int kResidRows = 16;           // RESID item: 16 rows of the residual part
constexpr int kMaxRhs = 32;

// Scalar blob of the vector kinds (TRSV / GEMV / AXPY / RESID / NRM).
struct VecArgs {
    int32_t nrhs;
    int32_t flags;    // bit 0: binary32 arithmetic (solves); bit 1: AXPY assigns / RESID with x = 0
    int32_t i;        // row block (RESID)
    int32_t T;        // number of row blocks
    int32_t b;        // rows per block (tile size)
};
constexpr int32_t kVecF32 = 1, kVecAssign = 2;
// GEMV with a triangular matrix M: only the 64-column blocks that can hold
// nonzeros are visited (lower: q <= r, upper: q >= r)
constexpr int32_t kVecLowerM = 4, kVecUpperM = 8;
// RESID: leave the |A| row-sum partials from an earlier residual in place
// (the norm of A does not change between refinement steps)
constexpr int32_t kVecKeepNorm = 16;

struct PanelArgs {
    int32_t b, pw, kk, jj, col0;
};
constexpr int kPanelWidth = 128;          // panel width used by the Cholesky helpers
constexpr int kPanelTrsmRows = 16;        // PANEL_TRSM item: rows below the diagonal block
constexpr int kPanelUpdRows = 16;         // PANEL_UPD item: rows x 64 columns

// Elements of one part of the residual work area: b*nrhs values, then per
// RESID item the maxima |r_j| and |x_j| and the largest row sum of |A|.
// RESID output part: b*nrhs residual values, then per item max|r_j|,
// max|x_j|, max|b_j| (nrhs each) and the largest |A| row sum
B3T_HD constexpr int64_t resid_part_elems(int b, int nrhs) {
    return (int64_t)b * nrhs + (int64_t)(b / kResidRows) * (3 * nrhs + 1);
}

enum : int32_t {
    kNoop = 0, kScalF32 = 1, kPotrf = 2, kTrsm = 3, kSyrk = 4, kGemm = 5,
    kPotrfMx = 6, kTrsmMx = 7, kSyrkMx = 8, kGemmMx = 9, kQuant = 10,
    kTrsvL = 11, kGemvL = 12, kTrsvLT = 13, kGemvLT = 14, kAxpy = 15, kResid = 16, kNrm = 17,
    kPotrfD = 18, kPanelTrsm = 19, kPanelUpd = 20, kCvt = 21, kTrtri = 22, kTrmmMx = 23,
    kSliceA = 24, kSliceX = 25, kResidSl = 26, kSliceW = 27, kSliceU = 28, kTrmmSl = 29, kTrtriCol = 30,
    kNumKinds = 31
};

// Sliced FP64 residual (the Ozaki scheme: exact products of integer digit
// slices on the tensor cores).  A value v of a block with scale exponent e
// (|v| < 2^(e-2)) is V = trunc(v 2^(60-e)), written in kSlDigits balanced
// base-32 digits d_s in [-16, 15], V = sum_s d_s 32^(11-s); every digit is an
// E4M3 integer.  Pairs of slices (s, t) with s + t <= kSlDigits - 1 are
// multiplied and each group m = s + t is summed in one binary32 accumulator:
// at most 12 pairs x b products of magnitude <= 256, so every partial sum is
// an integer below 2^24 (b <= 4096) and the sums are exact.
constexpr int kSlDigits = 12;
constexpr int kSlGroups = 12;             // m = s + t = 0 .. 11
constexpr int kSlRows = 128;              // RESID_SL item: 128 rows of R_i
constexpr int kSlNp = 16;                 // B operand rows: right-hand sides, padded to 16
constexpr uint32_t kSlChunk = 16384;      // A slice chunk: 128 rows x 128 bytes of K
constexpr uint32_t kSlXChunk = kSlNp * 128;   // X slice chunk: 16 rows x 128 bytes of K
// A slice part (one use-tile (I, J) of the symmetric matrix): chunks
// (rb, kc, s) at ((rb * nk + kc) * 12 + s) * 16 KiB, nk = b / 128; then b f64
// row sums of |A_IJ|; then the int32 scale exponent, padded to 16 bytes.
B3T_HD constexpr int64_t sl_a_part_bytes(int b) {
    return (int64_t)kSlDigits * b * b + 8 * (int64_t)b + 16;
}
// X slice part (part J): chunks (kc, t) at (kc * 12 + t) * 2 KiB; then 16
// int32 exponents (one per right-hand side); then per 16-row group and
// right-hand side max|x| (b / 16 x 16 f64).
B3T_HD constexpr int64_t sl_x_part_bytes(int b) {
    return (int64_t)kSlDigits * (b / 128) * kSlXChunk + 64 + (int64_t)(b / 16) * kSlNp * 8;
}

struct SliceArgs {
    int32_t i, j, T, b, nrhs;
};

// Sliced panel product of the mixed factorisation, L_ik = fp64(W_ik) U_k:
// W_ik sliced with one exponent per row (K = its columns), U_k with one
// exponent per column (K = its rows).  W slices: chunks (rb, kc, s) at
// ((rb * nk + kc) * 12 + s) * 16 KiB (128 rows x 128 bytes of K); U slices:
// for 32-column block cb, chunk set (cb, kc) of twelve 32 x 128-byte chunks
// at ((cb * nk + kc) * 12 + t) * 4 KiB.  Then b int32 exponents.
constexpr int kTsCols = 32;               // TRMM_SL item: 128 rows x 32 columns of L_ik
B3T_HD constexpr int64_t sl_w_bytes(int b) { return (int64_t)kSlDigits * b * b + 4 * (int64_t)b; }
B3T_HD constexpr int64_t sl_u_bytes(int b) { return (int64_t)kSlDigits * b * b + 4 * (int64_t)b; }

// One task as the device sees it: 64 bytes.
struct alignas(16) TaskRec {
    uint64_t buf[kMaxBuffers];   // device pointers, in the codelet's order
    int64_t n;                   // vector length (SCAL) or tile size b
    int32_t kind;
    int32_t nitems;              // work items the task is split into
    int32_t succ_off;            // first successor in the CSR array
    int32_t nsucc;
    int32_t aux;                 // POTRF: global column offset; MX: format; SCAL: item
                                 // chain (k > 0: head of k absorbed tasks, buf[1] = their
                                 // ids then their factor bits; -1: absorbed; 0: neither)
    uint32_t scal;               // SCAL: float factor bits
};
static_assert(sizeof(TaskRec) == 64, "TaskRec is 64 bytes");

// Device status + queue control block (one per launch arena).
struct alignas(128) Ctl {
    int32_t error;               // sticky: 0 or a positive errno
    int32_t err_task;            // task id that set it
    int32_t err_info;            // POTRF info (1-based global column)
    int32_t err_where;           // where it was raised (diagnostics)
    int32_t pad0[28];            // the error words alone on their line: every claim reads them
    unsigned long long retired;  // tasks retired in this launch (every retirement adds 1)
    unsigned long long subs_consumed;   // stream mode: submissions taken in
    int32_t pad1[28];
    // per-ring heads / tails (ring = level * nsub + sub), each on its own 128-byte line
    struct alignas(128) Level {
        unsigned long long head;
        unsigned long long tail;
        int32_t pad[28];
    } lvl[kMaxRings];
};

// Stream mode (a resident kernel fed with new task graphs while it runs).
// Written by the host through copies on a feed stream, read by the kernel.
struct alignas(128) StreamCtl {
    unsigned long long published_subs;   // submissions whose data is in place
    unsigned long long published_tasks;  // tasks in those submissions
    unsigned long long stop;             // host: no more submissions
    unsigned long long pad[13];
};

struct SubDesc {
    unsigned long long root_off;   // first root slot in the shared root array
    uint32_t nroots;
    uint32_t batch;
};

// One traced work item (globaltimer ns on the CTA's SM).
struct TraceRec {
    int32_t task, item, sm, kind;
    uint64_t t_start, t_end;
};
static_assert(sizeof(TraceRec) == 32, "TraceRec is 32 bytes");

// Kernel variants.  The executor is compiled once per family set below; a
// launch runs the smallest variant whose families cover its task kinds, so
// that a DAG of simple tasks is not compiled together with (and does not
// share registers with) the bodies it never runs.
constexpr uint32_t kFamScal = 1, kFamF64 = 2, kFamSolve = 4, kFamMx = 8;
constexpr uint32_t kVarScal = kFamScal, kVarF64 = kFamF64, kVarSolve = kFamSolve,
                   kVarNoMx = kFamScal | kFamF64 | kFamSolve, kVarAll = kVarNoMx | kFamMx;
B3T_HD constexpr uint32_t family_of(int kind) {
    return kind == kScalF32 ? kFamScal
         : (kind == kPotrf || kind == kTrsm || kind == kSyrk || kind == kGemm || kind == kPotrfD ||
            kind == kPanelTrsm || kind == kPanelUpd) ? kFamF64
         : ((kind >= kTrsvL && kind <= kNrm) || kind == kTrtri || kind == kTrtriCol || kind == kSliceA ||
            kind == kSliceX) ? kFamSolve
         : (kind == kSliceW || kind == kSliceU || kind == kTrmmSl) ? kFamMx
         : (kind >= kPotrfMx && kind <= kQuant) || kind == kCvt || kind == kTrmmMx || kind == kResidSl ? kFamMx
         : 0u;   // NOOP runs in every variant
}
B3T_HD constexpr uint32_t variant_of(uint32_t fams) {
    return (fams & kFamMx) ? kVarAll
         : (fams & ~kVarScal) == 0 ? kVarScal
         : (fams & ~kVarF64) == 0 ? kVarF64
         : (fams & ~kVarSolve) == 0 ? kVarSolve
         : kVarNoMx;
}

struct LaunchParams {
    const TaskRec *tasks;
    const int32_t *succ;         // CSR successor lists
    const int32_t *level;        // ready-queue level of each task
    int32_t *counters;           // remaining predecessors per task
    int32_t *done_items;         // finished items per task
    int32_t *next_item;          // next item to hand out, per task
    unsigned long long *slots;   // ready rings (one slot per task), rings back to back
    Ctl *ctl;
    unsigned long long ring_off[kMaxRings];   // first slot of each ring (ring = level * nsub + sub)
    unsigned long long ring_cap[kMaxRings];
    int64_t ntasks;
    int32_t nlevels;
    int32_t nsub;                // rings per level (task t of level l goes to ring l * nsub + t % nsub)
    int32_t has_mx;              // launch holds tcgen05 work: allocate TMEM
    uint32_t variant;            // kernel variant (family set) the launch runs
    uint32_t fams;               // families of the launch's kinds (0: empty tasks only)
    int64_t timeout_ns;
    int32_t debug;
    int32_t stream_mode;
    int32_t scal_stages;         // 16 KiB stages of the SCAL bulk-copy ring (fit the dynamic shared memory)
    // stream mode only
    const StreamCtl *sctl;
    const SubDesc *subs;
    const unsigned long long *sroots;
    const int32_t *task_batch;
    int32_t *batch_left;
    int32_t *batch_info;            // first POTRF info of a batch (device)
    volatile int32_t *batch_done;   // host-mapped: 1 when a batch retired, 2 + info if a
                                    // POTRF of it met a non-positive pivot
    int64_t deadline_ns;
    // tracing (null when off): one record per finished work item
    TraceRec *trace;
    unsigned long long *trace_n;
    int64_t trace_cap;
};

// Init-kernel parameters: reset counters, rings and status for a launch.
struct InitParams {
    const int32_t *indeg;        // initial counters
    int32_t *counters;
    int32_t *done_items;
    int32_t *next_item;
    unsigned long long *slots;
    unsigned long long nslots;
    const unsigned long long *roots;      // root task slots, per ring back to back
    unsigned long long root_off[kMaxRings];
    unsigned long long root_cnt[kMaxRings];
    Ctl *ctl;
    int64_t ntasks;
    int32_t nlevels;
    int32_t nrings;              // nlevels * nsub
};

constexpr unsigned long long kEmpty = ~0ull;

// A ready-ring slot names a task and carries its item count.
B3T_HD inline unsigned long long pack_slot(int64_t task, int32_t nitems) {
    return ((unsigned long long)task << 32) | (uint32_t)nitems;
}

}  // namespace b3t

// Launch entry points implemented in executor.cu.
extern "C" {
int b3t_internal_launch(const b3t::InitParams *ip, const b3t::LaunchParams *lp,
                        int nctas, size_t smem, void *stream, void *ev_start, void *ev_stop);
int b3t_internal_occupancy(int *ctas_per_sm, size_t smem, int *num_sms, uint32_t variant);
int b3t_internal_launch_exec(const b3t::LaunchParams *lp, int nctas, size_t smem, void *stream, void *ev_start);
size_t b3t_internal_smem_bytes(uint32_t variant, int32_t scal_stages);
int32_t b3t_internal_scal_stages(uint32_t variant, size_t smem);
}
