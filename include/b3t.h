/*
 * b3t: a task-DAG executor for one B300 GPU (sm_103a).
 *
 * The programming model is the one of Section 2 of the paper (Courtes,
 * "C Language Extensions for Hybrid CPU/GPU Programming with StarPU"):
 *   - a task is declared with its implementation, its number of buffer
 *     parameters and one access mode per buffer (read-only, write-only or
 *     read-write), like the paper's codelet structure;
 *   - buffers are registered before tasks use them;
 *   - invoking a task is asynchronous: it only adds the task to the
 *     scheduler's queue; the access modes together with the order of the
 *     invocations determine the dependency graph;
 *   - a wait joins every pending task.
 * Here every task has exactly one implementation, a CUDA device function
 * run by a persistent kernel; there is no CPU implementation and no
 * fallback.
 *
 * Conventions for every function below:
 *   - Return value: 0 on success, a negative errno value on failure (the
 *     generated task body of Section 3.2 turns a non-zero error into
 *     strerror(-err); this library never aborts, the caller decides).
 *     b3t_strerror() gives a message.
 *   - Pointers passed as buffers are DEVICE pointers, owned by the caller
 *     (for instance torch tensors).  The caller keeps them alive and
 *     unmodified by other work until the tasks using them have completed
 *     (b3t_task_wait, b3t_data_acquire or b3t_data_unregister): the
 *     ownership rule behind the paper's warning about registering automatic
 *     variables (Section 3.4).
 *   - The library owns handles, codelets, task records and its own device
 *     scratch (task table, dependency counters, ready queue, status word).
 *   - A context is not thread-safe; use one context per host thread.
 *   - All calls are non-blocking except b3t_task_wait, b3t_data_acquire,
 *     b3t_data_unregister, b3t_tiles_unregister and b3t_shutdown.
 */
#ifndef B3T_H
#define B3T_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define B3T_API __attribute__((visibility("default")))
#else
#define B3T_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct b3t_ctx b3t_ctx;
typedef int32_t b3t_handle;
typedef int32_t b3t_codelet;
typedef int32_t b3t_graph;

/* Access modes.  Section 3.2: the generated invocation passes a read-write
 * buffer with mode value 3; read and write are the two bits of it. */
enum { B3T_R = 1, B3T_W = 2, B3T_RW = 3 };

/* Task implementations.  Each kind fixes its buffers (in order), their
 * modes, their element types and the scalar argument blob; b3t_task_decl
 * checks a declaration against it (Section 3.2: a signature mismatch between
 * a task and its implementation is diagnosed).  Tiles are b x b, contiguous,
 * column-major inside the tile (element (r, c) at r + c*b), registered with
 * ld = b, b a multiple of 64 (128 for the mixed-precision kinds).
 *
 *  kind            buffers (mode, type)                       scalars
 *  B3T_NOOP        0..4 buffers of any mode                   none
 *  B3T_SCAL_F32    x (RW, f32 vector, 16-byte aligned)        float f
 *                  x[i] <- fl32(x[i] * f)   (Section 2 example)
 *  B3T_POTRF       A_kk (RW, f64 tile)                        int32 col0
 *                  lower Cholesky in place; a pivot <= 0 or NaN makes the
 *                  wait return -EDOM with info = col0 + 1-based column
 *  B3T_TRSM        L_kk (R), A_ik (RW)  f64 tiles             none
 *                  A_ik <- A_ik L_kk^{-T}
 *  B3T_SYRK        A_ik (R), A_ii (RW)  f64 tiles             none
 *                  A_ii <- A_ii - A_ik A_ik^T (lower triangle only)
 *  B3T_GEMM        A_ik (R), A_jk (R), A_ij (RW)  f64 tiles   none
 *                  A_ij <- A_ij - A_ik A_jk^T
 *  Mixed precision: W tiles binary32, L tiles f64, Q tiles quantised
 *  (fmt = B3T_FMT_BF16 or B3T_FMT_E4M3, layout below):
 *  B3T_POTRF_MX    W_kk (R, f32), L_kk (W, f64)               int32 col0
 *                  L_kk = chol(fp64(W_kk)); strict upper part of L_kk = 0
 *  B3T_TRSM_MX     L_kk (R), W_ik (R, f32), L_ik (W, f64)     none
 *                  L_ik = fp64(W_ik) L_kk^{-T} (substitution, row blocks)
 *  B3T_TRMM_MX     U_k (R, f64), W_ik (R, f32), L_ik (W, f64) none
 *                  L_ik = fp64(W_ik) U_k with U_k = L_kk^{-T} from B3T_TRTRI
 *                  (upper triangular, zeros below the diagonal): the same
 *                  panel solve as a product, in independent 64 x 64 blocks,
 *                  summed over p ascending with one FMA per term
 *  B3T_QUANT       L_ik (R, f64), Q_ik (W)                    int32 fmt
 *                  Q_ik = RN_fmt(L_ik / 2^e): one rounding from FP64 to the
 *                  format, to nearest, ties to even (E4M3 saturating at
 *                  448); e is the tile's scale exponent (0 for bf16; for
 *                  E4M3 the smallest e with max|L_ik| <= 448 * 2^e), so the
 *                  division is exact
 *  B3T_SYRK_MX     Q_ik (R), W_ii (RW, f32)                   int32 fmt
 *                  W_ii <- fl32(W_ii - 2^(2e) Q_ik Q_ik^T), lower triangle
 *  B3T_GEMM_MX     Q_ik (R), Q_jk (R), W_ij (RW, f32)         int32 fmt
 *                  W_ij <- fl32(W_ij - 2^(ei+ej) Q_ik Q_jk^T)
 *  The products of the MX updates are exact and are accumulated in binary32
 *  on the tensor cores (tcgen05).
 */
enum b3t_kind {
    B3T_NOOP = 0,
    B3T_SCAL_F32 = 1,
    B3T_POTRF = 2,
    B3T_TRSM = 3,
    B3T_SYRK = 4,
    B3T_GEMM = 5,
    B3T_POTRF_MX = 6,
    B3T_TRSM_MX = 7,
    B3T_SYRK_MX = 8,
    B3T_GEMM_MX = 9,
    B3T_QUANT = 10,
    B3T_TRSV_L = 11,
    B3T_GEMV_L = 12,
    B3T_TRSV_LT = 13,
    B3T_GEMV_LT = 14,
    B3T_AXPY = 15,
    B3T_RESID = 16,
    B3T_NRM = 17,
    B3T_POTRF_D = 18,
    B3T_PANEL_TRSM = 19,
    B3T_PANEL_UPD = 20,
    B3T_CVT = 21,
    B3T_TRTRI = 22,
    B3T_TRMM_MX = 23,
    B3T_SLICE_A = 24,
    B3T_SLICE_X = 25,
    B3T_RESID_SL = 26,
    B3T_SLICE_W = 27,
    B3T_SLICE_U = 28,
    B3T_TRMM_SL = 29,
    B3T_TRTRI_COL = 30
};

/* Diagonal tile split into column panels.  A b x b diagonal tile partitioned
 * (b3t_data_partition, the filters of Section 5.1) into np = b / pw column
 * panels of b x pw (pw = 64 or 128; panel kk is columns kk*pw.. of the tile,
 * leading dimension b) is factored by a small DAG instead of one POTRF, so
 * that several CTAs work on it:
 *   for kk: POTRF_D(P_kk); PANEL_TRSM(P_kk) (kk < np-1);
 *           for jj > kk: PANEL_UPD(P_kk, P_jj)
 *  B3T_POTRF_D     P_kk (RW)       Cholesky of the pw x pw block at row kk*pw
 *  B3T_PANEL_TRSM  P_kk (RW)       rows below it: X <- X L_d^{-T}
 *  B3T_PANEL_UPD   P_kk (R), P_jj (RW)
 *                  P_jj(r, :) -= P_kk(r, :) P_kk(jj*pw.., :)^T for rows
 *                  r >= jj*pw (lower part on the diagonal block)
 *  Scalars: struct b3t_panel_args; col0 offsets POTRF info like B3T_POTRF.
 *  B3T_TRTRI_COL   P_cb (R, panel part cb of L_kk, pw = 64), V_{cb-1} (R),
 *                  V_cb (W): column block cb (columns 64 cb ..) of U_k =
 *                  L_kk^{-T}, V_j being U_k's column blocks (a partition of
 *                  the U tile into b x 64 parts; cb = 0 names V_0 twice).  The
 *                  block needs the columns before it and rows 64 cb .. of
 *                  L_kk, final once panel cb is factored, so the blocks follow
 *                  the panel DAG instead of the whole diagonal factor; the
 *                  same per-element operations as B3T_TRTRI.  Scalars: struct
 *                  b3t_panel_args with kk = cb.
 *  B3T_CVT         W_kk (R, f32 tile), L_kk (W, f64 tile): L = fp64(W) on the
 *                  lower triangle, 0 above; no scalars.
 *  B3T_TRTRI       L_kk (R, f64 tile), U_k (W, f64 tile): U_k = L_kk^{-T}
 *                  (upper triangular; 0 below the diagonal), computed in FP64
 *                  by substitution against the identity; no scalars.  The
 *                  solves of the refinement use it so that every diagonal
 *                  step is a triangular multiply (Section 2's tasks over
 *                  registered buffers; the inverse is this build's choice). */
typedef struct b3t_panel_args {
    int32_t b, pw, kk, jj, col0;
} b3t_panel_args;

/* Vector kinds (solves and refinement).  A block vector with nrhs <= 32
 * right-hand sides is split into T parts of b rows; part k holds Y_k(r, j) at
 * j*b + r.  Scalars: struct b3t_vec_args below (20 bytes).
 *  B3T_TRSV_L   L_kk (R, f64 tile), Y_k (RW)          Y_k <- L_kk^{-1} Y_k
 *  B3T_GEMV_L   L_ik (R), Y_k (R), Y_i (RW)           Y_i <- Y_i - L_ik Y_k
 *  B3T_TRSV_LT  L_kk (R), Y_k (RW)                    Y_k <- L_kk^{-T} Y_k
 *  B3T_GEMV_LT  L_ki (R), Y_k (R), Y_i (RW)           Y_i <- Y_i - L_ki^T Y_k
 *               (flags bit 0: compute in binary32, store FP64; bit 1:
 *               assign Y_i <- M Y_k instead of subtracting; bit 2 / bit 3:
 *               M is lower / upper triangular, so zero blocks are skipped)
 *  B3T_AXPY     X_i (RW), D_i (R)                     X_i <- X_i + D_i
 *               (flags bit 1: X_i <- D_i)
 *  B3T_RESID    A (R, all T(T+1)/2 packed f64 tiles as one buffer), X (R,
 *               T parts), B (R, T parts), R_i (W, b3t_resid_part_elems
 *               elements): R_i <- B_i - (A X)_i in FP64 with A symmetric and
 *               only its lower tiles stored; after the b*nrhs values, R_i
 *               holds per 16-row item max|r_j|, max|x_j|, max|b_j| and the largest
 *               row sum of |A| (flags bit 1: X taken as 0, R_i <- B_i;
 *               bit 4: keep the row-sum partials an earlier residual wrote,
 *               for refinement steps after the first)
 *  B3T_NRM      R (R, the T residual parts back to back), B (R), eta (W,
 *               nrhs + 1 f64):
 *               eta_j = max|r_j| / (||A||_inf max|x_j| + max|b_j|),
 *               eta[nrhs] = max_j eta_j (normwise backward error) */
typedef struct b3t_vec_args {
    int32_t nrhs, flags, i, T, b;
} b3t_vec_args;

/* Sliced FP64 residual (the refinement's r = b - A x with the products on
 * the tensor cores; the Ozaki scheme, Ozaki, Ogita, Oishi and Rump, Numer.
 * Algorithms 59, 2012).  A value v of a block with scale exponent e (the
 * smallest e = ilogb(max|block|) + 3, so |v| < 2^(e-2); 0 for a zero block)
 * is V = trunc(v 2^(60-e)) written as twelve balanced base-32 digits d_s in
 * [-16, 15], V = sum_s d_s 32^(11-s), each an exact E4M3 value ("slice" s).
 * The product of an A tile and an X part keeps the slice pairs with
 * s + t <= 11, each group m = s + t summed exactly in binary32 on the tensor
 * cores, and adds it in FP64 with its scale 2^(eA + eX - 5 (m + 2)).  Per
 * product term a*x the error is below 2^(eA + eX - 58.3); the FP64 sum
 * takes two roundings per tile.  b a multiple of 128 (<= 4096), nrhs <= 16.
 * Scalars: struct b3t_slice_args.
 *  B3T_SLICE_A   A (R, all T(T+1)/2 packed f64 tiles), D_ij (W), D_ji (W):
 *                the slices of the stored tile (i, j), j <= i, for its two
 *                uses: D_ij for A_ij (rows of block i), D_ji for A_ij^T
 *                (rows of block j); a diagonal tile passes the same part
 *                twice and has the one symmetric use.  A part
 *                (b3t_slice_a_part_bytes) holds, for 128-row block rb,
 *                128-column block kc and slice s, a 16 KiB chunk at
 *                ((rb * b/128 + kc) * 12 + s) * 16384 in the quantised tile
 *                layout (row r at r*128, 16-byte group g at g ^ (r % 8));
 *                then the b row sums of |A_use| (f64), then the int32
 *                exponent (padded to 16 bytes).
 *  B3T_SLICE_X   X_j (R, part of b*nrhs f64), E_j (W): the slices of the
 *                part, right-hand sides as 16 rows (zero padded): chunk
 *                (kc, t) of 16 x 128 bytes at (kc * 12 + t) * 2048 (same
 *                swizzle), then 16 int32 exponents, then per 16-row group
 *                and right-hand side max|x| (b/16 x 16 f64).
 *  B3T_RESID_SL  D (R, the T x T parts of use (I, J) at (I*T + J) *
 *                b3t_slice_a_part_bytes), E (R, T parts), B (R, T parts),
 *                R_i (W, b3t_resid_part_elems f64): R_i <- B_i - (A X)_i,
 *                with the per-16-row maxima of B3T_RESID (row sums of |A|
 *                from the A slice parts); items of 128 rows. */
typedef struct b3t_slice_args {
    int32_t i, j, T, b, nrhs;
} b3t_slice_args;
B3T_API size_t b3t_slice_a_part_bytes(int32_t b);
B3T_API size_t b3t_slice_x_part_bytes(int32_t b);

/* Sliced panel product of the mixed factorisation, L_ik = fp64(W_ik) U_k
 * (the product of B3T_TRMM_MX) with the slices of both operands on the
 * tensor cores: row r of W_ik is sliced with its own exponent eW[r] (K = the
 * columns), column c of U_k with eU[c] (K = the rows); the kept pairs' group
 * sums are combined as for B3T_RESID_SL and each element of L_ik is
 * H 2^(eW+eU-35) + L 2^(eW+eU-65) with one rounding.  Per product term the
 * error is below 2^(eW[r]+eU[c]-58.3).  No scalars; b = the tile's leading
 * dimension (a multiple of 128, <= 4096).
 *  B3T_SLICE_W  W_ik (R, f32 tile), WS_ik (W, b3t_slice_w_bytes): chunks
 *               (rb, kc, s) of 128 rows x 128 bytes of K at
 *               ((rb * b/128 + kc) * 12 + s) * 16384 (quantised-tile swizzle),
 *               then b int32 row exponents; items of 128 rows.
 *  B3T_SLICE_U  U_k (R, f64 tile), US_k (W, b3t_slice_u_bytes): per
 *               32-column block cb and K chunk kc, twelve chunks of 32 rows
 *               (columns of U) x 128 bytes at ((cb * b/128 + kc) * 12 + t) *
 *               4096, then b int32 column exponents; items of 32 columns.
 *  B3T_TRMM_SL  US_k (R), WS_ik (R), L_ik (W, f64 tile): items of 128 x 32;
 *               U_k must be zero below its diagonal (B3T_TRTRI's output). */
B3T_API size_t b3t_slice_w_bytes(int32_t b);
B3T_API size_t b3t_slice_u_bytes(int32_t b);
enum { B3T_VEC_F32 = 1, B3T_VEC_ASSIGN = 2, B3T_VEC_LOWER_M = 4, B3T_VEC_UPPER_M = 8, B3T_VEC_KEEP_NORM = 16 };

/* Low-precision formats of the Q tiles. */
enum b3t_fmt { B3T_FMT_BF16 = 0, B3T_FMT_E4M3 = 1 };

/* Quantised tile layout (Q tiles).  A b x b tile is cut into 16 KiB chunks
 * of 128 rows x 128 bytes of K (64 bf16 or 128 E4M3 columns); with
 * nk = b * esize / 128, chunk (rb, kb) covers rows 128*rb.. and starts at byte
 * (rb * nk + kb) * 16384.  Inside a chunk, row r occupies bytes r*128.. and its
 * 16-byte group g (columns ascending) is stored at group position g ^ (r % 8).
 * After the b*b*esize data bytes: int32 scale exponent e, padded to 16 bytes.
 * b3t_q_bytes() gives the total size (0 for invalid arguments). */
B3T_API size_t b3t_q_bytes(int b, int fmt);

typedef struct b3t_config {
    int64_t timeout_ns;     /* bound on any device-side wait; 0 = 10 s */
    int32_t ctas_per_sm;    /* persistent CTAs per SM; 0 = automatic */
    int32_t prio_levels;    /* ready-queue priority levels 1..8; 0 = 8 */
    int32_t debug_checks;   /* 1: kernels bounds-check task ids and items */
    int32_t host_only;      /* 1: no CUDA device is touched; registration,
                               submission and DAG inspection work, flush /
                               wait / replay return -ENODEV (for tools and
                               CPU-only tests of the dependency logic) */
    int32_t prio_policy;    /* ready-queue order: B3T_PRIO_CRITICAL (0,
                               default): critical path first (Section 5.3's
                               upward and downward ranks): the tasks whose
                               upward plus downward rank is the graph's
                               longest path take the top level, the others
                               the levels below by upward rank;
                               B3T_PRIO_DEPTH (1): deepest task first, so a
                               successor runs right after its predecessor
                               while the data is in L2; B3T_PRIO_UPWARD (2):
                               longest remaining path first (upward rank
                               alone, over all levels).  Any other value is
                               taken as the default */
    int32_t stream_free_sms; /* stream mode: SMs the resident kernel leaves
                               free for other work issued meanwhile (input
                               generation, copies); 0 = 8 */
    int32_t stream_no_mx;    /* stream mode: 1 runs the resident kernel
                               without the tensor-memory path (two CTAs per
                               SM instead of one, for FP64-only streams); a
                               batch holding a mixed-precision kind is then
                               refused (-EINVAL) */
    int32_t item_chains;     /* 1: successor-first at item granularity for
                               vector-scaling chains (Section 2's scheduler
                               with a partial view of the graph).  A
                               B3T_SCAL_F32 task whose only successor is a
                               B3T_SCAL_F32 task on the same buffer, with no
                               other predecessor, passes item i of that
                               successor to the CTA running its own item i:
                               the item reads exactly what item i of the
                               task wrote, so the CTA applies both factors,
                               in submission order and each rounded, to the
                               chunk it holds, and stores it once.  A chain
                               is a head and up to 32 absorbed tasks after
                               it.  Results are bit for bit
                               those of task-by-task execution; every task
                               still retires, and edges leaving a chain are
                               released when its last task retires.  Applies
                               to launches without mixed-precision kinds
                               (not to stream mode).  0 (default): task by
                               task. */
} b3t_config;

enum { B3T_PRIO_CRITICAL = 0, B3T_PRIO_DEPTH = 1, B3T_PRIO_UPWARD = 2 };

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream; NULL = the
 * legacy default stream).  cfg may be NULL.  -ENODEV without a CUDA device
 * (unless cfg->host_only), -ENOMEM when host or device memory runs out. */
B3T_API int b3t_init(b3t_ctx **ctx, const b3t_config *cfg, void *cuda_stream);

/* Wait for all pending work, release every library-owned resource and the
 * context.  Registered buffers stay the caller's. */
B3T_API int b3t_shutdown(b3t_ctx *ctx);

/* Declare a task (the codelet of Section 2): its name (for debugging, like
 * the codelet's name field), its implementation kind, the number of buffer
 * parameters, their modes and the size of its scalar blob.  -EINVAL if the
 * declaration does not match the kind's signature (Section 3.2). */
B3T_API int b3t_task_decl(b3t_ctx *ctx, const char *name, int kind, int nbuffers,
                          const uint8_t *modes, size_t scalar_bytes, b3t_codelet *out);

/* Register a device buffer (Section 2: buffers passed to tasks must be
 * registered first): nelems elements of elemsize bytes starting at
 * dev_ptr; ld = 0 for a vector, ld = b for a b x b tile.  The same address
 * may not be registered twice (-EEXIST).  -EINVAL on a null pointer or zero
 * size. */
B3T_API int b3t_data_register(b3t_ctx *ctx, void *dev_ptr, size_t nelems,
                              size_t elemsize, int64_t ld, b3t_handle *out);

/* Handle of a registered pointer (Section 3.2: the generated task body looks
 * the pointer up and reports an unregistered pointer).  -ENOENT if none. */
B3T_API int b3t_data_lookup(b3t_ctx *ctx, const void *dev_ptr, b3t_handle *out);

/* Split a registered buffer into nparts consecutive parts of part_nelems
 * elements each (the filters of Section 5.1).  Each part gets a handle of
 * its own; a task that names the parent accesses every part.  The parent
 * may not be partitioned twice (-EEXIST), nor while pending tasks name it
 * (-EBUSY); nparts * part_nelems must fit in it (-EINVAL). */
B3T_API int b3t_data_partition(b3t_ctx *ctx, b3t_handle parent, int32_t nparts,
                               size_t part_nelems, b3t_handle *parts_out);

/* Submit one task (asynchronous, Section 3.3): handles in the codelet's
 * buffer order, with the modes the caller uses them in (NULL = the
 * declaration's; otherwise they must equal it: -EINVAL), and the scalar
 * blob.  Dependencies on earlier submissions are derived here from the
 * access modes: read-after-write, write-after-read and write-after-write,
 * per buffer, in submission order.  -ENOENT for an unregistered handle;
 * -EINVAL for buffers whose size, alignment or type does not fit the kind.
 * The task runs at the next b3t_task_flush / b3t_task_wait. */
B3T_API int b3t_task_submit(b3t_ctx *ctx, b3t_codelet cl, const b3t_handle *handles,
                            const uint8_t *modes, int nbuffers, const void *scalars,
                            size_t scalar_bytes);

/* Same, naming the buffers by device pointer; each pointer is looked up like
 * the generated task body of Section 3.2 does (-ENOENT: "attempt to use
 * unregistered pointer"). */
B3T_API int b3t_task_submit_ptrs(b3t_ctx *ctx, b3t_codelet cl, void *const *ptrs,
                                 int nbuffers, const void *scalars, size_t scalar_bytes);

/* Launch every pending task as one persistent-kernel run on the context's
 * stream and return without waiting.  Tasks submitted later depend on the
 * flushed ones through stream order. */
B3T_API int b3t_task_flush(b3t_ctx *ctx);

/* Flush, then wait for every submitted task (Section 2: wait for all;
 * Section 3.3: the wait pragma) and read the device status words of the
 * launches since the last wait.  timeout_ns bounds the host wait (0 = no
 * bound; -ETIMEDOUT when it expires with work still running).  Returns
 * -ETIMEDOUT if a device-side wait ran past the context's timeout, -EDOM if
 * a POTRF met a non-positive pivot (see b3t_last_error), -EIO on a CUDA
 * error. */
B3T_API int b3t_task_wait(b3t_ctx *ctx, int64_t timeout_ns);

/* Make a buffer safe for host-side use (Section 3.4, acquire pragma): waits
 * for the tasks that write it (mode R) or also read it (mode W / RW).  It
 * currently flushes and joins ALL pending and in-flight work of the context,
 * a superset of those tasks (one persistent launch runs the whole batch, so
 * a per-buffer wait would not return earlier).  -ENOENT for an unknown
 * handle, -EINVAL for a mode outside 1..3, -EBUSY while capturing. */
B3T_API int b3t_data_acquire(b3t_ctx *ctx, b3t_handle h, uint8_t mode);

/* Wait for the tasks using the buffer, then forget the handle (Section 2).
 * Unregistering a partitioned parent unregisters its parts.  In stream mode
 * it does not wait: -EBUSY while an unfinished batch uses the buffer. */
B3T_API int b3t_data_unregister(b3t_ctx *ctx, b3t_handle h);

/* Detail of the last device-side failure: the task id (in submission order
 * within its launch) and the POTRF info (1-based global column), or -1. */
B3T_API int b3t_last_error(b3t_ctx *ctx, int32_t *task_id, int32_t *info);

/* Static message for a return code of this library. */
B3T_API const char *b3t_strerror(int err);

/* Repeated DAGs.  Between capture_begin and capture_end, submissions are
 * recorded instead of launched; capture_end builds the task table and the
 * dependency graph once, uploads them, and captures the launch (counter
 * reset + persistent kernel) into a CUDA graph.  replay launches it on the
 * context's stream without waiting; b3t_task_wait joins it.  The graph names
 * the same buffers every time; their contents are whatever they hold at
 * replay.  -EBUSY if tasks are pending at capture_begin. */
B3T_API int b3t_graph_capture_begin(b3t_ctx *ctx);
B3T_API int b3t_graph_capture_end(b3t_ctx *ctx, b3t_graph *out);
B3T_API int b3t_graph_replay(b3t_ctx *ctx, b3t_graph g);
B3T_API int b3t_graph_destroy(b3t_ctx *ctx, b3t_graph g);

/* Introspection of the pending (not yet flushed) batch, for tests and
 * tools: number of tasks and derived edges, and the edges themselves as
 * (pred, succ) pairs of task indices in submission order (pred < succ).
 * Writes at most cap pairs. */
B3T_API int b3t_dag_stats(b3t_ctx *ctx, int64_t *ntasks, int64_t *nedges);
B3T_API int b3t_dag_edges(b3t_ctx *ctx, int32_t *pred, int32_t *succ, int64_t cap,
                          int64_t *count);

/* Scheduling priority of the pending batch's tasks, as the next flush will
 * use it (Section 5.3: upward rank as a scheduling hint): rank[t] is, under
 * B3T_PRIO_UPWARD and B3T_PRIO_CRITICAL, the longest path from task t to the
 * end of the graph weighted by the library's per-kind cost estimate (ns on
 * one CTA; t's own cost included), or, under B3T_PRIO_DEPTH, the number of
 * tasks on the longest path from a source to t; level[t] in
 * 0..prio_levels-1 is the ready queue level (higher is claimed first):
 * floor(L * rank / (max rank * 1.000001)) for upward rank, min(L - 1, rank)
 * for depth; for critical, L - 1 if the longest path through t (its
 * downward rank, the longest cost-weighted path from a source to t with t's
 * cost excluded, plus its upward rank) is the graph's longest path, else
 * min(L - 2, floor((L - 1) * rank / (max rank * 1.000001))); 0 with one
 * level.
 * Writes at most cap entries of each (either pointer may be NULL); *count =
 * number of pending tasks. */
B3T_API int b3t_dag_levels(b3t_ctx *ctx, float *rank, int32_t *level, int64_t cap, int64_t *count);

/* Item chains of the pending batch, as the next flush will form them (see
 * b3t_config.item_chains): aux[t] = k > 0 if task t heads a chain of k
 * absorbed B3T_SCAL_F32 tasks, -1 if t is absorbed, 0 otherwise (always 0
 * with item_chains off or when the batch holds a mixed-precision kind).
 * Writes at most cap entries; *count = number of pending tasks. */
B3T_API int b3t_dag_item_chains(b3t_ctx *ctx, int32_t *aux, int64_t cap, int64_t *count);

/* Launch statistics of the last launch (flush or replay): tasks, work
 * items, persistent CTAs, and the device time of the persistent kernel (or
 * of the replayed graph) in ns, measured with CUDA events on the context's
 * stream; valid after b3t_task_wait, -1 otherwise. */
B3T_API int b3t_last_launch(b3t_ctx *ctx, int64_t *ntasks, int64_t *nitems,
                            int32_t *nctas, int64_t *kernel_ns);

/* Add one phantom dependency to a pending task so that its counter never
 * reaches zero: the launch then ends through the device-side timeout
 * (-ETIMEDOUT), never by hanging.  For failure-detection tests. */
B3T_API int b3t_debug_block_task(b3t_ctx *ctx, int64_t task_index);

/* ---------------------------------------------------------------------
 * Tiled Cholesky helpers, built on the calls above.  Tiles are passed as an
 * array of T(T+1)/2 device pointers to b x b column-major tiles in packed
 * column order: tile (i, j), i >= j, at index j*T - j(j-1)/2 + (i - j).
 * Every tile is registered as its own buffer (the workaround Section 5.1
 * gives for partitioned matrices; already registered tiles are reused) and
 * the right-looking task order is submitted:
 *   for k: POTRF(A_kk); for i>k: TRSM(A_kk, A_ik);
 *          for i>k: SYRK(A_ik, A_ii); for k<j<i: GEMM(A_ik, A_jk, A_ij)
 * col0 is added to POTRF info values (global column of the first tile).
 * Several submissions before one wait run in one launch (batching). */
B3T_API int b3t_cholesky_submit(b3t_ctx *ctx, double *const *tiles, int32_t T, int32_t b,
                                int32_t col0);

/* Mixed precision, right-looking:
 *   for k: POTRF_MX(W_kk, L_kk);
 *          for i>k: TRSM_MX(L_kk, W_ik, L_ik), QUANT(L_ik, Q_ik);
 *          for i>k: SYRK_MX(Q_ik, W_ii); for k<j<i: GEMM_MX(Q_ik, Q_jk, W_ij)
 * W tiles (binary32, caller-initialised, e.g. to fl32(A)), L tiles (f64) and
 * Q tiles (b3t_q_bytes(b, fmt) bytes each; the diagonal ones are unused)
 * receive the results. */
B3T_API int b3t_cholesky_mx_submit(b3t_ctx *ctx, float *const *W, double *const *L,
                                   void *const *Q, int32_t T, int32_t b, int32_t fmt,
                                   int32_t col0);

/* Mixed precision with the panel solve as a product with the inverted
 * diagonal tile (the trailing updates as in b3t_cholesky_mx_submit):
 *   for k: POTRF_MX(W_kk, L_kk) (or CVT + the panel DAG for b >= 256);
 *          TRTRI(L_kk, U_k) (k < T-1);
 *          for i>k: TRMM_MX(U_k, W_ik, L_ik), QUANT(L_ik, Q_ik);
 *          for i>k: SYRK_MX(Q_ik, W_ii); for k<j<i: GEMM_MX(Q_ik, Q_jk, W_ij)
 * U: T pointers to b x b f64 tiles of caller-owned scratch (U_k = L_kk^{-T}
 * on return, for k < T-1).  An explicit inverse rounds differently from
 * substitution, and its error grows with the condition number of L_kk
 * (about kappa(L_kk) times the FP64 unit roundoff, relative): on the
 * well-conditioned diagonal tiles of A = B B^T / N + c I it agrees with
 * B3T_TRSM_MX to ~1e-15; for ill-conditioned tiles use
 * b3t_cholesky_mx_submit.  -EINVAL for a bad shape or format. */
B3T_API int b3t_cholesky_mx_inv_submit(b3t_ctx *ctx, float *const *W, double *const *L,
                                       void *const *Q, double *const *U, int32_t T, int32_t b,
                                       int32_t fmt, int32_t col0);

/* b3t_cholesky_mx_inv_submit with the panel product sliced onto the tensor
 * cores: per step k, TRTRI(L_kk -> U_k), SLICE_U(U_k -> US_k), and for every
 * i > k SLICE_W(W_ik -> WS_ik), TRMM_SL(US_k, WS_ik -> L_ik), QUANT(L_ik ->
 * Q_ik); the updates as in b3t_cholesky_mx_submit.  WS: T(T+1)/2 pointers
 * in the packed order (the diagonal entries are not used) to
 * b3t_slice_w_bytes(b) bytes each; US: T pointers to b3t_slice_u_bytes(b)
 * bytes (the last one is not used).  b a multiple of 128 (-EINVAL
 * otherwise). */
B3T_API int b3t_cholesky_mx_sliced_submit(b3t_ctx *ctx, float *const *W, double *const *L, void *const *Q,
                                          double *const *U, void *const *WS, void *const *US, int32_t T,
                                          int32_t b, int32_t fmt, int32_t col0);

/* Solves with a tiled Cholesky factor: Y <- (L L^T)^{-1} Y, submitted as
 * TRSV_L / GEMV_L tasks (forward, k ascending) then TRSV_LT / GEMV_LT tasks
 * (backward, k descending).  L: T(T+1)/2 f64 tile pointers (packed order;
 * only lower triangles read).  Y: device f64 block vector of T parts,
 * part_stride elements apart (>= b*nrhs); registered and partitioned here if
 * it is not already.  flags: B3T_VEC_F32 for binary32 arithmetic. */
B3T_API int b3t_chol_solve_submit(b3t_ctx *ctx, double *const *L, double *Y, int32_t T, int32_t b,
                                  int32_t nrhs, int64_t part_stride, int32_t flags);

/* Tracing.  While it is on, every launch built (flushed, captured or opened
 * in stream mode) records one b3t_trace_rec per finished work item: task id
 * (index in its launch, or in the stream's task arena), item, SM, kind, and
 * the item's start and end on the device clock (%globaltimer, ns).  Records
 * beyond the capacity are counted but dropped.
 *  b3t_trace_start  waits for pending work, (re)allocates room for capacity
 *                   records (device memory, owned by the context, freed by
 *                   b3t_shutdown), zeroes the count and turns tracing on.
 *  b3t_trace_read   waits, copies min(count, capacity) records to host
 *                   memory and sets *count to the number of items traced.
 *  b3t_trace_stop   turns tracing off for launches built afterwards.
 * -ENODEV on a host-only context, -ENOENT (read) before any start, -EBUSY
 * while a stream is open. */
typedef struct b3t_trace_rec {
    int32_t task, item, sm, kind;
    uint64_t t_start_ns, t_end_ns;
} b3t_trace_rec;
B3T_API int b3t_trace_start(b3t_ctx *ctx, int64_t capacity);
B3T_API int b3t_trace_read(b3t_ctx *ctx, void *records, int64_t capacity, int64_t *count);
B3T_API int b3t_trace_stop(b3t_ctx *ctx);

/* U_k <- L_kk^{-T} for the T diagonal tiles of a tiled Cholesky factor
 * (TRTRI tasks, one per tile, 32-row items).  L: T(T+1)/2 f64 tile pointers
 * (packed order); U: T f64 tile pointers (b x b each, caller-owned); both
 * registered here if they are not already.  Returns 0 or -EINVAL (shape,
 * b not a multiple of 64). */
B3T_API int b3t_chol_inv_submit(b3t_ctx *ctx, double *const *L, double *const *U, int32_t T, int32_t b);

/* Y <- (L L^T)^{-1} Y with the inverted diagonal tiles U (from
 * b3t_chol_inv_submit, which must have been submitted earlier on this
 * context; the dependency on it is derived from the U registrations):
 *   forward, k ascending:   Z_k = U_k^T Y_k (GEMV_LT, assign, lower M);
 *                           Y_i -= L_ik Z_k for i > k (GEMV_L)
 *   backward, k descending: Y_k = U_k Z_k (GEMV_L, assign, upper M);
 *                           Z_i -= L_ki^T Y_k for i < k (GEMV_LT)
 * Y, Z: device f64 block vectors of T parts part_stride elements apart
 * (>= b*nrhs); Z is scratch.  Every step splits into 16-row items, so no
 * task runs a row-by-row substitution.  flags: B3T_VEC_F32. */
B3T_API int b3t_chol_solve_inv_submit(b3t_ctx *ctx, double *const *L, double *const *U, double *Y,
                                      double *Z, int32_t T, int32_t b, int32_t nrhs, int64_t part_stride,
                                      int32_t flags);

/* Elements (f64) of one RESID output part R_i: the b*nrhs residual values,
 * then per 16-row item max|r_j|, max|x_j| and max|b_j| (nrhs each) and the
 * largest row sum of |A|.  NRM reads T such parts back to back.  0 for
 * invalid arguments. */
B3T_API size_t b3t_resid_part_elems(int32_t b, int32_t nrhs);

/* Elements (f64) of the work area b3t_ir_solve and b3t_ir_step_submit need:
 * the residual parts (b*nrhs values plus per-item norm partials each), a
 * scratch block vector and the T inverted diagonal tiles of the factor, each
 * region 256-byte aligned.  0 for invalid arguments. */
B3T_API size_t b3t_ir_work_elems(int32_t T, int32_t b, int32_t nrhs);

/* Forget the registrations the refinement helpers made inside the work area
 * R (residual parts, scratch vector, inverted tiles), so that the memory can
 * be freed and reused.  Waits for pending tasks (outside stream mode); in
 * stream mode returns -EBUSY while a batch still uses them. */
B3T_API int b3t_ir_release(b3t_ctx *ctx, double *R, int32_t T, int32_t b, int32_t nrhs);

/* Iterative refinement, each step a task graph run by the executor:
 *   x_0 = 0, r_0 = b, U_k = L_kk^{-T} (TRTRI);  repeat  d = (L L^T)^{-1} r
 *   (solve tasks with the inverted diagonal tiles),
 *   x += d (AXPY), r = b - A x in FP64 (RESID), eta (NRM)
 * until eta <= tol (returns 0), max_iter steps (-ERANGE) or no progress
 * (eta above 0.9 x its previous value: -ERANGE).  A_packed: the original
 * matrix as T(T+1)/2 contiguous packed lower f64 tiles; L: factor tile
 * pointers (any precision history, FP64 storage); B, X: T parts of b*nrhs
 * f64; R: b3t_ir_work_elems f64; eta: nrhs + 1 f64 (device).  flags:
 * B3T_VEC_F32 for binary32 correction solves.  iters and eta_out (nrhs + 1
 * host doubles) report the result.  Blocks until done. */
B3T_API int b3t_ir_solve(b3t_ctx *ctx, const double *A_packed, double *const *L, const double *B,
                         double *X, double *R, double *eta, int32_t T, int32_t b, int32_t nrhs,
                         int32_t flags, double tol, int32_t max_iter, int32_t *iters, double *eta_out);

/* Bytes of the slice area b3t_ir_solve_sliced needs: the T x T A slice
 * parts, then (256-byte aligned) the T X slice parts.  0 for invalid
 * arguments (b a multiple of 128 up to 4096, T <= 4096). */
B3T_API size_t b3t_ir_slice_bytes(int32_t T, int32_t b);

/* b3t_ir_solve with the sliced FP64 residual (B3T_RESID_SL) in place of
 * B3T_RESID: the first step also slices every stored tile of A (SLICE_A),
 * every step slices x (SLICE_X) before the residual.  S: device area of
 * b3t_ir_slice_bytes(T, b) bytes, 256-byte aligned, owned by the caller; its
 * registrations are dropped before returning.  nrhs <= 16, b a multiple of
 * 128 (-EINVAL otherwise). */
B3T_API int b3t_ir_solve_sliced(b3t_ctx *ctx, const double *A_packed, double *const *L, const double *B,
                                double *X, double *R, void *S, double *eta, int32_t T, int32_t b,
                                int32_t nrhs, int32_t flags, double tol, int32_t max_iter, int32_t *iters,
                                double *eta_out);

/* ---------------------------------------------------------------------
 * Stream mode: continuous submission into one resident persistent kernel.
 * b3t_stream_open launches the executor on the context's stream and leaves it
 * running; each b3t_stream_submit hands it the tasks submitted since the last
 * call as one self-contained batch (edges only inside the batch), uploaded
 * through a separate feed stream and published with a counter: the tasks of
 * the new batch join the ready queue while earlier batches are still running,
 * so their work overlaps on the device.  Capacities are fixed at open
 * (-ENOMEM beyond; a batch whose upload exceeds 64 MiB: -E2BIG).  While the
 * stream is open the caller must not make calls that synchronise the whole
 * device (cudaDeviceSynchronize, cudaFree, cudaFreeHost, ...): they would wait
 * for the resident kernel.  The resident kernel leaves stream_free_sms SMs
 * (b3t_config) free so that other kernels issued meanwhile can run.  A batch may not name a buffer that an unfinished batch
 * uses (-EBUSY; the tasks stay pending).  The kernel exits after
 * b3t_stream_close once everything published has retired, or at deadline_ns
 * after open (-ETIMEDOUT).  While the stream is open, flush / wait / replay
 * on this context return -EBUSY.  A POTRF that meets a non-positive pivot does
 * not stop the stream: its batch completes with info set. */
B3T_API int b3t_stream_open(b3t_ctx *ctx, int64_t max_tasks, int64_t max_edges, int32_t max_batches,
                            int64_t deadline_ns);
B3T_API int b3t_stream_submit(b3t_ctx *ctx, int32_t *batch_id);
/* 1 if the batch has finished (info: 0, or the 1-based global column of a
 * non-positive pivot), 0 if it is still running, a negative errno if the
 * resident kernel stopped before finishing it.  Non-blocking. */
B3T_API int b3t_stream_query(b3t_ctx *ctx, int32_t batch, int32_t *info);
B3T_API int b3t_stream_close(b3t_ctx *ctx);

/* Submit one refinement step of b3t_ir_solve without waiting (first != 0:
 * start from x = 0, r = b), for callers that drive the loop themselves, such
 * as a serving loop in stream mode.  eta is written by the step's NRM task. */
B3T_API int b3t_ir_step_submit(b3t_ctx *ctx, const double *A_packed, double *const *L, const double *B,
                               double *X, double *R, double *eta, int32_t T, int32_t b, int32_t nrhs,
                               int32_t flags, int32_t first);

/* Wait (or, in stream mode, check that no unfinished batch uses them), then
 * unregister the T(T+1)/2 tiles given (any registered set). */
B3T_API int b3t_tiles_unregister(b3t_ctx *ctx, void *const *tiles, int32_t T);

/* ---------------------------------------------------------------------
 * Allocation-free vector-scaling chains.  The paper has no counterpart: it
 * is an extra entry point for callers that cannot let a library allocate
 * device memory -- a process whose GPU memory is all reserved by a
 * framework's caching allocator, code that cannot afford the device-wide
 * synchronisation cudaMalloc / cudaFree may imply, or hosts that forbid
 * allocation after start-up.  It performs no cudaMalloc, cudaFree or other
 * allocating call; its scratch (a ticket counter, a status word and one
 * completion counter per task) is a fixed file-scope device array of
 * about 256 KiB that every GPU loading the library holds until exit.
 *
 * Computes, for every block i < nblocks and every step k < nchain in order,
 * x_i[e] <- fl32(x_i[e] * factors[i * nchain + k]), where block i is
 * x[i*n .. i*n + n): the same results, bit for bit, as submitting the
 * B3T_SCAL_F32 task chains through b3t_task_submit.  x and factors are
 * device pointers owned by the caller; x must be 16-byte aligned and n a
 * multiple of 4 (-EINVAL otherwise).  nblocks * nchain may not exceed 65536
 * (-E2BIG).  timeout_ns bounds every device-side wait (0 = 10 s;
 * -ETIMEDOUT).  Runs on cuda_stream and returns after it has finished.
 * The first call on a device looks up the array's device address and the
 * grid size (once per device, with that device current); make that first
 * call before any stream capture.  Every call on a device shares the one
 * array and clears what must start at zero; calls that overlap on the GPU
 * (other streams or host threads) race on it and must not be issued. */
B3T_API int b3t_scal_chains_noalloc(float *x, int64_t n, int32_t nblocks, int32_t nchain,
                                    const float *factors, int64_t timeout_ns, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* B3T_H */
