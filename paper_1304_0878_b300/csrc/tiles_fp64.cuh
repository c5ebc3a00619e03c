// FP64 tile task bodies for the persistent executor (256 threads per CTA).
//
// Tiles are b x b, column-major inside the tile: element (r, c) at r + c*b.
// Only the lower triangle of diagonal tiles is read or written.
//   POTRF : A_kk = L_kk L_kk^T            one work item per task
//   TRSM  : A_ik <- A_ik L_kk^{-T}        items of kTrsmRows rows
//   SYRK  : A_ii <- A_ii - A_ik A_ik^T    items of 64 x 64 lower blocks
//   GEMM  : A_ij <- A_ij - A_ik A_jk^T    items of 64 x 64 blocks
// FP64 on sm_103 is bound by the DFMA pipe (about two DFMA per clock per
// SM), not by memory: the bodies stage operands through shared memory in
// K-chunks and keep a small register tile per thread, which is enough to keep
// that pipe busy.  Data written by other tasks of the same launch is read
// with plain (coherent) loads, never through the read-only path.
#pragma once
#include "b3t_internal.h"

namespace b3t {

constexpr int kKc = 32;            // K chunk staged in shared memory

// a / d from r = 1 / d (one IEEE division per divisor, shared by every
// quotient with that divisor): q = RN(a r), the exact remainder
// e = a - q d by one FMA, then the correction RN(q + e r), which by
// Markstein's theorem (P. Markstein, IBM J. Res. Dev. 34(1), 1990; Muller et
// al., Handbook of Floating-Point Arithmetic, division with an FMA) is the
// correctly rounded quotient, bit for bit what a / d gives, for finite d != 0
// and no underflow.  A zero quotient keeps the sign of q (a / d would give
// -0 for a = -0).  On sm_103 a dependent FP64 operation takes ~64 cycles and a
// division ~640, so a substitution chain of k divisions by known pivots is
// k x 3 operations long instead of k divisions.
__device__ __forceinline__ double div_rcp(double a, double d, double r) {
    const double q = __dmul_rn(a, r);
    const double q1 = fma(fma(-q, d, a), r, q);
    return (__double_as_longlong(q) << 1) == 0 ? q : q1;
}

// C(crow0.., ccol0..) (64 x 64 block) -= A(arow0.., 0..K) * B(brow0.., 0..K)^T,
// all column-major with leading dimension ld.  lower_only: write only the
// entries with row - lower_shift >= column.
// C(crow0.., ccol0..) (RM x 64 block) -= A(arow0.., 0..K) * B(brow0.., 0..K)^T,
// all column-major with leading dimension ld.  lower_only: write only the
// entries with row - lower_shift >= column.  Thread (tx, ty) owns rows
// tx + 16 i (i < RM / 16) and columns ty + 16 j (j < 4); p ascending, one
// FMA per term.
template <int RM = 64>
__device__ __forceinline__ void gemm_rows_f64(const double *A, int arow0, const double *B, int brow0,
                                              double *C, int crow0, int ccol0, int K, int ld, bool lower_only,
                                              int lower_shift, double *smem) {
    static_assert(RM == 16 || RM == 32 || RM == 64, "rows per block");
    constexpr int NI = RM / 16;
    const int b = ld;
    double *As = smem;                   // [kKc][RM]
    double *Bs = smem + kKc * RM;        // [kKc][64]
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    double acc[NI][4];
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += kKc) {
#pragma unroll
        for (int q = 0; q < (kKc * RM) / kThreads; ++q) {
            const int e = tid + q * kThreads;
            const int r = e % RM, p = e / RM;
            As[p * RM + r] = A[(size_t)(arow0 + r) + (size_t)(k0 + p) * b];
        }
#pragma unroll
        for (int q = 0; q < (kKc * 64) / kThreads; ++q) {
            const int e = tid + q * kThreads;
            const int r = e & 63, p = e >> 6;
            Bs[p * 64 + r] = B[(size_t)(brow0 + r) + (size_t)(k0 + p) * b];
        }
        __syncthreads();
#pragma unroll 8
        for (int p = 0; p < kKc; ++p) {
            double a[NI], bb[4];
#pragma unroll
            for (int i = 0; i < NI; ++i) a[i] = As[p * RM + tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[p * 64 + ty + 16 * j];
#pragma unroll
            for (int i = 0; i < NI; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int r = crow0 + tx + 16 * i, c = ccol0 + ty + 16 * j;
            if (!lower_only || r - lower_shift >= c) {
                double *p = C + (size_t)r + (size_t)c * b;
                *p = *p - acc[i][j];
            }
        }
}

__device__ __forceinline__ void gemm64_f64(const double *A, int arow0, const double *B, int brow0,
                                           double *C, int crow0, int ccol0, int K, int ld, bool lower_only,
                                           int lower_shift, double *smem) {
    gemm_rows_f64<64>(A, arow0, B, brow0, C, crow0, ccol0, K, ld, lower_only, lower_shift, smem);
}

__device__ __forceinline__ void gemm_item(const TaskRec &t, int item, double *smem) {
    const int b = (int)t.n, m = b / kGemmBlk;
    const int bi = item / m, bj = item % m;
    if (b <= kSmallTile && t.nitems == (b / kSmallGemmRows) * m) {   // kSmallGemmRows x 64 blocks (the same FMAs per element)
        gemm_rows_f64<kSmallGemmRows>((const double *)t.buf[0], bi * kSmallGemmRows, (const double *)t.buf[1],
                                      bj * 64, (double *)t.buf[2], bi * kSmallGemmRows, bj * 64, b, b, false, 0,
                                      smem);
        return;
    }
    gemm64_f64((const double *)t.buf[0], bi * 64, (const double *)t.buf[1], bj * 64,
               (double *)t.buf[2], bi * 64, bj * 64, b, b, false, 0, smem);
}

// item -> (bi, bj), bi >= bj, enumerating the lower block triangle row by row
__device__ __forceinline__ void tri_index(int item, int &bi, int &bj) {
    int i = (int)((sqrtf(8.0f * item + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= item) ++i;
    while (i * (i + 1) / 2 > item) --i;
    bi = i;
    bj = item - i * (i + 1) / 2;
}

__device__ __forceinline__ void syrk_item(const TaskRec &t, int item, double *smem) {
    const int b = (int)t.n;
    if (b <= kSmallTile && t.nitems == (b / kSmallGemmRows) * (b / kGemmBlk)) {
        // kSmallGemmRows x 64 blocks; those wholly above the diagonal are empty
        const int m = b / kGemmBlk, bi = item / m, bj = item % m;
        if (bi * kSmallGemmRows + kSmallGemmRows - 1 < bj * 64) return;
        const double *A = (const double *)t.buf[0];
        gemm_rows_f64<kSmallGemmRows>(A, bi * kSmallGemmRows, A, bj * 64, (double *)t.buf[1], bi * kSmallGemmRows,
                                      bj * 64, b, b, true, 0, smem);
        return;
    }
    int bi, bj;
    tri_index(item, bi, bj);
    const double *A = (const double *)t.buf[0];
    gemm64_f64(A, bi * 64, A, bj * 64, (double *)t.buf[1], bi * 64, bj * 64, b, b, bi == bj, 0, smem);
}

// X L^T = A for rows [r0, r0 + 32) of an n-wide block (n a multiple of 64).
// Ain is the input (f64, or f32 for the mixed-precision panel), X the f64
// output (may alias Ain when Tin is double), L the n x n lower factor; all
// column-major with leading dimension ld.
// kIdent: the input rows are rows r0.. of the identity (Ain is not read), so
// X rows are rows of L^{-T}: columns before the 64-block holding r0 are zero
// and are written as zeros without being computed.
// kPipe: the next K chunk is loaded into registers while the current one is
// used (one memory latency per item instead of one per chunk; more
// registers, so only the out-of-line mixed-precision TRSM uses it).
// Columns c_lo .. c_hi - 1 (64-column blocks) of rows r0 .. r0 + RB - 1; the
// columns before c_lo must be final in X already (the column-block TRTRI).
template <typename Tin, bool kIdent = false, bool kPipe = false, int RB = kTrsmRows>
__device__ __forceinline__ void trsm_rows(const double *L, const Tin *Ain, double *X, int r0, int n, int ld,
                                          double *smem, int c_lo = 0, int c_hi = -1) {
    static_assert(RB == 8 || RB == 16 || RB == 32, "rows per item");
    const int b = ld;
    if (c_hi < 0) c_hi = n;
    const int cz = kIdent ? (r0 / 64) * 64 : 0;     // first column block that can be nonzero
    const int cs = cz > c_lo ? cz : c_lo;
    constexpr int RS = RB + 1;              // padded row stride of the row-major staging
    constexpr int NG = kThreads / RB;       // column groups: thread (tr, tw) owns row tr
    constexpr int NC = 64 / NG;             // and columns tw + NG j, j < NC, of a block
    double *Lcb = smem;                     // [64][65]  Lcb[c*65 + q] = L(c0+c, c0+q)
    double *Acc = Lcb + 64 * 65;            // [64][RS]  Acc[c*RS + r]
    double *Xs = Acc + 64 * RS;             // [kKc][RS] Xs[p*RS + r] = X(r0+r, k0+p)
    double *Ls = Xs + kKc * RS;             // [kKc][64] Ls[p*64 + c] = L(c0+c, k0+p)
    const int tid = threadIdx.x;
    const int tr = tid % RB, tw = tid / RB;
    if (kIdent) {
        for (int c0 = c_lo; c0 < cz && c0 < c_hi; c0 += 64) {
#pragma unroll
            for (int j = 0; j < NC; ++j) X[(size_t)(r0 + tr) + (size_t)(c0 + tw + NG * j) * b] = 0.0;
        }
    }
    for (int c0 = cs; c0 < c_hi; c0 += 64) {
        double acc[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            if (kIdent) acc[j] = (r0 + tr == c0 + tw + NG * j) ? 1.0 : 0.0;
            else acc[j] = (double)Ain[(size_t)(r0 + tr) + (size_t)(c0 + tw + NG * j) * b];
        }
        constexpr int NX = (RB * kKc) / kThreads, NL = (64 * kKc) / kThreads;
        double xv[kPipe ? NX : 1], lv[kPipe ? NL : 1];
        if (kPipe && cz < c0) {
#pragma unroll
            for (int q = 0; q < NX; ++q) {
                const int e = tid + q * kThreads;
                xv[q] = X[(size_t)(r0 + e % RB) + (size_t)(cz + e / RB) * b];
            }
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                const int e = tid + q * kThreads;
                lv[q] = L[(size_t)(c0 + (e & 63)) + (size_t)(cz + (e >> 6)) * b];
            }
        }
        // the sum runs over every column block that can be nonzero, also
        // those computed before c_lo
        for (int k0 = cz; k0 < c0; k0 += kKc) {
#pragma unroll
            for (int q = 0; q < NX; ++q) {
                const int e = tid + q * kThreads;
                const int r = e % RB, p = e / RB;
                Xs[p * RS + r] = kPipe ? xv[kPipe ? q : 0] : X[(size_t)(r0 + r) + (size_t)(k0 + p) * b];
            }
#pragma unroll
            for (int q = 0; q < NL; ++q) {
                const int e = tid + q * kThreads;
                const int c = e & 63, p = e >> 6;
                Ls[p * 64 + c] = kPipe ? lv[kPipe ? q : 0] : L[(size_t)(c0 + c) + (size_t)(k0 + p) * b];
            }
            __syncthreads();
            if (kPipe && k0 + kKc < c0) {
#pragma unroll
                for (int q = 0; q < NX; ++q) {
                    const int e = tid + q * kThreads;
                    xv[q] = X[(size_t)(r0 + e % RB) + (size_t)(k0 + kKc + e / RB) * b];
                }
#pragma unroll
                for (int q = 0; q < NL; ++q) {
                    const int e = tid + q * kThreads;
                    lv[q] = L[(size_t)(c0 + (e & 63)) + (size_t)(k0 + kKc + (e >> 6)) * b];
                }
            }
#pragma unroll 8
            for (int p = 0; p < kKc; ++p) {
                const double x = Xs[p * RS + tr];
#pragma unroll
                for (int j = 0; j < NC; ++j) acc[j] = fma(-x, Ls[p * 64 + tw + NG * j], acc[j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < NC; ++j) Acc[(tw + NG * j) * RS + tr] = acc[j];
        for (int e = tid; e < 64 * 64; e += kThreads) {
            const int c = e & 63, q = e >> 6;           // element (c0+c, c0+q)
            if (c >= q) Lcb[c * 65 + q] = L[(size_t)(c0 + c) + (size_t)(c0 + q) * b];
        }
        // 1 / L(c, c) in the padding slot of row c (every solve of the block
        // divides by these 64 pivots)
        if (tid < 64) Lcb[tid * 65 + 64] = 1.0 / L[(size_t)(c0 + tid) + (size_t)(c0 + tid) * b];
        __syncthreads();
        // small triangular solve, right-looking over the 64 columns in panels
        // of 8: warp 0 solves a panel (lane = row, the 8 columns in
        // registers), then every thread applies the panel to the columns to
        // its right.  Per element the operations and their order are those
        // of the column-by-column loop, so results are unchanged; the block
        // needs 16 barriers instead of 128.
        for (int p0 = 0; p0 < 64; p0 += 8) {
            if (tid < RB) {
                double x[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) x[j] = Acc[(p0 + j) * RS + tid];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    x[j] = div_rcp(x[j], Lcb[(p0 + j) * 65 + p0 + j], Lcb[(p0 + j) * 65 + 64]);
#pragma unroll
                    for (int jj = j + 1; jj < 8; ++jj) x[jj] = fma(-x[j], Lcb[(p0 + jj) * 65 + p0 + j], x[jj]);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) Acc[(p0 + j) * RS + tid] = x[j];
            }
            __syncthreads();
            const int rem = 56 - p0;
            for (int e = tid; e < RB * rem; e += kThreads) {
                const int r = e % RB, cc = p0 + 8 + e / RB;
                double v = Acc[cc * RS + r];
#pragma unroll
                for (int j = 0; j < 8; ++j) v = fma(-Acc[(p0 + j) * RS + r], Lcb[cc * 65 + p0 + j], v);
                Acc[cc * RS + r] = v;
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < NC; ++j)
            X[(size_t)(r0 + tr) + (size_t)(c0 + tw + NG * j) * b] = Acc[(tw + NG * j) * RS + tr];
        __syncthreads();
    }
}

__device__ __forceinline__ void trsm_item(const TaskRec &t, int item, double *smem) {
    double *A = (double *)t.buf[1];
    if (t.n <= kSmallTile && t.nitems == (int)t.n / kSmallTrsmRows)
        trsm_rows<double, false, false, kSmallTrsmRows>((const double *)t.buf[0], A, A, item * kSmallTrsmRows,
                                                        (int)t.n, (int)t.n, smem);
    else
        trsm_rows<double>((const double *)t.buf[0], A, A, item * kTrsmRows, (int)t.n, (int)t.n, smem);
}

// TRTRI: U_k <- L_kk^{-T} (upper triangular, the strict lower part zero),
// kTrtriRows rows of U_k (= columns of L_kk^{-1}) per item.  Row r of U_k
// needs the columns from r to b, so the first item is the longest: it is the
// step of the mixed factorisation that no other CTA can share, and short
// items keep it short.  Out of line, with the pipelined K loop (one CTA per
// SM in the mixed-precision launch).
__device__ __noinline__ void trtri_item(const TaskRec &t, int item, double *smem) {
    trsm_rows<double, true, true, kTrtriRows>((const double *)t.buf[0], (const double *)nullptr,
                                              (double *)t.buf[1], item * kTrtriRows, (int)t.n, (int)t.n,
                                              smem);
}

// Out of line with the pipelined K loop: the mixed-precision launch runs one
// CTA per SM, so a chunk's load latency is not hidden by a second CTA.
__device__ __noinline__ void trsm_mx_item(const TaskRec &t, int item, double *smem) {
    trsm_rows<float, false, true>((const double *)t.buf[0], (const float *)t.buf[1], (double *)t.buf[2],
                                  item * kTrsmRows, (int)t.n, (int)t.n, smem);
}

// TRMM_MX: L_ik <- fp64(W_ik) U_k with U_k = L_kk^{-T} (upper triangular,
// zero below the diagonal, from TRTRI), one kTrmmRows x 64 block of L_ik per
// item:
//   L(rows bi, cols bj) = sum_{p < 64 (bj + 1)} fp64(W(rows bi, p)) U(p, cols bj),
// p ascending, one FMA per term.  Unlike the substitution (TRSM_MX), every
// block is independent, so a tile's panel solve spreads over many CTAs and
// runs at the DFMA rate of a plain product; the longest item (the last block
// column, K = b) bounds the task's latency.  The mixed-precision launch runs
// one CTA per SM, so the next K chunk is loaded into registers while the
// current one is used.
__device__ __noinline__ void trmm_mx_item(const TaskRec &t, int item, double *smem) {
    constexpr int RM = kTrmmRows;
    constexpr int NI = RM / 16;                 // rows per thread
    const int b = (int)t.n, m = b / kGemmBlk;
    const int bi = item / m, bj = item % m;
    const double *U = (const double *)t.buf[0];
    const float *Wt = (const float *)t.buf[1];
    double *L = (double *)t.buf[2];
    double *As = smem;                   // [kKc][RM]  As[p*RM + r] = W(RM bi + r, k0 + p)
    double *Bs = smem + kKc * RM;        // [kKc][65]  Bs[p*65 + c] = U(k0 + p, 64 bj + c)
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int K = (bj + 1) * 64;
    constexpr int NA = (kKc * RM) / kThreads;   // elements of W per thread and chunk
    constexpr int NQ = (kKc * 64) / kThreads;   // elements of U per thread and chunk
    const float *Wb = Wt + (size_t)bi * RM;
    const double *Ub = U + (size_t)bj * 64 * b;
    float av[NA];
    double bv[NQ];
#pragma unroll
    for (int q = 0; q < NA; ++q) {
        const int e = tid + q * kThreads;
        av[q] = Wb[(size_t)(e % RM) + (size_t)(e / RM) * b];
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int e = tid + q * kThreads;
        bv[q] = Ub[(size_t)(e & 31) + (size_t)(e >> 5) * b];
    }
    double acc[NI][4];
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += kKc) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int e = tid + q * kThreads;
            As[(e / RM) * RM + e % RM] = (double)av[q];
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int e = tid + q * kThreads;
            Bs[(e & 31) * 65 + (e >> 5)] = bv[q];
        }
        __syncthreads();
        if (k0 + kKc < K) {
#pragma unroll
            for (int q = 0; q < NA; ++q) {
                const int e = tid + q * kThreads;
                av[q] = Wb[(size_t)(e % RM) + (size_t)(k0 + kKc + e / RM) * b];
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int e = tid + q * kThreads;
                bv[q] = Ub[(size_t)(k0 + kKc + (e & 31)) + (size_t)(e >> 5) * b];
            }
        }
#pragma unroll 8
        for (int p = 0; p < kKc; ++p) {
            double a[NI], bb[4];
#pragma unroll
            for (int i = 0; i < NI; ++i) a[i] = As[p * RM + tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[p * 65 + ty + 16 * j];
#pragma unroll
            for (int i = 0; i < NI; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < NI; ++i)
            L[(size_t)(bi * RM + tx + 16 * i) + (size_t)(bj * 64 + ty + 16 * j) * b] = acc[i][j];
}

// Panel update of potrf_block for RB rows from rr0 (all valid):
// A(rr0.., jb..jb+32) -= A(rr0.., 0..jb) A(jb..jb+32, 0..jb)^T on the lower
// part.  RB = 64: thread (tr, tc) owns row tr and 8 columns; RB = 32: row tr
// and 4 columns, so that a 32-row tail keeps all eight warps busy instead of
// issuing FP64 instructions whose lanes are rows past the block (the SM's
// FP64 pipe takes a warp instruction whatever its active lanes).  The
// per-element FMA order (k ascending) is the same.
template <int RB>
__device__ __forceinline__ void potrf_panel_rows(double *A, int ld, int rr0, int jb, double *Lr, double *Lc) {
    constexpr int PW = 32;
    constexpr int NG = kThreads / RB;          // column groups
    constexpr int NJ = PW / NG;                // columns per thread
    const int tid = threadIdx.x;
    const int tr = tid % RB, tc = tid / RB;
    double acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = 0.0;
    for (int k0 = 0; k0 < jb; k0 += kKc) {
#pragma unroll
        for (int q = 0; q < (RB * kKc) / kThreads; ++q) {
            const int e = tid + q * kThreads;
            const int r = e % RB, p = e / RB;
            Lr[p * RB + r] = A[(size_t)(rr0 + r) + (size_t)(k0 + p) * ld];
        }
#pragma unroll
        for (int q = 0; q < (PW * kKc) / kThreads; ++q) {
            const int e = tid + q * kThreads;
            const int c = e & 31, p = e >> 5;
            Lc[p * 32 + c] = A[(size_t)(jb + c) + (size_t)(k0 + p) * ld];
        }
        __syncthreads();
#pragma unroll 8
        for (int p = 0; p < kKc; ++p) {
            const double x = Lr[p * RB + tr];
#pragma unroll
            for (int j = 0; j < NJ; ++j) acc[j] = fma(x, Lc[p * 32 + tc + NG * j], acc[j]);
        }
        __syncthreads();
    }
    const int gr = rr0 + tr;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int gc = jb + tc + NG * j;
        if (gr >= gc) {
            double *p = A + (size_t)gr + (size_t)gc * ld;
            *p = *p - acc[j];
        }
    }
}

// Step (3) of potrf_block: rows jb + 32.. of the 32 columns from jb, solved
// against the factored 32 x 32 block Dg (with 1 / Dg(c, c) in the padding
// slot Dg[c * 33 + 32]), one row per thread.  Right-looking:
// once x[c] is final it is subtracted from every later column, so each x[c']
// takes the terms q = 0, 1, .. in the same order as a left-looking sum (the
// same roundings), but a row's dependent chain is one division and one FMA
// per column instead of c FMAs and a division (on B300 a dependent FP64 FMA
// takes 64 cycles whatever the number of active lanes).  Out of line: its 32
// live values stay out of the caller's register budget.
__device__ __noinline__ void potrf_rows_below(double *A, int b, int ld, int jb, const double *Dg) {
    constexpr int PW = 32;
    for (int i = jb + PW + (int)threadIdx.x; i < b; i += kThreads) {
        double x[PW];
#pragma unroll
        for (int c = 0; c < PW; ++c) x[c] = A[(size_t)i + (size_t)(jb + c) * ld];
#pragma unroll
        for (int c = 0; c < PW; ++c) {
            x[c] = div_rcp(x[c], Dg[c * 33 + c], Dg[c * 33 + 32]);
#pragma unroll
            for (int c2 = c + 1; c2 < PW; ++c2) x[c2] = fma(-x[c], Dg[c2 * 33 + c], x[c2]);
        }
#pragma unroll
        for (int c = 0; c < PW; ++c) A[(size_t)i + (size_t)(jb + c) * ld] = x[c];
    }
}

// Cholesky of one n x n block in place (lower, leading dimension ld), one
// CTA, left-looking over panels of 32 columns.  Returns 0 or the 1-based
// column (within the block) of the first pivot that is <= 0 or NaN.
__device__ __forceinline__ int potrf_block(double *A, int n, int ld, double *smem, int *s_info) {
    const int b = n;
    constexpr int PW = 32;
    double *Dg = smem;                     // [32][33]  Dg[i*33 + k] = A(jb+i, jb+k)
    double *Lr = Dg + PW * 33;             // [kKc][64] Lr[p*64 + r] = A(rr0+r, k0+p)
    double *Lc = Lr + kKc * 64;            // [kKc][32] Lc[p*32 + c] = A(jb+c, k0+p)
    const int tid = threadIdx.x;
    if (tid == 0) *s_info = 0;
    __syncthreads();
    for (int jb = 0; jb < b; jb += PW) {
        // (1) panel update: P = A(jb:, jb:jb+32) - A(jb:, :jb) A(jb:jb+32, :jb)^T,
        // in blocks of 64 rows and a 32-row tail (b and jb are multiples of 32)
        if (jb > 0) {
            for (int rr0 = jb; rr0 < b; rr0 += 64) {
                if (b - rr0 >= 64) potrf_panel_rows<64>(A, ld, rr0, jb, Lr, Lc);
                else potrf_panel_rows<32>(A, ld, rr0, jb, Lr, Lc);
            }
            __syncthreads();
        }
        // (2) factor the 32 x 32 diagonal block in shared memory
        for (int e = tid; e < PW * PW; e += kThreads) {
            const int i = e & 31, k = e >> 5;
            if (i >= k) Dg[i * 33 + k] = A[(size_t)(jb + i) + (size_t)(jb + k) * ld];
        }
        __syncthreads();
        for (int j = 0; j < PW; ++j) {
            if (tid == 0) {
                const double d = Dg[j * 33 + j];
                if (!(d > 0.0)) *s_info = jb + j + 1;
                else Dg[j * 33 + j] = sqrt(d);
            }
            __syncthreads();
            if (*s_info) return *s_info;
            if (tid > j && tid < PW) Dg[tid * 33 + j] = Dg[tid * 33 + j] / Dg[j * 33 + j];
            __syncthreads();
            for (int e = tid; e < PW * PW; e += kThreads) {
                const int i = e & 31, k = e >> 5;
                if (k > j && i >= k) Dg[i * 33 + k] = fma(-Dg[i * 33 + j], Dg[k * 33 + j], Dg[i * 33 + k]);
            }
            __syncthreads();
        }
        for (int e = tid; e < PW * PW; e += kThreads) {
            const int i = e & 31, k = e >> 5;
            if (i >= k) A[(size_t)(jb + i) + (size_t)(jb + k) * ld] = Dg[i * 33 + k];
        }
        // (3) rows below the block: X Dg^T = P, one row per thread, dividing
        // by the 32 pivots through their reciprocals (padding slot of row c)
        if (jb + PW < b) {
            if (tid < PW) Dg[tid * 33 + 32] = 1.0 / Dg[tid * 33 + tid];
            __syncthreads();
            potrf_rows_below(A, b, ld, jb, Dg);
        }
        __syncthreads();
    }
    return 0;
}

// Named barriers (ids 1..15; 0 is __syncthreads): sync waits for `count`
// threads, arrive counts the caller without waiting.  The fence before the
// arrival publishes the caller's shared-memory stores to the waiting threads.
// Ids are immediates, so that the kernel reserves only the barriers it uses.
template <int kId, int kCount>
__device__ __forceinline__ void nbar_sync() {
    asm volatile("bar.sync %0, %1;" ::"n"(kId), "n"(kCount) : "memory");
}
template <int kId, int kCount>
__device__ __forceinline__ void nbar_arrive() {
    __threadfence_block();
    asm volatile("bar.arrive %0, %1;" ::"n"(kId), "n"(kCount) : "memory");
}
// phase parity p selects barrier kId + p
template <int kId, int kCount>
__device__ __forceinline__ void nbar_sync2(int p) {
    if (p) nbar_sync<kId + 1, kCount>();
    else nbar_sync<kId, kCount>();
}
template <int kId, int kCount>
__device__ __forceinline__ void nbar_arrive2(int p) {
    if (p) nbar_arrive<kId + 1, kCount>();
    else nbar_arrive<kId, kCount>();
}

// Cholesky of one 64 x 64 block (lower, leading dimension ld) in shared
// memory, right-looking column by column: column j is scaled (a square root,
// then one division per row) and its contribution
// A(i, k) -= L(i, j) L(k, j) is applied to every later column, for
// j = 0, 1, .. in order, so every element takes its terms in ascending j with
// one rounding each.  On B300 the SM's FP64 pipe is shared by its four
// sub-partitions: it takes about one warp instruction every 16-19 cycles,
// whatever the number of active lanes, and a dependent FP64 operation waits
// 64 cycles (a square root ~680, a division ~650; measured with timing
// probes).  The column chain (square root, division, and the update of the
// next column) runs on warps 0 and 1 (one row per thread), while warps 2, 3,
// 6 and 7 apply column j to columns j + 2 .. 63 one column behind:
//   chain, column j:  (1) s = sqrt(d_j), L(i, j) = A(i, j) / s;
//                     (2) L_j ready -> update warps;
//                     (3) once the update warps have applied column j - 1 to
//                         column j + 1 (T_{j-1}): A(i, j + 1) -= L(i, j)
//                         L(j + 1, j) for i > j + 1, and d_{j+1} =
//                         A(j+1, j+1) - L(j+1, j)^2 the same way in every
//                         chain thread (no barrier before its square root);
//   update, column j: wait L_j; column j + 2; arrive T_j; columns j + 3 ..;
//                     barrier among the update warps.
// The update warps walk the trailing elements of columns j + 3 .. 63 as one
// packed range (the lower triangle stored column by column, an index table
// in shared memory), 128 elements per pass, so that every FP64 instruction
// they issue carries 32 useful lanes: a half-empty warp instruction costs the
// shared FP64 pipe as much as a full one.
// L_j and T_j alternate between two barrier ids each: neither side can run
// two columns ahead of the other, so an id is never reused before its
// previous phase completed.  Warps 4 and 5 wait at the final barrier.  A
// pivot that is <= 0 or NaN is recorded (1-based column) and the loops run to
// the end on NaNs, so every warp takes the same barriers.
__device__ __noinline__ int potrf64_pipelined(double *A, int ld, double *S, int *s_info) {
    constexpr int n = 64, SP = 65;               // S[c * SP + r] = A(r, c)
    constexpr int kChain = 64, kUpd = 128, kBoth = kChain + kUpd;
    // L(j, j) goes to Dg: every chain thread reads the updated A(j, j) while
    // forming d_j, so that element is not written again inside the loop
    double *Dg = S + n * SP;
    // packed lower triangle, column by column: element (r, c) at
    // off(c) + r - c with off(c) = 64 c - c (c - 1) / 2; tab[e] = r | c << 8
    unsigned short *tab = reinterpret_cast<unsigned short *>(Dg + n);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < n * n; e += kThreads) {
        const int r = e & 63, c = e >> 6;
        if (r >= c) {
            S[c * SP + r] = A[(size_t)r + (size_t)c * ld];
            tab[c * n - c * (c - 1) / 2 + r - c] = (unsigned short)(r | c << 8);
        }
    }
    if (tid == 0) *s_info = 0;
    __syncthreads();
    if (warp < 2) {
        const int i = tid;
        int info = 0;
        double d = S[0];
        for (int j = 0; j < n; ++j) {
            if (!(d > 0.0) && info == 0) info = j + 1;
            const double s = sqrt(d);
            double l = 0.0;
            if (i == j) {
                Dg[j] = s;
                l = s;
            } else if (i > j) {
                l = S[j * SP + i] / s;
                S[j * SP + i] = l;
            }
            nbar_sync<5, kChain>();
            if (j + 2 < n) nbar_arrive2<1, kBoth>(j & 1);
            if (j + 1 < n) {
                if (j >= 1) nbar_sync2<3, kBoth>((j - 1) & 1);
                const double lj1 = S[j * SP + j + 1];
                d = fma(-lj1, lj1, S[(j + 1) * SP + j + 1]);
                if (i > j + 1) S[(j + 1) * SP + i] = fma(-l, lj1, S[(j + 1) * SP + i]);
            }
        }
        if (tid == 0) *s_info = info;
    } else if (warp != 4 && warp != 5) {
        // u = 0..127 over warps 2, 3, 6, 7: each pass of 128 elements gives
        // every warp 32 of them
        const int u = ((warp & 1) | (warp >= 6 ? 2 : 0)) * 32 + lane;
        for (int j = 0; j + 2 < n; ++j) {
            nbar_sync2<1, kBoth>(j & 1);
            // column j + 2 first (rows j + 2 .., needed by the chain's next step)
            const int i2 = j + 2 + u;
            if (i2 < n) S[(j + 2) * SP + i2] = fma(-S[j * SP + i2], S[j * SP + j + 2], S[(j + 2) * SP + i2]);
            nbar_arrive2<3, kBoth>(j & 1);
            // columns j + 3 .. 63, four elements per thread at a time, loads
            // before the FMAs (one shared-memory latency per group)
            const int c3 = j + 3;
            for (int e0 = c3 * n - c3 * (c3 - 1) / 2 + u; e0 < n * (n + 1) / 2; e0 += 4 * kUpd) {
                double a[4], li[4], lk[4];
                int pos[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = e0 + q * kUpd;
                    const bool v = e < n * (n + 1) / 2;
                    const int rc = v ? tab[e] : 0, r = rc & 255, c = rc >> 8;
                    pos[q] = v ? c * SP + r : -1;
                    li[q] = v ? S[j * SP + r] : 0.0;
                    lk[q] = v ? S[j * SP + c] : 0.0;
                    a[q] = v ? S[c * SP + r] : 0.0;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (pos[q] >= 0) S[pos[q]] = fma(-li[q], lk[q], a[q]);
            }
            nbar_sync<6, kUpd>();
        }
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += kThreads) {
        const int r = e & 63, c = e >> 6;
        if (r >= c) A[(size_t)r + (size_t)c * ld] = r == c ? Dg[c] : S[c * SP + r];
    }
    const int info = *s_info;
    __syncthreads();
    return info;
}

__device__ __forceinline__ int potrf_tile(double *A, int b, double *smem, int *s_info) {
    // a 64 x 64 tile takes the pipelined right-looking factorisation
    return b == 64 ? potrf64_pipelined(A, b, smem, s_info) : potrf_block(A, b, b, smem, s_info);
}

// ---- diagonal tile split into column panels (partition parts of the tile)
// record: buf[0] = panel kk (and buf[1] = panel jj for updates), n = b,
// aux = global column offset of the tile (POTRF info), scal = kk | jj << 8 | pw << 16
__device__ __forceinline__ int pn_kk(const TaskRec &t) { return (int)(t.scal & 0xff); }
__device__ __forceinline__ int pn_jj(const TaskRec &t) { return (int)((t.scal >> 8) & 0xff); }
__device__ __forceinline__ int pn_pw(const TaskRec &t) { return (int)(t.scal >> 16); }

// POTRF of the diagonal block of panel kk (rows kk*pw.., pw x pw)
// TRTRI of one 64-column block cb of U_k = L_kk^{-T}: rows r0 .. r0 + 7 of
// columns 64 cb .. 64 cb + 63, from the columns before it (earlier TRTRI_COL
// tasks) and rows 64 cb .. 64 cb + 63 of L_kk, which are final once panel cb
// of the diagonal factor is done; rows below the block get zeros.  The same
// per-element operations as TRTRI.  Record: buf[0] = panel part cb of L_kk,
// buf[2] = column block cb of U_k (the tiles' bases are 64 cb columns before).
__device__ __noinline__ void trtri_col_item(const TaskRec &t, int item, double *smem) {
    const int b = (int)t.n, cb = pn_kk(t), c0 = cb * 64;
    const double *L = (const double *)t.buf[0] - (size_t)c0 * b;
    double *U = (double *)t.buf[2] - (size_t)c0 * b;
    trsm_rows<double, true, true, kTrtriRows>(L, (const double *)nullptr, U, item * kTrtriRows, b, b, smem, c0,
                                              c0 + 64);
}

__device__ __forceinline__ int potrf_d_item(const TaskRec &t, double *smem, int *s_info) {
    const int b = (int)t.n, kk = pn_kk(t), pw = pn_pw(t);
    double *P = (double *)t.buf[0];
    const int info = pw == 64 ? potrf64_pipelined(P + (size_t)kk * pw, b, smem, s_info)
                              : potrf_block(P + (size_t)kk * pw, pw, b, smem, s_info);
    return info ? kk * pw + info : 0;
}

// rows below the diagonal block of panel kk: X L_d^T = P, kPanelTrsmRows
// rows per item (the next panel's update waits for every item: short items
// keep the diagonal chain short)
__device__ __forceinline__ void panel_trsm_item(const TaskRec &t, int item, double *smem) {
    const int b = (int)t.n, kk = pn_kk(t), pw = pn_pw(t);
    double *P = (double *)t.buf[0];
    trsm_rows<double, false, false, kPanelTrsmRows>(P + (size_t)kk * pw, P, P,
                                                    (kk + 1) * pw + item * kPanelTrsmRows, pw, b, smem);
}

// panel jj -= panel kk(rows jj*pw.., :) panel kk(jj*pw..jj*pw+pw, :)^T, rows
// from jj*pw (lower part on the diagonal block); blocks of kPanelUpdRows x 64
// per item (the update of the next panel is on the diagonal chain)
__device__ __forceinline__ void panel_upd_item(const TaskRec &t, int item, double *smem) {
    const int b = (int)t.n, jj = pn_jj(t), pw = pn_pw(t);
    const double *Pk = (const double *)t.buf[0];
    double *Pj = (double *)t.buf[1];
    const int nc = pw / 64;
    const int bi = item / nc, bj = item % nc;
    const int row0 = jj * pw + bi * kPanelUpdRows;
    gemm_rows_f64<kPanelUpdRows>(Pk, row0, Pk, jj * pw + bj * 64, Pj, row0, bj * 64, pw, b,
                                 bi * kPanelUpdRows < pw, jj * pw, smem);
}

}  // namespace b3t
