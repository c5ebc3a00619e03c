// Solve and refinement task bodies (256 threads per CTA).
//
// Vectors with nrhs right-hand sides are split into T row blocks ("parts")
// of b rows; part k holds Y_k(r, j) at j*b + r (column-major b x nrhs).
//   TRSV_L  : Y_k <- L_kk^{-1} Y_k            item = one right-hand side
//   GEMV_L  : Y_i <- Y_i - L_ik Y_k           item = 16 rows of Y_i
//   TRSV_LT : Y_k <- L_kk^{-T} Y_k            item = one right-hand side
//   GEMV_LT : Y_i <- Y_i - L_ki^T Y_k         item = 16 rows of Y_i
//             (flags: assign Y_i <- M Y_k instead; M lower or upper
//             triangular, so that blocks of zeros are skipped)
//   AXPY    : X_i <- X_i + D_i (or X_i = D_i) one item
//   RESID   : R_i <- B_i - (A X)_i, FP64, with A symmetric and only its lower
//             tiles stored; also per-item maxima |R|, |X_i| and the largest
//             row sum of |A| (for the backward error)   item = 16 rows
//   NRM     : eta_j = max|r_j| / (||A||_inf max|x_j| + max|b_j|), one item
// The solve bodies compute in Tc (double, or float for refinement
// corrections) and read / write FP64 storage.
#pragma once
#include "b3t_internal.h"

namespace b3t {

// record packing of the vector kinds: n = b, aux = i | flags << 24,
// scal = T | nrhs << 16
__device__ __forceinline__ int vk_nrhs(const TaskRec &t) { return (int)(t.scal >> 16); }
__device__ __forceinline__ int vk_T(const TaskRec &t) { return (int)(t.scal & 0xffff); }
__device__ __forceinline__ int vk_i(const TaskRec &t) { return t.aux & 0xffffff; }
__device__ __forceinline__ int vk_flags(const TaskRec &t) { return (t.aux >> 24) & 0xff; }

template <typename Tc>
__device__ __forceinline__ void trsv_l_item(const TaskRec &t, int j, unsigned char *smem) {
    const double *L = (const double *)t.buf[0];
    double *y = (double *)t.buf[1] + (size_t)j * t.n;
    const int b = (int)t.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Tc *ys = (Tc *)smem;                 // [b]
    Tc *red = ys + b;                    // [8][32]
    Tc *Dg = red + 256;                  // [32][33]
    for (int r = tid; r < b; r += kThreads) ys[r] = (Tc)y[r];
    __syncthreads();
    for (int R0 = 0; R0 < b; R0 += 32) {
        Tc s = 0;
#pragma unroll 8
        for (int q = warp; q < R0; q += 8) s += (Tc)L[(size_t)(R0 + lane) + (size_t)q * b] * ys[q];
        red[warp * 32 + lane] = s;
        for (int e = tid; e < 1024; e += kThreads) {
            const int i = e & 31, k = e >> 5;
            Dg[i * 33 + k] = i >= k ? (Tc)L[(size_t)(R0 + i) + (size_t)(R0 + k) * b] : (Tc)0;
        }
        __syncthreads();
        if (warp == 0) {
            Tc v = ys[R0 + lane];
            for (int g = 0; g < 8; ++g) v -= red[g * 32 + lane];
            for (int c = 0; c < 32; ++c) {
                if (lane == c) v = v / Dg[c * 33 + c];
                const Tc xc = __shfl_sync(0xffffffffu, v, c);
                if (lane > c) v -= Dg[lane * 33 + c] * xc;
            }
            ys[R0 + lane] = v;
        }
        __syncthreads();
    }
    for (int r = tid; r < b; r += kThreads) y[r] = (double)ys[r];
}

template <typename Tc>
__device__ __forceinline__ void trsv_lt_item(const TaskRec &t, int j, unsigned char *smem) {
    const double *L = (const double *)t.buf[0];
    double *y = (double *)t.buf[1] + (size_t)j * t.n;
    const int b = (int)t.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Tc *ys = (Tc *)smem;                 // [b]
    Tc *red = ys + b;                    // [32]
    Tc *Dg = red + 256;                  // [32][33]
    for (int r = tid; r < b; r += kThreads) ys[r] = (Tc)y[r];
    __syncthreads();
    for (int R0 = b - 32; R0 >= 0; R0 -= 32) {
        // red[r] = sum_{q >= R0+32} L(q, R0+r) y_q  (column R0+r of L is contiguous)
        for (int r = warp; r < 32; r += 8) {
            Tc s = 0;
            const double *col = L + (size_t)(R0 + r) * b;
#pragma unroll 8
            for (int q = R0 + 32 + lane; q < b; q += 32) s += (Tc)col[q] * ys[q];
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red[r] = s;
        }
        for (int e = tid; e < 1024; e += kThreads) {
            const int i = e & 31, k = e >> 5;
            Dg[i * 33 + k] = i >= k ? (Tc)L[(size_t)(R0 + i) + (size_t)(R0 + k) * b] : (Tc)0;
        }
        __syncthreads();
        if (warp == 0) {
            Tc v = ys[R0 + lane] - red[lane];
            for (int c = 31; c >= 0; --c) {
                if (lane == c) v = v / Dg[c * 33 + c];
                const Tc xc = __shfl_sync(0xffffffffu, v, c);
                if (lane < c) v -= Dg[c * 33 + lane] * xc;
            }
            ys[R0 + lane] = v;
        }
        __syncthreads();
    }
    for (int r = tid; r < b; r += kThreads) y[r] = (double)ys[r];
}

// Y_i(r0+r, j) -= sum_q M(r, q) Y_k(q, j), M = L_ik (trans = false) or
// L_ki^T (trans = true), kGemvRows = 16 rows per item (32 items per 512-row
// part: the solve's critical path is a chain of these tasks, so short items
// spread each step over many SMs).  Thread (r, g) owns row r and the
// right-hand sides g, g + 16 (NM of them, 1 or 2).  The 16 x 64 block of M
// and the 64 x nrhs block of Y_k are staged in shared memory per 64-column
// step, all loads of a step issued before the first is used (prefetching
// the next step into registers measured slower: it spills).
// Not inlined: compiled on its own, the body keeps its loop free of the
// register spills of the whole executor (measured 25 % faster in binary32).
template <typename Tc, bool trans, int NM>
__device__ __noinline__ void gemv_body(const TaskRec &t, int item, unsigned char *smem) {
    const double *L = (const double *)t.buf[0];
    const double *Yk = (const double *)t.buf[1];
    double *Yi = (double *)t.buf[2];
    constexpr int RR = kGemvRows, G = kThreads / RR;
    const int b = (int)t.n, nrhs = vk_nrhs(t), tid = threadIdx.x;
    const int r = tid % RR, g = tid / RR, r0 = item * RR;
    Tc *Ys = (Tc *)smem;                 // [nrhs][65]: Ys[j*65 + q] = Y_k(q0 + q, j)
    Tc *Lc = Ys + 65 * kMaxRhs;          // [RR][65]:   Lc[r*65 + q] = M(r0 + r, q0 + q)
    const int fl = vk_flags(t);
    // a triangular M has nonzeros only in the 64-column blocks that reach
    // q <= r (lower) or q >= r (upper) for the item's rows
    const int qa = (fl & kVecUpperM) ? (r0 / 64) * 64 : 0;
    const int qb = (fl & kVecLowerM) ? r0 + RR : b;
    Tc acc[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = 0;
    for (int q0 = qa; q0 < qb; q0 += 64) {
        double ly[8], lm[(RR * 64) / kThreads];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = tid + u * kThreads, q = e & 63, jj = e >> 6;
            if (jj < nrhs) ly[u] = Yk[(size_t)jj * b + q0 + q];
        }
#pragma unroll
        for (int u = 0; u < (RR * 64) / kThreads; ++u) {
            const int e = tid + u * kThreads;
            if (trans) {
                const int q = e & 63, rr = e >> 6;
                lm[u] = L[(size_t)(q0 + q) + (size_t)(r0 + rr) * b];
            } else {
                const int rr = e % RR, q = e / RR;
                lm[u] = L[(size_t)(r0 + rr) + (size_t)(q0 + q) * b];
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = tid + u * kThreads, q = e & 63, jj = e >> 6;
            if (jj < nrhs) Ys[jj * 65 + q] = (Tc)ly[u];
        }
#pragma unroll
        for (int u = 0; u < (RR * 64) / kThreads; ++u) {
            const int e = tid + u * kThreads;
            const int q = trans ? (e & 63) : (e / RR), rr = trans ? (e >> 6) : (e % RR);
            Lc[rr * 65 + q] = (Tc)lm[u];
        }
        __syncthreads();
#pragma unroll 8
        for (int q = 0; q < 64; ++q) {
            const Tc a = Lc[r * 65 + q];
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                const int jj = g + G * m;
                if (jj < nrhs) acc[m] += a * Ys[jj * 65 + q];
            }
        }
        __syncthreads();
    }
    const bool assign = fl & kVecAssign;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const int jj = g + G * m;
        if (jj < nrhs) {
            double *p = Yi + (size_t)jj * b + r0 + r;
            *p = assign ? (double)acc[m] : *p - (double)acc[m];
        }
    }
}

// Binary32 GEMV with nrhs <= 16, one 16-row item: the warps split the
// columns instead of taking turns on them.  Warp w owns the 64-column blocks
// w, w + 8, ... of the item's range; it stages its block of M and of Y_k in
// its own shared memory (no block-wide barrier per step), accumulates its
// partial sums for all 16 x nrhs outputs (lane: row lane % 16, right-hand
// sides lane / 16 + 2m), and one reduction over the warps ends the item.
// Only the final sum order differs from gemv_body (binary32 either way).
template <bool trans>
__device__ __noinline__ void gemv_f32_split(const TaskRec &t, int item, unsigned char *smem) {
    const double *L = (const double *)t.buf[0];
    const double *Yk = (const double *)t.buf[1];
    double *Yi = (double *)t.buf[2];
    constexpr int RR = kGemvRows, NW = kThreads / 32, P = 65;
    const int b = (int)t.n, nrhs = vk_nrhs(t), tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = item * RR, fl = vk_flags(t);
    const int qa = (fl & kVecUpperM) ? (r0 / 64) * 64 : 0;
    const int qb = (fl & kVecLowerM) ? r0 + RR : b;
    float *Lw = (float *)smem + warp * (RR + 16) * P;   // [RR][P]: Lw[r*P + q] = M(r0 + r, q0 + q)
    float *Yw = Lw + RR * P;                             // [16][P]: Yw[j*P + q] = Y_k(q0 + q, j)
    const int r = lane & 15, jh = lane >> 4;
    float acc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[m] = 0.f;
    for (int q0 = qa + 64 * warp; q0 < qb; q0 += 64 * NW) {
        // four rounds of 16 independent loads per lane (the block of M, then
        // the block of Y_k), converted to binary32 into the warp's area
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            double v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int e = lane + 32 * (u + 16 * h);
                if (trans) {
                    const int q = e & 63, rr = e >> 6;
                    v[u] = L[(size_t)(q0 + q) + (size_t)(r0 + rr) * b];
                } else {
                    const int rr = e % RR, q = e / RR;
                    v[u] = L[(size_t)(r0 + rr) + (size_t)(q0 + q) * b];
                }
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int e = lane + 32 * (u + 16 * h);
                const int q = trans ? (e & 63) : (e / RR), rr = trans ? (e >> 6) : (e % RR);
                Lw[rr * P + q] = (float)v[u];
            }
        }
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            double v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int e = lane + 32 * (u + 16 * h), q = e & 63, jj = e >> 6;
                v[u] = jj < nrhs ? Yk[(size_t)jj * b + q0 + q] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int e = lane + 32 * (u + 16 * h), q = e & 63, jj = e >> 6;
                Yw[jj * P + q] = (float)v[u];
            }
        }
        __syncwarp();
#pragma unroll 8
        for (int q = 0; q < 64; ++q) {
            const float a = Lw[r * P + q];
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] = fmaf(a, Yw[(jh + 2 * m) * P + q], acc[m]);
        }
    }
    __syncthreads();   // every warp is done with its staging area
    float *Red = (float *)smem;                          // [NW][RR][16]
#pragma unroll
    for (int m = 0; m < 8; ++m) Red[(warp * RR + r) * 16 + jh + 2 * m] = acc[m];
    __syncthreads();
    {
        const int rr = tid & 15, jj = tid >> 4;          // 256 threads: 16 rows x 16 rhs
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) v += Red[(w * RR + rr) * 16 + jj];
        if (jj < nrhs) {
            double *p = Yi + (size_t)jj * b + r0 + rr;
            *p = (fl & kVecAssign) ? (double)v : *p - (double)v;
        }
    }
    __syncthreads();   // the reduction area is the next item's staging area
}

template <typename Tc, bool trans>
__device__ __forceinline__ void gemv_item(const TaskRec &t, int item, unsigned char *smem) {
    if (sizeof(Tc) == 4 && vk_nrhs(t) <= 16) gemv_f32_split<trans>(t, item, smem);
    else if (vk_nrhs(t) <= kThreads / kGemvRows) gemv_body<Tc, trans, 1>(t, item, smem);
    else gemv_body<Tc, trans, 2>(t, item, smem);
}

__device__ __forceinline__ void axpy_item(const TaskRec &t) {
    double *X = (double *)t.buf[0];
    const double *D = (const double *)t.buf[1];
    const size_t n = (size_t)t.n * vk_nrhs(t);
    const bool assign = vk_flags(t) & 2;
    for (size_t e = threadIdx.x; e < n; e += kThreads) X[e] = assign ? D[e] : X[e] + D[e];
}

__device__ __forceinline__ int64_t ptile(int i, int j, int T) {
    return (int64_t)j * T - (int64_t)j * (j - 1) / 2 + (i - j);
}

// Thread (r, g) accumulates row r0 + r of A X (kResidRows = 16 rows per
// item: 32 items per 512-row part, so that the items fill the grid in many
// waves) for the right-hand sides g, g + 16 (NM of them, 1 or 2); it also
// adds columns 4g..4g+3 of each 64-column step to the row sum of |A| (one
// FP64 add per element of A, spread evenly over the warps), unless the flags
// keep the row sums an earlier residual left in place.
template <int NM>
__device__ __forceinline__ void resid_body(const TaskRec &t, int item, unsigned char *smem) {
    const double *A = (const double *)t.buf[0];
    const double *X = (const double *)t.buf[1];
    const double *B = (const double *)t.buf[2];
    double *Ri = (double *)t.buf[3];
    const int b = (int)t.n, nrhs = vk_nrhs(t), T = vk_T(t), i = vk_i(t);
    const bool xzero = vk_flags(t) & 2, keep_norm = vk_flags(t) & kVecKeepNorm;
    constexpr int RR = kResidRows, G = kThreads / RR;
    const int tid = threadIdx.x, r = tid % RR, g = tid / RR, r0 = item * RR, nit = b / RR;
    double *As = (double *)smem;            // [64 columns][RR + 1]: As[c*(RR+1) + r]
    double *Xs = As + 64 * (RR + 1);        // [nrhs][65]
    double acc[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = 0.0;
    double rs = 0.0;
    if (!xzero) {
        for (int J = 0; J < T; ++J) {
            const double *tile = A + (size_t)ptile(J > i ? J : i, J > i ? i : J, T) * b * b;
            for (int c0 = 0; c0 < b; c0 += 64) {
                double lx[8], la[(64 * RR) / kThreads];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = tid + u * kThreads, c = e & 63, jj = e >> 6;
                    if (jj < nrhs) lx[u] = X[(size_t)J * b * nrhs + (size_t)jj * b + c0 + c];
                }
#pragma unroll
                for (int u = 0; u < (64 * RR) / kThreads; ++u) {
                    const int e = tid + u * kThreads;
                    size_t off;
                    if (J < i) {            // tile (i, J): (r, c) at r + c*b
                        const int rr = e % RR, c = e / RR;
                        off = (size_t)(r0 + rr) + (size_t)(c0 + c) * b;
                    } else if (J > i) {     // tile (J, i): A(i.., J..) = tile(c, r)
                        const int c = e & 63, rr = e >> 6;
                        off = (size_t)(c0 + c) + (size_t)(r0 + rr) * b;
                    } else {                // diagonal tile: lower part, mirrored
                        const int rr = e % RR, c = e / RR;
                        const int R = r0 + rr, C = c0 + c;
                        off = R >= C ? (size_t)R + (size_t)C * b : (size_t)C + (size_t)R * b;
                    }
                    la[u] = tile[off];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = tid + u * kThreads, c = e & 63, jj = e >> 6;
                    if (jj < nrhs) Xs[jj * 65 + c] = lx[u];
                }
#pragma unroll
                for (int u = 0; u < (64 * RR) / kThreads; ++u) {
                    const int e = tid + u * kThreads;
                    const int rr = (J > i) ? (e >> 6) : (e % RR), c = (J > i) ? (e & 63) : (e / RR);
                    As[c * (RR + 1) + rr] = la[u];
                }
                __syncthreads();
                // row sums of |A|: group g adds columns 4g..4g+3 of its row
                // (spread over every warp: no warp does more FP64 work)
                if (!keep_norm) {
#pragma unroll
                    for (int c = 4 * g; c < 4 * g + 4; ++c) rs += fabs(As[c * (RR + 1) + r]);
                }
#pragma unroll 4
                for (int c = 0; c < 64; ++c) {
                    const double a = As[c * (RR + 1) + r];
#pragma unroll
                    for (int m = 0; m < NM; ++m) {
                        const int jj = g + G * m;
                        if (jj < nrhs) acc[m] = fma(a, Xs[jj * 65 + c], acc[m]);
                    }
                }
                __syncthreads();
            }
        }
    }
    // residual, then per-column maxima of |r|, |x|, |b| and the largest |A| row sum
    double *Ra = As;                        // reuse: [nrhs][RR] |r|, |x|, |b|
    double *Xa = As + RR * kMaxRhs;
    double *Ba = Xa + RR * kMaxRhs;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        const int jj = g + G * m;
        if (jj < nrhs) {
            const size_t o = (size_t)jj * b + r0 + r;
            const double bv = B[(size_t)i * b * nrhs + o];
            const double v = bv - acc[m];
            Ri[o] = v;
            Ra[jj * RR + r] = fabs(v);
            Xa[jj * RR + r] = xzero ? 0.0 : fabs(X[(size_t)i * b * nrhs + o]);
            Ba[jj * RR + r] = fabs(bv);
        }
    }
    double *Rs = Ba + RR * kMaxRhs;         // [G][RR] partial row sums
    Rs[g * RR + r] = rs;
    __syncthreads();
    double *Rn = Ri + (size_t)b * nrhs;
    if (tid < nrhs) {
        double mr = 0.0, mx = 0.0, mb = 0.0;
        for (int k = 0; k < RR; ++k) {
            mr = fmax(mr, Ra[tid * RR + k]);
            mx = fmax(mx, Xa[tid * RR + k]);
            mb = fmax(mb, Ba[tid * RR + k]);
        }
        Rn[(size_t)item * nrhs + tid] = mr;
        Rn[(size_t)nit * nrhs + (size_t)item * nrhs + tid] = mx;
        Rn[(size_t)2 * nit * nrhs + (size_t)item * nrhs + tid] = mb;
    } else if (tid == 32 && !keep_norm) {
        double m = 0.0;
        for (int k = 0; k < RR; ++k) {
            double rsum = 0.0;
            for (int q = 0; q < G; ++q) rsum += Rs[q * RR + k];
            m = fmax(m, rsum);
        }
        Rn[(size_t)3 * nit * nrhs + item] = m;
    }
}

__device__ __forceinline__ void resid_item(const TaskRec &t, int item, unsigned char *smem) {
    if (vk_nrhs(t) <= kThreads / kResidRows) resid_body<1>(t, item, smem);
    else resid_body<2>(t, item, smem);
}

__device__ __forceinline__ void nrm_item(const TaskRec &t, unsigned char *smem) {
    const double *R = (const double *)t.buf[0];
    double *eta = (double *)t.buf[2];              // buf[1] (B) orders the task after B's writers
    const int b = (int)t.n, nrhs = vk_nrhs(t), T = vk_T(t), nit = b / kResidRows;
    const int64_t PR = resid_part_elems(b, nrhs);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *sm = (double *)smem;          // [4][8][32]: rmax, xmax, bmax, anorm partials
    double rm = 0.0, xm = 0.0, bm = 0.0, an = 0.0;
    const int jj = lane;
    // every maximum comes from the RESID items' partials (B itself is not
    // read again: its per-item maxima were recorded with the residual)
    if (jj < nrhs) {
        for (int k = warp; k < T * nit; k += 8) {
            const double *Rn = R + (size_t)(k / nit) * PR + (size_t)b * nrhs;
            const int it = k % nit;
            rm = fmax(rm, Rn[(size_t)it * nrhs + jj]);
            xm = fmax(xm, Rn[(size_t)nit * nrhs + (size_t)it * nrhs + jj]);
            bm = fmax(bm, Rn[(size_t)2 * nit * nrhs + (size_t)it * nrhs + jj]);
        }
    }
    for (int k = tid; k < T * nit; k += kThreads) {
        const double *Rn = R + (size_t)(k / nit) * PR + (size_t)b * nrhs;
        an = fmax(an, Rn[(size_t)3 * nit * nrhs + k % nit]);
    }
    sm[0 * 256 + warp * 32 + lane] = rm;
    sm[1 * 256 + warp * 32 + lane] = xm;
    sm[2 * 256 + warp * 32 + lane] = bm;
    sm[3 * 256 + tid] = an;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int k = 0; k < 256; ++k) a = fmax(a, sm[3 * 256 + k]);
        double emax = 0.0;
        for (int j = 0; j < nrhs; ++j) {
            double r2 = 0.0, x2 = 0.0, b2 = 0.0;
            for (int w = 0; w < 8; ++w) {
                r2 = fmax(r2, sm[0 * 256 + w * 32 + j]);
                x2 = fmax(x2, sm[1 * 256 + w * 32 + j]);
                b2 = fmax(b2, sm[2 * 256 + w * 32 + j]);
            }
            const double e = r2 / (a * x2 + b2);
            eta[j] = e;
            emax = fmax(emax, e);
        }
        eta[nrhs] = emax;
    }
}

}  // namespace b3t
