// Sliced FP64 residual: R_i = B_i - (A X)_i with the products on the tcgen05
// tensor cores (the Ozaki scheme: Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Every value of a block with scale exponent e (|v| < 2^(e-2): the tile of A,
// or one right-hand side of a part of X) becomes the integer
// V = trunc(v 2^(60-e)), |V| < 2^58, written in twelve balanced base-32
// digits d_s in [-16, 15] (V = sum_s d_s 32^(11-s)); every digit is an exact
// E4M3 value, so slice s of a block is an E4M3 matrix.  The product of a tile
// and a part is
//   sum_{s,t} 2^(eA + eX - 5 (s + t + 2)) A_s X_t,
// of which the pairs with m = s + t <= 11 are kept.  One MMA chain per group
// m sums its pairs' products (integers of magnitude <= 256) in a binary32
// accumulator: at most 12 pairs x b terms, below 2^24, so the sums are exact.
// The twelve group sums of a tile are combined in 64-bit integers,
//   H = sum_{m<6} G_m 32^(5-m),  L = sum_{m>=6} G_m 32^(11-m)  (|H|, |L| < 2^50),
// and added to the FP64 accumulator as H 2^(eA+eX-35) + L 2^(eA+eX-65): two
// roundings per tile, the only ones besides the final B - AX.  Error per
// product term (the truncation of both values and the dropped pairs):
// below 2^(eA+eX-58.3).
//
//   SLICE_A   one stored lower tile (i, j) -> the slices of its uses: A_ij
//             (rows of block i, K = its columns) and A_ij^T (rows of block
//             j); a diagonal tile has the one symmetric use.  Also the row
//             sums of |A_IJ| per use (for ||A||_inf) and the scale exponent.
//   SLICE_X   part J of X -> its slices (16 right-hand sides, zero padded),
//             one exponent per right-hand side, max|x| per 16-row group.
//   RESID_SL  128 rows of R_i: thread 0 streams A slice chunks (16 KiB,
//             bulk copies into a kSlStages ring) and the X slices of each
//             K-chunk (24 KiB, two slots); thread 32 issues the MMAs (M = 128,
//             K = 32; per A slice s one MMA of N = 16 (12 - s) against the
//             stacked X slices) into twelve group accumulators per tile, in
//             two tensor-memory buffers; warps 4-7 read a finished tile's
//             groups (one row per thread), combine them and accumulate in
//             FP64 while the next tile's MMAs run.  Then R_i = B_i - acc and
//             the per-16-row maxima that NRM reads (the RESID part layout).
#pragma once
#include <cuda_fp8.h>
#include "b3t_internal.h"
#include "mx.cuh"
#include "solve.cuh"

namespace b3t {

// record packing: n = b, aux = i | j << 16, scal = T | nrhs << 16
__device__ __forceinline__ int sl_i(const TaskRec &t) { return t.aux & 0xffff; }
__device__ __forceinline__ int sl_j(const TaskRec &t) { return (t.aux >> 16) & 0xffff; }
__device__ __forceinline__ int sl_T(const TaskRec &t) { return (int)(t.scal & 0xffff); }
__device__ __forceinline__ int sl_nrhs(const TaskRec &t) { return (int)(t.scal >> 16); }

constexpr int kSlStages = 7;                         // A chunk ring
constexpr uint32_t kSlXSet = kSlDigits * kSlXChunk;  // X slices of one K-chunk (24 KiB)
constexpr uint32_t kSlXOff = 0;                      // two X slots
constexpr uint32_t kSlAOff = 2 * kSlXSet;            // then the A ring (7 x 16 KiB)
static_assert(kSlAOff + kSlStages * kSlChunk <= 160 * 1024, "RESID_SL stages fit the MX data area");
// 16 (32^12 - 1) / 31: adds 16 to every base-32 digit, so that the balanced
// digits of V are the plain digits of V + kSlBias, minus 16
constexpr unsigned long long kSlBias = 595056260442243600ull;

// Scale exponent of a block with max |v| = amax: |v| < 2^(e-2); 0 if amax = 0.
__device__ __forceinline__ int sl_exp(double amax) {
    if (!(amax > 0.0)) return 0;
    return ilogb(amax) + 3;
}

// V + kSlBias for one value (V = trunc(v 2^(60-e)) from the significand;
// zeros and subnormals give V = 0).
__device__ __forceinline__ unsigned long long sl_u(double v, int e) {
    const long long bits = __double_as_longlong(v);
    const int E = (int)((bits >> 52) & 0x7ff);
    long long V = 0;
    if (E != 0) {
        const long long m = (bits & 0x000fffffffffffffll) | 0x0010000000000000ll;
        int sh = E - 1015 - e;                   // <= 5 when |v| < 2^(e-2)
        if (sh > 5) sh = 5;
        if (sh >= 0) V = m << sh;
        else if (sh > -64) V = m >> (-sh);
        if (bits < 0) V = -V;
    }
    return (unsigned long long)(V + (long long)kSlBias);
}

// Four digits (shift sh picks the slice) -> four E4M3 bytes, K ascending.
__device__ __forceinline__ uint32_t sl_pack4(const unsigned long long *u, int sh) {
    float2 a, c;
    a.x = (float)((int)((u[0] >> sh) & 31ull) - 16);
    a.y = (float)((int)((u[1] >> sh) & 31ull) - 16);
    c.x = (float)((int)((u[2] >> sh) & 31ull) - 16);
    c.y = (float)((int)((u[3] >> sh) & 31ull) - 16);
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(a, __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(c, __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

// Store the twelve slices of 16 values (one 16-byte group of a chunk row).
__device__ __forceinline__ void sl_store16(unsigned char *dst, size_t slice_stride, const unsigned long long *u) {
#pragma unroll
    for (int s = 0; s < kSlDigits; ++s) {
        const int sh = 5 * (kSlDigits - 1 - s);
        uint4 w;
        w.x = sl_pack4(u, sh);
        w.y = sl_pack4(u + 4, sh);
        w.z = sl_pack4(u + 8, sh);
        w.w = sl_pack4(u + 12, sh);
        *reinterpret_cast<uint4 *>(dst + (size_t)s * slice_stride) = w;
    }
}

// 2^k as a double (k may be below the normal range).
__device__ __forceinline__ double sl_pow2(int k) {
    if (k >= -1022 && k <= 1023) return __longlong_as_double((long long)(k + 1023) << 52);
    return ldexp(1.0, k);
}

__device__ __noinline__ void slice_a_item(const TaskRec &t, double *red, int *s_e) {
    const int b = (int)t.n, T = sl_T(t), i = sl_i(t), j = sl_j(t);
    const double *A = (const double *)t.buf[0] + (size_t)ptile(i, j, T) * b * b;
    unsigned char *D = (unsigned char *)t.buf[1];     // use (i, j)
    unsigned char *Dt = (unsigned char *)t.buf[2];    // use (j, i); D itself on the diagonal
    const bool diag = i == j;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nk = b / 128;
    const size_t sbytes = (size_t)kSlDigits * b * b;
    double *Pd = (double *)(D + sbytes), *Pt = (double *)(Dt + sbytes);
    // element (r, c) of the use (i, j): the stored tile, or on the diagonal
    // the symmetric tile from its lower triangle
    auto at = [&](int r, int c) -> double {
        return (!diag || r >= c) ? A[(size_t)r + (size_t)c * b] : A[(size_t)c + (size_t)r * b];
    };
    // row sums of |A_ij| (c ascending) and the tile's maximum
    double mx = 0.0;
    for (int r = tid; r < b; r += kThreads) {
        double s = 0.0;
        for (int c = 0; c < b; ++c) {
            const double a = fabs(at(r, c));
            s += a;
            mx = fmax(mx, a);
        }
        Pd[r] = s;
    }
    // column sums of |A_ij| = row sums of the use (j, i): a warp per column,
    // lane partials over rows lane, lane + 32, ..., then a fixed shuffle tree
    if (!diag) {
        for (int c = warp; c < b; c += kThreads / 32) {
            double s = 0.0;
            for (int r = lane; r < b; r += 32) s += fabs(A[(size_t)r + (size_t)c * b]);
#pragma unroll
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) Pt[c] = s;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) m = fmax(m, red[w]);
        *s_e = sl_exp(m);
    }
    __syncthreads();
    const int e = *s_e;
    // use (i, j): unit = (row r, 16-column group g16), consecutive threads on
    // consecutive rows (coalesced reads of the column-major tile)
    for (int u0 = tid; u0 < b * (b / 16); u0 += kThreads) {
        const int r = u0 % b, g16 = u0 / b;
        unsigned long long u[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) u[k] = sl_u(at(r, 16 * g16 + k), e);
        const int rb = r >> 7, rr = r & 127, kc = g16 >> 3, g = g16 & 7;
        sl_store16(D + (size_t)(rb * nk + kc) * kSlDigits * kSlChunk + (size_t)rr * 128 + ((g ^ (rr & 7)) << 4),
                   kSlChunk, u);
    }
    // use (j, i): row c of A_ij^T is column c of the tile; unit = (c, 16-row
    // group), a thread reads 16 consecutive doubles
    if (!diag) {
        for (int u0 = tid; u0 < b * (b / 16); u0 += kThreads) {
            const int c = u0 / (b / 16), g16 = u0 % (b / 16);
            unsigned long long u[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) u[k] = sl_u(A[(size_t)(16 * g16 + k) + (size_t)c * b], e);
            const int rb = c >> 7, rr = c & 127, kc = g16 >> 3, g = g16 & 7;
            sl_store16(Dt + (size_t)(rb * nk + kc) * kSlDigits * kSlChunk + (size_t)rr * 128 + ((g ^ (rr & 7)) << 4),
                       kSlChunk, u);
        }
    }
    if (tid == 0) {
        int *ed = (int *)(D + sbytes + 8 * (size_t)b);
        ed[0] = e; ed[1] = 0; ed[2] = 0; ed[3] = 0;
        if (!diag) {
            int *et = (int *)(Dt + sbytes + 8 * (size_t)b);
            et[0] = e; et[1] = 0; et[2] = 0; et[3] = 0;
        }
    }
}

__device__ __noinline__ void slice_x_item(const TaskRec &t, int *s_ex) {
    const int b = (int)t.n, nrhs = sl_nrhs(t);
    const double *X = (const double *)t.buf[0];
    unsigned char *D = (unsigned char *)t.buf[1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t sbytes = (size_t)kSlDigits * (b / 128) * kSlXChunk;
    int *ex = (int *)(D + sbytes);
    double *xm = (double *)(D + sbytes + 64);         // [b / 16][kSlNp]
    // a warp per right-hand side: max |x| per 16-row group and over the part
    for (int c = warp; c < kSlNp; c += kThreads / 32) {
        double m = 0.0;
        for (int r0 = 0; r0 < b; r0 += 32) {
            double v = c < nrhs ? fabs(X[(size_t)c * b + r0 + lane]) : 0.0;
#pragma unroll
            for (int o = 8; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
            if ((lane & 15) == 0) xm[(size_t)((r0 + lane) >> 4) * kSlNp + c] = v;
            m = fmax(m, v);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_ex[c] = sl_exp(m);
    }
    __syncthreads();
    // unit = (right-hand side n, 16-row group): 16 consecutive doubles
    for (int u0 = tid; u0 < kSlNp * (b / 16); u0 += kThreads) {
        const int n = u0 / (b / 16), g16 = u0 % (b / 16);
        const int e = s_ex[n];
        unsigned long long u[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) u[k] = n < nrhs ? sl_u(X[(size_t)n * b + 16 * g16 + k], e) : kSlBias;
        const int kc = g16 >> 3, g = g16 & 7;
        sl_store16(D + (size_t)kc * kSlDigits * kSlXChunk + (size_t)n * 128 + ((g ^ (n & 7)) << 4), kSlXChunk, u);
    }
    if (tid < kSlNp) ex[tid] = s_ex[tid];
}

// Instruction descriptor: f32 accumulate, E4M3 A and B, K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t sl_idesc(uint32_t n) {
    return (1u << 4) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Per-CTA pipeline state of RESID_SL, persistent across items.
struct SlState {
    uint64_t *full, *empty;     // [kSlStages] A chunk ring
    uint64_t *xfull, *xempty;   // [2] X slots
    uint64_t *done, *tfree;     // [2] accumulator buffers: MMAs finished / read out
    uint64_t *drain;            // [1] after a failed wait: every MMA issued has finished
    uint32_t fa, fx;            // A / X fills so far (thread 0)
    uint32_t nj;                // tiles accumulated so far (every thread)
};
constexpr int kSlBars = 2 * kSlStages + 2 + 2 + 2 + 2 + 1;

// Returns 0, or ETIMEDOUT when a pipeline wait ran out (block-wide).
__device__ __noinline__ int resid_sl_item(const TaskRec &t, int item, SlState &st, unsigned char *smem,
                                             uint32_t tmem, int64_t limit_ns, int *s_fail) {
    const int b = (int)t.n, T = sl_T(t), nrhs = sl_nrhs(t), i = sl_i(t), rb = item;
    const int nk = b / 128;
    const size_t PB = (size_t)sl_a_part_bytes(b), XB = (size_t)sl_x_part_bytes(b);
    const size_t a_sbytes = (size_t)kSlDigits * b * b, x_sbytes = (size_t)kSlDigits * nk * kSlXChunk;
    const unsigned char *AS = (const unsigned char *)t.buf[0];
    const unsigned char *XS = (const unsigned char *)t.buf[1];
    const double *B = (const double *)t.buf[2];
    double *Rp = (double *)t.buf[3];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t Q = (uint32_t)T * nk * kSlDigits;    // steps: (J, kc, s)
    if (tid == 0) *s_fail = 0;
    __syncthreads();
    bool ok = true;
    if (tid == 0) {
        // producer: the A chunks of every step into the ring, the X set of
        // each (J, kc) into its slot, as soon as the slot is free
        asm volatile("fence.proxy.async.global;" ::: "memory");
        uint32_t issued = 0, xissued = 0;
        auto a_src = [&](uint32_t q) -> const unsigned char * {
            const uint32_t s = q % kSlDigits, jk = q / kSlDigits, J = jk / nk, kc = jk % nk;
            return AS + ((size_t)i * T + J) * PB + ((size_t)(rb * nk + kc) * kSlDigits + s) * kSlChunk;
        };
        for (uint32_t q = 0; q < Q && ok; ++q) {
            const uint32_t s = q % kSlDigits, jk = q / kSlDigits, J = jk / nk, kc = jk % nk;
            if (s == 0) {
                const uint32_t gx = st.fx + jk, xs = gx & 1;
                if (gx >= 2 && !mbar_wait(&st.xempty[xs], ((gx >> 1) - 1) & 1, limit_ns)) { ok = false; break; }
                mbar_expect_tx(&st.xfull[xs], kSlXSet);
                bulk_g2s(smem + kSlXOff + xs * kSlXSet, XS + (size_t)J * XB + (size_t)kc * kSlXSet, kSlXSet,
                         &st.xfull[xs]);
                ++xissued;
            }
            const uint32_t ga = st.fa + q, slot = ga % kSlStages;
            if (ga >= (uint32_t)kSlStages && !mbar_wait(&st.empty[slot], ((ga / kSlStages) - 1) & 1, limit_ns)) {
                ok = false;
                break;
            }
            mbar_expect_tx(&st.full[slot], kSlChunk);
            bulk_g2s(smem + kSlAOff + slot * kSlChunk, a_src(q), kSlChunk, &st.full[slot]);
            ++issued;
        }
        if (!ok) {
            *s_fail = 1;
            // the copies in flight land before shared memory is given up: the
            // latest fill of each slot
            for (uint32_t q = issued > (uint32_t)kSlStages ? issued - kSlStages : 0; q < issued; ++q) {
                const uint32_t ga = st.fa + q;
                mbar_wait(&st.full[ga % kSlStages], (ga / kSlStages) & 1, limit_ns);
            }
            for (uint32_t x = xissued > 2 ? xissued - 2 : 0; x < xissued; ++x) {
                const uint32_t gx = st.fx + x;
                mbar_wait(&st.xfull[gx & 1], (gx >> 1) & 1, limit_ns);
            }
        }
    } else if (tid == 32) {
        // MMA issuer: per step, once its chunks have landed, one MMA per K
        // step over the stacked X slices
        for (uint32_t J = 0; J < (uint32_t)T && ok; ++J) {
            const uint32_t jt = st.nj + J, buf = jt & 1;
            // the buffer is free once the epilogue of tile jt - 2 has read it
            if (jt >= 2 && !mbar_wait(&st.tfree[buf], ((jt >> 1) - 1) & 1, limit_ns)) { ok = false; break; }
            tc_fence_after();
            const uint32_t dbase = tmem + buf * (kSlGroups * kSlNp);
            for (uint32_t kc = 0; kc < (uint32_t)nk && ok; ++kc) {
                for (uint32_t s = 0; s < (uint32_t)kSlDigits; ++s) {
                    const uint32_t q = (J * nk + kc) * kSlDigits + s;
                    const uint32_t ga = st.fa + q, slot = ga % kSlStages;
                    const uint32_t gx = st.fx + J * nk + kc, xs = gx & 1;
                    if (s == 0 && !mbar_wait(&st.xfull[xs], (gx >> 1) & 1, limit_ns)) { ok = false; break; }
                    if (!mbar_wait(&st.full[slot], (ga / kSlStages) & 1, limit_ns)) { ok = false; break; }
                    tc_fence_after();
                    // all pairs (s, t), t = 0 .. 11 - s, in one MMA per K step: the
                    // X set is [t][16 rows][128 bytes], i.e. one K-major operand of
                    // 192 rows, and group m = s + t sits at columns 16 m, so the
                    // first 16 (12 - s) rows land on the groups s .. 11
                    const uint64_t ad = sw128_desc(smem_u32(smem + kSlAOff + slot * kSlChunk));
                    const uint64_t bd = sw128_desc(smem_u32(smem + kSlXOff + xs * kSlXSet));
                    const uint32_t idesc = sl_idesc((uint32_t)kSlNp * (kSlGroups - s));
#pragma unroll
                    for (uint32_t k4 = 0; k4 < 4; ++k4)
                        mma_e4m3(dbase + s * kSlNp, ad + 2 * k4, bd + 2 * k4, idesc, (kc | s | k4) ? 1u : 0u);
                    mma_commit(&st.empty[slot]);
                    if (s == kSlDigits - 1) mma_commit(&st.xempty[xs]);
                }
            }
            if (ok) mma_commit(&st.done[buf]);
        }
        if (!ok) {
            *s_fail = 1;
            // every MMA issued finishes before tensor memory is given up
            mma_commit(st.drain);
            mbar_wait(st.drain, 0, limit_ns);
        }
    } else if (warp >= 4) {
        const int q = warp & 3, row = 32 * q + lane;        // TMEM lane = row of the item
        const int gr = rb * kSlRows + row;                   // row within part i
        double acc[kSlNp];
#pragma unroll
        for (int c = 0; c < kSlNp; ++c) acc[c] = 0.0;
        for (int J = 0; J < T; ++J) {
            const uint32_t jt = st.nj + J, buf = jt & 1;
            const int ea = *(const int *)(AS + ((size_t)i * T + J) * PB + a_sbytes + 8 * (size_t)b);
            const int *ex = (const int *)(XS + (size_t)J * XB + x_sbytes);
            if (ok && !mbar_wait(&st.done[buf], (jt >> 1) & 1, limit_ns)) ok = false;
            if (ok) {
                tc_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + buf * (kSlGroups * kSlNp);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    long long Hs[8], Ls[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) { Hs[c] = 0; Ls[c] = 0; }
#pragma unroll
                    for (int m = 0; m < kSlGroups; ++m) {
                        float v[8];
                        tmem_ld8(tb + m * kSlNp + 8 * h, v);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const long long g = (long long)__float2int_rz(v[c]);
                            if (m < 6) Hs[c] += g << (5 * (5 - m));
                            else Ls[c] += g << (5 * (11 - m));
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int e = ea + ex[8 * h + c];
                        acc[8 * h + c] = fma((double)Hs[c], sl_pow2(e - 35), acc[8 * h + c]);
                        acc[8 * h + c] = fma((double)Ls[c], sl_pow2(e - 65), acc[8 * h + c]);
                    }
                }
                tc_fence_before();
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&st.tfree[buf]);
        }
        // R_i = B_i - acc and the per-16-row maxima of the RESID part layout
        const double *Bi = B + (size_t)i * b * nrhs;
        double *Rn = Rp + (size_t)b * nrhs;
        const int nit = b / kResidRows, it16 = gr >> 4;
        double rs = 0.0;
        for (int J = 0; J < T; ++J) rs += ((const double *)(AS + ((size_t)i * T + J) * PB + a_sbytes))[gr];
        const double *xmax = (const double *)(XS + (size_t)i * XB + x_sbytes + 64);
#pragma unroll
        for (int c = 0; c < kSlNp; ++c) {
            if (c < nrhs) {
                const double bv = Bi[(size_t)c * b + gr];
                const double r = bv - acc[c];
                Rp[(size_t)c * b + gr] = r;
                double mr = fabs(r), mb = fabs(bv);
#pragma unroll
                for (int o = 8; o; o >>= 1) {
                    mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
                    mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
                }
                if ((lane & 15) == 0) {
                    Rn[(size_t)it16 * nrhs + c] = mr;
                    Rn[(size_t)nit * nrhs + (size_t)it16 * nrhs + c] = xmax[(size_t)it16 * kSlNp + c];
                    Rn[(size_t)2 * nit * nrhs + (size_t)it16 * nrhs + c] = mb;
                }
            }
        }
#pragma unroll
        for (int o = 8; o; o >>= 1) rs = fmax(rs, __shfl_xor_sync(0xffffffffu, rs, o));
        if ((lane & 15) == 0) Rn[(size_t)3 * nit * nrhs + it16] = rs;
    }
    st.fa += Q;
    st.fx += (uint32_t)T * nk;
    st.nj += (uint32_t)T;
    if (__syncthreads_or(*s_fail || !ok)) return ETIMEDOUT;
    return 0;
}

// ---------------------------------------------------------------------
// Sliced panel product of the mixed factorisation: L_ik = fp64(W_ik) U_k
// (U_k = L_kk^{-T}, upper triangular), the product of TRMM_MX with the
// slices of both operands on the tensor cores.  Row r of W_ik has the scale
// exponent eW[r] (its maximum), column c of U_k the exponent eU[c]; with the
// group sums G_m of the kept pairs (s + t <= 11),
//   L(r, c) = H 2^(eW[r]+eU[c]-35) + L 2^(eW[r]+eU[c]-65)   (one rounding),
// H and L combined from G_m as in RESID_SL.  Per product term the error is
// below 2^(eW+eU-58.3), as for the residual.
//   SLICE_W   128 rows of W_ik per item: row exponents, then the slices
//             (chunks (rb, kc, s) of 128 rows x 128 bytes of K).
//   SLICE_U   32 columns of U_k per item: column exponents, then the
//             slices as chunk sets (cb, kc) of 12 x (32 rows x 128 bytes).
//   TRMM_SL   a 128 x 32 block of L_ik per item.  Thread 0 streams the W
//             chunks of the block's rows (16 KiB, 4-stage ring) and the U
//             chunk set of each K chunk (48 KiB, two slots); thread 32
//             issues per W slice s the MMAs against the stacked U slices: group m =
//             s + t at TMEM columns 32 m, N = 32 (12 - s) (two MMAs, 256 and
//             32 (4 - s) columns, for s < 4).  U_k is zero below the
//             diagonal, so the K range stops at the block's last column.
//             All eight warps then combine the groups and write L.

constexpr int kTsStages = 4;
constexpr uint32_t kTsBChunk = kTsCols * 128;            // 4 KiB: 32 rows x 128 bytes
constexpr uint32_t kTsBSet = kSlDigits * kTsBChunk;      // 48 KiB: the 12 U slices of a K chunk
constexpr uint32_t kTsBOff = 0;                          // two U slots
constexpr uint32_t kTsAOff = 2 * kTsBSet;                // then the W ring (4 x 16 KiB)
static_assert(kTsAOff + kTsStages * kSlChunk <= 160 * 1024, "TRMM_SL stages fit the MX data area");

__device__ __noinline__ void slice_w_item(const TaskRec &t, int item, unsigned char *smem) {
    const int b = (int)t.n, nk = b / 128, rb = item;
    const float *W = (const float *)t.buf[0];
    unsigned char *D = (unsigned char *)t.buf[1];
    int *eW = (int *)(D + (size_t)kSlDigits * b * b);
    float *hm = (float *)smem;                 // [2][128] maxima over half a row
    int *re = (int *)(smem + 1024);            // [128] row exponents
    const int tid = threadIdx.x;
    {
        const int rr = tid & 127, h = tid >> 7, r = rb * 128 + rr;
        float m = 0.0f;
        for (int c = h * (b / 2); c < (h + 1) * (b / 2); ++c) m = fmaxf(m, fabsf(W[(size_t)r + (size_t)c * b]));
        hm[h * 128 + rr] = m;
    }
    __syncthreads();
    if (tid < 128) {
        const int e = sl_exp((double)fmaxf(hm[tid], hm[128 + tid]));
        re[tid] = e;
        eW[rb * 128 + tid] = e;
    }
    __syncthreads();
    for (int u0 = tid; u0 < 128 * (b / 16); u0 += kThreads) {
        const int rr = u0 & 127, g16 = u0 >> 7, r = rb * 128 + rr;
        const int e = re[rr];
        unsigned long long u[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) u[k] = sl_u((double)W[(size_t)r + (size_t)(16 * g16 + k) * b], e);
        const int kc = g16 >> 3, g = g16 & 7;
        sl_store16(D + (size_t)(rb * nk + kc) * kSlDigits * kSlChunk + (size_t)rr * 128 + ((g ^ (rr & 7)) << 4),
                   kSlChunk, u);
    }
}

__device__ __noinline__ void slice_u_item(const TaskRec &t, int item, unsigned char *smem) {
    const int b = (int)t.n, nk = b / 128, cb = item, c0 = cb * kTsCols;
    const double *U = (const double *)t.buf[0];
    unsigned char *D = (unsigned char *)t.buf[1];
    int *eU = (int *)(D + (size_t)kSlDigits * b * b);
    int *ce = (int *)smem;                     // [32] column exponents
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int cc = warp; cc < kTsCols; cc += kThreads / 32) {
        double m = 0.0;
        for (int p = lane; p < b; p += 32) m = fmax(m, fabs(U[(size_t)p + (size_t)(c0 + cc) * b]));
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            const int e = sl_exp(m);
            ce[cc] = e;
            eU[c0 + cc] = e;
        }
    }
    __syncthreads();
    for (int u0 = tid; u0 < kTsCols * (b / 16); u0 += kThreads) {
        const int cc = u0 / (b / 16), g16 = u0 % (b / 16);
        const int e = ce[cc];
        unsigned long long u[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) u[k] = sl_u(U[(size_t)(16 * g16 + k) + (size_t)(c0 + cc) * b], e);
        const int kc = g16 >> 3, g = g16 & 7;
        sl_store16(D + (size_t)(cb * nk + kc) * kSlDigits * kTsBChunk + (size_t)cc * 128 + ((g ^ (cc & 7)) << 4),
                   kTsBChunk, u);
    }
}

// Per-CTA pipeline state of TRMM_SL, persistent across items.
struct TsState {
    uint64_t *full, *empty;     // [kTsStages] W chunk ring
    uint64_t *bfull, *bempty;   // [2] U chunk sets
    uint64_t *done;             // [1] the item's MMAs have finished
    uint64_t *drain;            // [1] after a failed wait
    uint32_t fa, fb;            // W / U fills so far (thread 0)
    uint32_t nd;                // items completed so far (every thread)
};
constexpr int kTsBars = 2 * kTsStages + 2 + 2 + 1 + 1;

// Returns 0, or ETIMEDOUT when a pipeline wait ran out (block-wide).
__device__ __noinline__ int trmm_sl_item(const TaskRec &t, int item, TsState &st, unsigned char *smem,
                                         uint32_t tmem, int64_t limit_ns, int *s_fail) {
    const int b = (int)t.n, nk = b / 128, ncb = b / kTsCols;
    const int rb = item / ncb, cb = item % ncb, c0 = cb * kTsCols;
    const unsigned char *US = (const unsigned char *)t.buf[0];
    const unsigned char *WS = (const unsigned char *)t.buf[1];
    double *L = (double *)t.buf[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t nks = (uint32_t)cb + 1;                 // K steps of 32: rows p < c0 + 32 of U_k
    const uint32_t nkc = (nks + 3) / 4;                    // K chunks of 128
    const uint32_t Q = nkc * kSlDigits;                    // steps (kc, s)
    if (tid == 0) *s_fail = 0;
    __syncthreads();
    if (tid == 0) {
        // producer: the W chunks of the block's rows and the U chunk set of
        // each K chunk, as soon as their slots are free
        asm volatile("fence.proxy.async.global;" ::: "memory");
        bool ok = true;
        uint32_t issued = 0, bissued = 0;
        auto w_src = [&](uint32_t q) -> const unsigned char * {
            return WS + ((size_t)(rb * nk + q / kSlDigits) * kSlDigits + q % kSlDigits) * kSlChunk;
        };
        for (uint32_t q = 0; q < Q && ok; ++q) {
            const uint32_t s = q % kSlDigits, kc = q / kSlDigits;
            if (s == 0) {
                const uint32_t gb = st.fb + kc, bs = gb & 1;
                if (gb >= 2 && !mbar_wait(&st.bempty[bs], ((gb >> 1) - 1) & 1, limit_ns)) { ok = false; break; }
                mbar_expect_tx(&st.bfull[bs], kTsBSet);
                bulk_g2s(smem + kTsBOff + bs * kTsBSet, US + (size_t)(cb * nk + kc) * kTsBSet, kTsBSet,
                         &st.bfull[bs]);
                ++bissued;
            }
            const uint32_t ga = st.fa + q, slot = ga % kTsStages;
            if (ga >= (uint32_t)kTsStages && !mbar_wait(&st.empty[slot], ((ga / kTsStages) - 1) & 1, limit_ns)) {
                ok = false;
                break;
            }
            mbar_expect_tx(&st.full[slot], kSlChunk);
            bulk_g2s(smem + kTsAOff + slot * kSlChunk, w_src(q), kSlChunk, &st.full[slot]);
            ++issued;
        }
        if (!ok) {
            *s_fail = 1;
            for (uint32_t q = issued > (uint32_t)kTsStages ? issued - kTsStages : 0; q < issued; ++q) {
                const uint32_t ga = st.fa + q;
                mbar_wait(&st.full[ga % kTsStages], (ga / kTsStages) & 1, limit_ns);
            }
            for (uint32_t x = bissued > 2 ? bissued - 2 : 0; x < bissued; ++x) {
                const uint32_t gb = st.fb + x;
                mbar_wait(&st.bfull[gb & 1], (gb >> 1) & 1, limit_ns);
            }
        }
    } else if (tid == 32) {
        // MMA issuer
        bool ok = true;
        for (uint32_t kc = 0; kc < nkc && ok; ++kc) {
            const uint32_t ksteps = min(4u, nks - 4 * kc);
            for (uint32_t s = 0; s < (uint32_t)kSlDigits; ++s) {
                const uint32_t q = kc * kSlDigits + s;
                const uint32_t ga = st.fa + q, slot = ga % kTsStages;
                const uint32_t gb = st.fb + kc, bs = gb & 1;
                if (s == 0 && !mbar_wait(&st.bfull[bs], (gb >> 1) & 1, limit_ns)) { ok = false; break; }
                if (!mbar_wait(&st.full[slot], (ga / kTsStages) & 1, limit_ns)) { ok = false; break; }
                tc_fence_after();
                const uint64_t ad = sw128_desc(smem_u32(smem + kTsAOff + slot * kSlChunk));
                const uint64_t bd = sw128_desc(smem_u32(smem + kTsBOff + bs * kTsBSet));
                for (uint32_t k4 = 0; k4 < ksteps; ++k4) {
                    const uint32_t acc = (kc | s | k4) ? 1u : 0u;
                    if (s < 4) {
                        // U slices t = 0..7 (256 rows), then t = 8..11-s from row 256
                        mma_e4m3(tmem + kTsCols * s, ad + 2 * k4, bd + 2 * k4, sl_idesc(256), acc);
                        mma_e4m3(tmem + kTsCols * (s + 8), ad + 2 * k4, bd + ((256u * 128u) >> 4) + 2 * k4,
                                 sl_idesc(kTsCols * (4 - s)), acc);
                    } else {
                        mma_e4m3(tmem + kTsCols * s, ad + 2 * k4, bd + 2 * k4, sl_idesc(kTsCols * (12 - s)), acc);
                    }
                }
                mma_commit(&st.empty[slot]);
                if (s == kSlDigits - 1) mma_commit(&st.bempty[bs]);
            }
        }
        if (!ok) {
            *s_fail = 1;
            mma_commit(st.drain);
            mbar_wait(st.drain, 0, limit_ns);
        } else {
            mma_commit(st.done);
        }
    }
    st.fa += Q;
    st.fb += nkc;
    __syncthreads();
    bool ok = *s_fail == 0;
    if (ok && !mbar_wait(st.done, st.nd & 1, limit_ns)) ok = false;
    if (ok) st.nd++;
    if (__syncthreads_or(!ok)) return ETIMEDOUT;
    tc_fence_after();
    // epilogue: warp w reads TMEM lanes 32 (w & 3).. (its rows) and 16 of the
    // block's 32 columns (w >> 2)
    const int q = warp & 3, h = warp >> 2, rr = 32 * q + lane, r = rb * 128 + rr;
    const int ew = *(const int *)(WS + (size_t)kSlDigits * b * b + 4 * (size_t)r);
    const int *eU = (const int *)(US + (size_t)kSlDigits * b * b);
    const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + 16 * h;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        long long Hs[8], Ls[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) { Hs[c] = 0; Ls[c] = 0; }
#pragma unroll
        for (int m = 0; m < kSlGroups; ++m) {
            float v[8];
            tmem_ld8(tb + kTsCols * m + 8 * half, v);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const long long g = (long long)__float2int_rz(v[c]);
                if (m < 6) Hs[c] += g << (5 * (5 - m));
                else Ls[c] += g << (5 * (11 - m));
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int cc = 16 * h + 8 * half + c;
            const int e = ew + eU[c0 + cc];
            const double v = fma((double)Ls[c], sl_pow2(e - 65), (double)Hs[c] * sl_pow2(e - 35));
            L[(size_t)r + (size_t)(c0 + cc) * b] = v;
        }
    }
    tc_fence_before();
    __syncthreads();
    return 0;
}

}  // namespace b3t
