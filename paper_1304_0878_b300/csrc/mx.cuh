// Mixed-precision tile bodies: quantisation of a panel tile and the
// low-precision trailing update on the tcgen05 tensor cores.
//
// Q tile layout (written by QUANT, read by the updates): a b x b tile is cut
// into 16 KiB chunks of 128 rows x 128 bytes of K; chunk (rb, kb) sits at
// (rb * nk + kb) * 16 KiB with nk = b * esize / 128.  Inside a chunk row r
// takes 128 bytes at r * 128 and its 16-byte group g is stored at group
// position g ^ (r % 8): the 128-byte swizzled, K-major operand layout of the
// tensor cores, so one bulk copy of a chunk into a 1024-byte aligned shared
// buffer is directly an MMA operand.  After the data: int32 scale exponent e
// (scale 2^e).
//
// Update item (SYRK_MX / GEMM_MX): a 128 x 128 block of the binary32 tile W,
//   W <- fl32(W - 2^(ea+eb) * QA QB^T),
// QA = rows 128*bi.. of the first operand, QB = rows 128*bj.. of the second.
// One thread issues bulk copies (cp.async.bulk, completion on an mbarrier)
// into a kMxStages ring and the MMAs (M = 128, N = 128, 4 per 128-byte K
// chunk); the accumulator lives in tensor memory (128 columns), starts from
// the W block (all eight warps write it there) and is read back by all eight
// warps for the epilogue.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include "b3t_internal.h"

namespace b3t {

constexpr int kMxStages = 5;
constexpr uint32_t kChunkBytes = 16384;
// 128 columns for the MX update's accumulator, 2 x 192 for RESID_SL's group
// accumulators (the MX launch runs one CTA per SM)
constexpr uint32_t kTmemCols = 512;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase did not complete within limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int64_t limit_ns) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t n = 0;; ++n) {
        if (mbar_try(bar, parity)) return true;
        if ((n & 255) == 255 && (int64_t)(gtimer() - t0) > limit_ns) return false;
    }
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_s2g_mx(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor: f32 accumulate, K-major A and B, M = 128, N = 128;
// operand format 1 = bf16 (kind::f16) or 0 = E4M3 (kind::f8f6f4).
__host__ __device__ constexpr uint32_t mx_idesc(uint32_t opfmt) {
    return (1u << 4) | (opfmt << 7) | (opfmt << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_e4m3(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Per-CTA state of the tensor-core pipeline, persistent across items.
struct MxState {
    uint64_t *full;       // [kMxStages]
    uint64_t *empty;      // [kMxStages]
    uint64_t *done;       // [1]
    unsigned char *stage; // kMxStages x 32 KiB, 1024-aligned
    uint32_t tmem;        // accumulator base address
    uint32_t fills;       // stage fills issued so far (kept by thread 0 only)
    uint32_t items;       // items completed so far (all threads)
};

// Smallest e with amax <= 448 * 2^e (exact comparisons); 0 for amax = 0.
__device__ __forceinline__ int e4m3_scale_exp(double amax) {
    if (!(amax > 0.0)) return 0;
    int e = ilogb(amax) - 8;
    while (amax > ldexp(448.0, e)) ++e;
    while (amax <= ldexp(448.0, e - 1)) --e;
    return e;
}

__device__ __forceinline__ int q_esize(int fmt) { return fmt == 0 ? 2 : 1; }

// FP64 -> bfloat16, one rounding to nearest even (the PTX conversion from
// .f64 to .bf16 rounds once; overflow gives infinity).
__device__ __forceinline__ uint32_t bf16_bits_rn(double x) {
    unsigned short h;
    asm("cvt.rn.bf16.f64 %0, %1;" : "=h"(h) : "d"(x));
    return h;
}

// FP64 -> the nearest value of the E4M3 grid (4 significant bits, smallest
// normal 2^-6, so a quantum of 2^-9 below it), ties to even, as a binary32
// holding that value exactly.  One rounding, done on the FP64 significand:
// with m the 53-bit significand and k the bits to drop (49 in the normal
// range, more below 2^-6), RN-even is (m + 2^(k-1) - 1 + bit_k(m)) >> k.
// Magnitudes above 448 are left to the saturating conversion that follows;
// the tile's scale keeps them out (max |x / 2^e| <= 448).
__device__ __forceinline__ float e4m3_round_f64(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned long long sgn = u & 0x8000000000000000ull, a = u ^ sgn;
    if (a >= 0x7ff0000000000000ull) return (float)x;           // inf / NaN: left to the conversion
    const int E = (int)(a >> 52);
    const int ex = E - 1023;
    const int k = 49 + max(0, -6 - ex);
    if (E == 0 || k >= 54) return sgn ? -0.0f : 0.0f;          // below half the smallest subnormal
    const unsigned long long m = (a & 0x000fffffffffffffull) | 0x0010000000000000ull;
    const unsigned long long r = (m + (1ull << (k - 1)) - 1ull + ((m >> k) & 1ull)) >> k;
    // r * 2^(ex - 52 + k); the exponent is >= -9, so the power of two is a
    // normal double and the product is exact
    const double y = (double)r * __longlong_as_double((long long)(1023 + ex - 52 + k) << 52);
    return (float)(sgn ? -y : y);
}

// QUANT: L (f64 tile) -> Q (layout above).  One work item per tile.
// QUANT, one 16 KiB chunk of the Q layout per item (128 rows x 128 bytes of
// K): chunk-parallel, so that a tile's quantisation is not one CTA's serial
// pass on the factorisation's critical path.  For E4M3 every item forms the
// tile's max|L| itself (the same value in every item, from an L2-resident
// tile) so that no second pass or cross-item reduction is needed.
__device__ __forceinline__ void quant_item(const TaskRec &t, int item, double *red, int *s_e) {
    const double *L = (const double *)t.buf[0];
    unsigned char *Q = (unsigned char *)t.buf[1];
    const int b = (int)t.n, fmt = t.aux, es = q_esize(fmt);
    const int tid = threadIdx.x;
    if (fmt == 1) {
        double m = 0.0;
        for (size_t i = tid; i < (size_t)b * b; i += kThreads) m = fmax(m, fabs(L[i]));
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((tid & 31) == 0) red[tid >> 5] = m;
        __syncthreads();
        if (tid == 0) {
            double a = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) a = fmax(a, red[w]);
            *s_e = e4m3_scale_exp(a);
        }
    } else if (tid == 0) {
        *s_e = 0;
    }
    __syncthreads();
    const int e = *s_e;
    const int G = 16 / es;                  // values per 16-byte group
    const int cpc = 128 / es;               // K values per chunk
    const int nk = b / cpc;
    const int rb = item / nk, kb = item % nk;
    // 128 rows x 8 groups of the chunk: 1024 (row, group) pairs, 4 per thread
    for (int p = tid; p < 128 * (cpc / G); p += kThreads) {
        const int rr = p & 127, g = p >> 7;
        const int r = rb * 128 + rr, c0 = kb * cpc + g * G;
        uint32_t w[4];
        if (fmt == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t lo = bf16_bits_rn(L[(size_t)r + (size_t)(c0 + 2 * j) * b]);
                const uint32_t hi = bf16_bits_rn(L[(size_t)r + (size_t)(c0 + 2 * j + 1) * b]);
                w[j] = lo | (hi << 16);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t word = 0;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // the rounded values are on the E4M3 grid: the conversion is exact
                    float2 f;
                    f.x = e4m3_round_f64(ldexp(L[(size_t)r + (size_t)(c0 + 4 * j + 2 * h) * b], -e));
                    f.y = e4m3_round_f64(ldexp(L[(size_t)r + (size_t)(c0 + 4 * j + 2 * h + 1) * b], -e));
                    const __nv_fp8x2_storage_t q = __nv_cvt_float2_to_fp8x2(f, __NV_SATFINITE, __NV_E4M3);
                    word |= (uint32_t)q << (16 * h);
                }
                w[j] = word;
            }
        }
        unsigned char *dst = Q + ((size_t)rb * nk + kb) * kChunkBytes + (size_t)rr * 128 + ((g ^ (rr & 7)) << 4);
        *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (item == 0 && tid == 0) {
        int *tr = (int *)(Q + (size_t)b * b * es);
        tr[0] = e; tr[1] = 0; tr[2] = 0; tr[3] = 0;
    }
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
        "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
        "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
        "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
        "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
        "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}

// SYRK_MX (syrk = true, lower blocks only) / GEMM_MX update of one 128 x 128
// block.  The accumulator starts from the W block itself:
//   D = -W / s + QA QB^T   (tensor cores, binary32 accumulation),
//   W <- -s D,
// with s = 2^(ea+eb): dividing by a power of two and negating are exact and
// round-to-nearest is symmetric, so this is W - s QA QB^T with the block's
// old value as the first term of the sum.  Every thread owns one row of the
// block (TMEM lane) and 64 of its columns: it loads them from global memory
// (a warp reads 32 consecutive floats of a column: coalesced), writes them
// into tensor memory (tcgen05.st), and after the MMAs reads the result back
// (tcgen05.ld) and stores it, so the W block never passes through shared
// memory.  Thread 0 streams the operand chunks through the kMxStages ring
// (bulk copies) and issues the MMAs.  Returns 0, or ETIMEDOUT when a
// pipeline wait ran out (block-wide).
__device__ __forceinline__ int mx_update_item(const TaskRec &t, int item, bool syrk, MxState &st,
                                              int64_t limit_ns, int *s_fail) {
    const int b = (int)t.n, fmt = t.aux, es = q_esize(fmt);
    const unsigned char *QA = (const unsigned char *)t.buf[0];
    const unsigned char *QB = syrk ? QA : (const unsigned char *)t.buf[1];
    float *W = (float *)(syrk ? t.buf[1] : t.buf[2]);
    int bi, bj;
    if (syrk) {
        int i = (int)((sqrtf(8.0f * item + 1.0f) - 1.0f) * 0.5f);
        while ((i + 1) * (i + 2) / 2 <= item) ++i;
        while (i * (i + 1) / 2 > item) --i;
        bi = i; bj = item - i * (i + 1) / 2;
    } else {
        const int m = b / kMxBlk;
        bi = item / m; bj = item % m;
    }
    const int nk = b * es / 128;
    const uint32_t idesc = mx_idesc(fmt == 0 ? 1u : 0u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, h = warp >> 2;
    const int rr = 32 * q + lane;                            // row of the block = TMEM lane
    int es_sum = 0;
    if (fmt == 1) {
        es_sum = *(const int *)(QA + (size_t)b * b * es) + *(const int *)(QB + (size_t)b * b * es);
    }
    const uint32_t G = st.fills;
    uint32_t issued = 0;
    if (tid == 0) {
        *s_fail = 0;
        // make generic-proxy writes of the producer tasks visible to the bulk copies
        asm volatile("fence.proxy.async.global;" ::: "memory");
        // the first chunks start loading while the W block goes into tensor memory
        while ((int)issued < nk && (int)issued < kMxStages) {
            const uint32_t g = G + issued, slot = g % kMxStages;
            if (g >= (uint32_t)kMxStages && !mbar_wait(&st.empty[slot], ((g / kMxStages) - 1) & 1, limit_ns)) {
                *s_fail = 1;
                break;
            }
            unsigned char *sa = st.stage + slot * 2 * kChunkBytes;
            mbar_expect_tx(&st.full[slot], 2 * kChunkBytes);
            bulk_g2s(sa, QA + ((size_t)bi * nk + issued) * kChunkBytes, kChunkBytes, &st.full[slot]);
            bulk_g2s(sa + kChunkBytes, QB + ((size_t)bj * nk + issued) * kChunkBytes, kChunkBytes, &st.full[slot]);
            ++issued;
        }
    }
    // D = -W / s: row rr, columns 64 h .. 64 h + 63 of the block
    float *Wg = W + (size_t)(bi * kMxBlk + rr) + (size_t)(bj * kMxBlk + 64 * h) * b;
    const uint32_t tl = st.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(64 * h);
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
        float v[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = Wg[(size_t)(32 * i + c) * b];
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = -ldexpf(v[c], -es_sum);
        tmem_st32(tl + 32 * i, v);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        bool fail = *s_fail != 0;
        for (int kk = 0; kk < nk && !fail; ++kk) {
            while ((int)issued < nk && (int)issued < kk + kMxStages) {
                const uint32_t g = G + issued, slot = g % kMxStages;
                if (g >= (uint32_t)kMxStages && !mbar_wait(&st.empty[slot], ((g / kMxStages) - 1) & 1, limit_ns)) {
                    fail = true;
                    break;
                }
                unsigned char *sa = st.stage + slot * 2 * kChunkBytes;
                mbar_expect_tx(&st.full[slot], 2 * kChunkBytes);
                bulk_g2s(sa, QA + ((size_t)bi * nk + issued) * kChunkBytes, kChunkBytes, &st.full[slot]);
                bulk_g2s(sa + kChunkBytes, QB + ((size_t)bj * nk + issued) * kChunkBytes, kChunkBytes,
                         &st.full[slot]);
                ++issued;
            }
            if (fail) break;
            const uint32_t g = G + kk, slot = g % kMxStages;
            if (!mbar_wait(&st.full[slot], (g / kMxStages) & 1, limit_ns)) { fail = true; break; }
            tc_fence_after();
            const uint32_t sa = smem_u32(st.stage + slot * 2 * kChunkBytes);
            const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + kChunkBytes);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                // advance 32 bytes of K per MMA inside the swizzle atom; every
                // MMA accumulates (the accumulator holds -W / s)
                if (fmt == 0) mma_bf16(st.tmem, ad + 2 * i, bd + 2 * i, idesc, 1u);
                else mma_e4m3(st.tmem, ad + 2 * i, bd + 2 * i, idesc, 1u);
            }
            mma_commit(&st.empty[slot]);
        }
        if (fail) {
            *s_fail = 1;
            // let copies already issued land before shared memory is reused
            for (uint32_t k2 = 0; k2 < issued; ++k2) {
                const uint32_t g = G + k2;
                mbar_wait(&st.full[g % kMxStages], (g / kMxStages) & 1, limit_ns);
            }
        }
        st.fills = G + issued;
        mma_commit(st.done);
    }
    __syncthreads();
    const bool ok = mbar_wait(st.done, st.items & 1, limit_ns);
    st.items++;
    tc_fence_after();
    // every thread takes the same branch: each one's wait may end differently
    if (__syncthreads_or(*s_fail || !ok)) return ETIMEDOUT;
    // epilogue: W <- -s D, row rr, the thread's 64 columns (SYRK: the upper
    // part of a diagonal block is left as it was)
    const int gr = bi * kMxBlk + rr;
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
        float v[32];
        tmem_ld32(tl + 32 * i, v);
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const int gc = bj * kMxBlk + 64 * h + 32 * i + c;
            if (!syrk || gr >= gc) Wg[(size_t)(32 * i + c) * b] = -ldexpf(v[c], es_sum);
        }
    }
    tc_fence_before();
    __syncthreads();
    return 0;
}

// GEMM_MX on 256 x 256 blocks (b a multiple of 256; 4 items per 512-wide
// tile): the same update as mx_update_item, with two accumulators of
// M = 128, N = 256 (tensor-memory columns 0..255 for rows 0..127 of the
// block, 256..511 for rows 128..255) that share every B chunk, so an item
// moves 1 MiB (operands 512 KiB, W 256 KiB in and out) for four 128 x 128
// blocks instead of 1.5 MiB, and pays the per-item claim once for four.
// A K-chunk takes two ring slots (the two A chunks, then the two B chunks,
// 32 KiB each); thread 0 issues a chunk's MMAs before topping up the ring,
// so the slots it refills belong to chunks whose MMAs were issued one chunk
// earlier.  Thread (q, h) owns row 128 h + 32 q + lane of the block (TMEM
// lane 32 q + lane of accumulator h) and its 256 columns, loaded two 32-column
// batches ahead of the tensor-memory stores.  Per element the arithmetic is
// that of mx_update_item.  Returns 0, or ETIMEDOUT when a pipeline wait ran
// out (block-wide).
constexpr int kMxWide = kMxWideBlk;

__device__ __forceinline__ void mx_wide_fill(MxState &st, uint32_t g, int s, const unsigned char *QA,
                                             const unsigned char *QB, int bi, int bj, int nk) {
    const uint32_t slot = g % kMxStages;
    unsigned char *sa = st.stage + slot * 2 * kChunkBytes;
    const int kk = s >> 1;
    const unsigned char *Q = (s & 1) ? QB : QA;
    const int rb = 2 * ((s & 1) ? bj : bi);
    mbar_expect_tx(&st.full[slot], 2 * kChunkBytes);
    bulk_g2s(sa, Q + ((size_t)rb * nk + kk) * kChunkBytes, kChunkBytes, &st.full[slot]);
    bulk_g2s(sa + kChunkBytes, Q + ((size_t)(rb + 1) * nk + kk) * kChunkBytes, kChunkBytes, &st.full[slot]);
}

__device__ __noinline__ int mx_gemm_wide_item(const TaskRec &t, int item, MxState &st, int64_t limit_ns,
                                              int *s_fail) {
    const int b = (int)t.n, fmt = t.aux, es = q_esize(fmt);
    const unsigned char *QA = (const unsigned char *)t.buf[0];
    const unsigned char *QB = (const unsigned char *)t.buf[1];
    float *W = (float *)t.buf[2];
    const int m = b / kMxWide;
    const int bi = item / m, bj = item % m;
    const int nk = b * es / 128;
    const int nfill = 2 * nk;
    constexpr uint32_t idesc = (mx_idesc(1u) & ~(0x3Fu << 17)) | ((uint32_t)(kMxWide >> 3) << 17);
    constexpr uint32_t idesc8 = (mx_idesc(0u) & ~(0x3Fu << 17)) | ((uint32_t)(kMxWide >> 3) << 17);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, h = warp >> 2;
    int es_sum = 0;
    if (fmt == 1) {
        es_sum = *(const int *)(QA + (size_t)b * b * es) + *(const int *)(QB + (size_t)b * b * es);
    }
    const uint32_t G = st.fills;
    int issued = 0;
    if (tid == 0) {
        *s_fail = 0;
        asm volatile("fence.proxy.async.global;" ::: "memory");
        while (issued < nfill && issued < kMxStages) {
            const uint32_t g = G + issued;
            if (g >= (uint32_t)kMxStages &&
                !mbar_wait(&st.empty[g % kMxStages], ((g / kMxStages) - 1) & 1, limit_ns)) {
                *s_fail = 1;
                break;
            }
            mx_wide_fill(st, g, issued, QA, QB, bi, bj, nk);
            ++issued;
        }
    }
    // D = -W / s: row 128 h + 32 q + lane of the block, its 256 columns
    const int rr = 128 * h + 32 * q + lane;
    float *Wg = W + (size_t)(bi * kMxWide + rr) + (size_t)(bj * kMxWide) * b;
    const uint32_t tl = st.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kMxWide * h);
    {
        float va[32], vb[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) va[c] = Wg[(size_t)c * b];
#pragma unroll 1
        for (int i = 0; i < kMxWide / 32; i += 2) {
#pragma unroll
            for (int c = 0; c < 32; ++c) vb[c] = Wg[(size_t)(32 * (i + 1) + c) * b];
#pragma unroll
            for (int c = 0; c < 32; ++c) va[c] = -ldexpf(va[c], -es_sum);
            tmem_st32(tl + 32 * i, va);
            if (i + 2 < kMxWide / 32) {
#pragma unroll
                for (int c = 0; c < 32; ++c) va[c] = Wg[(size_t)(32 * (i + 2) + c) * b];
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) vb[c] = -ldexpf(vb[c], -es_sum);
            tmem_st32(tl + 32 * (i + 1), vb);
        }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        bool fail = *s_fail != 0;
        for (int kk = 0; kk < nk && !fail; ++kk) {
            const uint32_t ga = G + 2 * kk, gb = ga + 1;
            if (!mbar_wait(&st.full[ga % kMxStages], (ga / kMxStages) & 1, limit_ns) ||
                !mbar_wait(&st.full[gb % kMxStages], (gb / kMxStages) & 1, limit_ns)) {
                fail = true;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(st.stage + (ga % kMxStages) * 2 * kChunkBytes);
            const uint32_t sb = smem_u32(st.stage + (gb % kMxStages) * 2 * kChunkBytes);
            const uint64_t a0 = sw128_desc(sa), a1 = sw128_desc(sa + kChunkBytes), bd = sw128_desc(sb);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (fmt == 0) {
                    mma_bf16(st.tmem, a0 + 2 * i, bd + 2 * i, idesc, 1u);
                    mma_bf16(st.tmem + kMxWide, a1 + 2 * i, bd + 2 * i, idesc, 1u);
                } else {
                    mma_e4m3(st.tmem, a0 + 2 * i, bd + 2 * i, idesc8, 1u);
                    mma_e4m3(st.tmem + kMxWide, a1 + 2 * i, bd + 2 * i, idesc8, 1u);
                }
            }
            mma_commit(&st.empty[ga % kMxStages]);
            mma_commit(&st.empty[gb % kMxStages]);
            // fills up to 2 kk + 4: their slots held chunk kk - 1, whose MMAs
            // were issued one chunk ago (and the next chunk's two fills are
            // among them)
            while (issued < nfill && issued < 2 * kk + kMxStages) {
                const uint32_t g = G + issued;
                if (g >= (uint32_t)kMxStages &&
                    !mbar_wait(&st.empty[g % kMxStages], ((g / kMxStages) - 1) & 1, limit_ns)) {
                    fail = true;
                    break;
                }
                mx_wide_fill(st, g, issued, QA, QB, bi, bj, nk);
                ++issued;
            }
        }
        if (fail) {
            *s_fail = 1;
            for (int k2 = 0; k2 < issued; ++k2) {
                const uint32_t g = G + k2;
                mbar_wait(&st.full[g % kMxStages], (g / kMxStages) & 1, limit_ns);
            }
        }
        st.fills = G + issued;
        mma_commit(st.done);
    }
    __syncthreads();
    const bool ok = mbar_wait(st.done, st.items & 1, limit_ns);
    st.items++;
    tc_fence_after();
    if (__syncthreads_or(*s_fail || !ok)) return ETIMEDOUT;
#pragma unroll 1
    for (int i = 0; i < kMxWide / 32; ++i) {
        float v[32];
        tmem_ld32(tl + 32 * i, v);
#pragma unroll
        for (int c = 0; c < 32; ++c) Wg[(size_t)(32 * i + c) * b] = -ldexpf(v[c], es_sum);
    }
    tc_fence_before();
    __syncthreads();
    return 0;
}

}  // namespace b3t
