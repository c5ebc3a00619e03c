// Device executor: one persistent kernel runs a whole task graph.
//
// Section 2 of the paper: the runtime learns the task graph from the access
// modes and the invocation order, and schedules tasks as their inputs become
// ready.  Here that schedule runs on the GPU itself:
//   * every CTA of a grid sized to full residency loops: claim a work item from
//     the device-resident ready queue, run the task body on it, and count the
//     item done;
//   * the CTA that finishes the last item of a task retires it: one warp
//     decrements the dependency counters of its successors (one lane per
//     successor, atomics issued by the whole warp) and pushes every successor
//     whose counter reached zero into the ready queue (one slot per task);
//   * the ready queue has up to kMaxLevels levels (upward-rank buckets, the
//     scheduling hint of Section 5.3, or depth from the sources); a claim
//     takes the next item of the oldest task of the highest non-empty level,
//     found with one warp-wide scan; a CTA that finishes an item of a task
//     with several items asks for the task's next item in the same round trip
//     as its done count, so it scans the queue only once the task runs dry;
//   * SCAL items stream through a ring of shared-memory stages with bulk
//     copies (cp.async.bulk and mbarriers) in the variant without tensor
//     memory, through double-buffered registers in the other;
//   * every wait is bounded by %globaltimer: an idle CTA that sees no work for
//     longer than the launch's timeout sets ETIMEDOUT in the status word and
//     the whole grid exits; nothing spins forever.
#include <cuda_runtime.h>
#include <cerrno>

#include "b3t_internal.h"
#include "mx.cuh"
#include "solve.cuh"
#include "tiles_fp64.cuh"
#include "sliced.cuh"

namespace b3t {

// dynamic shared memory per CTA: tensor-core stages and the W block need
// 160 KB; without them the largest body (FP64 TRSM) needs 75 KB, which
// leaves room for two CTAs
constexpr size_t kSmemData = 164 * 1024;   // kMxStages (5) x 32 KiB operand stages + slack
constexpr size_t kSmemDataNoMx = 76 * 1024;

__device__ __forceinline__ unsigned long long ld_acq(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_rlx(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_rlx_i32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void set_error(Ctl *ctl, int err, int task, int info, int where) {
    if (atomicCAS(&ctl->error, 0, err) == 0) {
        ctl->err_task = task;
        ctl->err_info = info;
        ctl->err_where = where;
        __threadfence();
    }
}

// ------------------------------------------------------------- SCAL
// x[i] <- fl32(x[i] * f) over one chunk, 128-bit loads and stores.  Each
// thread walks batches of U float4 at a stride of the CTA; two register
// batches alternate, so the loads of the next batch are in flight while the
// current one is scaled and stored.
__device__ __forceinline__ float4 mul4(float4 a, float f) {
    a.x = __fmul_rn(a.x, f); a.y = __fmul_rn(a.y, f);
    a.z = __fmul_rn(a.z, f); a.w = __fmul_rn(a.w, f);
    return a;
}

__device__ __forceinline__ void scal_item(const TaskRec &t, int item) {
    float *x = (float *)t.buf[0];
    const float f = __uint_as_float(t.scal);
    const int64_t start = (int64_t)item * kScalChunk;
    const int64_t end = min(t.n, start + kScalChunk);
    const int64_t nv = (end - start) >> 2;
    float4 *v = reinterpret_cast<float4 *>(x + start);
    constexpr int U = 8;
    constexpr int64_t B = (int64_t)kThreads * U;   // float4 per batch
    const int tid = threadIdx.x;
    const int64_t nfull = nv / B;
    float4 a[U], b[U];
    int64_t j = 0;
    if (nfull > 0) {
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = __ldcg(v + tid + u * kThreads);
    }
    for (; j + 2 <= nfull; j += 2) {
        const int64_t o0 = j * B + tid, o1 = o0 + B;
#pragma unroll
        for (int u = 0; u < U; ++u) b[u] = __ldcg(v + o1 + u * kThreads);
#pragma unroll
        for (int u = 0; u < U; ++u) __stcg(v + o0 + u * kThreads, mul4(a[u], f));
        if (j + 2 < nfull) {
#pragma unroll
            for (int u = 0; u < U; ++u) a[u] = __ldcg(v + o1 + B + u * kThreads);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) __stcg(v + o1 + u * kThreads, mul4(b[u], f));
    }
    if (j < nfull) {   // an odd batch count leaves the last batch in a
#pragma unroll
        for (int u = 0; u < U; ++u) __stcg(v + j * B + tid + u * kThreads, mul4(a[u], f));
    }
    for (int64_t i = nfull * B + tid; i < nv; i += kThreads) __stcg(v + i, mul4(__ldcg(v + i), f));
    const int64_t tail = (end - start) & 3;
    if (tid < tail) {
        float *p = x + start + nv * 4 + tid;
        *p = __fmul_rn(*p, f);
    }
}

// SCAL through bulk copies: 16 KiB chunks stream through a ring of S shared
// memory stages (global -> shared with an mbarrier, multiply in place,
// shared -> global).  Thread 0 issues every copy.  The loads of a CTA form one
// sequence across items: load q goes into stage q % S and completes phase
// q / S of that stage's mbarrier.  So that the ring does not drain at item
// boundaries, the item reserves the next item of the same task at its start
// (the same next-item counter the claims use) and, once the current item's
// chunks are all issued, its loads continue with that item's chunks; the
// executor runs the reserved item next.  A stage is refilled one chunk late:
// after chunk c is stored, the stage of chunk c - 1 is refilled once its
// store has read it (cp.async.bulk.wait_group.read 1), so the store just
// issued never holds up a load.  An item ends when its own stores have
// completed (wait_group 0); the next item's loads stay in flight.
// Every wait is bounded; the first that gives up stops the item (no further
// copies) after the loads already issued are drained, again with a bound
// (drain_ns).  Returns 0 or the 1-based chunk whose wait gave up; the caller
// then takes no further item on this CTA (the ring's phases are no longer
// known), so nothing touches the shared area again.
constexpr int kSbMaxStages = 12;
constexpr uint32_t kSbBytes = 16384;

struct ScalRing {
    uint64_t *full;          // [S] mbarriers
    unsigned char *stage;    // S x 16 KiB
    uint32_t S;              // stages of this launch
    uint32_t issued;         // loads issued so far (sequence number of the next one; thread 0's copy counts)
    uint32_t consumed;       // chunks processed so far (sequence number of the next one)
    int64_t nx_task;         // task and item whose first chunks are already loading
    int32_t nx_item;
};

__device__ __forceinline__ void bulk_s2g_commit(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// bytes moved by bulk copies for item `it` of a SCAL task over n floats, and
// the item's first element
__device__ __forceinline__ uint32_t scal_bulk_bytes(int64_t n, int it, int64_t *start) {
    *start = (int64_t)it * kScalChunk;
    const int64_t end = min(n, *start + kScalChunk);
    return (uint32_t)(((end - *start) & ~(int64_t)3) * 4);
}

// fch / nf: factor bits of the task's item-chain members (nf = 0 for a
// task alone), applied after the task's own factor, each rounded.
__device__ __forceinline__ int scal_item_bulk(const TaskRec &t, int64_t task, int item, int next_item,
                                              ScalRing &ring, int64_t limit_ns, int64_t drain_ns,
                                              const uint32_t *fch, int nf) {
    float *x = (float *)t.buf[0];
    const float f = __uint_as_float(t.scal);
    int64_t start, start2 = 0;
    const uint32_t bytes = scal_bulk_bytes(t.n, item, &start);
    const int nch = (int)((bytes + kSbBytes - 1) / kSbBytes);
    uint32_t bytes2 = 0;
    if (next_item >= 0) bytes2 = scal_bulk_bytes(t.n, next_item, &start2);
    const int nch2 = (int)((bytes2 + kSbBytes - 1) / kSbBytes);
    const int64_t end = min(t.n, start + kScalChunk);
    const int tid = threadIdx.x;
    char *gx = (char *)(x + start);
    char *gx2 = (char *)(x + start2);
    const uint32_t S = ring.S;
    const uint32_t base = ring.consumed;            // sequence number of this item's chunk 0
    if (!(ring.nx_task == task && ring.nx_item == item)) ring.issued = base;   // nothing of it loading yet
    const uint32_t total = (uint32_t)(nch + nch2);  // chunks in the sequence this item may issue
    // issue load q (sequence number) into stage q % S
    auto issue = [&](uint32_t q) {
        const uint32_t k = q - base;
        const uint32_t sl = q % S;
        const uint32_t nb = k < (uint32_t)nch ? min(kSbBytes, bytes - k * kSbBytes)
                                              : min(kSbBytes, bytes2 - (k - nch) * kSbBytes);
        const char *src = k < (uint32_t)nch ? gx + (size_t)k * kSbBytes : gx2 + (size_t)(k - nch) * kSbBytes;
        mbar_expect_tx(&ring.full[sl], nb);
        bulk_g2s(ring.stage + sl * kSbBytes, src, nb, &ring.full[sl]);
    };
    if (tid == 0) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        while (ring.issued - base < total && ring.issued - base < S) issue(ring.issued++);
    }
    int failed = 0, c = 0;
    for (; c < nch; ++c) {
        const uint32_t q = base + c, sl = q % S;
        const uint32_t nb = min(kSbBytes, bytes - (uint32_t)c * kSbBytes);
        const bool ok = mbar_wait(&ring.full[sl], (q / S) & 1, limit_ns);
        if (ok) {
            float4 *v = reinterpret_cast<float4 *>(ring.stage + sl * kSbBytes);
            if (nf == 0) {
                for (uint32_t i = tid; i < nb / 16; i += kThreads) v[i] = mul4(v[i], f);
            } else {
                for (uint32_t i = tid; i < nb / 16; i += kThreads) {
                    float4 a = mul4(v[i], f);
                    for (int j = 0; j < nf; ++j) a = mul4(a, __uint_as_float(fch[j]));
                    v[i] = a;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        if (__syncthreads_or(!ok)) {
            failed = c + 1;
            break;
        }
        if (tid == 0) {
            bulk_s2g_commit(gx + (size_t)c * kSbBytes, ring.stage + sl * kSbBytes, nb);
            // refill the stage of the previous chunk (q - 1) with load q - 1 + S
            // once its store has read it; the store just issued may still be reading
            const uint32_t target = q - 1 + S;
            if (ring.issued <= target && ring.issued - base < total) {
                asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                while (ring.issued <= target && ring.issued - base < total) issue(ring.issued++);
            }
        }
    }
    if (tid == 0 && failed) {
        // loads already issued (this item's and the next one's) land before
        // the CTA stops touching its shared memory
        for (uint32_t q = base + c; q != ring.issued; ++q) mbar_wait(&ring.full[q % S], (q / S) & 1, drain_ns);
    }
    ring.consumed = base + (uint32_t)nch;
    ring.nx_task = task;
    ring.nx_item = next_item;
    const int64_t tail = (end - start) - (int64_t)(bytes / 4);
    if (!failed && tid < tail) {
        float *p = x + start + bytes / 4 + tid;
        float y = __fmul_rn(*p, f);
        for (int j = 0; j < nf; ++j) y = __fmul_rn(y, __uint_as_float(fch[j]));
        *p = y;
    }
    if (tid == 0) {
        // this item's stores are complete before its done count is published
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
    return failed;
}

// POTRF_MX: L_kk = chol(fp64(W_kk)), strict upper part of L_kk zeroed.
__device__ __forceinline__ int potrf_mx_item(const TaskRec &t, double *smem, int *s_info) {
    const float *Wt = (const float *)t.buf[0];
    double *L = (double *)t.buf[1];
    const int b = (int)t.n;
    for (size_t e = threadIdx.x; e < (size_t)b * b; e += kThreads) {
        const int r = (int)(e % b), c = (int)(e / b);
        L[e] = r >= c ? (double)Wt[e] : 0.0;
    }
    __syncthreads();
    return potrf_tile(L, b, smem, s_info);
}

// CVT: L_kk = fp64(W_kk) on the lower triangle, 0 above.
// CVT, kCvtCols columns per item (column-parallel: the conversion of a
// diagonal tile sits on the factorisation's critical path).
__device__ __forceinline__ void cvt_item(const TaskRec &t, int item) {
    const float *Wt = (const float *)t.buf[0];
    double *L = (double *)t.buf[1];
    const int b = (int)t.n;
    for (int c = item * kCvtCols; c < (item + 1) * kCvtCols; ++c)
        for (int r = threadIdx.x; r < b; r += kThreads)
            L[(size_t)r + (size_t)c * b] = r >= c ? (double)Wt[(size_t)r + (size_t)c * b] : 0.0;
}

// ------------------------------------------------------------- queue
// Each ready-ring slot names one task and its item count.  Warp 0 claims a
// work item: one warp-wide scan finds the highest non-empty level; the task
// at that level's head hands out its items through an atomicAdd on its
// next_item counter, and whoever takes (or overshoots) the last item
// advances the head with a CAS, so the head moves once per task, not once per
// item.  Returns the packed (task, item), or kEmpty when the launch is over
// (all tasks retired, an error was raised, or the wait timed out: the last
// two leave the reason in ctl).
__device__ __forceinline__ void push_roots(const LaunchParams &p, const SubDesc &sd) {
    const int lane = threadIdx.x & 31;
    for (uint32_t k = lane; k < sd.nroots; k += 32) {
        const unsigned long long v = p.sroots[sd.root_off + k];
        const int64_t t = (int64_t)(v >> 32);
        const int lv = p.level[t] * p.nsub + (int)(t % p.nsub);
        const unsigned long long pos = atomicAdd(&p.ctl->lvl[lv].tail, 1ull);
        if (p.debug && pos >= p.ring_cap[lv]) set_error(p.ctl, EPROTO, (int)t, -1, 7);
        else st_rel(p.slots + p.ring_off[lv] + pos, v);
    }
    __syncwarp();
}

// Up to kBatch (8) ready single-item tasks are taken with one CAS of the head
// when the level holds more than twice as many of them as the grid has CTAs
// (the head is the serialisation point of a DAG of short tasks); the extra
// ones are kept in pend[] (shared, warp 0 only) and run next.
constexpr int kBatch = 8;

__device__ __forceinline__ unsigned long long claim(const LaunchParams &p, uint64_t kstart, uint32_t &nclaims,
                                                    unsigned long long *pend, int *npend) {
    const int lane = threadIdx.x & 31;
    Ctl *ctl = p.ctl;
    const uint64_t t0 = gtimer();
    uint32_t backoff = 0;
    // the sticky error word is read on every 16th claim and on every retry:
    // a launch that failed stops within a few items, and a claim that wins
    // costs one round trip for the level heads.  After losing the race for a
    // single-item head the word is read first, alone: the extra round trip
    // spaces out the contenders (measured: 1.76 M against 1.62 M empty
    // tasks/s); after an exhausted multi-item task it rides along with the
    // heads (an extra trip there cost 8 % on streaming chains).
    const bool check = (nclaims++ & 15) == 0;
    bool lost = false;
    for (uint32_t spin = 0;; ++spin) {
        int err = 0;
        if (lost) {
            if (lane == 0) err = ld_rlx_i32(&ctl->error);
            err = __shfl_sync(0xffffffffu, err, 0);
            if (err) return kEmpty;
        }
        // lane l reads rings l and l + 32
        unsigned long long h = 0, tl = 0, h2 = 0, tl2 = 0;
        const int nrings = p.nlevels * p.nsub;
        const bool mine = lane < nrings, mine2 = lane + 32 < nrings;
        if (mine) {
            h = ld_rlx(&ctl->lvl[lane].head);
            tl = ld_rlx(&ctl->lvl[lane].tail);
        }
        if (mine2) {
            h2 = ld_rlx(&ctl->lvl[lane + 32].head);
            tl2 = ld_rlx(&ctl->lvl[lane + 32].tail);
        }
        if (lane == 31 && !lost && (check || spin > 0)) err = ld_rlx_i32(&ctl->error);
        err = __shfl_sync(0xffffffffu, err, 31);
        if (err) return kEmpty;
        lost = false;
        const unsigned long long mask = (unsigned long long)__ballot_sync(0xffffffffu, mine && h < tl) |
                                        ((unsigned long long)__ballot_sync(0xffffffffu, mine2 && h2 < tl2) << 32);
        if (mask) {
            // the highest non-empty level; among its rings the CTA's own
            // (blockIdx mod nsub) first, then the next ones in turn
            const int ns = p.nsub;                                       // 1..64
            const int top = (63 - __clzll((long long)mask)) / ns;
            const unsigned long long all = ns == 64 ? ~0ull : (1ull << ns) - 1ull;
            const unsigned long long sub = (mask >> (top * ns)) & all;
            const int home = (int)(blockIdx.x % (unsigned)ns);
            const unsigned long long rot = home == 0 ? sub : ((sub >> home) | (sub << (ns - home))) & all;
            const int lv = top * ns + (home + __ffsll((long long)rot) - 1) % ns;
            const unsigned long long hv = __shfl_sync(0xffffffffu, lv < 32 ? h : h2, lv & 31);
            const unsigned long long tv = __shfl_sync(0xffffffffu, lv < 32 ? tl : tl2, lv & 31);
            unsigned long long item = kEmpty;
            int got = 0;
            if (lane == 0) {
                if (p.debug && hv >= p.ring_cap[lv]) {
                    set_error(ctl, EPROTO, -1, -1, 3);
                    got = 2;
                } else {
                    unsigned long long *slot = p.slots + p.ring_off[lv] + hv;
                    // a producer reserves the slot (tail) before it fills it
                    unsigned long long v = ld_acq(slot);
                    const uint64_t ts = gtimer();
                    for (uint32_t n = 0; v == kEmpty; ++n) {
                        __nanosleep(32);
                        v = ld_acq(slot);
                        if ((n & 63) == 63 && (int64_t)(gtimer() - ts) > p.timeout_ns) {
                            set_error(ctl, ETIMEDOUT, -1, -1, 2);
                            got = 2;
                            break;
                        }
                    }
                    if (!got) {
                        const int64_t t = (int64_t)(v >> 32);
                        const int n = (int)(v & 0xffffffffu);
                        if (n == 1) {
                            // single-item task: taking the head slot is taking the task;
                            // with many ready, the next filled single-item slots too
                            int k = 1;
                            unsigned long long more[kBatch - 1];
                            if (tv - hv > 2ull * gridDim.x / (unsigned)p.nsub) {
                                while (k < kBatch && hv + k < tv) {
                                    const unsigned long long w = ld_acq(slot + k);
                                    if (w == kEmpty || (int)(w & 0xffffffffu) != 1) break;
                                    more[k - 1] = w;
                                    ++k;
                                }
                            }
                            if (atomicCAS(&ctl->lvl[lv].head, hv, hv + k) == hv) {
                                item = (unsigned long long)t << 32;
                                got = 1;
                                for (int q = k - 1; q >= 1; --q) pend[(*npend)++] = (more[q - 1] >> 32) << 32;
                            } else {
                                got = 3;   // lost the race for the head
                            }
                        } else {
                            const int i = atomicAdd(&p.next_item[t], 1);
                            if (i >= n - 1) atomicCAS(&ctl->lvl[lv].head, hv, hv + 1);
                            if (i < n) {
                                item = ((unsigned long long)t << 32) | (uint32_t)i;
                                got = 1;
                            }
                        }
                    }
                }
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            if (got == 1) return __shfl_sync(0xffffffffu, item, 0);
            if (got == 2) return kEmpty;
            lost = got == 3;
            continue;
        }
        if (p.stream_mode) {
            // take in a newly published task graph, or stop when told to and
            // everything published has retired; bounded by the deadline
            unsigned long long cs = 0, ps = 0;
            int took = 0, done = 0;
            if (lane == 0) {
                ps = ld_acq(&p.sctl->published_subs);
                cs = ld_rlx(&ctl->subs_consumed);
                if (cs < ps) {
                    took = atomicCAS(&ctl->subs_consumed, cs, cs + 1) == cs;
                } else if (ld_acq(&p.sctl->stop)) {
                    done = ld_acq(&ctl->retired) >= ld_acq(&p.sctl->published_tasks);
                }
            }
            took = __shfl_sync(0xffffffffu, took, 0);
            done = __shfl_sync(0xffffffffu, done, 0);
            cs = __shfl_sync(0xffffffffu, cs, 0);
            if (took) {
                const SubDesc sd = p.subs[cs];
                push_roots(p, sd);
                continue;
            }
            if (done) return kEmpty;
            if ((spin & 15) == 15 && (int64_t)(gtimer() - kstart) > p.deadline_ns) {
                if (lane == 0) set_error(ctl, ETIMEDOUT, -1, -1, 8);
                return kEmpty;
            }
            __nanosleep(backoff);
            backoff = backoff < 256 ? backoff + 32 : 256;
            continue;
        }
        unsigned long long r = 0;
        if (lane == 0) r = ld_acq(&ctl->retired);
        r = __shfl_sync(0xffffffffu, r, 0);
        if ((int64_t)r >= p.ntasks) return kEmpty;
        if ((spin & 15) == 15 && (int64_t)(gtimer() - t0) > p.timeout_ns) {
            if (lane == 0) set_error(ctl, ETIMEDOUT, -1, -1, 1);
            return kEmpty;
        }
        __nanosleep(backoff);
        backoff = backoff < 256 ? backoff + 32 : 256;
    }
}

// Warp 0 retires task t: successors' counters (one lane per successor),
// one ready-ring slot per successor that became ready, retired count.  A task
// whose one successor it absorbed into an item chain releases none (nsucc
// given as 0).
__device__ __forceinline__ void retire(const LaunchParams &p, int64_t t, const TaskRec &rec, int nsucc) {
    const int lane = threadIdx.x & 31;
    __threadfence();
    for (int base = 0; base < nsucc; base += 32) {
        const int k = base + lane;
        if (k < nsucc) {
            const int s = p.succ[rec.succ_off + k];
            const int prev = atomicSub(&p.counters[s], 1);
            if (prev == 1) {
                const int lv = p.level[s] * p.nsub + s % p.nsub;
                const unsigned long long pos = atomicAdd(&p.ctl->lvl[lv].tail, 1ull);
                if (p.debug && pos >= p.ring_cap[lv]) set_error(p.ctl, EPROTO, s, -1, 4);
                else st_rel(p.slots + p.ring_off[lv] + pos, pack_slot(s, p.tasks[s].nitems));
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        if (p.stream_mode) {
            const int b = p.task_batch[t];
            if (atomicSub(&p.batch_left[b], 1) == 1) {
                const int info = atomicAdd(&p.batch_info[b], 0);
                __threadfence_system();
                p.batch_done[b] = info ? 2 + info : 1;
                __threadfence_system();
            }
        }
        atomicAdd(&p.ctl->retired, 1ull);
    }
}

// One variant per family set (kVarScal, kVarF64, kVarSolve, kVarNoMx,
// kVarAll): only the bodies of the variant's families are compiled in.  The
// variant with the tcgen05 tensor-memory path (kVarAll: mixed-precision
// launches and stream mode) runs one CTA per SM, as a kernel that allocates
// tensor memory does; the others run two (120 registers keep two 256-thread
// CTAs in the register file).
template <uint32_t kVar>
__global__ void __maxnreg__(120) exec_kernel(const LaunchParams p) {
    constexpr bool kMx = (kVar & kFamMx) != 0;
    extern __shared__ __align__(1024) unsigned char dsmem[];
    // align the dynamic area to 1024 bytes (128-byte swizzled operands)
    unsigned char *smem = (unsigned char *)(((uintptr_t)dsmem + 1023) & ~(uintptr_t)1023);
    __shared__ unsigned long long s_item;
    __shared__ int s_fresh;
    __shared__ int s_info, s_fail, s_e;
    __shared__ __align__(8) uint64_t s_bars[2 * kMxStages + 1];
    __shared__ uint32_t s_tmem;
    __shared__ double s_red[kThreads / 32];
    const int tid = threadIdx.x, warp = tid >> 5;

    MxState mx;
    mx.full = s_bars;
    mx.empty = s_bars + kMxStages;
    mx.done = s_bars + 2 * kMxStages;
    mx.stage = smem;
    mx.fills = 0;
    mx.items = 0;
    mx.tmem = 0;
    // RESID_SL pipeline (its own barriers: the phases of the MX ring above
    // are tracked separately, only the stage bytes are shared)
    __shared__ __align__(8) uint64_t s_slbars[kSlBars];
    SlState sl;
    sl.full = s_slbars;
    sl.empty = s_slbars + kSlStages;
    sl.xfull = s_slbars + 2 * kSlStages;
    sl.xempty = sl.xfull + 2;
    sl.done = sl.xempty + 2;
    sl.tfree = sl.done + 2;
    sl.drain = sl.tfree + 2;
    sl.fa = sl.fx = sl.nj = 0;
    // TRMM_SL pipeline (its own barriers as well)
    __shared__ __align__(8) uint64_t s_tsbars[kTsBars];
    TsState ts;
    ts.full = s_tsbars;
    ts.empty = s_tsbars + kTsStages;
    ts.bfull = s_tsbars + 2 * kTsStages;
    ts.bempty = ts.bfull + 2;
    ts.done = ts.bempty + 2;
    ts.drain = ts.done + 1;
    ts.fa = ts.fb = ts.nd = 0;
    if (kMx && p.has_mx) {
        if (tid == 0) {
            for (int i = 0; i < 2 * kMxStages + 1; ++i) mbar_init(&s_bars[i], 1);
            for (int i = 0; i < kSlBars; ++i) mbar_init(&s_slbars[i], 1);
            for (int i = 0; i < kTsBars; ++i) mbar_init(&s_tsbars[i], 1);
            // each of the four epilogue warps frees an accumulator buffer
            mbar_init(&sl.tfree[0], 4);
            mbar_init(&sl.tfree[1], 4);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (warp == 0) tmem_alloc(&s_tmem, kTmemCols);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        mx.tmem = s_tmem;
    }

    // SCAL bulk-copy ring (the variants without the tensor-memory path)
    __shared__ __align__(8) uint64_t s_sbar[kSbMaxStages];
    __shared__ int s_resv;      // next item of the same task reserved by a SCAL item, or -1
    // item chain of the SCAL task last run here: its id, members and factors
    __shared__ int64_t s_cht;
    __shared__ int32_t s_chid[kMaxChain];
    __shared__ uint32_t s_chf[kMaxChain];
    if (tid == 0) s_cht = -1;
    ScalRing ring;
    ring.full = s_sbar;
    ring.stage = smem;
    ring.S = (uint32_t)min(max(p.scal_stages, 2), kSbMaxStages);
    ring.issued = ring.consumed = 0;
    ring.nx_task = -1;
    ring.nx_item = -1;
    if ((kVar & kFamScal) && !kMx) {
        if (tid == 0) {
            for (uint32_t i = 0; i < ring.S; ++i) mbar_init(&s_sbar[i], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    const uint64_t kstart = gtimer();
    __shared__ TaskRec s_rec;
    // warp 0: an item of the previous task taken when that item finished,
    // and single-item tasks taken together with an earlier claim
    unsigned long long fi = kEmpty;
    uint32_t nclaims = 0;
    __shared__ unsigned long long s_pend[kBatch];
    __shared__ int s_npend;
    if (tid == 0) s_npend = 0;
    for (;;) {
        if (warp == 0) {
            const int lane = tid & 31;
            const bool same = fi != kEmpty;
            __syncwarp();
            const int np = s_npend;
            unsigned long long it;
            if (same) {
                it = fi;
            } else if (np > 0) {
                it = s_pend[np - 1];
                __syncwarp();
                if (lane == 0) s_npend = np - 1;
            } else {
                it = claim(p, kstart, nclaims, s_pend, &s_npend);
            }
            const int64_t t = (int64_t)(it >> 32);
            if (!same && it != kEmpty && (!p.debug || t < p.ntasks) && lane < 4)
                reinterpret_cast<uint4 *>(&s_rec)[lane] = __ldcg(reinterpret_cast<const uint4 *>(p.tasks + t) + lane);
            if (lane == 0) { s_item = it; s_fresh = !same; }
        }
        __syncthreads();
        const unsigned long long item = s_item;
        if (item == kEmpty) break;
        // acquire side for every thread of the CTA, when the item starts a
        // task this CTA has not run yet: the next item of the same task reads
        // the inputs the first one acquired (the release side is warp 0's
        // fence after the CTA barrier that ends every item)
        if (s_fresh) __threadfence();
        const int64_t t = (int64_t)(item >> 32);
        const int it = (int)(item & 0xffffffffu);
        const uint64_t t_item = (p.trace && tid == 0) ? gtimer() : 0;
        if (p.debug && (t >= p.ntasks || it >= s_rec.nitems)) {
            if (tid == 0) set_error(p.ctl, EPROTO, (int)t, -1, 5);
            __syncthreads();
            break;
        }
        const TaskRec rec = s_rec;
        int st = 0;
        constexpr bool kScal = (kVar & kFamScal) != 0, kF64 = (kVar & kFamF64) != 0,
                       kSolve = (kVar & kFamSolve) != 0, kScalRing = kScal && !kMx;
        const uint32_t fam = family_of(rec.kind);
        if (fam && !(fam & kVar)) {
            st = -EPROTO;   // the runtime picks a variant that covers every kind of the launch
        } else {
            switch (rec.kind) {
            case kScalF32:
                if constexpr (kScal && !kMx) {
                    // reserve the task's next item so that its loads start
                    // while this one drains (the executor runs it next)
                    if (tid == 0) s_resv = rec.nitems > 1 ? atomicAdd(&p.next_item[t], 1) : -1;
                    // head of an item chain: its members' ids and factors,
                    // read once per run of the task's items on this CTA
                    const int nf = rec.aux > 0 ? min(rec.aux, kMaxChain) : 0;
                    if (nf && s_cht != t && tid < nf) {
                        const int32_t *ch = (const int32_t *)rec.buf[1];
                        s_chid[tid] = __ldcg(ch + tid);
                        s_chf[tid] = (uint32_t)__ldcg(ch + rec.aux + tid);
                    }
                    __syncthreads();
                    if (tid == 0) s_cht = nf ? t : -1;
                    const int nxt = s_resv < rec.nitems ? s_resv : -1;
                    // each wait of the ring gives up after 50 ms (a 16 KiB copy
                    // takes microseconds) and the launch reports ETIMEDOUT
                    const int fc = scal_item_bulk(rec, t, it, nxt, ring, min(p.timeout_ns, (int64_t)50000000),
                                                  p.timeout_ns, s_chf, nf);
                    if (fc) {
                        if (tid == 0) set_error(p.ctl, ETIMEDOUT, (int)t, fc, 20);
                        st = -ETIMEDOUT;
                    }
                } else if constexpr (kScal) {
                    scal_item(rec, it);
                }
                break;
            case kPotrf:
                if constexpr (kF64) {
                    const int info = potrf_tile((double *)rec.buf[0], (int)rec.n, (double *)smem, &s_info);
                    if (info) st = rec.aux + info;
                }
                break;
            case kTrsm: if constexpr (kF64) trsm_item(rec, it, (double *)smem); break;
            case kSyrk: if constexpr (kF64) syrk_item(rec, it, (double *)smem); break;
            case kGemm: if constexpr (kF64) gemm_item(rec, it, (double *)smem); break;
            case kPotrfD:
                if constexpr (kF64) {
                    const int info = potrf_d_item(rec, (double *)smem, &s_info);
                    if (info) st = rec.aux + info;
                }
                break;
            case kPanelTrsm: if constexpr (kF64) panel_trsm_item(rec, it, (double *)smem); break;
            case kPanelUpd: if constexpr (kF64) panel_upd_item(rec, it, (double *)smem); break;
            case kPotrfMx:
                if constexpr (kMx) {
                    const int info = potrf_mx_item(rec, (double *)smem, &s_info);
                    if (info) st = rec.aux + info;
                }
                break;
            case kTrsmMx: if constexpr (kMx) trsm_mx_item(rec, it, (double *)smem); break;
            case kTrmmMx: if constexpr (kMx) trmm_mx_item(rec, it, (double *)smem); break;
            case kCvt: if constexpr (kMx) cvt_item(rec, it); break;
            case kQuant: if constexpr (kMx) quant_item(rec, it, s_red, &s_e); break;
            case kSyrkMx:
            case kGemmMx:
                if constexpr (kMx) {
                    if (!p.has_mx) { st = -EPROTO; break; }
                    const bool wide = rec.kind == kGemmMx && rec.n % kMxWide == 0;
                    if (wide ? mx_gemm_wide_item(rec, it, mx, p.timeout_ns, &s_fail)
                             : mx_update_item(rec, it, rec.kind == kSyrkMx, mx, p.timeout_ns, &s_fail))
                        st = -ETIMEDOUT;
                }
                break;
            case kTrtri: if constexpr (kSolve) trtri_item(rec, it, (double *)smem); break;
            case kTrtriCol: if constexpr (kSolve) trtri_col_item(rec, it, (double *)smem); break;
            case kSliceW: if constexpr (kMx) slice_w_item(rec, it, smem); break;
            case kSliceU: if constexpr (kMx) slice_u_item(rec, it, smem); break;
            case kTrmmSl:
                if constexpr (kMx) {
                    if (!p.has_mx) { st = -EPROTO; break; }
                    if (trmm_sl_item(rec, it, ts, smem, mx.tmem, min(p.timeout_ns, (int64_t)200000000), &s_fail)) {
                        if (tid == 0) set_error(p.ctl, ETIMEDOUT, (int)t, 0, 31);
                        st = -ETIMEDOUT;
                    }
                }
                break;
            case kSliceA: if constexpr (kSolve) slice_a_item(rec, s_red, &s_e); break;
            case kSliceX: if constexpr (kSolve) slice_x_item(rec, (int *)s_red); break;
            case kResidSl:
                if constexpr (kMx) {
                    if (!p.has_mx) { st = -EPROTO; break; }
                    // a chunk copy or a tile's MMAs take microseconds: each wait of
                    // the pipeline gives up after 200 ms and the launch reports ETIMEDOUT
                    if (resid_sl_item(rec, it, sl, smem, mx.tmem, min(p.timeout_ns, (int64_t)200000000), &s_fail)) {
                        if (tid == 0) set_error(p.ctl, ETIMEDOUT, (int)t, 0, 30);
                        st = -ETIMEDOUT;
                    }
                }
                break;
            case kTrsvL:
                if constexpr (kSolve) {
                    if (vk_flags(rec) & kVecF32) trsv_l_item<float>(rec, it, smem);
                    else trsv_l_item<double>(rec, it, smem);
                }
                break;
            case kTrsvLT:
                if constexpr (kSolve) {
                    if (vk_flags(rec) & kVecF32) trsv_lt_item<float>(rec, it, smem);
                    else trsv_lt_item<double>(rec, it, smem);
                }
                break;
            case kGemvL:
                if constexpr (kSolve) {
                    if (vk_flags(rec) & kVecF32) gemv_item<float, false>(rec, it, smem);
                    else gemv_item<double, false>(rec, it, smem);
                }
                break;
            case kGemvLT:
                if constexpr (kSolve) {
                    if (vk_flags(rec) & kVecF32) gemv_item<float, true>(rec, it, smem);
                    else gemv_item<double, true>(rec, it, smem);
                }
                break;
            case kAxpy: if constexpr (kSolve) axpy_item(rec); break;
            case kResid: if constexpr (kSolve) resid_item(rec, it, smem); break;
            case kNrm: if constexpr (kSolve) nrm_item(rec, smem); break;
            default: break;   // NOOP
            }
        }
        // generic-proxy writes of this body to the dynamic shared area are
        // ordered before any bulk copy (async proxy) a later item issues into
        // the same bytes; the barrier below hands them to the issuing thread
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();   // every thread is done with the item
        if (warp == 0) {
            // warp 0 alone finishes the item; the other warps go on to the
            // barrier at the top of the loop
            int flag = 0, nj = -1;
            if (tid == 0) {
                if (st > 0 && p.stream_mode) {
                    // a served request that is not positive definite fails
                    // alone: its info is reported with the batch, the graph drains
                    atomicCAS(&p.batch_info[p.task_batch[t]], 0, st);
                    st = 0;
                }
                if (st > 0) {
                    set_error(p.ctl, EDOM, (int)t, st, 0);   // not positive definite: no retire
                } else if (st < 0) {
                    set_error(p.ctl, -st, (int)t, -1, 6);
                } else if (rec.nitems == 1) {
                    flag = 1;   // the only item: retire (which fences) at once
                } else {
                    __threadfence();
                    // the next item of the same task is asked for together
                    // with the done count (the two round trips overlap); a
                    // SCAL item of the streaming variants reserved it already
                    const bool resv = rec.kind == kScalF32 && (kVar & kFamScal) && !kMx;
                    nj = resv ? s_resv : atomicAdd(&p.next_item[t], 1);
                    const int d = atomicAdd(&p.done_items[t], 1) + 1;
                    flag = d == rec.nitems;
                }
            }
            if (p.trace && tid == 0) {
                const unsigned long long k = atomicAdd(p.trace_n, 1ull);
                if ((int64_t)k < p.trace_cap) {
                    uint32_t sm;
                    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
                    p.trace[k] = TraceRec{(int32_t)t, it, (int32_t)sm, rec.kind, t_item, gtimer()};
                }
            }
            flag = __shfl_sync(0xffffffffu, flag, 0);
            nj = __shfl_sync(0xffffffffu, nj, 0);
            const bool chain = kScalRing && rec.kind == kScalF32 && rec.aux > 0;
            if (flag) retire(p, t, rec, chain ? 0 : rec.nsucc);
            if (chain && st == 0) {
                // the item was also item `it` of every chain member: count it
                // done for each (lane j for member j); members that finished
                // retire in chain order, the last one with its successors
                const int lane = tid & 31, k = rec.aux;
                uint32_t fin = 0;
                __threadfence();   // the chunk's stores before each member's done count
                for (int j0 = 0; j0 < k; j0 += 32) {
                    const int j = j0 + lane;
                    const bool last = j < k && atomicAdd(&p.done_items[s_chid[j]], 1) + 1 == rec.nitems;
                    fin = __ballot_sync(0xffffffffu, last);
                    for (uint32_t m = fin; m; m &= m - 1) {
                        const int jj = j0 + __ffs(m) - 1;
                        const int64_t mt = s_chid[jj];
                        TaskRec mr = rec;
                        if (jj == k - 1) {
                            mr.succ_off = __ldcg(&p.tasks[mt].succ_off);
                            mr.nsucc = __ldcg(&p.tasks[mt].nsucc);
                        }
                        retire(p, mt, mr, jj == k - 1 ? mr.nsucc : 0);
                    }
                }
                if (p.trace && lane == 0) {
                    const uint64_t t_end = gtimer();
                    for (int j = 0; j < k; ++j) {
                        const unsigned long long q = atomicAdd(p.trace_n, 1ull);
                        if ((int64_t)q < p.trace_cap) {
                            uint32_t sm;
                            asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
                            p.trace[q] = TraceRec{s_chid[j], it, (int32_t)sm, rec.kind, t_item, t_end};
                        }
                    }
                }
            }
            fi = (nj >= 0 && nj < rec.nitems) ? (((unsigned long long)t << 32) | (uint32_t)nj) : kEmpty;
        }
        // a bulk-copy or tensor-core pipeline whose bounded wait gave up
        // leaves its mbarrier phases unknown (and, after a failed drain,
        // copies possibly still landing in shared memory): the CTA takes no
        // further item, neither its pending ones nor a claim (st is the same
        // in every thread: the pipeline bodies return a block-wide result)
        if (st == -ETIMEDOUT) break;
    }

    if (kMx && p.has_mx) {
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (warp == 0) tmem_dealloc(mx.tmem, kTmemCols);
    }
}

__global__ void init_kernel(const InitParams ip, const LaunchParams lp) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = gid; i < ip.ntasks; i += stride) {
        ip.counters[i] = ip.indeg[i];
        ip.done_items[i] = 0;
        ip.next_item[i] = 0;
    }
    for (int64_t i = gid; i < (int64_t)ip.nslots; i += stride) {
        int l = 0;
        while (l + 1 < ip.nrings && (unsigned long long)i >= lp.ring_off[l + 1]) ++l;
        const unsigned long long k = (unsigned long long)i - lp.ring_off[l];
        ip.slots[i] = k < ip.root_cnt[l] ? ip.roots[ip.root_off[l] + k] : kEmpty;
    }
    if (gid == 0) {
        for (int l = 0; l < kMaxRings; ++l) {
            ip.ctl->lvl[l].head = 0;
            ip.ctl->lvl[l].tail = l < ip.nrings ? ip.root_cnt[l] : 0;
        }
        ip.ctl->retired = 0;
    }
}

}  // namespace b3t

using namespace b3t;

extern "C" size_t b3t_internal_smem_bytes(uint32_t variant, int32_t scal_stages) {
    // the vector variant needs only the SCAL ring: scal_stages x 16 KiB (4
    // stages let three CTAs share an SM, 12 fill one CTA per SM)
    if (variant == kVarScal) return (size_t)min(max(scal_stages, 2), kSbMaxStages) * kSbBytes + 1024;
    return ((variant & kFamMx) ? kSmemData : kSmemDataNoMx) + 1024;
}

extern "C" int32_t b3t_internal_scal_stages(uint32_t variant, size_t smem) {
    // stages of the SCAL ring that fit the launch's dynamic shared memory
    if (variant & kFamMx) return 0;
    const size_t n = (smem - 1024) / kSbBytes;
    return (int32_t)(n > (size_t)kSbMaxStages ? kSbMaxStages : n);
}

template <uint32_t kVar>
static int occupancy_of(int *ctas_per_sm, size_t smem) {
    // the largest dynamic area a launch of this variant may ask for
    const size_t most = kVar == kVarScal ? (size_t)kSbMaxStages * kSbBytes + 1024 : kSmemData + 1024;
    if (cudaFuncSetAttribute(exec_kernel<kVar>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most) !=
            cudaSuccess ||
        cudaFuncSetAttribute(exec_kernel<kVar>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) !=
            cudaSuccess)
        return -EIO;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, exec_kernel<kVar>, kThreads, smem) ==
                   cudaSuccess
               ? 0
               : -EIO;
}

extern "C" int b3t_internal_occupancy(int *ctas_per_sm, size_t smem, int *num_sms, uint32_t variant) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -EIO;
    switch (variant) {
    case kVarScal: return occupancy_of<kVarScal>(ctas_per_sm, smem);
    case kVarF64: return occupancy_of<kVarF64>(ctas_per_sm, smem);
    case kVarSolve: return occupancy_of<kVarSolve>(ctas_per_sm, smem);
    case kVarNoMx: return occupancy_of<kVarNoMx>(ctas_per_sm, smem);
    case kVarAll: return occupancy_of<kVarAll>(ctas_per_sm, smem);
    }
    return -EINVAL;
}

static void launch_exec(const LaunchParams *lp, int nctas, size_t smem, cudaStream_t s) {
    switch (lp->variant) {
    case kVarScal: exec_kernel<kVarScal><<<nctas, kThreads, smem, s>>>(*lp); break;
    case kVarF64: exec_kernel<kVarF64><<<nctas, kThreads, smem, s>>>(*lp); break;
    case kVarSolve: exec_kernel<kVarSolve><<<nctas, kThreads, smem, s>>>(*lp); break;
    case kVarNoMx: exec_kernel<kVarNoMx><<<nctas, kThreads, smem, s>>>(*lp); break;
    default: exec_kernel<kVarAll><<<nctas, kThreads, smem, s>>>(*lp); break;
    }
}

extern "C" int b3t_internal_launch(const InitParams *ip, const LaunchParams *lp, int nctas, size_t smem,
                                   void *stream, void *ev_start, void *ev_stop) {
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t work = ip->ntasks > (int64_t)ip->nslots ? ip->ntasks : (int64_t)ip->nslots;
    int ib = (int)((work + 255) / 256);
    ib = ib < 1 ? 1 : (ib > 4096 ? 4096 : ib);
    init_kernel<<<ib, 256, 0, s>>>(*ip, *lp);
    if (ev_start) cudaEventRecord((cudaEvent_t)ev_start, s);
    launch_exec(lp, nctas, smem, s);
    if (ev_stop) cudaEventRecord((cudaEvent_t)ev_stop, s);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : -EIO;
}

extern "C" int b3t_internal_launch_exec(const LaunchParams *lp, int nctas, size_t smem, void *stream,
                                        void *ev_start) {
    cudaStream_t s = (cudaStream_t)stream;
    if (ev_start) cudaEventRecord((cudaEvent_t)ev_start, s);
    launch_exec(lp, nctas, smem, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -EIO;
}
