// Allocation-free runner for chains of vector-scaling tasks.
//
// The task executor in executor.cu keeps its task table, dependency counters
// and ready queue in device memory that the library allocates with
// cudaMalloc.  Some callers cannot let a library do that: a process whose
// device memory is owned by a framework's caching allocator (every byte
// reserved up front, out-of-band cudaMalloc fails or breaks the budget),
// code that must not trigger the implicit device synchronisation cudaMalloc
// and cudaFree can cause, or embedded/real-time hosts that forbid allocation
// after start-up.  For them, b3t_scal_chains_noalloc runs the same chained
// x[i] <- fl32(x[i] * f) tasks with all of its scratch in one file-scope
// device array of fixed size, reserved when the library is loaded.
//
// The array is shared by every call in the process on a given device and
// keeps the previous call's contents, so each call clears the parts that must
// start at zero, and calls that overlap on the GPU (two streams, two host
// threads) race on it.
#include <cuda_runtime.h>

#include <cerrno>
#include <mutex>

#include "b3t.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int64_t kNaChunk = 1 << 16;            // f32 elements per work item
constexpr int kNaMaxTasks = 65536;               // nblocks * nchain limit
constexpr int kNaMaxDevices = 64;

// Scratch: [0] ticket counter, [1] error flag, [2..] per-task finished-item
// counters (one 32-bit counter per task, packed two per word).
constexpr size_t kNaWords = 2 + kNaMaxTasks / 2;
static __device__ __align__(256) unsigned long long g_b3t_noalloc_scratch[kNaWords];

struct NaScratch {
    unsigned long long ticket;
    unsigned long long error;
    unsigned int done[kNaMaxTasks];
};
static_assert(sizeof(NaScratch) == kNaWords * 8, "scratch layout");

__device__ __forceinline__ unsigned int na_ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long na_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void na_clear(NaScratch *s, int ntasks) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) { s->ticket = 0; s->error = 0; }
    for (int k = i; k < ntasks; k += gridDim.x * blockDim.x) s->done[k] = 0;
}

// Tickets are handed out in chain-step-major order (all blocks' step k
// before any step k+1), so an item of step k only ever waits for items with
// smaller tickets, held by CTAs that are already running: with every CTA
// resident the waits end.  Each wait is still bounded by timeout_ns.
__global__ void __launch_bounds__(kNaThreads) na_chains(float *x, int64_t n, int nblocks, int nchain,
                                                        const float *factors, int items, NaScratch *s,
                                                        long long timeout_ns) {
    __shared__ long long s_tk;
    const long long total = (long long)nblocks * nchain * items;
    for (;;) {
        if (threadIdx.x == 0) {
            long long tk = (long long)atomicAdd(&s->ticket, 1ull);
            if (tk >= total || *(volatile unsigned long long *)&s->error) tk = -1;
            if (tk >= 0) {
                const long long task = tk / items;
                const int k = (int)(task / nblocks), blk = (int)(task % nblocks);
                if (k > 0) {
                    const unsigned int *dep = &s->done[(size_t)(k - 1) * nblocks + blk];
                    const unsigned long long t0 = na_now();
                    for (unsigned n2 = 0; na_ld_acquire(dep) < (unsigned)items; ++n2) {
                        __nanosleep(64);
                        if ((n2 & 63) == 63 && (long long)(na_now() - t0) > timeout_ns) {
                            atomicExch(&s->error, (unsigned long long)ETIMEDOUT);
                            tk = -1;
                            break;
                        }
                    }
                }
            }
            s_tk = tk;
        }
        __syncthreads();
        const long long tk = s_tk;
        if (tk < 0) break;
        __threadfence();
        const long long task = tk / items;
        const int it = (int)(tk % items);
        const int k = (int)(task / nblocks), blk = (int)(task % nblocks);
        const float f = factors[(size_t)blk * nchain + k];
        float4 *v = reinterpret_cast<float4 *>(x + (size_t)blk * n + (size_t)it * kNaChunk);
        const int64_t cnt = (min(n, (int64_t)(it + 1) * kNaChunk) - (int64_t)it * kNaChunk) / 4;
        for (int64_t i = threadIdx.x; i < cnt; i += kNaThreads) {
            float4 a = __ldcg(v + i);
            a.x = __fmul_rn(a.x, f); a.y = __fmul_rn(a.y, f);
            a.z = __fmul_rn(a.z, f); a.w = __fmul_rn(a.w, f);
            __stcg(v + i, a);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&s->done[task], 1u);
        }
    }
}

struct NaDevice {
    bool ready = false;
    NaScratch *scratch = nullptr;   // device address of g_b3t_noalloc_scratch
    int nctas = 0;
};
NaDevice g_na_dev[kNaMaxDevices];
std::mutex g_na_mutex;

// One-time set-up per device, with that device current: the device address
// of the scratch array (its name in host code is only a host-side stand-in)
// and the resident grid size.
int na_setup(NaDevice **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return -ENODEV; }
    if (dev < 0 || dev >= kNaMaxDevices) return -ENODEV;
    std::lock_guard<std::mutex> lk(g_na_mutex);
    NaDevice &d = g_na_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_b3t_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return -EIO;
        }
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, na_chains, kNaThreads, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            return -EIO;
        }
        d.scratch = (NaScratch *)p;
        d.nctas = per_sm * sms;
        d.ready = true;
    }
    *out = &d;
    return 0;
}

}  // namespace

extern "C" B3T_API int b3t_scal_chains_noalloc(float *x, int64_t n, int32_t nblocks, int32_t nchain,
                                               const float *factors, int64_t timeout_ns, void *cuda_stream) {
    if (!x || !factors || n <= 0 || nblocks <= 0 || nchain <= 0) return -EINVAL;
    if (n % 4 || ((uintptr_t)x) % 16) return -EINVAL;
    if ((int64_t)nblocks * nchain > kNaMaxTasks) return -E2BIG;
    const int64_t items = (n + kNaChunk - 1) / kNaChunk;
    if (items > 0x7fffffff || items * (int64_t)nblocks * nchain > ((int64_t)1 << 40)) return -E2BIG;
    NaDevice *d = nullptr;
    int rc = na_setup(&d);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int ntasks = nblocks * nchain;
    na_clear<<<(ntasks + 255) / 256, 256, 0, s>>>(d->scratch, ntasks);
    na_chains<<<d->nctas, kNaThreads, 0, s>>>(x, n, nblocks, nchain, factors, (int)items, d->scratch,
                                               timeout_ns > 0 ? timeout_ns : 10'000'000'000LL);
    if (cudaGetLastError() != cudaSuccess) return -EIO;
    unsigned long long err = 0;
    if (cudaMemcpyAsync(&err, &d->scratch->error, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return -EIO;
    }
    return err ? -(int)err : 0;
}
