// pg_micro.cu -- measured ceilings for the roofline: throughput of scalar
// FP32 FMA chains, packed FP32x2 FMA chains, MUFU rsqrt chains, the Newton
// pair term's exact instruction mix with every operand in registers (no
// shared or global memory), and random 8-byte gathers from a 4096-entry
// table in shared memory (the tabulated force's lookup, Section 3.4, with
// indices spread like those of pairs inside the cutoff), the same gathers
// from four interleaved copies and through the read-only global path (the
// placements that could raise that ceiling), each timed with CUDA events.
#include <cuda_runtime.h>

#include "pg.h"
#include "pg_device.cuh"

namespace pg {
namespace {

constexpr int kChains = 8;
constexpr int kMicroThreads = 256;
constexpr int kSinkSize = 8192;

// destination of the (practically never taken) store that keeps the work alive
__device__ float g_micro_sink[kSinkSize];

constexpr int kGatherTable = 4096;   // entries of the gather table (float2, 32 KB)

// kind 0: scalar FFMA; 1: packed FFMA2; 2: MUFU rsqrt; 3: the Newton pair
// mix; 4: random 8-byte shared-memory gathers (kGatherTable entries)
__global__ void __launch_bounds__(kMicroThreads) k_micro(int kind, int iters, float seed)
{
    extern __shared__ float2 gtab[];
    const float s = seed + threadIdx.x * 1e-7f;
    float acc = 0.0f;
    if (kind == 4) {
        for (int k = threadIdx.x; k < kGatherTable; k += kMicroThreads)
            gtab[k] = make_float2(1e-30f * k, 0.0f);
        __syncthreads();
        // kChains independent chains per thread; each gather's index comes
        // from a per-lane pseudo-random sequence mixed with the value just
        // loaded (zero here), so no load can be hoisted or merged
        unsigned h[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) h[c] = (threadIdx.x + 1) * 2654435761u + c * 40503u + blockIdx.x;
        float sum = 0.0f;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                const float2 v = gtab[(h[c] >> 12) & (kGatherTable - 1)];
                h[c] = h[c] * 1664525u + 1013904223u + __float_as_uint(v.y);
                sum += v.x;
            }
        acc = sum;
    } else if (kind == 0) {
        float x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = s + c;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], 0.999999f, 1e-7f);
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += x[c];
    } else if (kind == 1) {
        u64 x[kChains];
        const u64 a = pk2(0.999999f, 0.999998f), b = pk2(1e-7f, 2e-7f);
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = pk2(s + c, s - c);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = f2fma(x[c], a, b);
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float lo, hi;
            up2(x[c], lo, hi);
            acc += lo + hi;
        }
    } else if (kind == 2) {
        float x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = 1.5f + s + c;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = rsq(x[c]) + 1.0f;
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc += x[c];
    } else {
        // four i-pairs against a j that moves a little each iteration: the
        // pair term of the all-pairs kernel (13 FP32x2 + 2 MUFU per pair)
        u64 xi[4], yi[4], zi[4], ax[4], ay[4], az[4], ph[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            xi[p] = pk2(s + p, s - p);
            yi[p] = pk2(0.5f * p, -0.25f * p);
            zi[p] = pk2(0.1f, 0.2f * p);
            ax[p] = ay[p] = az[p] = ph[p] = 0ull;
        }
        u64 xj = pk2(0.3f, 0.3f), yj = pk2(0.7f, 0.7f), zj = pk2(-0.2f, -0.2f), mj = pk2(1e-3f, 1e-3f);
        const u64 e2 = pk2(1e-4f, 1e-4f), step = pk2(1e-6f, 1e-6f);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const u64 dx = f2sub(xj, xi[p]), dy = f2sub(yj, yi[p]), dz = f2sub(zj, zi[p]);
                u64 r2 = f2fma(dx, dx, e2);
                r2 = f2fma(dy, dy, r2);
                r2 = f2fma(dz, dz, r2);
                float ra, rb;
                up2(r2, ra, rb);
                const u64 q = pk2(rsq(ra), rsq(rb));
                const u64 mq = f2mul(mj, q);
                const u64 mq3 = f2mul(mq, f2mul(q, q));
                ph[p] = f2sub(ph[p], mq);
                ax[p] = f2fma(mq3, dx, ax[p]);
                ay[p] = f2fma(mq3, dy, ay[p]);
                az[p] = f2fma(mq3, dz, az[p]);
            }
            xj = f2add(xj, step);
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            float a0, a1, b0, b1;
            up2(f2add(f2add(ax[p], ay[p]), f2add(az[p], ph[p])), a0, a1);
            up2(xi[p], b0, b1);
            acc += a0 + a1 + b0 * 0.0f + b1 * 0.0f;
        }
    }
    if (acc == 12345.678f && blockIdx.x < kSinkSize) g_micro_sink[blockIdx.x] = acc;
}

// The same random 8-byte gathers from other placements of the table:
// C > 0: C interleaved copies in shared memory, entry e of copy c in 8-byte
// slot C e + c (copy c on bank pairs c, c + C, ...), lane l reading copy
// l mod C, so that the lanes of a warp spread over C disjoint bank sets;
// C = 0: the read-only global path (L1) on a table in device memory.
template <int C, int NTH>
__global__ void __launch_bounds__(NTH) k_micro_gather(int iters, const float2 *__restrict__ gtab_dev)
{
    extern __shared__ float2 gtab[];
    if (C > 0) {
        for (int k = threadIdx.x; k < kGatherTable * C; k += NTH) gtab[k] = make_float2(1e-30f * (k / C), 0.0f);
        __syncthreads();
    }
    const int copy = C > 0 ? (threadIdx.x & 31) % C : 0;
    unsigned h[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) h[c] = (threadIdx.x + 1) * 2654435761u + c * 40503u + blockIdx.x;
    float sum = 0.0f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            const unsigned e = (h[c] >> 12) & (kGatherTable - 1);
            const float2 v = C > 0 ? gtab[e * C + copy] : __ldg(gtab_dev + e);
            h[c] = h[c] * 1664525u + 1013904223u + __float_as_uint(v.y);
            sum += v.x;
        }
    if (sum == 12345.678f && blockIdx.x < kSinkSize) g_micro_sink[blockIdx.x] = sum;
}

// kind 5: four interleaved shared copies (1024-thread blocks, one per SM:
// 128 KB of table); kind 6: the read-only global path
int micro_gather(int kind, int sms, float *ms, double *gathers)
{
    constexpr int kCopies = 4, kThreadsC = 1024;
    const int iters = kind == 5 ? 4096 : 512;
    float2 *dtab = nullptr;
    int nth = kMicroThreads, blocks = 0;
    size_t smem = 0;
    cudaError_t e = cudaSuccess;
    if (kind == 5) {
        smem = (size_t)kGatherTable * kCopies * sizeof(float2);
        e = cudaFuncSetAttribute(k_micro_gather<kCopies, kThreadsC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        nth = kThreadsC;
        blocks = sms;
    } else {
        e = cudaMalloc(&dtab, kGatherTable * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemset(dtab, 0, kGatherTable * sizeof(float2));
        blocks = sms * 8;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {   // warm-up, then the timed launch
        const int n = pass ? iters : 16;
        if (pass) cudaEventRecord(e0);
        if (kind == 5)
            k_micro_gather<kCopies, kThreadsC><<<blocks, nth, smem>>>(n, nullptr);
        else
            k_micro_gather<0, kMicroThreads><<<blocks, nth>>>(n, dtab);
        if (pass) cudaEventRecord(e1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (dtab) cudaFree(dtab);
    *gathers = (double)blocks * nth * iters * kChains;
    if (e != cudaSuccess) { (void)cudaGetLastError(); return PG_ECUDA; }
    return PG_OK;
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" int pg_microbench(int kind, double *per_sm_clock, double *per_second)
{
    if (kind < 0 || kind > 6 || !per_sm_clock || !per_second) return PG_EINVAL;
    int dev = 0, sms = 0, clk_khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return PG_ECUDA; }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    if (kind >= 5) {
        float ms = 0;
        double g = 0;
        const int rc = micro_gather(kind, sms, &ms, &g);
        if (rc) return rc;
        if (ms <= 0) return PG_ECUDA;
        *per_second = g / (ms * 1e-3);
        *per_sm_clock = *per_second / ((double)sms * clk_khz * 1e3);
        return PG_OK;
    }
    const int blocks = sms * 8;
    const int iters = kind == 2 || kind == 4 ? 4096 : 16384;
    // lane operations per thread per iteration: FFMA 8, FFMA2 16, rsqrt 8,
    // Newton mix: 8 interactions (4 pairs x 2 lanes), gathers 8
    const double per_iter = kind == 0 ? 8.0 : kind == 1 ? 16.0 : 8.0;
    const size_t smem = kind == 4 ? kGatherTable * sizeof(float2) : 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        (void)cudaGetLastError();
        return PG_ECUDA;
    }
    k_micro<<<blocks, kMicroThreads, smem>>>(kind, 64, 0.5f);   // warm-up
    cudaEventRecord(e0);
    k_micro<<<blocks, kMicroThreads, smem>>>(kind, iters, 0.5f);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || ms <= 0) { (void)cudaGetLastError(); return PG_ECUDA; }
    const double ops = (double)blocks * kMicroThreads * iters * per_iter;
    *per_second = ops / (ms * 1e-3);
    *per_sm_clock = *per_second / ((double)sms * clk_khz * 1e3);
    return PG_OK;
}

namespace pg {

// The failure path of a bounded device wait: one thread waits on a fresh
// mbarrier that nothing arrives at, with the library's time-bounded wait and
// the given limit; the wait gives up and records a timeout in the status
// word, as a force kernel whose bulk copies never land would.
__global__ void k_wait_selftest(int *status, unsigned long long limit_ns)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    mbar_fence_init();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!mbar_wait(&bar, 0u, limit_ns)) report(status, kStatusTimeout, 9);
        mbar_inval(&bar);
    }
}

cudaError_t launch_wait_selftest(int *status, unsigned long long limit_ns, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(status, limit_ns);
    return cudaGetLastError();
}

}  // namespace pg
