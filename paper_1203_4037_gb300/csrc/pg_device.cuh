// pg_device.cuh -- device-side building blocks shared by the pg kernels:
// packed FP32x2 arithmetic, the MUFU reciprocal square root, mbarriers with
// time-limited waits, bulk global->shared copies, and the status word the
// kernels report errors through. sm_100-family only (f32x2 needs sm_100+).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pg_internal.h"

namespace pg {

typedef unsigned long long u64;

// ---------------------------------------------------------------- f32x2
// A u64 holds two FP32 lanes {lo, hi}; one instruction processes both.
__device__ __forceinline__ u64 pk2(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(u64 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 f2fma(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 f2add(u64 a, u64 b)
{
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 f2sub(u64 a, u64 b)
{
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 f2mul(u64 a, u64 b)
{
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// MUFU reciprocal square root, the hardware approximation (the GPU's
// counterpart of the paper's VRSQRTPS); flushes subnormals.
__device__ __forceinline__ float rsq(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no overflow).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Packed TwoSum on both lanes.
__device__ __forceinline__ void two_sum2(u64 a, u64 b, u64 &s, u64 &e)
{
    s = f2add(a, b);
    u64 bb = f2sub(s, a);
    e = f2add(f2sub(a, f2sub(s, bb)), f2sub(b, bb));
}

// Fold a tile partial p into the running compensated pair (hi, lo).
__device__ __forceinline__ void fold2(u64 &hi, u64 &lo, u64 p)
{
    u64 s, e;
    two_sum2(hi, p, s, e);
    hi = s;
    lo = f2add(lo, e);
}

// ---------------------------------------------------------------- timers
__device__ __forceinline__ u64 global_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// first error wins; the host reads the word after the launch sequence
__device__ __forceinline__ void report(int *status, int code, int where)
{
    if (status) {
        if (atomicCAS(status, 0, code) == 0) atomicExch(status + 1, where);
    }
}

// ---------------------------------------------------------------- mbarrier
// one {A, G1} table entry for s in [2, s_max]: byte offset from the FP32
// bits of s by shift and mask, then a shared load (no integer multiply);
// tbase = the table's shared address minus 8 times the index of s = 2
__device__ __forceinline__ float2 tab_at(unsigned tbase, unsigned bits, int shift3)
{
    float2 v;
    const unsigned addr = tbase + ((bits >> shift3) & ~7u);
    asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

// the same for a table with a potential half: {A, G1, A_p, P1} per knot,
// 16 bytes; tbase = the table's shared address minus 16 times the index of
// s = 2
__device__ __forceinline__ float4 tab4_at(unsigned tbase, unsigned bits, int shift4)
{
    float4 v;
    const unsigned addr = tbase + ((bits >> shift4) & ~15u);
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

// min(s, s_max) for s > 0 as the integer minimum of the FP32 bit patterns
// (positive floats order like their bits; a NaN also maps to s_max): the
// clamp then runs on the ALU pipe instead of the busier FMA pipe
__device__ __forceinline__ float clamp_pos(float s, unsigned smax_bits)
{
    return __uint_as_float(min(__float_as_uint(s), smax_bits));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// arrive once and announce `bytes` of transaction for the current phase
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n"
                 " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete, giving up after
// `limit_ns` nanoseconds of wall time. Returns false on time-out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, u64 limit_ns)
{
    if (mbar_try(bar, parity)) return true;
    u64 t0 = global_ns();
    for (unsigned it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63u) == 63u && global_ns() - t0 > limit_ns) return false;
    }
}

// make prior generic-proxy accesses to shared memory ordered before later
// async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// ---------------------------------------------------------------- misc
__device__ __forceinline__ double4 ldg_d4(const double4 *p)
{
    double4 r;
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
    return r;
}

// The potential term i's own pair added in the loop (d = 0 exactly; i-particle
// k is j record k + self_off), as the
// loop computed it, so that subtracting it leaves no cancellation error:
// Newton -m_k rsqrt(eps^2) (eps of the global setting or of i itself; at
// eps = 0 the pair added nothing); table with a potential m_k psi~(s = 2),
// knot 0's value A_p + 2 P1.
__device__ __forceinline__ double self_potential(const CombineArgs &c, long long k)
{
    const float mk = (float)c.jrec[k + c.self_off].w;
    if (c.newton) {
        const float e2 = c.epsi ? (float)c.xi[k].w : c.eps2;
        return e2 > 0.0f ? -(double)__fmul_rn(mk, rsq(e2)) : 0.0;
    }
    if (c.tabpot) {
        const float4 t0 = c.agp[0];
        return (double)__fmul_rn(mk, __fmaf_rn(2.0f, t0.w, t0.z));
    }
    return 0.0;
}

}  // namespace pg
