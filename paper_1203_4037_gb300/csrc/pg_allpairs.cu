// pg_allpairs.cu -- the i-particle x j-particle force loop, all pairs.
//
// Method (Tanikawa et al. 2012): for each i, sum over all j
//   Newton, Eq. (1) with G = 1:  a_i += m_j d / (r^2 + eps^2)^{3/2},
//                                phi_i -= m_j / (r^2 + eps^2)^{1/2}
//     (the steps of Section 3.3: difference, r^2 + eps^2, inverse square
//      root, m/r, m/r^3, accumulate);
//   tabulated, Eq. (2): a_i += m_j g(r) d with g read from the bit-pattern
//     table of Section 3.4 (s = min(|d~|^2 + 2, s_max), index from the FP32
//     bits of s, linear interpolation), positions in the scaled units of
//     Section 3.4.2 and the result rescaled at the end.
//
// GB300 mapping (not the paper's AVX layout):
//  * work is split stream-K style: the (i-tile, j-sub-tile) units are cut
//    into equal contiguous ranges, one per CTA, so every SM gets the same
//    number of pair evaluations whatever the tile counts;
//  * i-particles sit in registers, 2*NP per thread, packed in pairs for the
//    FP32x2 instructions; j sub-tiles of kTJ records arrive in shared memory
//    by bulk copies (double-buffered, completion on an mbarrier);
//  * precision: the FP64 j record minus the FP64 i-tile centre is rounded to
//    FP32 once per (j, tile) while staging; the pair loop runs in FP32 with
//    the MUFU rsqrt; each sub-tile's FP32 partial is folded into a TwoSum
//    (hi, lo) pair; the per-CTA partials are combined in FP64.
//
// DF selects double-float differencing, for i-tiles that are not compact
// (i-particles not in Morton order, or few i against many more j): each
// FP32 offset x~ = fp32(x - c) is staged with its FP32 residual
// e = fp32((x - c) - x~), and a pair's difference is formed as
// (x~_j - x~_i) + (e_j - e_i). Its error is then a few units of FP32
// rounding of |d| itself, whatever the tile's extent; with one FP32 offset
// per particle it is a few units of the offsets' magnitude, which for a
// close pair inside a wide tile is far more (3 more lane operations per
// component and pair).
//
// EXT selects the extended form of each mode: in Newton mode the softening
// of each i-particle read from its record (w = eps_i^2: the i-particle
// structure of Section 3.1 carries eps^2 per i), with a guard that gives a
// coincident pair at eps_i = 0 no contribution; in table mode a potential
// phi_i += m_j psi~(s) from a second table on the same knots, interleaved
// with the force table as {A, G1, A_p, P1} (the paper's tabulated kernel
// stores accelerations only).
#include "pg_device.cuh"

namespace pg {

// Bulk-copy the raw j records of sub-tile s (32 bytes each: FP64 (x, m), or
// the double-float pairs) into a buffer slot.
__device__ __forceinline__ void issue_jsub(const void *jrec, long long nj, int s, double4 *dst,
                                           uint64_t *bar)
{
    long long j0 = (long long)s * kTJ;
    long long nv = nj - j0;
    if (nv > kTJ) nv = kTJ;
    unsigned bytes = (unsigned)(nv * 32);
    mbar_arrive_tx(bar, bytes);
    bulk_g2s(dst, reinterpret_cast<const unsigned char *>(jrec) + j0 * 32, bytes, bar);
}

// which CTA owns unit u under the equal split of W units over `grid` CTAs
__host__ __device__ __forceinline__ long long stream_k_owner(long long u, long long grid,
                                                             long long W)
{
    return ((u + 1) * grid - 1) / W;
}

long long stream_k_first(long long u, int grid, long long W)
{
    return stream_k_owner(u, grid, W);
}

template <int NP>
struct Bi_of {
    static constexpr int value = kNT * 2 * NP;
};

int allpairs_bi(int np) { return kNT * 2 * np; }

// Pair arithmetic on two FP32 lanes: packed f32x2 instructions (PK) or two
// scalar instructions per operation (the same roundings either way).
template <bool PK>
struct Lanes;

template <>
struct Lanes<true> {
    static __device__ __forceinline__ u64 fma(u64 a, u64 b, u64 c) { return f2fma(a, b, c); }
    static __device__ __forceinline__ u64 add(u64 a, u64 b) { return f2add(a, b); }
    static __device__ __forceinline__ u64 sub(u64 a, u64 b) { return f2sub(a, b); }
    static __device__ __forceinline__ u64 mul(u64 a, u64 b) { return f2mul(a, b); }
};

template <>
struct Lanes<false> {
    static __device__ __forceinline__ u64 fma(u64 a, u64 b, u64 c)
    {
        float a0, a1, b0, b1, c0, c1;
        up2(a, a0, a1); up2(b, b0, b1); up2(c, c0, c1);
        return pk2(__fmaf_rn(a0, b0, c0), __fmaf_rn(a1, b1, c1));
    }
    static __device__ __forceinline__ u64 add(u64 a, u64 b)
    {
        float a0, a1, b0, b1;
        up2(a, a0, a1); up2(b, b0, b1);
        return pk2(__fadd_rn(a0, b0), __fadd_rn(a1, b1));
    }
    static __device__ __forceinline__ u64 sub(u64 a, u64 b)
    {
        float a0, a1, b0, b1;
        up2(a, a0, a1); up2(b, b0, b1);
        return pk2(__fsub_rn(a0, b0), __fsub_rn(a1, b1));
    }
    static __device__ __forceinline__ u64 mul(u64 a, u64 b)
    {
        float a0, a1, b0, b1;
        up2(a, a0, a1); up2(b, b0, b1);
        return pk2(__fmul_rn(a0, b0), __fmul_rn(a1, b1));
    }
};

// CTAs per SM the register budget is sized for
#ifndef PG_NP4_MIN_BLOCKS
#define PG_NP4_MIN_BLOCKS 3
#endif
#ifndef PG_TABLE_NP4_MIN_BLOCKS
#define PG_TABLE_NP4_MIN_BLOCKS 3
#endif
// unroll depth of the j loop: independent pair terms in flight per thread
// (measured on GB300: 16 beats 4 by 6 % in table mode and 4 % in Newton
// mode; 32 falls back in table mode)
#ifndef PG_AP_UNROLL
#define PG_AP_UNROLL 16
#endif
#define PG_STR_(x) #x
#define PG_UNROLL(n) _Pragma(PG_STR_(unroll n))
// (the double-float variant holds three more i-pair registers per pair and
// the residuals in flight: one block fewer, so that it does not spill)
template <int NP, bool TABLE, bool DF>
struct MinBlocks {
    static constexpr int value = DF ? (NP == 1 ? 6 : NP == 2 ? 4 : 2)
                               : NP == 1 ? 8 : NP == 2 ? 5
                               : TABLE ? PG_TABLE_NP4_MIN_BLOCKS : PG_NP4_MIN_BLOCKS;
};

// u64 words staged per j record: {x, y, z, m} (each value in both lanes),
// with DF also {e_x, e_y, e_z, 0}
template <bool DF> struct CvtWords { static constexpr int value = DF ? 8 : 4; };

// (hi + lo) - (chi + clo) rounded once to FP32, from a double-float value
// and a double-float centre: TwoSum gives hi - chi = s + t exactly, and the
// small remainder (lo - clo) + t is added to s with one rounding (its own
// rounding is far below s's last place), as exact a rounding as forming the
// difference in FP64
__device__ __forceinline__ float df_offset(float hi, float lo, float chi, float clo)
{
    float s, t;
    two_sum(hi, -chi, s, t);
    return __fadd_rn(s, __fadd_rn(__fsub_rn(lo, clo), t));
}

template <int NP, bool TABLE, bool EXT, bool PK, bool DF>
__global__ void __launch_bounds__(kNT, MinBlocks<NP, TABLE, DF>::value) k_allpairs(AllPairsArgs a)
{
    using V = Lanes<PK>;
    constexpr int Bi = Bi_of<NP>::value;
    constexpr int kW = CvtWords<DF>::value;
    extern __shared__ __align__(128) unsigned char smem[];
    double4 *raw = reinterpret_cast<double4 *>(smem);                       // [2][kTJ]
    u64 *cvt = reinterpret_cast<u64 *>(smem + 2 * kTJ * sizeof(double4));   // [kTJ][kW]
    // compensated running sums (hi, lo) of every thread's i, [2 kComp NP][kNT]
    // (kComp = 4: a and phi; 3 in table mode without a potential): they
    // change once per sub-tile, so they live in shared memory
    constexpr int kComp = TABLE && !EXT ? 3 : 4;
    u64 *run = cvt + kTJ * kW;
    uint64_t *bar = reinterpret_cast<uint64_t *>(run + 2 * kComp * NP * kNT);
    int *flag = reinterpret_cast<int *>(bar + 2);
    float2 *tab = reinterpret_cast<float2 *>(bar + 4);

    // Newton with single offsets stages double-float records and forms each
    // offset in FP32 (df_offset, rounded once): no FP64 instruction in the
    // steady state (GB300 issues FP64 at about two operations per SM-clock,
    // and the conversion runs between the barriers around the pair loop)
    constexpr bool HLJ = !TABLE && !DF;
    const void *jsrc = HLJ ? (const void *)a.jhl : (const void *)a.jrec;

    const int tid = threadIdx.x;
    const long long G = gridDim.x;
    const long long b = blockIdx.x;
    const long long u0 = b * a.W / G, u1 = (b + 1) * a.W / G;
    if (u0 >= u1) return;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    if (TABLE && !EXT)
        for (int k = tid; k < a.tab.n; k += kNT) tab[k] = a.tab.AG1[k];
    if (TABLE && EXT)
        for (int k = tid; k < a.tab.n; k += kNT) reinterpret_cast<float4 *>(tab)[k] = a.tab.AGP[k];
    __syncthreads();

    // prefetch the first two sub-tiles
    unsigned pending = 0; // bit k: a copy into buffer k is in flight (thread 0)
    if (tid == 0) {
        issue_jsub(jsrc, a.nj, (int)(u0 % a.njsub), raw, &bar[0]);
        pending = 1u;
        if (u0 + 1 < u1) {
            issue_jsub(jsrc, a.nj, (int)((u0 + 1) % a.njsub), raw + kTJ, &bar[1]);
            pending |= 2u;
        }
    }
    unsigned phase = 0;   // bit k: parity of the next completion of buffer k

    // per-thread state
    u64 xi[NP], yi[NP], zi[NP];
    u64 exi[DF ? NP : 1], eyi[DF ? NP : 1], ezi[DF ? NP : 1];   // DF: the offsets' residuals
    u64 e2i[NP];                                 // Newton EXT: each i-pair's eps^2
    u64 ax[NP], ay[NP], az[NP], ph[NP];          // sub-tile partials
    // running sum k of pair p: hi at run[(2 kComp p + k) kNT + tid], lo at k + kComp
    auto RH = [&](int p, int k) -> u64 & { return run[(2 * kComp * p + k) * kNT + tid]; };
    auto RL = [&](int p, int k) -> u64 & { return run[(2 * kComp * p + kComp + k) * kNT + tid]; };
    double cx = 0, cy = 0, cz = 0;
    float chx = 0, chy = 0, chz = 0, clx = 0, cly = 0, clz = 0;   // HLJ: the centre as hi + lo
    long long cur = -1;

    const u64 zero2 = 0ull;
    const float c0 = TABLE ? 2.0f : a.eps2;
    const u64 c0v = pk2(c0, c0);
    const double sc = TABLE ? a.tab.scale : 1.0;
    const unsigned smax_bits = __float_as_uint(a.tab.s_max);
    const int sh3 = a.tab.shift - (EXT ? 4 : 3);
    const unsigned tb0 = smem_u32(tab) - (a.tab.base << (EXT ? 4 : 3));
    bool failed = false;

    auto flush = [&](long long t) {
        long long slot = b - stream_k_owner(t * a.njsub, G, a.W);
        double4 *dst = a.part + ((size_t)t * a.smax_slots + (size_t)slot) * Bi;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float h[8] = {0, 0, 0, 0, 0, 0, 0, 0}, l[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int k = 0; k < kComp; ++k) {
                up2(RH(p, k), h[2 * k], h[2 * k + 1]);
                up2(RL(p, k), l[2 * k], l[2 * k + 1]);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                int li = (2 * p + q) * kNT + tid;
                if (t * Bi + li < a.ni)
                    dst[li] = make_double4((double)h[q] + (double)l[q], (double)h[2 + q] + (double)l[2 + q],
                                           (double)h[4 + q] + (double)l[4 + q],
                                           (double)h[6 + q] + (double)l[6 + q]);
            }
        }
    };

    for (long long u = u0; u < u1; ++u) {
        const long long t = u / a.njsub;
        const int s = (int)(u % a.njsub);
        const int buf = (int)((u - u0) & 1);

        if (t != cur) {
            if (cur >= 0) flush(cur);
            cur = t;
            double4 c = a.ctr[t];
            cx = c.x; cy = c.y; cz = c.z;
            chx = (float)cx; clx = (float)(cx - (double)chx);
            chy = (float)cy; cly = (float)(cy - (double)chy);
            chz = (float)cz; clz = (float)(cz - (double)chz);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float fx[2], fy[2], fz[2], fe[2], rx[2], ry[2], rz[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    long long i = t * Bi + (2 * p + q) * kNT + tid;
                    if (i < a.ni) {
                        double4 v = a.xi[i];
                        const double ox = (v.x - cx) * sc, oy = (v.y - cy) * sc, oz = (v.z - cz) * sc;
                        fx[q] = (float)ox;
                        fy[q] = (float)oy;
                        fz[q] = (float)oz;
                        if (HLJ) {   // the j records' formula, so the own pair differences to 0
                            const float hx = (float)v.x, hy = (float)v.y, hz = (float)v.z;
                            fx[q] = df_offset(hx, (float)(v.x - (double)hx), chx, clx);
                            fy[q] = df_offset(hy, (float)(v.y - (double)hy), chy, cly);
                            fz[q] = df_offset(hz, (float)(v.z - (double)hz), chz, clz);
                        }
                        rx[q] = (float)(ox - (double)fx[q]);
                        ry[q] = (float)(oy - (double)fy[q]);
                        rz[q] = (float)(oz - (double)fz[q]);
                        fe[q] = (float)v.w;
                    } else {
                        fx[q] = fy[q] = fz[q] = fe[q] = rx[q] = ry[q] = rz[q] = 0.0f;
                    }
                }
                xi[p] = pk2(fx[0], fx[1]);
                yi[p] = pk2(fy[0], fy[1]);
                zi[p] = pk2(fz[0], fz[1]);
                if (DF) {
                    exi[p] = pk2(rx[0], rx[1]);
                    eyi[p] = pk2(ry[0], ry[1]);
                    ezi[p] = pk2(rz[0], rz[1]);
                }
                e2i[p] = pk2(fe[0], fe[1]);
#pragma unroll
                for (int k = 0; k < kComp; ++k) RH(p, k) = RL(p, k) = zero2;
            }
        }

        // wait for this sub-tile's raw records (one thread waits, all learn)
        if (tid == 0) {
            bool ok = mbar_wait(&bar[buf], (phase >> buf) & 1u, kWaitLimitNs);
            if (ok) pending &= ~(1u << buf);
            *flag = ok ? 1 : 0;
        }
        __syncthreads();
        if (*flag == 0) { failed = true; break; }
        phase ^= 1u << buf;

        // convert: FP64 record minus FP64 tile centre, rounded once to FP32
        // (DF: and the residual of that rounding; HLJ: the same rounding
        // formed in FP32 from the double-float record); each value is stored twice so one
        // 16-byte load yields f32x2 pairs
        {
            const long long j0 = (long long)s * kTJ;
            long long nv = a.nj - j0;
            if (nv > kTJ) nv = kTJ;
            const double4 *r = raw + buf * kTJ;
            const float4 *r4 = reinterpret_cast<const float4 *>(r);
            for (int e = tid; e < kTJ; e += kNT) {
                float x, y, z, m, rx = 0.0f, ry = 0.0f, rz = 0.0f;
                if (HLJ && e < nv) {
                    const float4 h = r4[2 * e], l = r4[2 * e + 1];
                    x = df_offset(h.x, l.x, chx, clx);
                    y = df_offset(h.y, l.y, chy, cly);
                    z = df_offset(h.z, l.z, chz, clz);
                    m = h.w;
                } else if (e < nv) {
                    double4 v = r[e];
                    const double ox = (v.x - cx) * sc, oy = (v.y - cy) * sc, oz = (v.z - cz) * sc;
                    x = (float)ox;
                    y = (float)oy;
                    z = (float)oz;
                    if (DF) {
                        rx = (float)(ox - (double)x);
                        ry = (float)(oy - (double)y);
                        rz = (float)(oz - (double)z);
                    }
                    m = (float)v.w;
                } else {   // padding: zero mass far away contributes exactly 0
                    x = y = z = 1.0e4f;
                    m = 0.0f;
                }
                cvt[kW * e + 0] = pk2(x, x);
                cvt[kW * e + 1] = pk2(y, y);
                cvt[kW * e + 2] = pk2(z, z);
                cvt[kW * e + 3] = pk2(m, m);
                if (DF) {
                    cvt[kW * e + 4] = pk2(rx, rx);
                    cvt[kW * e + 5] = pk2(ry, ry);
                    cvt[kW * e + 6] = pk2(rz, rz);
                    cvt[kW * e + 7] = 0ull;
                }
            }
        }
        __syncthreads();
        // refill the raw buffer just consumed with unit u + 2
        if (tid == 0 && u + 2 < u1) {
            fence_proxy_async();
            issue_jsub(jsrc, a.nj, (int)((u + 2) % a.njsub), raw + buf * kTJ, &bar[buf]);
            pending |= 1u << buf;
        }

#pragma unroll
        for (int p = 0; p < NP; ++p) ax[p] = ay[p] = az[p] = ph[p] = zero2;

        PG_UNROLL(PG_AP_UNROLL)
        for (int e = 0; e < kTJ; ++e) {
            const ulonglong2 xy = reinterpret_cast<const ulonglong2 *>(cvt)[(kW / 2) * e];
            const ulonglong2 zm = reinterpret_cast<const ulonglong2 *>(cvt)[(kW / 2) * e + 1];
            ulonglong2 rxy = make_ulonglong2(0ull, 0ull), rz0 = rxy;
            if (DF) {
                rxy = reinterpret_cast<const ulonglong2 *>(cvt)[(kW / 2) * e + 2];
                rz0 = reinterpret_cast<const ulonglong2 *>(cvt)[(kW / 2) * e + 3];
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                u64 dx = V::sub(xy.x, xi[p]);
                u64 dy = V::sub(xy.y, yi[p]);
                u64 dz = V::sub(zm.x, zi[p]);
                if (DF) {
                    dx = V::add(dx, V::sub(rxy.x, exi[p]));
                    dy = V::add(dy, V::sub(rxy.y, eyi[p]));
                    dz = V::add(dz, V::sub(rz0.x, ezi[p]));
                }
                u64 r2 = V::fma(dx, dx, !TABLE && EXT ? e2i[p] : c0v);
                r2 = V::fma(dy, dy, r2);
                r2 = V::fma(dz, dz, r2);
                float ra, rb;
                up2(r2, ra, rb);
                if (!TABLE) {
                    float qa = rsq(ra), qb = rsq(rb);
                    if (EXT) {     // eps_i = 0: a coincident pair contributes nothing
                        qa = ra > 0.0f ? qa : 0.0f;
                        qb = rb > 0.0f ? qb : 0.0f;
                    }
                    const u64 q = pk2(qa, qb);
                    const u64 mq = V::mul(zm.y, q);
                    const u64 q2 = V::mul(q, q);
                    const u64 mq3 = V::mul(mq, q2);
                    ph[p] = V::sub(ph[p], mq);
                    ax[p] = V::fma(mq3, dx, ax[p]);
                    ay[p] = V::fma(mq3, dy, ay[p]);
                    az[p] = V::fma(mq3, dz, az[p]);
                } else {
                    ra = clamp_pos(ra, smax_bits);
                    rb = clamp_pos(rb, smax_bits);
                    // the entry's shared address by shift and mask of the
                    // bits (7 % faster than indexing on GB300); each lane's
                    // {A, G1} arrives as a pair: two scalar FMAs write the
                    // packed g without register moves
                    u64 g;
                    if (EXT) {
                        const float4 ta = tab4_at(tb0, __float_as_uint(ra), sh3);
                        const float4 tb = tab4_at(tb0, __float_as_uint(rb), sh3);
                        g = pk2(__fmaf_rn(ra, ta.y, ta.x), __fmaf_rn(rb, tb.y, tb.x));
                        const u64 pp = pk2(__fmaf_rn(ra, ta.w, ta.z), __fmaf_rn(rb, tb.w, tb.z));
                        ph[p] = V::fma(zm.y, pp, ph[p]);
                    } else {
                        const float2 ta = tab_at(tb0, __float_as_uint(ra), sh3);
                        const float2 tb = tab_at(tb0, __float_as_uint(rb), sh3);
                        g = pk2(__fmaf_rn(ra, ta.y, ta.x), __fmaf_rn(rb, tb.y, tb.x));
                    }
                    const u64 mg = V::mul(zm.y, g);
                    ax[p] = V::fma(mg, dx, ax[p]);
                    ay[p] = V::fma(mg, dy, ay[p]);
                    az[p] = V::fma(mg, dz, az[p]);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            fold2(RH(p, 0), RL(p, 0), ax[p]);
            fold2(RH(p, 1), RL(p, 1), ay[p]);
            fold2(RH(p, 2), RL(p, 2), az[p]);
            if (!TABLE || EXT) fold2(RH(p, 3), RL(p, 3), ph[p]);
        }
    }

    if (failed) {
        // let copies still in flight land before the CTA's shared memory goes
        if (tid == 0) {
            report(a.status, kStatusTimeout, 1);
            for (int k = 0; k < 2; ++k)
                if (pending & (1u << k)) mbar_wait(&bar[k], (phase >> k) & 1u, kWaitLimitNs / 4);
        }
        return;
    }
    if (cur >= 0) flush(cur);
}

// ------------------------------------------------------------------ host

size_t allpairs_smem(int np, bool table, int ntab, bool ext, bool df)
{
    size_t s = 2 * kTJ * sizeof(double4) + (size_t)kTJ * (df ? 8 : 4) * sizeof(u64) +
               2 * (table && !ext ? 3 : 4) * np * kNT * sizeof(u64) + 4 * sizeof(uint64_t);
    if (table) s += (size_t)ntab * sizeof(float2);
    return s;
}

// raise the kernel's dynamic shared memory limit once per device (outside
// any capture); the attribute belongs to the device's context
template <int NP, bool TABLE, bool EXT, bool PK, bool DF>
static cudaError_t configure_one()
{
    static bool done[kMaxDevices] = {};
    return once_per_device(done, [] {
        return cudaFuncSetAttribute(k_allpairs<NP, TABLE, EXT, PK, DF>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)allpairs_smem(NP, TABLE, 2 << 13, EXT, DF));
    });
}

template <int NP, bool TABLE, bool EXT, bool PK, bool DF>
static cudaError_t launch_one(const AllPairsArgs &a, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = configure_one<NP, TABLE, EXT, PK, DF>();
    if (e != cudaSuccess) return e;
    k_allpairs<NP, TABLE, EXT, PK, DF><<<grid, kNT, smem, st>>>(a);
    return cudaGetLastError();
}

template <int NP, bool TABLE, bool EXT, bool PK, bool DF>
static int occupancy_one(size_t smem)
{
    auto k = k_allpairs<NP, TABLE, EXT, PK, DF>;
    if (configure_one<NP, TABLE, EXT, PK, DF>() != cudaSuccess) return 1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kNT, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

// the double-float variant exists in packed form only (the same roundings)
template <int NP, bool PK, bool DF>
static int occupancy_pk(bool table, bool ext, size_t smem)
{
    if (table) return ext ? occupancy_one<NP, true, true, PK, DF>(smem) : occupancy_one<NP, true, false, PK, DF>(smem);
    return ext ? occupancy_one<NP, false, true, PK, DF>(smem) : occupancy_one<NP, false, false, PK, DF>(smem);
}

template <int NP>
static int occupancy_np(bool table, bool packed, bool ext, bool df, size_t smem)
{
    if (df) return occupancy_pk<NP, true, true>(table, ext, smem);
    return packed ? occupancy_pk<NP, true, false>(table, ext, smem) : occupancy_pk<NP, false, false>(table, ext, smem);
}

int allpairs_max_blocks_per_sm(int np, bool table, int ntab, bool packed, bool ext, bool df)
{
    size_t smem = allpairs_smem(np, table, ntab, ext, df);
    return np == 1 ? occupancy_np<1>(table, packed, ext, df, smem)
         : np == 4 ? occupancy_np<4>(table, packed, ext, df, smem)
                   : occupancy_np<2>(table, packed, ext, df, smem);
}

template <int NP, bool PK, bool DF>
static cudaError_t launch_np(const AllPairsArgs &a, int grid, bool table, bool ext, size_t smem,
                             cudaStream_t st)
{
    if (table) return ext ? launch_one<NP, true, true, PK, DF>(a, grid, smem, st)
                          : launch_one<NP, true, false, PK, DF>(a, grid, smem, st);
    return ext ? launch_one<NP, false, true, PK, DF>(a, grid, smem, st)
               : launch_one<NP, false, false, PK, DF>(a, grid, smem, st);
}

template <int NP>
static cudaError_t launch_np_any(const AllPairsArgs &a, int grid, bool table, bool ext, bool packed,
                                 bool df, size_t smem, cudaStream_t st)
{
    if (df) return launch_np<NP, true, true>(a, grid, table, ext, smem, st);
    return packed ? launch_np<NP, true, false>(a, grid, table, ext, smem, st)
                  : launch_np<NP, false, false>(a, grid, table, ext, smem, st);
}

cudaError_t launch_allpairs(const AllPairsArgs &a, int grid, int np, bool table, bool ext,
                            bool packed, bool df, size_t smem, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    if (np == 1) return launch_np_any<1>(a, grid, table, ext, packed, df, smem, st);
    if (np == 2) return launch_np_any<2>(a, grid, table, ext, packed, df, smem, st);
    if (np == 4) return launch_np_any<4>(a, grid, table, ext, packed, df, smem, st);
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ combine
// One thread per i (tile order): add the CTA partials of its tile in slot
// order in FP64, take out the self pair's potential term, rescale, scatter.
__global__ void k_combine(CombineArgs c)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= c.ni) return;
    long long t = p / c.Bi;
    int li = (int)(p % c.Bi);
    double ax = 0, ay = 0, az = 0, ph = 0;
    if (c.njsub > 0) {
        long long bf = stream_k_owner(t * c.njsub, c.grid, c.W);
        long long bl = stream_k_owner((t + 1) * c.njsub - 1, c.grid, c.W);
        for (long long s = 0; s <= bl - bf; ++s) {
            double4 v = c.part[((size_t)t * c.smax_slots + (size_t)s) * c.Bi + li];
            ax += v.x; ay += v.y; az += v.z; ph += v.w;
        }
    }
    long long k = c.perm ? (long long)c.perm[p] : p;
    if (c.self && c.njsub > 0) ph -= self_potential(c, k);
    if (c.fail_nan && *c.fail_nan != 0) ax = ay = az = ph = __longlong_as_double(0x7ff8000000000000ll);
    c.acc[3 * k] = ax * c.accscale;
    c.acc[3 * k + 1] = ay * c.accscale;
    c.acc[3 * k + 2] = az * c.accscale;
    if (c.pot) c.pot[k] = c.newton || c.tabpot ? ph : 0.0;
}

// The same sum with a 128-thread block per i, for few i-particles with many
// partial slots (a single thread per i would walk hundreds of dependent
// loads): thread t adds slots t, t + 128, ..., a fixed butterfly adds each
// warp's lanes and thread 0 the four warps in order, so the result does not
// depend on the run.
constexpr int kWideThreads = 128;

__global__ void __launch_bounds__(kWideThreads) k_combine_wide(CombineArgs c)
{
    __shared__ double4 wsum[kWideThreads / 32];
    const long long p = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const long long t = p / c.Bi;
    const int li = (int)(p % c.Bi);
    double ax = 0, ay = 0, az = 0, ph = 0;
    if (c.njsub > 0) {
        const long long bf = stream_k_owner(t * c.njsub, c.grid, c.W);
        const long long bl = stream_k_owner((t + 1) * c.njsub - 1, c.grid, c.W);
        for (long long s = threadIdx.x; s <= bl - bf; s += kWideThreads) {
            const double4 v = c.part[((size_t)t * c.smax_slots + (size_t)s) * c.Bi + li];
            ax += v.x; ay += v.y; az += v.z; ph += v.w;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
        ph += __shfl_xor_sync(0xffffffffu, ph, o);
    }
    if (lane == 0) wsum[threadIdx.x >> 5] = make_double4(ax, ay, az, ph);
    __syncthreads();
    if (threadIdx.x != 0) return;
    ax = ay = az = ph = 0;
    for (int w = 0; w < kWideThreads / 32; ++w) {
        ax += wsum[w].x; ay += wsum[w].y; az += wsum[w].z; ph += wsum[w].w;
    }
    const long long k = c.perm ? (long long)c.perm[p] : p;
    if (c.self && c.njsub > 0) ph -= self_potential(c, k);
    if (c.fail_nan && *c.fail_nan != 0) ax = ay = az = ph = __longlong_as_double(0x7ff8000000000000ll);
    c.acc[3 * k] = ax * c.accscale;
    c.acc[3 * k + 1] = ay * c.accscale;
    c.acc[3 * k + 2] = az * c.accscale;
    if (c.pot) c.pot[k] = c.newton || c.tabpot ? ph : 0.0;
}

cudaError_t launch_combine(const CombineArgs &c, cudaStream_t st)
{
    if (c.ni <= 0) return cudaSuccess;
    if (c.smax_slots >= 32)
        k_combine_wide<<<(unsigned)c.ni, kWideThreads, 0, st>>>(c);
    else
        k_combine<<<(unsigned)((c.ni + 255) / 256), 256, 0, st>>>(c);
    return cudaGetLastError();
}

}  // namespace pg
