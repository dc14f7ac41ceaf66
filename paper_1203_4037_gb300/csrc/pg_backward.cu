// pg_backward.cu -- gradients of L = sum_i w_i . a_i for the all-pairs force
// (an extension: the paper has no backward pass). Pair terms are recomputed,
// never stored.
//
// With d_kj = x_j - x_k, the pair kernel K(r^2) (Newton: (r^2+eps^2)^(-3/2);
// table: the interpolant g(s), s = scale^2 r^2 + 2) and J(d) = K I +
// 2 dK/d(r^2) d d^T (symmetric, even in d):
//   dL/dx_k = sum_{j != k} J(d_kj) (m_k w_j - m_j w_k)
//   dL/dm_k = -sum_{j != k} K(r_kj) w_j . d_kj
//   dL/dv_b = sum_{i, j != i} m_j (w_i . d_ij) dK/dv_b   (table knot values)
// In the table's scaled units (d~ = scale d) the position term is
// g u + 2 G1 (d~ . u) d~ with no further factor; the mass and knot terms
// carry one factor 1/scale, applied at the end.
//
// Layout as the forward all-pairs kernel: stream-K units of (i-tile,
// j-sub-tile), i in registers (KI per thread; scalar FP32 for the table,
// whose per-lane knot gathers and histogram atomics do not pack; packed
// FP32x2 for Newton, k_backward_newton below), j positions,
// masses and weights bulk-copied to shared memory and converted to FP32
// offsets from the FP64 tile centre, TwoSum folding per sub-tile, FP64
// combine. The knot gradient goes through a per-CTA shared-memory histogram
// (pairs inside the cutoff only) and one FP64 atomic per knot per CTA.
#include "pg_device.cuh"

namespace pg {

constexpr int kKI = 4;                      // i per thread
constexpr float kFltMinNormal = 1.17549435e-38f;   // smallest normal FP32
constexpr int kBiB = kNT * kKI;

int backward_bi() { return kBiB; }

__device__ __forceinline__ void issue_bw(const double4 *jx, const double4 *jw, long long nj, int s,
                                         double4 *dx, double4 *dw, uint64_t *bar)
{
    long long j0 = (long long)s * kTJ;
    long long nv = nj - j0;
    if (nv > kTJ) nv = kTJ;
    unsigned bytes = (unsigned)(nv * sizeof(double4));
    mbar_arrive_tx(bar, 2 * bytes);
    bulk_g2s(dx, jx + j0, bytes, bar);
    bulk_g2s(dw, jw + j0, bytes, bar);
}

__host__ __device__ __forceinline__ long long sk_owner(long long u, long long grid, long long W)
{
    return ((u + 1) * grid - 1) / W;
}

// The table's backward (scalar FP32, kKI i per thread)
__global__ void __launch_bounds__(kNT) k_backward_table(BackwardArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    double4 *rawx = reinterpret_cast<double4 *>(smem);                 // [2][kTJ]
    double4 *raww = rawx + 2 * kTJ;                                     // [2][kTJ]
    float4 *cv = reinterpret_cast<float4 *>(raww + 2 * kTJ);            // [kTJ][2]
    uint64_t *bar = reinterpret_cast<uint64_t *>(cv + 2 * kTJ);
    int *flag = reinterpret_cast<int *>(bar + 2);
    float2 *tab = reinterpret_cast<float2 *>(bar + 4);
    float *hist = reinterpret_cast<float *>(tab + a.tab.n);

    const int tid = threadIdx.x;
    const long long G = gridDim.x, b = blockIdx.x;
    const long long u0 = b * a.W / G, u1 = (b + 1) * a.W / G;
    if (u0 >= u1) return;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    for (int k = tid; k < a.tab.n; k += kNT) {
        tab[k] = a.tab.AG1[k];
        hist[k] = 0.0f;
    }
    __syncthreads();

    unsigned pending = 0, phase = 0;
    if (tid == 0) {
        issue_bw(a.jx, a.jwv, a.n, (int)(u0 % a.njsub), rawx, raww, &bar[0]);
        pending = 1u;
        if (u0 + 1 < u1) {
            issue_bw(a.jx, a.jwv, a.n, (int)((u0 + 1) % a.njsub), rawx + kTJ, raww + kTJ, &bar[1]);
            pending |= 2u;
        }
    }

    const float c0 = 2.0f;
    const double sc = a.tab.scale;
    float xk[kKI], yk[kKI], zk[kKI], mk[kKI], wkx[kKI], wky[kKI], wkz[kKI];
    float gx[kKI], gy[kKI], gz[kKI], gm[kKI];
    float hx[kKI], hy[kKI], hz[kKI], hm[kKI], lx[kKI], ly[kKI], lz[kKI], lm[kKI];
    double cx = 0, cy = 0, cz = 0;
    long long cur = -1;
    bool failed = false;

    auto flush = [&](long long t) {
        long long slot = b - sk_owner(t * a.njsub, G, a.W);
        double4 *dst = a.part + ((size_t)t * a.smax_slots + (size_t)slot) * kBiB;
#pragma unroll
        for (int q = 0; q < kKI; ++q) {
            int li = q * kNT + tid;
            if (t * kBiB + li < a.n)
                dst[li] = make_double4((double)hx[q] + lx[q], (double)hy[q] + ly[q],
                                       (double)hz[q] + lz[q], (double)hm[q] + lm[q]);
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
#pragma unroll
            for (int q = 0; q < kKI; ++q) {
                long long i = t * kBiB + q * kNT + tid;
                if (i < a.n) {
                    double4 v = a.xi[i], w = a.wv[i];
                    xk[q] = (float)((v.x - cx) * sc);
                    yk[q] = (float)((v.y - cy) * sc);
                    zk[q] = (float)((v.z - cz) * sc);
                    mk[q] = (float)v.w;
                    wkx[q] = (float)w.x; wky[q] = (float)w.y; wkz[q] = (float)w.z;
                } else {
                    xk[q] = yk[q] = zk[q] = mk[q] = wkx[q] = wky[q] = wkz[q] = 0.0f;
                }
                hx[q] = hy[q] = hz[q] = hm[q] = lx[q] = ly[q] = lz[q] = lm[q] = 0.0f;
            }
        }
        if (tid == 0) {
            bool ok = mbar_wait(&bar[buf], (phase >> buf) & 1u, kWaitLimitNs);
            if (ok) pending &= ~(1u << buf);
            *flag = ok ? 1 : 0;
        }
        __syncthreads();
        if (*flag == 0) { failed = true; break; }
        phase ^= 1u << buf;
        {
            const long long j0 = (long long)s * kTJ;
            long long nv = a.n - j0;
            if (nv > kTJ) nv = kTJ;
            for (int e = tid; e < kTJ; e += kNT) {
                float4 p, w;
                if (e < nv) {
                    double4 v = rawx[buf * kTJ + e], ww = raww[buf * kTJ + e];
                    p = make_float4((float)((v.x - cx) * sc), (float)((v.y - cy) * sc),
                                    (float)((v.z - cz) * sc), (float)v.w);
                    w = make_float4((float)ww.x, (float)ww.y, (float)ww.z, 0.0f);
                } else {
                    p = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.0f);
                    w = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
                cv[2 * e] = p;
                cv[2 * e + 1] = w;
            }
        }
        __syncthreads();
        if (tid == 0 && u + 2 < u1) {
            fence_proxy_async();
            issue_bw(a.jx, a.jwv, a.n, (int)((u + 2) % a.njsub), rawx + buf * kTJ, raww + buf * kTJ,
                     &bar[buf]);
            pending |= 1u << buf;
        }
#pragma unroll
        for (int q = 0; q < kKI; ++q) gx[q] = gy[q] = gz[q] = gm[q] = 0.0f;
#pragma unroll 2
        for (int e = 0; e < kTJ; ++e) {
            const float4 p = cv[2 * e], w = cv[2 * e + 1];
#pragma unroll
            for (int q = 0; q < kKI; ++q) {
                const float dx = p.x - xk[q], dy = p.y - yk[q], dz = p.z - zk[q];
                float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, c0)));
                // u = m_k w_j - m_j w_k with separate roundings: exactly 0 for j = k
                const float ux = __fsub_rn(__fmul_rn(mk[q], w.x), __fmul_rn(p.w, wkx[q]));
                const float uy = __fsub_rn(__fmul_rn(mk[q], w.y), __fmul_rn(p.w, wky[q]));
                const float uz = __fsub_rn(__fmul_rn(mk[q], w.z), __fmul_rn(p.w, wkz[q]));
                const float du = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
                const float wd = fmaf(dx, w.x, fmaf(dy, w.y, dz * w.z));
                const float sv = fminf(r2, a.tab.s_max);
                const unsigned bits = __float_as_uint(sv);
                const unsigned idx = (bits >> a.tab.shift) - a.tab.base;
                const float2 ag = tab[idx];
                const float K = fmaf(sv, ag.y, ag.x);
                const float c2 = 2.0f * ag.y * du;
                if (sv < a.tab.s_max) {
                    // hat weights of the bin's two knots; the knot spacing
                    // is 2^(exponent of s_k - F)
                    const unsigned kb = bits & ~((1u << a.tab.shift) - 1u);
                    const float sk = __uint_as_float(kb);
                    const float ds = __uint_as_float((kb & 0x7f800000u) -
                                                     ((unsigned)(23 - a.tab.shift) << 23));
                    const float tt = (sv - sk) / ds;
                    const float pw = p.w * fmaf(dx, wkx[q], fmaf(dy, wky[q], dz * wkz[q]));
                    atomicAdd(&hist[idx], pw * (1.0f - tt));
                    atomicAdd(&hist[idx + 1], pw * tt);
                }
                gx[q] = fmaf(K, ux, fmaf(c2, dx, gx[q]));
                gy[q] = fmaf(K, uy, fmaf(c2, dy, gy[q]));
                gz[q] = fmaf(K, uz, fmaf(c2, dz, gz[q]));
                gm[q] = fmaf(-K, wd, gm[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < kKI; ++q) {
            float sx, ex;
            two_sum(hx[q], gx[q], sx, ex); hx[q] = sx; lx[q] += ex;
            two_sum(hy[q], gy[q], sx, ex); hy[q] = sx; ly[q] += ex;
            two_sum(hz[q], gz[q], sx, ex); hz[q] = sx; lz[q] += ex;
            two_sum(hm[q], gm[q], sx, ex); hm[q] = sx; lm[q] += ex;
        }
    }
    if (failed) {
        if (tid == 0) {
            report(a.status, kStatusTimeout, 3);
            for (int k = 0; k < 2; ++k)
                if (pending & (1u << k)) mbar_wait(&bar[k], (phase >> k) & 1u, kWaitLimitNs / 4);
        }
        return;
    }
    if (cur >= 0) flush(cur);
    if (a.dv) {
        __syncthreads();
        for (int k = tid; k < a.tab.n; k += kNT)
            if (hist[k] != 0.0f) atomicAdd(&a.dv[k], (double)hist[k]);
    }
}

// ---------------------------------------------------------------- Newton, packed
// The Newton backward in packed FP32x2, two i-pairs per thread. With
// d = x_j - x_k, q = (r^2 + eps^2)^(-1/2), K = q^3 and u = m_k w_j - m_j w_k,
// J(d) u = K u - 3 K q^2 (d . u) d, so
//   dL/dx_k = m_k A_k - w_k B_k - 3 C_k,   dL/dm_k = -G_k,
//   A = sum_j K w_j, B = sum_j m_j K, C = sum_j K q^2 (d . u) d,
//   G = sum_j K (d . w_j), with d . u = m_k (d . w_j) - m_j (d . w_k):
// 26 FP32-pipe lane operations per interaction (difference 3, r^2 3,
// d . w_j 3, d . w_k 3, d . u 2, q^2 and K 2, K q^2 (d . u) 2, A 3, B 1,
// C 3, G 1) and one MUFU rsqrt, against 33 for J(d) u formed from u. The
// own pair (j index = i's index) is left out by zeroing its q, so its large
// K never enters the FP32 sums; a coincident pair at eps = 0 likewise.
constexpr int kNPB = 2;                       // i-pairs per thread
static_assert(2 * kNPB == kKI, "the packed kernel keeps the tile of the scalar one");

// The pair loop over one staged sub-tile of kTJ j (jb its first index). The
// j records are in the i-particles' (tile) order, so the own pair can only
// sit in the sub-tiles that overlap the thread's i-tile: CHECK (those, and
// every sub-tile at eps = 0, where a coincident pair has r^2 = 0) zeroes q
// for j = the i's own index and for r^2 = 0; elsewhere r^2 >= eps^2 > 0 and
// no pair is the own one, so the tests are left out.
template <bool CHECK>
__device__ __forceinline__ void bw_newton_tile(const ulonglong2 *__restrict__ cv, int jb, u64 c0v,
                                               const u64 (&xi)[kNPB], const u64 (&yi)[kNPB],
                                               const u64 (&zi)[kNPB], const u64 (&mk)[kNPB],
                                               const u64 (&wkx)[kNPB], const u64 (&wky)[kNPB],
                                               const u64 (&wkz)[kNPB], const int (&self0)[kNPB],
                                               const int (&self1)[kNPB], u64 (&acc)[kNPB][8])
{
#pragma unroll 4
    for (int e = 0; e < kTJ; ++e) {
        const ulonglong2 xy = cv[4 * e], zm = cv[4 * e + 1], wxy = cv[4 * e + 2], wz0 = cv[4 * e + 3];
        const int j = jb + e;
#pragma unroll
        for (int p = 0; p < kNPB; ++p) {
            const u64 dx = f2sub(xy.x, xi[p]), dy = f2sub(xy.y, yi[p]), dz = f2sub(zm.x, zi[p]);
            u64 r2 = f2fma(dx, dx, c0v);
            r2 = f2fma(dy, dy, r2);
            r2 = f2fma(dz, dz, r2);
            u64 wd = f2mul(dx, wxy.x);
            wd = f2fma(dy, wxy.y, wd);
            wd = f2fma(dz, wz0.x, wd);
            u64 dk = f2mul(dx, wkx[p]);
            dk = f2fma(dy, wky[p], dk);
            dk = f2fma(dz, wkz[p], dk);
            const u64 du = f2fma(mk[p], wd, f2mul(zm.y, dk));   // m_k d.w_j - m_j d.w_k
            float ra, rb;
            up2(r2, ra, rb);
            float qa = rsq(ra), qb = rsq(rb);
            if (CHECK) {
                qa = (ra > 0.0f && j != self0[p]) ? qa : 0.0f;
                qb = (rb > 0.0f && j != self1[p]) ? qb : 0.0f;
            }
            const u64 q = pk2(qa, qb);
            const u64 q2 = f2mul(q, q);
            const u64 K = f2mul(q, q2);
            const u64 tt = f2mul(f2mul(K, q2), du);
            acc[p][0] = f2fma(K, wxy.x, acc[p][0]);
            acc[p][1] = f2fma(K, wxy.y, acc[p][1]);
            acc[p][2] = f2fma(K, wz0.x, acc[p][2]);
            acc[p][3] = f2fma(zm.y, K, acc[p][3]);    // -sum m_j K
            acc[p][4] = f2fma(tt, dx, acc[p][4]);
            acc[p][5] = f2fma(tt, dy, acc[p][5]);
            acc[p][6] = f2fma(tt, dz, acc[p][6]);
            acc[p][7] = f2fma(K, wd, acc[p][7]);
        }
    }
}

__global__ void __launch_bounds__(kNT, 2) k_backward_newton(BackwardArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    double4 *rawx = reinterpret_cast<double4 *>(smem);                 // [2][kTJ]
    double4 *raww = rawx + 2 * kTJ;                                     // [2][kTJ]
    u64 *cvt = reinterpret_cast<u64 *>(raww + 2 * kTJ);                 // [kTJ][8]
    uint64_t *bar = reinterpret_cast<uint64_t *>(cvt + 8 * kTJ);
    int *flag = reinterpret_cast<int *>(bar + 2);

    const int tid = threadIdx.x;
    const long long G = gridDim.x, b = blockIdx.x;
    const long long u0 = b * a.W / G, u1 = (b + 1) * a.W / G;
    if (u0 >= u1) return;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    unsigned pending = 0, phase = 0;
    if (tid == 0) {
        issue_bw(a.jx, a.jwv, a.n, (int)(u0 % a.njsub), rawx, raww, &bar[0]);
        pending = 1u;
        if (u0 + 1 < u1) {
            issue_bw(a.jx, a.jwv, a.n, (int)((u0 + 1) % a.njsub), rawx + kTJ, raww + kTJ, &bar[1]);
            pending |= 2u;
        }
    }

    const u64 c0v = pk2(a.eps2, a.eps2);
    u64 xi[kNPB], yi[kNPB], zi[kNPB], mk[kNPB], wkx[kNPB], wky[kNPB], wkz[kNPB];
    int self0[kNPB], self1[kNPB];
    // compensated sums (hi, lo) of A (3), B, C (3), G per i-pair
    u64 sh[kNPB][8], sl[kNPB][8];
    double cx = 0, cy = 0, cz = 0;
    long long cur = -1;
    bool failed = false;

    auto flush = [&](long long t) {
        long long slot = b - sk_owner(t * a.njsub, G, a.W);
        double4 *dst = a.part + ((size_t)t * a.smax_slots + (size_t)slot) * kBiB;
#pragma unroll
        for (int p = 0; p < kNPB; ++p) {
            float h[16], l[16];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                up2(sh[p][k], h[2 * k], h[2 * k + 1]);
                up2(sl[p][k], l[2 * k], l[2 * k + 1]);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int li = (2 * p + q) * kNT + tid;
                const long long i = t * kBiB + li;
                if (i >= a.n) continue;
                double v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = (double)h[2 * k + q] + (double)l[2 * k + q];
                const double m = a.xi[i].w;
                const double4 w = a.wv[i];
                // v[3] holds -B (the staged masses are negated)
                dst[li] = make_double4(m * v[0] + w.x * v[3] - 3.0 * v[4],
                                       m * v[1] + w.y * v[3] - 3.0 * v[5],
                                       m * v[2] + w.z * v[3] - 3.0 * v[6], -v[7]);
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
            const double4 c = a.ctr[t];
            cx = c.x; cy = c.y; cz = c.z;
#pragma unroll
            for (int p = 0; p < kNPB; ++p) {
                float fx[2], fy[2], fz[2], fm[2], gx[2], gy[2], gz[2];
                int sf[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const long long i = t * kBiB + (2 * p + q) * kNT + tid;
                    if (i < a.n) {
                        const double4 v = a.xi[i], w = a.wv[i];
                        fx[q] = (float)(v.x - cx);
                        fy[q] = (float)(v.y - cy);
                        fz[q] = (float)(v.z - cz);
                        fm[q] = (float)v.w;
                        gx[q] = (float)w.x; gy[q] = (float)w.y; gz[q] = (float)w.z;
                        sf[q] = (int)i;        // j records in the same order
                    } else {
                        fx[q] = fy[q] = fz[q] = fm[q] = gx[q] = gy[q] = gz[q] = 0.0f;
                        sf[q] = -1;
                    }
                }
                xi[p] = pk2(fx[0], fx[1]);
                yi[p] = pk2(fy[0], fy[1]);
                zi[p] = pk2(fz[0], fz[1]);
                mk[p] = pk2(fm[0], fm[1]);
                wkx[p] = pk2(gx[0], gx[1]);
                wky[p] = pk2(gy[0], gy[1]);
                wkz[p] = pk2(gz[0], gz[1]);
                self0[p] = sf[0];
                self1[p] = sf[1];
#pragma unroll
                for (int k = 0; k < 8; ++k) sh[p][k] = sl[p][k] = 0ull;
            }
        }
        if (tid == 0) {
            bool ok = mbar_wait(&bar[buf], (phase >> buf) & 1u, kWaitLimitNs);
            if (ok) pending &= ~(1u << buf);
            *flag = ok ? 1 : 0;
        }
        __syncthreads();
        if (*flag == 0) { failed = true; break; }
        phase ^= 1u << buf;
        const long long j0 = (long long)s * kTJ;
        {
            long long nv = a.n - j0;
            if (nv > kTJ) nv = kTJ;
            for (int e = tid; e < kTJ; e += kNT) {
                float x = 1.0e4f, y = 1.0e4f, z = 1.0e4f, mn = 0.0f, wx = 0.0f, wy = 0.0f, wz = 0.0f;
                if (e < nv) {
                    const double4 v = rawx[buf * kTJ + e], ww = raww[buf * kTJ + e];
                    x = (float)(v.x - cx);
                    y = (float)(v.y - cy);
                    z = (float)(v.z - cz);
                    mn = -(float)v.w;
                    wx = (float)ww.x; wy = (float)ww.y; wz = (float)ww.z;
                }
                cvt[8 * e + 0] = pk2(x, x);
                cvt[8 * e + 1] = pk2(y, y);
                cvt[8 * e + 2] = pk2(z, z);
                cvt[8 * e + 3] = pk2(mn, mn);
                cvt[8 * e + 4] = pk2(wx, wx);
                cvt[8 * e + 5] = pk2(wy, wy);
                cvt[8 * e + 6] = pk2(wz, wz);
                cvt[8 * e + 7] = 0ull;
            }
        }
        __syncthreads();
        if (tid == 0 && u + 2 < u1) {
            fence_proxy_async();
            issue_bw(a.jx, a.jwv, a.n, (int)((u + 2) % a.njsub), rawx + buf * kTJ, raww + buf * kTJ,
                     &bar[buf]);
            pending |= 1u << buf;
        }
        u64 acc[kNPB][8];
#pragma unroll
        for (int p = 0; p < kNPB; ++p)
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[p][k] = 0ull;
        const ulonglong2 *cv = reinterpret_cast<const ulonglong2 *>(cvt);
        const bool diag = j0 < (t + 1) * kBiB && j0 + kTJ > t * kBiB;
        if (diag || !(a.eps2 >= kFltMinNormal))
            bw_newton_tile<true>(cv, (int)j0, c0v, xi, yi, zi, mk, wkx, wky, wkz, self0, self1, acc);
        else
            bw_newton_tile<false>(cv, (int)j0, c0v, xi, yi, zi, mk, wkx, wky, wkz, self0, self1, acc);
#pragma unroll
        for (int p = 0; p < kNPB; ++p)
#pragma unroll
            for (int k = 0; k < 8; ++k) fold2(sh[p][k], sl[p][k], acc[p][k]);
    }
    if (failed) {
        if (tid == 0) {
            report(a.status, kStatusTimeout, 3);
            for (int k = 0; k < 2; ++k)
                if (pending & (1u << k)) mbar_wait(&bar[k], (phase >> k) & 1u, kWaitLimitNs / 4);
        }
        return;
    }
    if (cur >= 0) flush(cur);
}

size_t backward_newton_smem() { return 4 * kTJ * sizeof(double4) + 8 * kTJ * sizeof(u64) + 4 * sizeof(uint64_t); }

size_t backward_smem(bool table, int ntab)
{
    size_t s = 4 * kTJ * sizeof(double4) + 2 * kTJ * sizeof(float4) + 4 * sizeof(uint64_t);
    if (table) s += (size_t)ntab * (sizeof(float2) + sizeof(float));
    return s;
}

static cudaError_t configure_b()
{
    static bool done[kMaxDevices] = {};
    return once_per_device(done, [] {
        return cudaFuncSetAttribute(k_backward_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)backward_smem(true, 1 << 13));
    });
}

static cudaError_t configure_bn()
{
    static bool done[kMaxDevices] = {};
    return once_per_device(done, [] {
        return cudaFuncSetAttribute(k_backward_newton, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)backward_newton_smem());
    });
}

// Newton: the packed kernel; table: the scalar one with the knot histogram
int backward_max_blocks_per_sm(bool table, int ntab)
{
    cudaError_t e = table ? configure_b() : configure_bn();
    if (e != cudaSuccess) return 1;
    int nb = 0;
    e = table ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_backward_table, kNT,
                                                             backward_smem(true, ntab))
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_backward_newton, kNT,
                                                             backward_newton_smem());
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

cudaError_t launch_backward(const BackwardArgs &a, int grid, bool table, size_t smem,
                            cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    cudaError_t e = table ? configure_b() : configure_bn();
    if (e != cudaSuccess) return e;
    if (table) k_backward_table<<<grid, kNT, smem, st>>>(a);
    else k_backward_newton<<<grid, kNT, backward_newton_smem(), st>>>(a);
    return cudaGetLastError();
}

// gather loss weights (FP64 [n][3]) into (a) record order and (b) tile order
__global__ void k_pack_w(const double *__restrict__ w, const unsigned *__restrict__ perm, long long n,
                         double4 *__restrict__ wj, double4 *__restrict__ wt)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    wj[p] = make_double4(w[3 * p], w[3 * p + 1], w[3 * p + 2], 0.0);
    long long k = perm ? (long long)perm[p] : p;
    wt[p] = make_double4(w[3 * k], w[3 * k + 1], w[3 * k + 2], 0.0);
}

cudaError_t launch_pack_w(const double *w, const unsigned *perm, long long n, double4 *wj,
                          double4 *wt, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_pack_w<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, perm, n, wj, wt);
    return cudaGetLastError();
}

__global__ void k_bw_combine(const double4 *__restrict__ part, const unsigned *__restrict__ perm,
                             long long n, int njsub, int slots, int grid, long long W, double mscale,
                             double *__restrict__ dx, double *__restrict__ dm)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    long long t = p / kBiB;
    int li = (int)(p % kBiB);
    double gx = 0, gy = 0, gz = 0, gm = 0;
    if (njsub > 0) {
        long long bf = sk_owner(t * njsub, grid, W), bl = sk_owner((t + 1) * njsub - 1, grid, W);
        for (long long s = 0; s <= bl - bf; ++s) {
            double4 v = part[((size_t)t * slots + (size_t)s) * kBiB + li];
            gx += v.x; gy += v.y; gz += v.z; gm += v.w;
        }
    }
    long long k = perm ? (long long)perm[p] : p;
    dx[3 * k] = gx;
    dx[3 * k + 1] = gy;
    dx[3 * k + 2] = gz;
    dm[k] = gm * mscale;
}

cudaError_t launch_backward_combine(const double4 *part, const unsigned *perm, long long n, int njsub,
                                    int slots, int grid, long long W, double mscale, double *dx,
                                    double *dm, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_bw_combine<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, perm, n, njsub, slots,
                                                              grid > 0 ? grid : 1, W > 0 ? W : 1,
                                                              mscale, dx, dm);
    return cudaGetLastError();
}

__global__ void k_dv_out(const double *__restrict__ acc, int n, double scale, float *__restrict__ dv)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dv[k] = (float)(acc[k] * scale);
}

cudaError_t launch_dv_out(const double *acc, int n, double scale, float *dv, cudaStream_t st)
{
    k_dv_out<<<(n + 255) / 256, 256, 0, st>>>(acc, n, scale, dv);
    return cudaGetLastError();
}

}  // namespace pg
