// pg_small.cu -- the all-pairs Newton force loop for small i-sets in one
// launch.
//
// For a few thousand particles (the 4096-body Plummer workload of Section
// 4.1's accuracy runs) the pair work is a few microseconds of the GPU, so
// separate launches for tile preparation, the force loop and the combine
// cost more than the work. Here one kernel does all of it:
//
//  * the i-particles (caller order, 256 per tile: 128 threads, one packed
//    pair of i each) and the j records are cut into ntiles x nchunk blocks,
//    nchunk chosen so that the grid fills the SMs;
//  * positions arrive as double-float records (FP32 hi, FP32 lo = x - hi,
//    packed once when they are set), and a pair's difference is formed as
//    (hi_j - hi_i) + (lo_j - lo_i): FP32 precision relative to |d| itself,
//    with no FP64 instruction in the kernel's loops (GB300 issues FP64 at
//    about two operations per SM-clock, so per-block FP64 conversions cost
//    more than the pair loop at this size);
//  * the pair loop of Eq. (1) (difference, r^2 + eps^2, MUFU rsqrt, m/r,
//    m/r^3, accumulate; Section 3.3's steps) runs in packed FP32x2, folding
//    each 256-j sub-tile into a compensated (hi, lo) pair;
//  * each block writes its (hi, lo) partial sums and takes a ticket of its
//    tile; the block that takes the last ticket adds the tile's partials in
//    chunk order with TwoSum (so the sum does not depend on which block
//    finished first), removes the own pair's potential in self mode, writes
//    the FP64 outputs and resets the ticket for the next call.
//
// Nothing in it waits on another block: the last block is simply the one
// whose atomic increment returns nchunk - 1, after every block has made its
// partials visible with a fence.
#include "pg_device.cuh"

namespace pg {

namespace {

constexpr int kSmallNT = 128;              // threads: one i-pair each
constexpr int kSmallBi = 2 * kSmallNT;     // i per tile
constexpr int kSmallSub = 256;             // j per compensated sub-tile

// the own pair's potential as the loop added it (d = 0 exactly): -m rsqrt(eps^2),
// nothing at eps = 0
__device__ __forceinline__ double small_self_pot(const SmallArgs &a, long long k, float e2)
{
    const float mk = a.jhl[2 * (k + a.self_off)].w;
    return e2 > 0.0f ? -(double)__fmul_rn(mk, rsq(e2)) : 0.0;
}

template <bool EXT>
__global__ void __launch_bounds__(kSmallNT) k_small(SmallArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ulonglong2 *cv = reinterpret_cast<ulonglong2 *>(smem);    // [jchunk][4]
    __shared__ int last;

    const int tid = threadIdx.x;
    const long long tile = blockIdx.x / a.nchunk;
    const int chunk = (int)(blockIdx.x - tile * a.nchunk);
    const long long i0 = tile * kSmallBi;

    // this thread's i-pair and each i's eps^2
    float hx[2], hy[2], hz[2], lx[2], ly[2], lz[2], fe[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const long long i = i0 + q * kSmallNT + tid;
        float4 h = make_float4(0.0f, 0.0f, 0.0f, 0.0f), l = h;
        fe[q] = a.eps2;
        if (i < a.ni) {
            h = a.ihl[2 * i];
            l = a.ihl[2 * i + 1];
            if (EXT && a.epsi) fe[q] = (float)a.xi[i].w;
        }
        hx[q] = h.x; hy[q] = h.y; hz[q] = h.z;
        lx[q] = l.x; ly[q] = l.y; lz[q] = l.z;
    }
    const u64 xi = pk2(hx[0], hx[1]), yi = pk2(hy[0], hy[1]), zi = pk2(hz[0], hz[1]);
    const u64 exi = pk2(lx[0], lx[1]), eyi = pk2(ly[0], ly[1]), ezi = pk2(lz[0], lz[1]);
    const u64 r0 = pk2(fe[0], fe[1]);

    // stage the chunk's j records: {hi_x, hi_y}, {hi_z, m}, {lo_x, lo_y},
    // {lo_z, 0}, each value in both lanes (padding: zero mass far away, an
    // exact zero term)
    const long long jb = (long long)chunk * a.jchunk;
    long long je = jb + a.jchunk;
    if (je > a.nj) je = a.nj;
    const int nv = (int)(je - jb);
    const int nvp = (nv + 15) & ~15;             // the loop's unroll
    for (int e = tid; e < nvp; e += kSmallNT) {
        float4 h = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.0f), l = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (e < nv) {
            h = a.jhl[2 * (jb + e)];
            l = a.jhl[2 * (jb + e) + 1];
        }
        cv[4 * e + 0] = make_ulonglong2(pk2(h.x, h.x), pk2(h.y, h.y));
        cv[4 * e + 1] = make_ulonglong2(pk2(h.z, h.z), pk2(h.w, h.w));
        cv[4 * e + 2] = make_ulonglong2(pk2(l.x, l.x), pk2(l.y, l.y));
        cv[4 * e + 3] = make_ulonglong2(pk2(l.z, l.z), 0ull);
    }

    __syncthreads();

    // the pair loop, compensated per sub-tile
    u64 sh[4] = {0, 0, 0, 0}, sl[4] = {0, 0, 0, 0};
    for (int s0 = 0; s0 < nvp; s0 += kSmallSub) {
        const int s1 = min(nvp, s0 + kSmallSub);
        u64 ax = 0, ay = 0, az = 0, ph = 0;
#pragma unroll 16
        for (int e = s0; e < s1; ++e) {
            const ulonglong2 hxy = cv[4 * e], hzm = cv[4 * e + 1], lxy = cv[4 * e + 2], lz0 = cv[4 * e + 3];
            const u64 dx = f2add(f2sub(hxy.x, xi), f2sub(lxy.x, exi));
            const u64 dy = f2add(f2sub(hxy.y, yi), f2sub(lxy.y, eyi));
            const u64 dz = f2add(f2sub(hzm.x, zi), f2sub(lz0.x, ezi));
            u64 r2 = f2fma(dx, dx, r0);
            r2 = f2fma(dy, dy, r2);
            r2 = f2fma(dz, dz, r2);
            float ra, rb;
            up2(r2, ra, rb);
            float qa = rsq(ra), qb = rsq(rb);
            if (EXT) {     // eps = 0: a coincident pair contributes nothing
                qa = ra > 0.0f ? qa : 0.0f;
                qb = rb > 0.0f ? qb : 0.0f;
            }
            const u64 q = pk2(qa, qb);
            const u64 mq = f2mul(hzm.y, q);
            const u64 mq3 = f2mul(mq, f2mul(q, q));
            ph = f2sub(ph, mq);
            ax = f2fma(mq3, dx, ax);
            ay = f2fma(mq3, dy, ay);
            az = f2fma(mq3, dz, az);
        }
        fold2(sh[0], sl[0], ax);
        fold2(sh[1], sl[1], ay);
        fold2(sh[2], sl[2], az);
        fold2(sh[3], sl[3], ph);
    }

    // this block's (hi, lo) partials, then a ticket of the tile
    {
        float h[8], l[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            up2(sh[k], h[2 * k], h[2 * k + 1]);
            up2(sl[k], l[2 * k], l[2 * k + 1]);
        }
        float4 *dst = a.part + 2 * (((size_t)tile * a.nchunk + chunk) * kSmallBi);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int li = q * kSmallNT + tid;
            dst[2 * li] = make_float4(h[q], h[2 + q], h[4 + q], h[6 + q]);
            dst[2 * li + 1] = make_float4(l[q], l[2 + q], l[4 + q], l[6 + q]);
        }
    }
    __threadfence();           // this thread's partials visible before the ticket
    __syncthreads();
    if (tid == 0) last = atomicAdd(a.ticket + tile, 1u) == (unsigned)(a.nchunk - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();

    // the last block of the tile: the partials in chunk order (TwoSum), FP64 out
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const long long i = i0 + q * kSmallNT + tid;
        if (i >= a.ni) continue;
        float H[4] = {0, 0, 0, 0}, L[4] = {0, 0, 0, 0};
        const float4 *src = a.part + 2 * ((size_t)tile * a.nchunk * kSmallBi + q * kSmallNT + tid);
        // eight chunks' partials in flight at a time (L2 reads: other blocks
        // wrote them), added in chunk order
        constexpr int kBatch = 8;
        for (int c0 = 0; c0 < a.nchunk; c0 += kBatch) {
            float4 vh[kBatch], vl[kBatch];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const int c = c0 + b < a.nchunk ? c0 + b : c0;
                vh[b] = __ldcg(src + 2 * (size_t)c * kSmallBi);
                vl[b] = __ldcg(src + 2 * (size_t)c * kSmallBi + 1);
            }
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                if (c0 + b >= a.nchunk) break;
                const float ph[4] = {vh[b].x, vh[b].y, vh[b].z, vh[b].w};
                const float pl[4] = {vl[b].x, vl[b].y, vl[b].z, vl[b].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float s, e;
                    two_sum(H[k], ph[k], s, e);
                    H[k] = s;
                    L[k] = __fadd_rn(L[k], __fadd_rn(pl[k], e));
                }
            }
        }
        double ph = (double)H[3] + (double)L[3];
        if (a.self) ph -= small_self_pot(a, i, fe[q]);
        a.acc[3 * i] = (double)H[0] + (double)L[0];
        a.acc[3 * i + 1] = (double)H[1] + (double)L[1];
        a.acc[3 * i + 2] = (double)H[2] + (double)L[2];
        if (a.pot) a.pot[i] = ph;
    }
    if (tid == 0) a.ticket[tile] = 0u;   // ready for the next call
}

template <bool EXT>
cudaError_t configure_small()
{
    static bool done[kMaxDevices] = {};
    return once_per_device(done, [] {
        return cudaFuncSetAttribute(k_small<EXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)small_smem(kSmallMaxChunk));
    });
}

template <bool EXT>
cudaError_t launch_small_one(const SmallArgs &a, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = configure_small<EXT>();
    if (e != cudaSuccess) return e;
    k_small<EXT><<<grid, kSmallNT, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

int small_bi() { return kSmallBi; }

// Shared memory per block: the staged chunk, but at least a quarter of an
// SM's shared memory less the per-block reserve, so that at most four blocks
// share an SM. The grid is about four blocks per SM and fits in one wave; left
// to the register limit (nine blocks), the block scheduler stacked up to 2.3
// times the average work on some SMs (measured: busiest SM 75k cycles
// against 33k on average for the 4096-body call).
constexpr size_t kSmallMinSmem = 50 * 1024;

size_t small_smem(int jchunk)
{
    const int nvp = (jchunk + 15) & ~15;
    const size_t need = (size_t)nvp * 8 * sizeof(u64);
    return need > kSmallMinSmem ? need : kSmallMinSmem;
}

cudaError_t launch_small(const SmallArgs &a, bool ext, cudaStream_t st)
{
    const long long ntiles = (a.ni + kSmallBi - 1) / kSmallBi;
    const long long grid = ntiles * a.nchunk;
    if (grid <= 0) return cudaSuccess;
    if (a.jchunk < 1 || a.jchunk > kSmallMaxChunk || grid >= (1LL << 31)) return cudaErrorInvalidValue;
    const size_t smem = small_smem(a.jchunk);
    return ext ? launch_small_one<true>(a, (int)grid, smem, st) : launch_small_one<false>(a, (int)grid, smem, st);
}

}  // namespace pg
