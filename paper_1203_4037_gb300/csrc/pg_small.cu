// pg_small.cu -- the all-pairs Newton force loop for small i-sets in one
// launch.
//
// For a few thousand particles (the 4096-body Plummer workload of Section
// 4.1's accuracy runs) the pair work is a few microseconds of the GPU, so
// separate launches for tile preparation, the force loop and the combine
// cost more than the work. Here one kernel does all of it:
//
//  * the i-particles (caller order, 256 per tile) and the j records are cut
//    into ntiles x nchunk blocks, about two per SM; each of a block's four
//    warps holds all 256 i of its tile (four packed i-pairs per lane, the
//    independent work the pair loop needs to hide its latencies) and takes
//    every fourth j of the block's chunk; the warps' sums are added in
//    shared memory in warp order;
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

constexpr int kSmallNT = 128;              // threads: four warps
constexpr int kSmallWarps = kSmallNT / 32;
constexpr int kSmallNP = 4;                // i-pairs per lane
constexpr int kSmallBi = 64 * kSmallNP;    // i per tile: every warp holds all of them
constexpr int kSmallBlocksPerSM = 3;       // resident blocks per SM (the register limit)
// blocks per cluster (chunks of one tile): 4 pack three blocks on every
// SM of GB300 (measured: with 8, 48 clusters fit at once, 384 blocks, and
// the SMs holding three of them set the time)
constexpr int kSmallCluster = 4;
constexpr int kSliceI = kSmallBi / kSmallCluster;          // i reduced by each block of a cluster
static_assert(kSmallBi % kSmallCluster == 0 && (kSliceI * 4) % kSmallNT == 0,
              "a block reduces its cluster's slice, (i, component) pairs spread over its threads");

// the own pair's potential as the loop added it (d = 0 exactly): -m rsqrt(eps^2),
// nothing at eps = 0
__device__ __forceinline__ double small_self_pot(const SmallArgs &a, long long k, float e2)
{
    const float mk = a.jhl[2 * (k + a.self_off)].w;
    return e2 > 0.0f ? -(double)__fmul_rn(mk, rsq(e2)) : 0.0;
}

// the cluster (distributed shared memory) primitives
__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// every thread of every block of the cluster arrives; shared-memory writes
// before it are visible to the cluster's blocks after it
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the float at this block's shared address p, in the shared memory of the
// cluster's block `rank`
__device__ __forceinline__ float ld_cluster(const float *p, unsigned rank)
{
    const unsigned a = smem_u32(p);
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(r) : "memory");
    return v;
}

// Lane l of every warp holds the tile's i-particles i0 + 64 p + l and
// i0 + 64 p + 32 + l (p < kSmallNP) as packed pairs; warp w takes every
// kSmallWarps-th staged j from w on. The kSmallCluster blocks of a cluster
// hold consecutive chunks of one tile (nchunk is a multiple of it).
template <bool EXT>
__global__ void __launch_bounds__(kSmallNT, kSmallBlocksPerSM) k_small(SmallArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ulonglong2 *cv = reinterpret_cast<ulonglong2 *>(smem);    // [jchunk][4]
    float *red = reinterpret_cast<float *>(smem);             // reuse: [warps][4][kSmallBi]
    __shared__ float bp[8 * kSmallBi];                        // the block's sums: hi [4][Bi], lo [4][Bi]
    __shared__ int last;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long tile = blockIdx.x / a.nchunk;
    const int chunk = (int)(blockIdx.x - tile * a.nchunk);
    const long long i0 = tile * kSmallBi;
    const int ncl = a.nchunk / kSmallCluster;                 // clusters per tile
    const int cl = chunk / kSmallCluster;                     // this block's cluster in the tile

    // this lane's i-pairs: double-float positions, each i's eps^2
    u64 xi[kSmallNP], yi[kSmallNP], zi[kSmallNP], exi[kSmallNP], eyi[kSmallNP], ezi[kSmallNP];
    u64 r0[kSmallNP];
#pragma unroll
    for (int p = 0; p < kSmallNP; ++p) {
        float hx[2], hy[2], hz[2], lx[2], ly[2], lz[2], fe[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const long long i = i0 + 64 * p + 32 * q + lane;
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
        xi[p] = pk2(hx[0], hx[1]); yi[p] = pk2(hy[0], hy[1]); zi[p] = pk2(hz[0], hz[1]);
        exi[p] = pk2(lx[0], lx[1]); eyi[p] = pk2(ly[0], ly[1]); ezi[p] = pk2(lz[0], lz[1]);
        r0[p] = pk2(fe[0], fe[1]);
    }

    // stage the chunk's j records: {hi_x, hi_y}, {hi_z, m}, {lo_x, lo_y},
    // {lo_z, 0}, each value in both lanes (padding, and chunks past the last
    // j: zero mass far away, an exact zero term)
    const long long jb = (long long)chunk * a.jchunk;
    long long je = jb + a.jchunk;
    if (je > a.nj) je = a.nj;
    const int nv = je > jb ? (int)(je - jb) : 0;
    const int nvp = (nv + 4 * kSmallWarps - 1) & ~(4 * kSmallWarps - 1);   // the warps' unroll
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

    // the pair loop: at most kSmallMaxChunk / kSmallWarps = 256 j per warp,
    // one FP32 sum each
    u64 ax[kSmallNP], ay[kSmallNP], az[kSmallNP], ph[kSmallNP];
#pragma unroll
    for (int p = 0; p < kSmallNP; ++p) ax[p] = ay[p] = az[p] = ph[p] = 0ull;
#pragma unroll 4
    for (int e = warp; e < nvp; e += kSmallWarps) {
        const ulonglong2 hxy = cv[4 * e], hzm = cv[4 * e + 1], lxy = cv[4 * e + 2], lz0 = cv[4 * e + 3];
#pragma unroll
        for (int p = 0; p < kSmallNP; ++p) {
            const u64 dx = f2add(f2sub(hxy.x, xi[p]), f2sub(lxy.x, exi[p]));
            const u64 dy = f2add(f2sub(hxy.y, yi[p]), f2sub(lxy.y, eyi[p]));
            const u64 dz = f2add(f2sub(hzm.x, zi[p]), f2sub(lz0.x, ezi[p]));
            u64 r2 = f2fma(dx, dx, r0[p]);
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
            ph[p] = f2sub(ph[p], mq);
            ax[p] = f2fma(mq3, dx, ax[p]);
            ay[p] = f2fma(mq3, dy, ay[p]);
            az[p] = f2fma(mq3, dz, az[p]);
        }
    }
    __syncthreads();           // every warp done with the staged records

    // the warps' sums: red[w][k][i], k = x, y, z, phi
#pragma unroll
    for (int p = 0; p < kSmallNP; ++p) {
        float v[8];
        up2(ax[p], v[0], v[1]); up2(ay[p], v[2], v[3]); up2(az[p], v[4], v[5]); up2(ph[p], v[6], v[7]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int q = 0; q < 2; ++q)
                red[(warp * 4 + k) * kSmallBi + 64 * p + 32 * q + lane] = v[2 * k + q];
    }
    __syncthreads();
    // the block's sums, warps in order with TwoSum: bp[k][i] hi, bp[4 + k][i] lo
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int li = q * kSmallNT + tid;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float H = 0.0f, L = 0.0f;
#pragma unroll
            for (int w = 0; w < kSmallWarps; ++w) {
                float s2, e2;
                two_sum(H, red[(w * 4 + k) * kSmallBi + li], s2, e2);
                H = s2;
                L = __fadd_rn(L, e2);
            }
            bp[k * kSmallBi + li] = H;
            bp[(4 + k) * kSmallBi + li] = L;
        }
    }

    // the cluster's sum: block rank r adds the tile's i-slice
    // [r kSliceI, (r + 1) kSliceI) over the cluster's blocks in rank order
    // (distributed shared memory, (i, component) pairs spread over the
    // threads) and stores it as this cluster's partial of those i
    cluster_sync();
    {
        const unsigned r = cluster_rank();
        float *dst = a.part + 8 * ((size_t)(tile * ncl + cl) * kSmallBi);
#pragma unroll
        for (int t = tid; t < 4 * kSliceI; t += kSmallNT) {
            const int li = (int)r * kSliceI + (t % kSliceI);
            const int k = t / kSliceI;
            float H = 0.0f, L = 0.0f;
#pragma unroll
            for (unsigned b = 0; b < (unsigned)kSmallCluster; ++b) {
                const float h = ld_cluster(bp + k * kSmallBi + li, b);
                const float l = ld_cluster(bp + (4 + k) * kSmallBi + li, b);
                float s2, e2;
                two_sum(H, h, s2, e2);
                H = s2;
                L = __fadd_rn(L, __fadd_rn(l, e2));
            }
            dst[k * kSmallBi + li] = H;
            dst[(4 + k) * kSmallBi + li] = L;
        }
    }
    cluster_sync();            // no block leaves while another reads its shared memory

    __threadfence();           // this thread's partial visible before the ticket
    __syncthreads();
    if (tid == 0) last = atomicAdd(a.ticket + tile, 1u) == (unsigned)(a.nchunk - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();

    // the last block of the tile: the clusters' partials in order (TwoSum), FP64 out
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int li = q * kSmallNT + tid;
        const long long i = i0 + li;
        if (i >= a.ni) continue;
        float H[4] = {0, 0, 0, 0}, L[4] = {0, 0, 0, 0};
        for (int c = 0; c < ncl; ++c) {
            const float *src = a.part + 8 * ((size_t)(tile * ncl + c) * kSmallBi);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float s2, e2;
                two_sum(H[k], __ldcg(src + k * kSmallBi + li), s2, e2);
                H[k] = s2;
                L[k] = __fadd_rn(L[k], __fadd_rn(__ldcg(src + (4 + k) * kSmallBi + li), e2));
            }
        }
        const float e2i = EXT && a.epsi ? (float)a.xi[i].w : a.eps2;
        double phv = (double)H[3] + (double)L[3];
        if (a.self) phv -= small_self_pot(a, i, e2i);
        a.acc[3 * i] = (double)H[0] + (double)L[0];
        a.acc[3 * i + 1] = (double)H[1] + (double)L[1];
        a.acc[3 * i + 2] = (double)H[2] + (double)L[2];
        if (a.pot) a.pot[i] = phv;
    }
    if (tid == 0) a.ticket[tile] = 0u;   // ready for the next call
}

template <bool EXT>
cudaError_t configure_small()
{
    static bool done[kMaxDevices] = {};
    return once_per_device(done, [] {
        cudaError_t e = cudaFuncSetAttribute(k_small<EXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)small_smem(kSmallMaxChunk));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_small<EXT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        return e;
    });
}

template <bool EXT>
cudaError_t launch_small_one(const SmallArgs &a, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = configure_small<EXT>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kSmallNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kSmallCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_small<EXT>, a);
}

// clusters of kSmallCluster blocks resident at once on this device
template <bool EXT>
int clusters_one(size_t smem)
{
    if (configure_small<EXT>() != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kSmallCluster);
    cfg.blockDim = dim3(kSmallNT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kSmallCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_small<EXT>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace

int small_bi() { return kSmallBi; }
int small_cluster() { return kSmallCluster; }
int small_max_clusters(bool ext)
{
    const size_t smem = small_smem(kSmallMaxChunk);
    return ext ? clusters_one<true>(smem) : clusters_one<false>(smem);
}

// Shared memory per block: the staged chunk and the warps' sums after it,
// but at least kSmallMinSmem so that at most small_blocks_per_sm() blocks
// share an SM. The grid is that many blocks per SM, in one wave; left to the
// register limit the block scheduler placed one to three blocks on an SM
// (measured: busiest SM 57k cycles against 31k on average for the 4096-body
// call), and the busiest SM sets the time.
constexpr size_t kSmallMinSmem = 60 * 1024;          // 4 x (60 KB + reserve) > 228 KB

int small_blocks_per_sm() { return kSmallBlocksPerSM; }

size_t small_smem(int jchunk)
{
    const int nvp = (jchunk + 4 * kSmallWarps - 1) & ~(4 * kSmallWarps - 1);
    size_t s = (size_t)nvp * 8 * sizeof(u64);
    const size_t red = (size_t)kSmallWarps * 4 * kSmallBi * sizeof(float);
    if (s < red) s = red;
    return s > kSmallMinSmem ? s : kSmallMinSmem;
}

cudaError_t launch_small(const SmallArgs &a, bool ext, cudaStream_t st)
{
    const long long ntiles = (a.ni + kSmallBi - 1) / kSmallBi;
    const long long grid = ntiles * a.nchunk;
    if (grid <= 0) return cudaSuccess;
    if (a.jchunk < 1 || a.jchunk > kSmallMaxChunk || grid >= (1LL << 31) || a.nchunk % kSmallCluster != 0)
        return cudaErrorInvalidValue;
    const size_t smem = small_smem(a.jchunk);
    return ext ? launch_small_one<true>(a, (int)grid, smem, st) : launch_small_one<false>(a, (int)grid, smem, st);
}

}  // namespace pg
