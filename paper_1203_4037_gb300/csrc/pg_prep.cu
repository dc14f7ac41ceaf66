// pg_prep.cu -- data staging ahead of the force kernels:
//  * packing of FP64 positions/masses into 32-byte records (the paper's
//    Jpdata/Ipdata packing, Section 3.1, kept in FP64 for the differencing
//    step);
//  * spatial ordering of the i-particles along a Morton curve so that each
//    i-tile is compact and its FP32 offsets from the FP64 tile centre are small;
//  * a stable LSD radix sort (8-bit digits, warp-level ranking) used for that
//    ordering and for the cell list;
//  * gather into tile order with per-tile FP64 centres.
#include "pg_device.cuh"

namespace pg {

// ---------------------------------------------------------------- packing
__global__ void k_pack_j(const double *__restrict__ x, const double *__restrict__ m,
                         double4 *__restrict__ out, long long n, float4 *__restrict__ hl)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 v = make_double4(x[3 * i], x[3 * i + 1], x[3 * i + 2], m ? m[i] : 0.0);
    out[i] = v;
    if (hl) {   // double-float pairs: hi = fp32(x), lo = fp32(x - hi)
        const float hx = (float)v.x, hy = (float)v.y, hz = (float)v.z;
        hl[2 * i] = make_float4(hx, hy, hz, (float)v.w);
        hl[2 * i + 1] = make_float4((float)(v.x - (double)hx), (float)(v.y - (double)hy),
                                    (float)(v.z - (double)hz), (float)v.w);
    }
}

// i records' fourth value: eps_k^2 with per-i softening (eps == nullptr: 0)
__global__ void k_set_w(double4 *__restrict__ x, const double *__restrict__ eps, long long n)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double e = eps ? eps[i] : 0.0;
    x[i].w = e * e;
}

cudaError_t launch_set_w(double4 *x, const double *eps, long long n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_set_w<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, eps, n);
    return cudaGetLastError();
}

cudaError_t launch_pack_j(const double *x, const double *m, double4 *jrec, long long n,
                          cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_pack_j<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, m, jrec, n, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_pack_i(const double *x, double4 *xi, long long n, cudaStream_t st, float4 *ihl)
{
    if (n <= 0) return cudaSuccess;
    k_pack_j<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, nullptr, xi, n, ihl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- bbox
// order-preserving map of a double onto an unsigned 64-bit integer
__device__ __forceinline__ unsigned long long ord_d(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord_d(unsigned long long u)
{
    unsigned long long b = (u & 0x8000000000000000ull) ? (u & 0x7fffffffffffffffull) : ~u;
    return __longlong_as_double((long long)b);
}

__global__ void k_bbox_init(unsigned long long *bb)
{
    if (threadIdx.x < 3) bb[threadIdx.x] = ~0ull;          // min
    else if (threadIdx.x < 6) bb[threadIdx.x] = 0ull;      // max
}

__global__ void k_bbox(const double4 *__restrict__ x, long long n, unsigned long long *bb)
{
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0, 0, 0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double4 p = x[i];
        unsigned long long o[3] = {ord_d(p.x), ord_d(p.y), ord_d(p.z)};
        for (int c = 0; c < 3; ++c) {
            lo[c] = o[c] < lo[c] ? o[c] : lo[c];
            hi[c] = o[c] > hi[c] ? o[c] : hi[c];
        }
    }
    for (int c = 0; c < 3; ++c) {
        for (int off = 16; off; off >>= 1) {
            unsigned long long a = __shfl_xor_sync(0xffffffffu, lo[c], off);
            unsigned long long b = __shfl_xor_sync(0xffffffffu, hi[c], off);
            lo[c] = a < lo[c] ? a : lo[c];
            hi[c] = b > hi[c] ? b : hi[c];
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int c = 0; c < 3; ++c) {
            atomicMin(bb + c, lo[c]);
            atomicMax(bb + 3 + c, hi[c]);
        }
    }
}

// spread the low 10 bits of v so that two zero bits separate each
__device__ __forceinline__ unsigned spread10(unsigned v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_morton(const double4 *__restrict__ x, long long n,
                         const unsigned long long *__restrict__ bb,
                         unsigned *__restrict__ keys, unsigned *__restrict__ vals)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo0 = unord_d(bb[0]), lo1 = unord_d(bb[1]), lo2 = unord_d(bb[2]);
    double s0 = unord_d(bb[3]) - lo0, s1 = unord_d(bb[4]) - lo1, s2 = unord_d(bb[5]) - lo2;
    double span = fmax(fmax(s0, s1), fmax(s2, 1e-300));
    double q = 1023.0 / span;
    double4 p = x[i];
    unsigned a = (unsigned)fmin(fmax((p.x - lo0) * q, 0.0), 1023.0);
    unsigned b = (unsigned)fmin(fmax((p.y - lo1) * q, 0.0), 1023.0);
    unsigned c = (unsigned)fmin(fmax((p.z - lo2) * q, 0.0), 1023.0);
    keys[i] = (spread10(a) << 2) | (spread10(b) << 1) | spread10(c);
    vals[i] = (unsigned)i;
}

// ---------------------------------------------------------------- radix sort
// Each warp owns a chunk of kChunk consecutive elements; a pass histograms
// the chunk's 8-bit digits, a scan turns the digit-major histogram into
// global offsets, and the scatter re-reads the chunk in order and ranks
// equal digits by lane order, which keeps the sort stable. A lane loads
// kBatch rounds' elements before it uses them, so a warp has kBatch loads
// in flight instead of one (about seven warps per SM hold the 2^20-key
// sorts' chunks; one load at a time left each pass latency-bound).
constexpr int kRounds = 32;
constexpr int kChunk = 32 * kRounds;
constexpr int kWarpsPerBlock = 4;
constexpr int kBatch = 8;
static_assert(kRounds % kBatch == 0, "rounds come in whole batches");

size_t sort_hist_entries(long long n)
{
    long long nchunks = (n + kChunk - 1) / kChunk;
    return (size_t)(256 * nchunks);
}

__global__ void k_rs_hist(const unsigned *__restrict__ keys, long long n, int shift,
                          long long nchunks, unsigned *__restrict__ hist)
{
    __shared__ unsigned cnt[kWarpsPerBlock][256];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long chunk = blockIdx.x * (long long)kWarpsPerBlock + w;
    for (int d = lane; d < 256; d += 32) cnt[w][d] = 0;
    __syncwarp();
    if (chunk < nchunks) {
        const long long base = chunk * kChunk;
#pragma unroll 1
        for (int r0 = 0; r0 < kRounds; r0 += kBatch) {
            unsigned k[kBatch];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const long long e = base + (r0 + b) * 32 + lane;
                k[b] = e < n ? keys[e] : 0u;
            }
#pragma unroll
            for (int b = 0; b < kBatch; ++b)
                if (base + (r0 + b) * 32 + lane < n) atomicAdd(&cnt[w][(k[b] >> shift) & 255u], 1u);
        }
    }
    __syncwarp();
    if (chunk < nchunks)
        for (int d = lane; d < 256; d += 32) hist[(long long)d * nchunks + chunk] = cnt[w][d];
}

// The scatter ranks each key as before (its destination: the chunk's
// offset for its digit plus the lane-ordered rank of equal digits before
// it), but places it in shared memory first, at its destination's position
// within the block's range for its digit (a block's chunks are adjacent in
// the digit-major offsets, so each digit's keys of a block go to one
// contiguous range). The block then writes its keys out in that order:
// runs of consecutive addresses instead of up to 32 scattered words per
// warp round.
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_rs_scatter(const unsigned *__restrict__ kin,
                                                                    const unsigned *__restrict__ vin,
                                                                    unsigned *__restrict__ kout,
                                                                    unsigned *__restrict__ vout, long long n,
                                                                    int shift, long long nchunks,
                                                                    const unsigned *__restrict__ offs)
{
    __shared__ unsigned cnt[kWarpsPerBlock][256];
    __shared__ unsigned sk[kWarpsPerBlock * kChunk], sv[kWarpsPerBlock * kChunk];
    __shared__ unsigned gstart[256], lstart[256];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long chunk0 = blockIdx.x * (long long)kWarpsPerBlock, chunk = chunk0 + w;
    const long long last = min(chunk0 + kWarpsPerBlock, nchunks);       // the block's chunks [chunk0, last)
    // per digit: the block's first destination and its key count; the
    // offsets are an exclusive scan, so the entry after the block's last
    // chunk of digit d ends the block's run of d (n after the array)
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        const long long e = (long long)d * nchunks + last;
        gstart[d] = offs[(long long)d * nchunks + chunk0];
        lstart[d] = (e < 256 * nchunks ? offs[e] : (unsigned)n) - gstart[d];
    }
    __syncthreads();
    if (w == 0) {        // lstart: exclusive scan of the counts over the digits
        unsigned v[8], tot = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v[q] = lstart[8 * lane + q];
            tot += v[q];
        }
        unsigned incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        unsigned run = incl - tot;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            lstart[8 * lane + q] = run;
            run += v[q];
        }
    }
    if (chunk < nchunks)
        for (int d = lane; d < 256; d += 32) cnt[w][d] = offs[(long long)d * nchunks + chunk];
    __syncthreads();
    const long long base = chunk * kChunk;
    const unsigned lt = (1u << lane) - 1u;
    if (chunk < nchunks) {
#pragma unroll 1
        for (int r0 = 0; r0 < kRounds; r0 += kBatch) {
            unsigned kk[kBatch], vv[kBatch];
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const long long e = base + (r0 + b) * 32 + lane;
                kk[b] = e < n ? kin[e] : 0u;
                vv[b] = e < n ? vin[e] : 0u;
            }
#pragma unroll
            for (int b = 0; b < kBatch; ++b) {
                const bool valid = base + (r0 + b) * 32 + lane < n;
                const unsigned key = kk[b], val = vv[b];
                const unsigned d = valid ? ((key >> shift) & 255u) : 256u + lane;   // invalid lanes never match
                const unsigned peers = __match_any_sync(0xffffffffu, d);
                const int leader = __ffs(peers) - 1;
                const unsigned rank = __popc(peers & lt);
                unsigned start = 0;
                if (valid && lane == leader) start = cnt[w][d];
                start = __shfl_sync(0xffffffffu, start, leader);
                __syncwarp();
                if (valid) {
                    const unsigned p = lstart[d] + (start + rank - gstart[d]);
                    sk[p] = key;
                    sv[p] = val;
                    if (lane == leader) cnt[w][d] = start + __popc(peers);
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    // the block's keys in destination order
    const long long b0 = chunk0 * kChunk;
    const int nb = (int)(min(n, last * (long long)kChunk) - b0);
    for (int p = threadIdx.x; p < nb; p += blockDim.x) {
        const unsigned key = sk[p], d = (key >> shift) & 255u;
        const unsigned g = gstart[d] + ((unsigned)p - lstart[d]);
        kout[g] = key;
        vout[g] = sv[p];
    }
}

// exclusive scan of n unsigned values in place: blocks of 1024 threads scan
// 4096 values each, a single block scans the block totals, a third pass adds
constexpr int kScanPer = 4096;

__device__ unsigned block_excl_scan(unsigned v, unsigned *sh)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t;
    }
    __syncthreads();
    unsigned pre = w ? sh[w - 1] : 0u;
    unsigned total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    sh[32] = total;
    return pre + x - v;
}

__global__ void k_scan1(unsigned *a, long long n, unsigned *sums)
{
    __shared__ unsigned sh[33];
    long long base = blockIdx.x * (long long)kScanPer + threadIdx.x * 4;
    unsigned v[4], s = 0;
    for (int q = 0; q < 4; ++q) {
        v[q] = base + q < n ? a[base + q] : 0u;
        s += v[q];
    }
    unsigned ex = block_excl_scan(s, sh);
    for (int q = 0; q < 4; ++q) {
        if (base + q < n) a[base + q] = ex;
        ex += v[q];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = sh[32];
}

__global__ void k_scan2(unsigned *sums, int nb)
{
    __shared__ unsigned sh[33];
    unsigned carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + threadIdx.x;
        unsigned v = i < nb ? sums[i] : 0u;
        unsigned ex = block_excl_scan(v, sh);
        if (i < nb) sums[i] = carry + ex;
        carry += sh[32];
        __syncthreads();
    }
}

__global__ void k_scan3(unsigned *a, long long n, const unsigned *sums)
{
    long long base = blockIdx.x * (long long)kScanPer + threadIdx.x * 4;
    unsigned add = sums[blockIdx.x];
    for (int q = 0; q < 4; ++q)
        if (base + q < n) a[base + q] += add;
}

static cudaError_t excl_scan(unsigned *a, long long n, unsigned *sums, cudaStream_t st)
{
    long long nb = (n + kScanPer - 1) / kScanPer;
    if (nb <= 0) return cudaSuccess;
    k_scan1<<<(unsigned)nb, 1024, 0, st>>>(a, n, sums);
    k_scan2<<<1, 1024, 0, st>>>(sums, (int)nb);
    k_scan3<<<(unsigned)nb, 1024, 0, st>>>(a, n, sums);
    return cudaGetLastError();
}

cudaError_t launch_excl_scan(unsigned *a, long long n, unsigned *sums, cudaStream_t st)
{
    return excl_scan(a, n, sums, st);
}

cudaError_t launch_radix_sort(unsigned *keys, unsigned *vals, long long n, int key_bits,
                              SortScratch &s, unsigned **keys_out, unsigned **vals_out,
                              cudaStream_t st)
{
    long long nchunks = (n + kChunk - 1) / kChunk;
    unsigned *kin = keys, *vin = vals;
    unsigned *kb = (keys == s.keys[0]) ? s.keys[1] : s.keys[0];
    unsigned *vb = (vals == s.vals[0]) ? s.vals[1] : s.vals[0];
    unsigned blocks = (unsigned)((nchunks + kWarpsPerBlock - 1) / kWarpsPerBlock);
    for (int shift = 0; shift < key_bits && n > 0; shift += 8) {
        k_rs_hist<<<blocks, 32 * kWarpsPerBlock, 0, st>>>(kin, n, shift, nchunks, s.hist);
        cudaError_t e = excl_scan(s.hist, 256 * nchunks, s.sums, st);
        if (e != cudaSuccess) return e;
        k_rs_scatter<<<blocks, 32 * kWarpsPerBlock, 0, st>>>(kin, vin, kb, vb, n, shift, nchunks,
                                                              s.hist);
        unsigned *t = kin; kin = kb; kb = t;
        t = vin; vin = vb; vb = t;
    }
    *keys_out = kin;
    *vals_out = vin;
    return cudaGetLastError();
}

cudaError_t launch_morton_sort(const double4 *xi, long long n, SortScratch &s, unsigned **perm_out,
                               cudaStream_t st)
{
    k_bbox_init<<<1, 32, 0, st>>>(s.bbox);
    unsigned g = (unsigned)((n + 255) / 256);
    k_bbox<<<g < 1024 ? g : 1024, 256, 0, st>>>(xi, n, s.bbox);
    k_morton<<<g, 256, 0, st>>>(xi, n, s.bbox, s.keys[0], s.vals[0]);
    unsigned *ko;
    return launch_radix_sort(s.keys[0], s.vals[0], n, 30, s, &ko, perm_out, st);
}

// ---------------------------------------------------------------- tiles
// One CTA per tile of Bi consecutive (sorted) i: gather the positions and
// take the midpoint of the tile's bounding box as its FP64 centre.
__global__ void k_tile_prep(const double4 *__restrict__ xi, const unsigned *__restrict__ perm,
                            long long n, int Bi, double4 *__restrict__ xt,
                            double4 *__restrict__ ctr)
{
    __shared__ double red[6][32];
    long long t = blockIdx.x;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = threadIdx.x; k < Bi; k += blockDim.x) {
        long long p = t * Bi + k;
        if (p >= n) break;
        double4 v = xi[perm ? (long long)perm[p] : p];
        xt[p] = v;
        lo[0] = fmin(lo[0], v.x); lo[1] = fmin(lo[1], v.y); lo[2] = fmin(lo[2], v.z);
        hi[0] = fmax(hi[0], v.x); hi[1] = fmax(hi[1], v.y); hi[2] = fmax(hi[2], v.z);
    }
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o; o >>= 1) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int c = 0; c < 3; ++c) { red[c][w] = lo[c]; red[3 + c][w] = hi[c]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = blockDim.x >> 5;
        for (int q = 1; q < nw; ++q)
            for (int c = 0; c < 3; ++c) {
                red[c][0] = fmin(red[c][0], red[c][q]);
                red[3 + c][0] = fmax(red[3 + c][0], red[3 + c][q]);
            }
        double c0 = 0.5 * (red[0][0] + red[3][0]);
        double c1 = 0.5 * (red[1][0] + red[4][0]);
        double c2 = 0.5 * (red[2][0] + red[5][0]);
        ctr[t] = make_double4(c0, c1, c2, 0.0);
    }
}

cudaError_t launch_tile_prep(const double4 *xi, const unsigned *perm, long long n, int Bi,
                             double4 *xi_tiled, double4 *ctr, cudaStream_t st)
{
    long long nt = (n + Bi - 1) / Bi;
    if (nt <= 0) return cudaSuccess;
    k_tile_prep<<<(unsigned)nt, 256, 0, st>>>(xi, perm, n, Bi, xi_tiled, ctr);
    return cudaGetLastError();
}

}  // namespace pg
