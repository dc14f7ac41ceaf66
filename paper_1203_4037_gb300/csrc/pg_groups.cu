// pg_groups.cu -- batched i-groups, each with its own j-list (the tree usage
// of Section 5.1: a group of nearby i-particles shares one interaction list
// of particles and pseudo-particles), and the periodic cell list that turns
// the cutoff force into the same shape of work.
//
// One persistent launch: every CTA takes work items (group, i-chunk) from an
// atomic queue ordered longest-first, gathers the group's j records by index
// into shared memory (converted once per record to FP32 offsets from the
// group's FP64 centre, with the periodic image shift applied in FP64), and
// evaluates the Newton or tabulated pair term with the i-particles in
// registers. A small group splits each set of i-particles across L lanes,
// each taking every L-th j, and combines the lanes with warp shuffles.
#include "pg_device.cuh"

namespace pg {

constexpr int kTJG = 512;          // j entries staged per step
constexpr int kPerThread = kTJG / kNT;

__device__ __forceinline__ void shift_of(int code, double box, double &sx, double &sy, double &sz)
{
    // code = 9 (dx+1) + 3 (dy+1) + (dz+1), dx, dy, dz in {-1, 0, 1}
    int dx = code / 9 - 1, dy = (code / 3) % 3 - 1, dz = code % 3 - 1;
    sx = dx * box;
    sy = dy * box;
    sz = dz * box;
}

template <int NP, bool TABLE>
__global__ void __launch_bounds__(kNT) k_groups(GroupArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    u64 *cvt = reinterpret_cast<u64 *>(smem);                            // [kTJG][4]
    int *sh = reinterpret_cast<int *>(smem + kTJG * 4 * sizeof(u64));   // item slot
    float2 *tab = reinterpret_cast<float2 *>(smem + kTJG * 4 * sizeof(u64) + 16);

    const int tid = threadIdx.x;
    if (TABLE)
        for (int k = tid; k < a.tab.n; k += kNT) tab[k] = a.tab.AG1[k];

    const float c0 = TABLE ? 2.0f : a.eps2;
    const u64 c0v = pk2(c0, c0);
    const double sc = TABLE ? a.tab.scale : 1.0;
    const int nitems = a.nitems >= 0 ? a.nitems : *a.nitems_dev;

    for (;;) {
        __syncthreads();   // previous item fully done with shared memory
        if (tid == 0) sh[0] = atomicAdd(a.queue, 1);
        __syncthreads();
        const int item = sh[0];
        if (item >= nitems) break;
        const GroupItem it = a.items[item];
        const double4 c = a.gctr[it.group];
        const long long jb = a.j_off[it.group], je = a.j_off[it.group + 1];

        // thread layout: nsets sets of 2*NP i-particles, L lanes per set
        const int nsets = (it.ni + 2 * NP - 1) / (2 * NP);
        int L = kNT / (nsets > 0 ? nsets : 1);
        L = L >= 32 ? 32 : L >= 16 ? 16 : L >= 8 ? 8 : L >= 4 ? 4 : L >= 2 ? 2 : 1;
        const int set = tid / L, lane = tid % L;
        const bool active = set < nsets;

        u64 xi[NP], yi[NP], zi[NP];
        u64 ax[NP], ay[NP], az[NP], ph[NP];
        u64 hx[NP], hy[NP], hz[NP], hp[NP], lx[NP], ly[NP], lz[NP], lp[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float fx[2] = {0, 0}, fy[2] = {0, 0}, fz[2] = {0, 0};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                int k = set * 2 * NP + 2 * p + q;
                if (active && k < it.ni) {
                    double4 v = a.xi[it.i0 + k];
                    fx[q] = (float)((v.x - c.x) * sc);
                    fy[q] = (float)((v.y - c.y) * sc);
                    fz[q] = (float)((v.z - c.z) * sc);
                }
            }
            xi[p] = pk2(fx[0], fx[1]);
            yi[p] = pk2(fy[0], fy[1]);
            zi[p] = pk2(fz[0], fz[1]);
            hx[p] = hy[p] = hz[p] = hp[p] = 0ull;
            lx[p] = ly[p] = lz[p] = lp[p] = 0ull;
        }

        // register prefetch of the first tile's records (and their shift codes)
        double4 rec[kPerThread];
        int code[kPerThread];
        auto fetch = [&](long long t0) {
#pragma unroll
            for (int r = 0; r < kPerThread; ++r) {
                long long e = t0 + r * kNT + tid;
                code[r] = 13;                  // no image shift
                if (e < je) {
                    int raw = a.jlist[e];
                    long long j = raw & 0x07ffffff;
                    if (j >= a.nj) {           // bad index: record and contribute nothing
                        report(a.status, kStatusBadIndex, 2);
                        rec[r] = make_double4(0, 0, 0, -1.0);
                        continue;
                    }
                    rec[r] = ldg_d4(a.jrec + j);
                    if (a.box > 0.0) code[r] = (int)(((unsigned)raw) >> 27);
                } else {
                    rec[r] = make_double4(0, 0, 0, -1.0);   // padding marker
                }
            }
        };
        fetch(jb);
        for (long long t0 = jb; t0 < je; t0 += kTJG) {
            // publish the prefetched tile: FP64 record + image shift - centre -> FP32
#pragma unroll
            for (int r = 0; r < kPerThread; ++r) {
                const int e = r * kNT + tid;
                float x, y, z, m;
                if (rec[r].w >= 0.0) {
                    double sx, sy, sz;
                    shift_of(code[r], a.box, sx, sy, sz);
                    x = (float)((rec[r].x + sx - c.x) * sc);
                    y = (float)((rec[r].y + sy - c.y) * sc);
                    z = (float)((rec[r].z + sz - c.z) * sc);
                    m = (float)rec[r].w;
                } else {
                    x = y = z = 1.0e4f;
                    m = 0.0f;
                }
                cvt[4 * e + 0] = pk2(x, x);
                cvt[4 * e + 1] = pk2(y, y);
                cvt[4 * e + 2] = pk2(z, z);
                cvt[4 * e + 3] = pk2(m, m);
            }
            __syncthreads();
            if (t0 + kTJG < je) fetch(t0 + kTJG);   // loads in flight during the compute
            long long nv = je - t0;
            if (nv > kTJG) nv = kTJG;
            if (active) {
#pragma unroll
                for (int p = 0; p < NP; ++p) ax[p] = ay[p] = az[p] = ph[p] = 0ull;
                const int nv_lane = (int)nv;
#pragma unroll 2
                for (int e = lane; e < nv_lane; e += L) {
                    const ulonglong2 xy = reinterpret_cast<const ulonglong2 *>(cvt)[2 * e];
                    const ulonglong2 zm = reinterpret_cast<const ulonglong2 *>(cvt)[2 * e + 1];
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        const u64 dx = f2sub(xy.x, xi[p]);
                        const u64 dy = f2sub(xy.y, yi[p]);
                        const u64 dz = f2sub(zm.x, zi[p]);
                        u64 r2 = f2fma(dx, dx, c0v);
                        r2 = f2fma(dy, dy, r2);
                        r2 = f2fma(dz, dz, r2);
                        float ra, rb;
                        up2(r2, ra, rb);
                        if (!TABLE) {
                            float qa = rsq(ra), qb = rsq(rb);
                            qa = ra > 0.0f ? qa : 0.0f;     // eps = 0: coincident pair adds nothing
                            qb = rb > 0.0f ? qb : 0.0f;
                            const u64 q = pk2(qa, qb);
                            const u64 mq = f2mul(zm.y, q);
                            const u64 mq3 = f2mul(mq, f2mul(q, q));
                            ph[p] = f2sub(ph[p], mq);
                            ax[p] = f2fma(mq3, dx, ax[p]);
                            ay[p] = f2fma(mq3, dy, ay[p]);
                            az[p] = f2fma(mq3, dz, az[p]);
                        } else {
                            ra = fminf(ra, a.tab.s_max);
                            rb = fminf(rb, a.tab.s_max);
                            const float2 ta = tab[(__float_as_uint(ra) >> a.tab.shift) - a.tab.base];
                            const float2 tb = tab[(__float_as_uint(rb) >> a.tab.shift) - a.tab.base];
                            const u64 g = f2fma(pk2(ra, rb), pk2(ta.y, tb.y), pk2(ta.x, tb.x));
                            const u64 mg = f2mul(zm.y, g);
                            ax[p] = f2fma(mg, dx, ax[p]);
                            ay[p] = f2fma(mg, dy, ay[p]);
                            az[p] = f2fma(mg, dz, az[p]);
                        }
                    }
                }
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    fold2(hx[p], lx[p], ax[p]);
                    fold2(hy[p], ly[p], ay[p]);
                    fold2(hz[p], lz[p], az[p]);
                    if (!TABLE) fold2(hp[p], lp[p], ph[p]);
                }
            }
            __syncthreads();   // everyone done with this tile before it is overwritten
        }

        // combine the L lanes of each set in FP64, write the set's outputs
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float h[8], l[8];
            up2(hx[p], h[0], h[1]); up2(hy[p], h[2], h[3]);
            up2(hz[p], h[4], h[5]); up2(hp[p], h[6], h[7]);
            up2(lx[p], l[0], l[1]); up2(ly[p], l[2], l[3]);
            up2(lz[p], l[4], l[5]); up2(lp[p], l[6], l[7]);
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = (double)h[k] + (double)l[k];
            for (int off = L >> 1; off > 0; off >>= 1)
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
            if (active && lane == 0) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    int k = set * 2 * NP + 2 * p + q;
                    if (k < it.ni) {
                        long long i = it.i0 + k;
                        long long o = a.perm ? (long long)a.perm[i] : i;
                        a.acc[3 * o] = v[0 + q] * a.accscale;
                        a.acc[3 * o + 1] = v[2 + q] * a.accscale;
                        a.acc[3 * o + 2] = v[4 + q] * a.accscale;
                        if (a.pot) a.pot[o] = TABLE ? 0.0 : v[6 + q];
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------------ host
size_t groups_smem(bool table, int ntab)
{
    size_t s = kTJG * 4 * sizeof(u64) + 16;
    if (table) s += (size_t)ntab * sizeof(float2);
    return s;
}

int groups_bi(int np) { return kNT * 2 * np; }

template <int NP, bool TABLE>
static cudaError_t configure_g()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_groups<NP, TABLE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)groups_smem(TABLE, 1 << 13));
    done = e == cudaSuccess;
    return e;
}

template <int NP, bool TABLE>
static int occ_g(size_t smem)
{
    if (configure_g<NP, TABLE>() != cudaSuccess) return 1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_groups<NP, TABLE>, kNT, smem) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

int groups_max_blocks_per_sm(int np, bool table, int ntab)
{
    size_t smem = groups_smem(table, ntab);
    if (table) return np == 1 ? occ_g<1, true>(smem) : np == 4 ? occ_g<4, true>(smem) : occ_g<2, true>(smem);
    return np == 1 ? occ_g<1, false>(smem) : np == 4 ? occ_g<4, false>(smem) : occ_g<2, false>(smem);
}

cudaError_t launch_groups(const GroupArgs &g, int grid, int np, bool table, size_t smem,
                          cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
#define PG_G(NP_)                                                        \
    if (np == NP_) {                                                     \
        cudaError_t e = table ? configure_g<NP_, true>() : configure_g<NP_, false>(); \
        if (e != cudaSuccess) return e;                                  \
        if (table) k_groups<NP_, true><<<grid, kNT, smem, st>>>(g);      \
        else k_groups<NP_, false><<<grid, kNT, smem, st>>>(g);           \
        return cudaGetLastError();                                       \
    }
    PG_G(1)
    PG_G(2)
    PG_G(4)
#undef PG_G
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ prep
// FP64 centre of each group: midpoint of its i-particles' bounding box
__global__ void k_group_ctr(const double4 *__restrict__ xi, const long long *__restrict__ i_off,
                            long long ngroups, double4 *__restrict__ ctr)
{
    long long g = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (g >= ngroups) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long long i = i_off[g] + lane; i < i_off[g + 1]; i += 32) {
        double4 v = xi[i];
        lo[0] = fmin(lo[0], v.x); lo[1] = fmin(lo[1], v.y); lo[2] = fmin(lo[2], v.z);
        hi[0] = fmax(hi[0], v.x); hi[1] = fmax(hi[1], v.y); hi[2] = fmax(hi[2], v.z);
    }
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o; o >>= 1) {
            lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    if (lane == 0) {
        bool empty = !(lo[0] <= hi[0]);
        ctr[g] = empty ? make_double4(0, 0, 0, 0)
                       : make_double4(0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]),
                                      0.5 * (lo[2] + hi[2]), 0.0);
    }
}

cudaError_t launch_group_ctr(const double4 *xi, const long long *i_off, long long ngroups,
                             double4 *ctr, cudaStream_t st)
{
    if (ngroups <= 0) return cudaSuccess;
    k_group_ctr<<<(unsigned)((ngroups + 3) / 4), 128, 0, st>>>(xi, i_off, ngroups, ctr);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ cell list
// Periodic cube of side box, nc cells per axis (side box/nc >= r_cut).
__device__ __forceinline__ int cell_axis(double x, double box, int nc)
{
    double w = x - box * floor(x / box);          // wrap into [0, box)
    int c = (int)(w * (nc / box));
    return c < 0 ? 0 : c >= nc ? nc - 1 : c;
}

// wrapped positions (x, y, z, m) and the cell key of every particle
__global__ void k_cell_key(const double4 *__restrict__ jrec, long long n, double box, int nc,
                           unsigned *__restrict__ key, unsigned *__restrict__ idx,
                           double4 *__restrict__ wrapped)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double4 v = jrec[i];
    double wx = v.x - box * floor(v.x / box);
    double wy = v.y - box * floor(v.y / box);
    double wz = v.z - box * floor(v.z / box);
    // floor can leave w == box for tiny negative inputs; fold it back
    if (wx >= box) wx -= box;
    if (wy >= box) wy -= box;
    if (wz >= box) wz -= box;
    wrapped[i] = make_double4(wx, wy, wz, v.w);
    int cx = cell_axis(wx, box, nc), cy = cell_axis(wy, box, nc), cz = cell_axis(wz, box, nc);
    key[i] = (unsigned)((cx * nc + cy) * nc + cz);
    idx[i] = (unsigned)i;
}

__global__ void k_cell_count(const unsigned *__restrict__ key, long long n, unsigned *__restrict__ cnt)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[key[i]], 1u);
}

// particles in cell order
__global__ void k_cell_gather(const double4 *__restrict__ wrapped, const unsigned *__restrict__ perm,
                              long long n, double4 *__restrict__ xs)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p < n) xs[p] = wrapped[perm[p]];
}

// per cell: number of j entries (27 neighbour cells) and number of items
__global__ void k_cell_sizes(const unsigned *__restrict__ start, int nc, int Bi,
                             unsigned *__restrict__ jcount, unsigned *__restrict__ icount)
{
    long long ncell = (long long)nc * nc * nc;
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= ncell) return;
    int cx = (int)(g / (nc * nc)), cy = (int)((g / nc) % nc), cz = (int)(g % nc);
    unsigned s = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int x = (cx + dx + nc) % nc, y = (cy + dy + nc) % nc, z = (cz + dz + nc) % nc;
                long long nb = ((long long)x * nc + y) * nc + z;
                s += start[nb + 1] - start[nb];
            }
    unsigned ni = start[g + 1] - start[g];
    jcount[g] = ni ? s : 0u;
    icount[g] = (ni + Bi - 1) / Bi;
}

__global__ void k_joff_widen(const unsigned *__restrict__ in, long long n, long long *__restrict__ out)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) out[k] = in[k];
}

__global__ void k_fill_iota(unsigned *__restrict__ v, long long n)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) v[k] = (unsigned)k;
}

// evaluated pairs of the cell decomposition: sum over cells of n_i * n_j
__global__ void k_cell_pairs(const unsigned *__restrict__ start, const unsigned *__restrict__ jcount,
                             long long ncell, unsigned long long *__restrict__ pairs)
{
    unsigned long long s = 0;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ncell;
         g += (long long)gridDim.x * blockDim.x)
        s += (unsigned long long)(start[g + 1] - start[g]) * jcount[g];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(pairs, s);
}

// one CTA per cell: its j-list, neighbour by neighbour; a neighbour reached
// across the box boundary carries the shift code of its periodic image
__global__ void k_cell_lists(const unsigned *__restrict__ start, int nc,
                             const unsigned *__restrict__ joff, int *__restrict__ jlist)
{
    long long g = blockIdx.x;
    unsigned ni = start[g + 1] - start[g];
    if (ni == 0) return;
    int cx = (int)(g / (nc * nc)), cy = (int)((g / nc) % nc), cz = (int)(g % nc);
    unsigned pos = joff[g];
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz) {
                int x = cx + dx, y = cy + dy, z = cz + dz;
                // the image of a wrapped neighbour sits one box length over
                int sx = x < 0 ? -1 : x >= nc ? 1 : 0;
                int sy = y < 0 ? -1 : y >= nc ? 1 : 0;
                int sz = z < 0 ? -1 : z >= nc ? 1 : 0;
                x = (x + nc) % nc; y = (y + nc) % nc; z = (z + nc) % nc;
                long long nb = ((long long)x * nc + y) * nc + z;
                int code = 9 * (sx + 1) + 3 * (sy + 1) + (sz + 1);
                unsigned b = start[nb], cnt = start[nb + 1] - b;
                for (unsigned k = threadIdx.x; k < cnt; k += blockDim.x)
                    jlist[pos + k] = (int)((b + k) | ((unsigned)code << 27));
                pos += cnt;
            }
}

// one item per (cell, chunk of <= Bi i-particles), keyed longest-first
__global__ void k_cell_items(const unsigned *__restrict__ start, long long ncell, int Bi,
                             const unsigned *__restrict__ ioff, const unsigned *__restrict__ jcount,
                             GroupItem *__restrict__ items, unsigned *__restrict__ keys,
                             unsigned *__restrict__ vals)
{
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= ncell) return;
    unsigned b = start[g], ni = start[g + 1] - b;
    unsigned o = ioff[g];
    for (unsigned k = 0; k * Bi < ni; ++k) {
        GroupItem it;
        it.group = (int)g;
        it.i0 = (int)(b + k * Bi);
        it.ni = (int)min((unsigned)Bi, ni - k * Bi);
        it.pad = 0;
        items[o + k] = it;
        unsigned long long cost = (unsigned long long)it.ni * jcount[g];
        unsigned cq = cost > 0xffffffull ? 0xffffffu : (unsigned)cost;
        keys[o + k] = 0xffffffu - cq;     // ascending sort = longest first
        vals[o + k] = o + k;
    }
}

__global__ void k_items_permute(const GroupItem *__restrict__ in, const unsigned *__restrict__ order,
                                const unsigned *__restrict__ nitems, GroupItem *__restrict__ out)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < (long long)*nitems) out[k] = in[order[k]];
}

__global__ void k_cell_ctr(int nc, double box, double4 *__restrict__ ctr)
{
    long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long ncell = (long long)nc * nc * nc;
    if (g >= ncell) return;
    int cx = (int)(g / (nc * nc)), cy = (int)((g / nc) % nc), cz = (int)(g % nc);
    double h = box / nc;
    ctr[g] = make_double4((cx + 0.5) * h, (cy + 0.5) * h, (cz + 0.5) * h, 0.0);
}

cudaError_t launch_cell_build(const double4 *jrec, long long n, double box, int nc, int Bi,
                              CellScratch &s, SortScratch &sort, cudaStream_t st)
{
    long long ncell = (long long)nc * nc * nc;
    unsigned gb = (unsigned)((n + 255) / 256);
    unsigned gc = (unsigned)((ncell + 255) / 256);
    k_cell_key<<<gb, 256, 0, st>>>(jrec, n, box, nc, sort.keys[0], sort.vals[0], s.wrapped);
    unsigned *ko, *perm;
    int bits = 0;
    while ((1LL << bits) < ncell) ++bits;
    cudaError_t e = launch_radix_sort(sort.keys[0], sort.vals[0], n, bits, sort, &ko, &perm, st);
    if (e != cudaSuccess) return e;
    // the item sort below reuses the sort buffers: keep our own copy
    cudaMemcpyAsync(s.perm, perm, n * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    perm = s.perm;
    // counts -> start (exclusive scan of ncell + 1 entries)
    cudaMemsetAsync(s.start, 0, (ncell + 1) * sizeof(unsigned), st);
    k_cell_count<<<gb, 256, 0, st>>>(ko, n, s.start);
    if ((e = launch_excl_scan(s.start, ncell + 1, sort.sums, st)) != cudaSuccess) return e;
    k_cell_gather<<<gb, 256, 0, st>>>(s.wrapped, perm, n, s.xs);
    k_cell_sizes<<<gc, 256, 0, st>>>(s.start, nc, Bi, s.jcount, s.icount);
    cudaMemsetAsync(s.pairs, 0, sizeof(unsigned long long), st);
    k_cell_pairs<<<gc < 1024 ? gc : 1024, 256, 0, st>>>(s.start, s.jcount, ncell, s.pairs);
    // j offsets (exclusive scan of jcount, ncell + 1 entries with a zero tail)
    cudaMemcpyAsync(s.joff32, s.jcount, ncell * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(s.joff32 + ncell, 0, sizeof(unsigned), st);
    if ((e = launch_excl_scan(s.joff32, ncell + 1, sort.sums, st)) != cudaSuccess) return e;
    k_joff_widen<<<(unsigned)((ncell + 1 + 255) / 256), 256, 0, st>>>(s.joff32, ncell + 1, s.joff);
    k_cell_lists<<<(unsigned)ncell, 128, 0, st>>>(s.start, nc, s.joff32, s.jlist);
    // items
    cudaMemcpyAsync(s.ioff, s.icount, ncell * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(s.ioff + ncell, 0, sizeof(unsigned), st);
    if ((e = launch_excl_scan(s.ioff, ncell + 1, sort.sums, st)) != cudaSuccess) return e;
    // unused item slots sort last
    cudaMemsetAsync(sort.keys[0], 0xff, s.item_cap * sizeof(unsigned), st);
    k_fill_iota<<<(unsigned)((s.item_cap + 255) / 256), 256, 0, st>>>(sort.vals[0], s.item_cap);
    k_cell_items<<<gc, 256, 0, st>>>(s.start, ncell, Bi, s.ioff, s.jcount, s.items_raw,
                                     sort.keys[0], sort.vals[0]);
    unsigned *order;
    if ((e = launch_radix_sort(sort.keys[0], sort.vals[0], s.item_cap, 24, sort, &ko, &order, st)) !=
        cudaSuccess)
        return e;
    k_items_permute<<<(unsigned)((s.item_cap + 255) / 256), 256, 0, st>>>(s.items_raw, order,
                                                                          s.ioff + ncell, s.items);
    k_cell_ctr<<<gc, 256, 0, st>>>(nc, box, s.ctr);
    return cudaGetLastError();
}

}  // namespace pg
