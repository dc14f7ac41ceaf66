// pg_tree.cu -- the tree front end: a Barnes-Hut tree over the j-particles,
// i-particles taken in groups that traverse it once and share one
// interaction list (the tree usage of Section 5.1: vacuum boundary,
// monopole moments, lists shared by a group after Makino's grouping), built
// on the GPU and fed to the batched-group kernel.
//
// The construction:
//  - the root is the cube at the per-axis minimum with side span = the
//    largest extent (1 if all particles coincide);
//  - keys: q = floor((x - lo) / span * 1024) per axis, clamped to 1023,
//    interleaved (x at bit 3b+2, y at 3b+1, z at 3b); a stable radix sort;
//  - the nodes of level L (0 .. 10) are the runs of equal 3L-bit prefix,
//    numbered level by level; a node's children are the next level's runs
//    inside it; its side is span / 2^L;
//  - monopoles bottom-up: M = sum m, S = sum m x over the particles (finest
//    level, in key order) or over the children in order; centre S / M;
//  - groups: nodes with at most ncrit particles whose parent has more (the
//    root if small), and finest-level nodes whose parent has more; in
//    particle order;
//  - a group with box [blo, bhi] accepts node N as one pseudo-particle if N
//    holds none of the group's particles and side^2 < theta^2 d^2 (d from
//    N's centre of mass to the box); else a leaf (at most nleaf particles,
//    or the finest level) gives its particles, else N is opened, children
//    in order, depth first.
// Every FP64 operation of the decisions uses an explicitly rounded
// intrinsic (no fused multiply-add), so the lists are reproducible bit for
// bit by any implementation that rounds the same operations the same way.
#include "pg_device.cuh"

namespace pg {

namespace {

constexpr int kLevels = 11;      // levels 0 .. 10
constexpr int kBits = 10;        // key bits per axis
constexpr int kStack = 8 * kLevels + 8;

// order-preserving map of a double onto 64-bit unsigned integers
__device__ __forceinline__ unsigned long long ord_of(double v)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ double val_of(unsigned long long o)
{
    const unsigned long long u = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
    return __longlong_as_double((long long)u);
}

__global__ void k_tree_bbox_init(unsigned long long *bb)
{
    if (threadIdx.x < 3) {
        bb[threadIdx.x] = ~0ull;         // min
        bb[3 + threadIdx.x] = 0ull;      // max
    }
}

__global__ void k_tree_bbox(const double4 *__restrict__ x, long long n, unsigned long long *bb)
{
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0, 0, 0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double4 v = x[i];
        const unsigned long long o[3] = {ord_of(v.x), ord_of(v.y), ord_of(v.z)};
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], o[a]);
            hi[a] = max(hi[a], o[a]);
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int s = 16; s; s >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], s));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], s));
        }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bb[a], lo[a]);
            atomicMax(&bb[3 + a], hi[a]);
        }
}

// geo = {lo_x, lo_y, lo_z, span}
__global__ void k_tree_span(const unsigned long long *bb, double *geo)
{
    if (threadIdx.x != 0) return;
    double span = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double lo = val_of(bb[a]), hi = val_of(bb[3 + a]);
        geo[a] = lo;
        const double e = __dsub_rn(hi, lo);
        if (e > span) span = e;
    }
    if (!(span > 0.0)) span = 1.0;
    geo[3] = span;
}

__device__ __forceinline__ unsigned spread10(unsigned v)
{
    unsigned r = 0;
#pragma unroll
    for (int b = 0; b < kBits; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

__global__ void k_tree_keys(const double4 *__restrict__ x, long long n, const double *geo,
                            unsigned *__restrict__ key, unsigned *__restrict__ idx)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 v = x[i];
    const double c[3] = {v.x, v.y, v.z};
    const double span = geo[3];
    unsigned k = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double u = __ddiv_rn(__dsub_rn(c[a], geo[a]), span);
        const double f = floor(__dmul_rn(u, 1024.0));
        const unsigned q = f >= 1023.0 ? 1023u : (unsigned)f;
        k |= spread10(q) << (2 - a);
    }
    key[i] = k;
    idx[i] = (unsigned)i;
}

// particles in key order (x, y, z, m) and the i records (x, y, z, 0)
__global__ void k_tree_gather(const double4 *__restrict__ x, const unsigned *__restrict__ perm,
                              long long n, double4 *__restrict__ xs, double4 *__restrict__ xi0)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 v = x[perm[i]];
    xs[i] = v;
    xi0[i] = make_double4(v.x, v.y, v.z, 0.0);
}

// flag[i] = 1 where a run of equal 3L-bit prefix starts; flag[n] = 0
__global__ void k_tree_flags(const unsigned *__restrict__ key, long long n, int sh,
                             unsigned *__restrict__ flag)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i > n) return;
    flag[i] = i == n ? 0u : (i == 0 || (key[i] >> sh) != (key[i - 1] >> sh)) ? 1u : 0u;
}

// after the exclusive scan of the flags: each run's first particle, and
// (below) the counts and children
__global__ void k_tree_starts(const unsigned *__restrict__ key, const unsigned *__restrict__ scan,
                              long long n, int sh, long long off, int *__restrict__ first)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0 || (key[i] >> sh) != (key[i - 1] >> sh)) first[off + scan[i]] = (int)i;
}

// run id at level L of particle i: the inclusive scan minus one = scan[i + 1] - 1
__global__ void k_tree_nodes(long long off, long long runs, long long n,
                             const unsigned *__restrict__ scan_next, long long off_next, int level,
                             int *__restrict__ first, int *__restrict__ count,
                             int *__restrict__ child0, int *__restrict__ childn,
                             unsigned char *__restrict__ lev)
{
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= runs) return;
    const long long k = off + r;
    const int f = first[k];
    const int e = r + 1 < runs ? first[k + 1] : (int)n;
    count[k] = e - f;
    lev[k] = (unsigned char)level;
    if (scan_next) {
        child0[k] = (int)(off_next + scan_next[f]);
        childn[k] = (int)(scan_next[e] - scan_next[f]);
    } else {
        child0[k] = 0;
        childn[k] = 0;
    }
}

// monopoles of the finest level from the particles, in key order
__global__ void k_tree_moments_leaf(long long off, long long runs, const int *__restrict__ first,
                                    const int *__restrict__ count, const double4 *__restrict__ xs,
                                    double *__restrict__ M, double *__restrict__ S)
{
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= runs) return;
    const long long k = off + r;
    double m = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = first[k]; i < first[k] + count[k]; ++i) {
        const double4 v = xs[i];
        m = __dadd_rn(m, v.w);
        s0 = __dadd_rn(s0, __dmul_rn(v.w, v.x));
        s1 = __dadd_rn(s1, __dmul_rn(v.w, v.y));
        s2 = __dadd_rn(s2, __dmul_rn(v.w, v.z));
    }
    M[k] = m;
    S[3 * k] = s0;
    S[3 * k + 1] = s1;
    S[3 * k + 2] = s2;
}

// monopoles of a coarser level from the children, in order
__global__ void k_tree_moments_up(long long off, long long runs, const int *__restrict__ child0,
                                  const int *__restrict__ childn, double *__restrict__ M,
                                  double *__restrict__ S)
{
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= runs) return;
    const long long k = off + r;
    double m = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int c = child0[k]; c < child0[k] + childn[k]; ++c) {
        m = __dadd_rn(m, M[c]);
        s0 = __dadd_rn(s0, S[3 * c]);
        s1 = __dadd_rn(s1, S[3 * c + 1]);
        s2 = __dadd_rn(s2, S[3 * c + 2]);
    }
    M[k] = m;
    S[3 * k] = s0;
    S[3 * k + 1] = s1;
    S[3 * k + 2] = s2;
}

// group marks at their first particle: gat[i] = node, else -1 (set before)
__global__ void k_tree_group_marks(long long off, long long runs, int level,
                                   const unsigned *__restrict__ scan_prev, long long off_prev,
                                   const int *__restrict__ first, const int *__restrict__ count,
                                   int ncrit, int *__restrict__ gat)
{
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= runs) return;
    const long long k = off + r;
    long long pc = -1;
    if (level > 0) {
        const long long p = off_prev + scan_prev[first[k] + 1] - 1;
        pc = count[p];
    }
    const bool grp = (count[k] <= ncrit && (level == 0 || pc > ncrit)) ||
                     (level == kLevels - 1 && pc > ncrit);
    if (grp) gat[first[k]] = (int)k;
}

__global__ void k_tree_group_flags(const int *__restrict__ gat, long long n, unsigned *__restrict__ f)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i > n) return;
    f[i] = i < n && gat[i] >= 0 ? 1u : 0u;
}

// groups in particle order with their boxes; i_off[g] (ngroups + 1 entries)
__global__ void k_tree_groups(const int *__restrict__ gat, const unsigned *__restrict__ gscan,
                              long long n, const int *__restrict__ count,
                              const double4 *__restrict__ xs, int *__restrict__ g_i0,
                              int *__restrict__ g_ni, double *__restrict__ gbox,
                              long long *__restrict__ i_off)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i == n) i_off[gscan[n]] = n;
    if (i >= n || gat[i] < 0) return;
    const unsigned g = gscan[i];
    const int ni = count[gat[i]];
    g_i0[g] = (int)i;
    g_ni[g] = ni;
    i_off[g] = i;
    double lo[3] = {xs[i].x, xs[i].y, xs[i].z}, hi[3] = {lo[0], lo[1], lo[2]};
    for (long long k = i; k < i + ni; ++k) {
        const double4 v = xs[k];
        const double c[3] = {v.x, v.y, v.z};
        for (int a = 0; a < 3; ++a) {
            if (c[a] < lo[a]) lo[a] = c[a];
            if (c[a] > hi[a]) hi[a] = c[a];
        }
    }
    for (int a = 0; a < 3; ++a) {
        gbox[6 * g + a] = lo[a];
        gbox[6 * g + 3 + a] = hi[a];
    }
}

struct WalkArgs {
    long long n, ngroups;
    const int *g_i0, *g_ni;
    const double *gbox;
    const int *first, *count, *child0, *childn;
    const unsigned char *lev;
    const double4 *com;        // per node: centre of mass S / M, mass
    const double *geo;         // {lo, span}
    double theta2;
    int nleaf;
    const long long *j_off;    // fill pass: offsets; count pass: nullptr
    unsigned *jcount;          // count pass output
    int *jlist;                // fill pass output
    int *status;
};

// one thread per group, depth first with an explicit stack
__global__ void k_tree_walk(WalkArgs w)
{
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= w.ngroups) return;
    const int i0 = w.g_i0[g];
    const double span = w.geo[3];
    double blo[3], bhi[3];
    for (int a = 0; a < 3; ++a) {
        blo[a] = w.gbox[6 * g + a];
        bhi[a] = w.gbox[6 * g + 3 + a];
    }
    int stack[kStack];
    int sp = 0;
    stack[sp++] = 0;
    long long cnt = 0;
    const long long base = w.j_off ? w.j_off[g] : 0;
    // the fill pass writes exactly what the count pass counted; the bound
    // turns any disagreement into a reported error instead of a stray write
    const long long cap = w.j_off ? w.j_off[g + 1] - base : 0;
    while (sp > 0) {
        const int k = stack[--sp];
        double d2 = 0.0;
        const double4 cm = w.com[k];
        for (int a = 0; a < 3; ++a) {
            const double c = a == 0 ? cm.x : a == 1 ? cm.y : cm.z;
            double d = 0.0;
            if (c < blo[a]) d = __dsub_rn(blo[a], c);
            else if (c > bhi[a]) d = __dsub_rn(c, bhi[a]);
            d2 = __dadd_rn(d2, __dmul_rn(d, d));
        }
        const double side = ldexp(span, -(int)w.lev[k]);
        const double side2 = __dmul_rn(side, side);
        const double lim = __dmul_rn(w.theta2, d2);
        const bool holds = w.first[k] <= i0 && i0 < w.first[k] + w.count[k];
        if (!holds && side2 < lim) {
            if (w.jlist) {
                if (cnt >= cap) {
                    report(w.status, kStatusBadIndex, 10);
                    break;
                }
                w.jlist[base + cnt] = (int)(w.n + k);
            }
            ++cnt;
        } else if (w.lev[k] == kLevels - 1 || w.count[k] <= w.nleaf) {
            if (w.jlist && cnt + w.count[k] > cap) {
                report(w.status, kStatusBadIndex, 10);
                break;
            }
            for (int j = w.first[k]; j < w.first[k] + w.count[k]; ++j) {
                if (w.jlist) w.jlist[base + cnt] = j;
                ++cnt;
            }
        } else {
            if (sp + w.childn[k] > kStack) {       // cannot happen: at most 8 per level
                report(w.status, kStatusBadIndex, 9);
                break;
            }
            for (int c = w.child0[k] + w.childn[k] - 1; c >= w.child0[k]; --c) stack[sp++] = c;
        }
    }
    if (w.jcount) w.jcount[g] = (unsigned)cnt;
}

__global__ void k_tree_widen(const unsigned *__restrict__ in, long long n, long long *__restrict__ out)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < n) out[k] = in[k];
}

// the pseudo-particles: (S / M, M), after the n particles of the j records
__global__ void k_tree_pseudo(const double *__restrict__ M, const double *__restrict__ S,
                              long long nnodes, double4 *__restrict__ out)
{
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= nnodes) return;
    const double m = M[k];
    out[k] = make_double4(__ddiv_rn(S[3 * k], m), __ddiv_rn(S[3 * k + 1], m),
                          __ddiv_rn(S[3 * k + 2], m), m);
}

// items: the groups cut into chunks of at most Bi particles; pairs = sum ni nj
__global__ void k_tree_items(const int *__restrict__ g_i0, const int *__restrict__ g_ni,
                             const unsigned *__restrict__ item_off, const long long *__restrict__ j_off,
                             long long ngroups, int Bi, GroupItem *__restrict__ items,
                             unsigned long long *__restrict__ pairs)
{
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned long long p = 0;
    if (g < ngroups) {
        const int ni = g_ni[g];
        unsigned o = item_off[g];
        for (int k = 0; k * Bi < ni; ++k) {
            GroupItem it;
            it.group = (int)g;
            it.i0 = g_i0[g] + k * Bi;
            it.ni = min(Bi, ni - k * Bi);
            it.pad = 0;
            items[o + k] = it;
        }
        p = (unsigned long long)ni * (unsigned long long)(j_off[g + 1] - j_off[g]);
    }
    for (int s = 16; s; s >>= 1) p += __shfl_xor_sync(0xffffffffu, p, s);
    if ((threadIdx.x & 31) == 0 && p) atomicAdd(pairs, p);
}

__global__ void k_tree_item_counts(const int *__restrict__ g_ni, long long ngroups, int Bi,
                                   unsigned *__restrict__ c)
{
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g > ngroups) return;
    c[g] = g < ngroups ? (unsigned)((g_ni[g] + Bi - 1) / Bi) : 0u;
}

unsigned blocks_of(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t tree_stage_keys(const double4 *jrec, long long n, TreeScratch &t, SortScratch &sort,
                            cudaStream_t st)
{
    k_tree_bbox_init<<<1, 32, 0, st>>>(t.bbox);
    k_tree_bbox<<<min(blocks_of(n), 1024u), 256, 0, st>>>(jrec, n, t.bbox);
    k_tree_span<<<1, 32, 0, st>>>(t.bbox, t.geo);
    k_tree_keys<<<blocks_of(n), 256, 0, st>>>(jrec, n, t.geo, sort.keys[0], sort.vals[0]);
    unsigned *ko = nullptr, *perm = nullptr;
    cudaError_t e = launch_radix_sort(sort.keys[0], sort.vals[0], n, 3 * kBits, sort, &ko, &perm, st);
    if (e != cudaSuccess) return e;
    cudaMemcpyAsync(t.key, ko, n * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(t.perm, perm, n * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    k_tree_gather<<<blocks_of(n), 256, 0, st>>>(jrec, t.perm, n, t.xs, t.xi0);
    // the run flags and their scans, every level
    for (int L = 0; L < kLevels; ++L) {
        unsigned *sc = t.scan + (size_t)L * (n + 1);
        k_tree_flags<<<blocks_of(n + 1), 256, 0, st>>>(t.key, n, 3 * (kBits - L), sc);
        if ((e = launch_excl_scan(sc, n + 1, sort.sums, st)) != cudaSuccess) return e;
        cudaMemcpyAsync(t.runs_dev + L, sc + n, sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    }
    return cudaGetLastError();
}

cudaError_t tree_stage_nodes(long long n, const long long *lev_off, int ncrit, TreeScratch &t,
                             SortScratch &sort, cudaStream_t st)
{
    for (int L = 0; L < kLevels; ++L) {
        const unsigned *sc = t.scan + (size_t)L * (n + 1);
        k_tree_starts<<<blocks_of(n), 256, 0, st>>>(t.key, sc, n, 3 * (kBits - L), lev_off[L], t.first);
    }
    for (int L = 0; L < kLevels; ++L) {
        const long long runs = lev_off[L + 1] - lev_off[L];
        const unsigned *next = L + 1 < kLevels ? t.scan + (size_t)(L + 1) * (n + 1) : nullptr;
        k_tree_nodes<<<blocks_of(runs), 256, 0, st>>>(lev_off[L], runs, n, next,
                                                      L + 1 < kLevels ? lev_off[L + 1] : 0, L,
                                                      t.first, t.count, t.child0, t.childn, t.lev);
    }
    {
        const long long L = kLevels - 1, runs = lev_off[L + 1] - lev_off[L];
        k_tree_moments_leaf<<<blocks_of(runs), 256, 0, st>>>(lev_off[L], runs, t.first, t.count, t.xs,
                                                             t.M, t.S);
    }
    for (int L = kLevels - 2; L >= 0; --L) {
        const long long runs = lev_off[L + 1] - lev_off[L];
        k_tree_moments_up<<<blocks_of(runs), 256, 0, st>>>(lev_off[L], runs, t.child0, t.childn,
                                                           t.M, t.S);
    }
    cudaMemsetAsync(t.gat, 0xff, n * sizeof(int), st);
    for (int L = 0; L < kLevels; ++L) {
        const long long runs = lev_off[L + 1] - lev_off[L];
        const unsigned *prev = L > 0 ? t.scan + (size_t)(L - 1) * (n + 1) : nullptr;
        k_tree_group_marks<<<blocks_of(runs), 256, 0, st>>>(lev_off[L], runs, L, prev,
                                                            L > 0 ? lev_off[L - 1] : 0, t.first,
                                                            t.count, ncrit, t.gat);
    }
    k_tree_group_flags<<<blocks_of(n + 1), 256, 0, st>>>(t.gat, n, t.gscan);
    cudaError_t e = launch_excl_scan(t.gscan, n + 1, sort.sums, st);
    if (e != cudaSuccess) return e;
    k_tree_groups<<<blocks_of(n + 1), 256, 0, st>>>(t.gat, t.gscan, n, t.count, t.xs, t.g_i0, t.g_ni,
                                                    t.gbox, t.i_off);
    cudaMemcpyAsync(t.runs_dev + kLevels, t.gscan + n, sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError();
}

cudaError_t tree_stage_walk(long long n, long long ngroups, double theta, int nleaf, bool fill,
                            TreeScratch &t, SortScratch &sort, int *status, cudaStream_t st)
{
    WalkArgs w{};
    w.n = n;
    w.ngroups = ngroups;
    w.g_i0 = t.g_i0;
    w.g_ni = t.g_ni;
    w.gbox = t.gbox;
    w.first = t.first;
    w.count = t.count;
    w.child0 = t.child0;
    w.childn = t.childn;
    w.lev = t.lev;
    w.com = t.jrec2 + n;       // the pseudo-particles, written before the walk
    w.theta2 = theta * theta;
    w.nleaf = nleaf;
    w.status = status;
    w.geo = t.geo;
    cudaError_t e = cudaSuccess;
    if (!fill) {
        w.jcount = t.jcount;
        k_tree_walk<<<blocks_of(ngroups), 256, 0, st>>>(w);
        cudaMemsetAsync(t.jcount + ngroups, 0, sizeof(unsigned), st);
        if ((e = launch_excl_scan(t.jcount, ngroups + 1, sort.sums, st)) != cudaSuccess) return e;
        k_tree_widen<<<blocks_of(ngroups + 1), 256, 0, st>>>(t.jcount, ngroups + 1, t.j_off);
    } else {
        w.j_off = t.j_off;
        w.jlist = t.jlist;
        k_tree_walk<<<blocks_of(ngroups), 256, 0, st>>>(w);
    }
    return cudaGetLastError();
}

// the j records: particles in key order, then one pseudo-particle per node
// (centre of mass S / M, mass); the walk reads the centres from here
cudaError_t tree_stage_jrec(long long n, long long nnodes, TreeScratch &t, cudaStream_t st)
{
    cudaMemcpyAsync(t.jrec2, t.xs, n * sizeof(double4), cudaMemcpyDeviceToDevice, st);
    k_tree_pseudo<<<blocks_of(nnodes), 256, 0, st>>>(t.M, t.S, nnodes, t.jrec2 + n);
    return cudaGetLastError();
}

cudaError_t tree_stage_records(long long n, long long nnodes, long long ngroups, int Bi,
                               TreeScratch &t, SortScratch &sort, cudaStream_t st)
{
    k_tree_item_counts<<<blocks_of(ngroups + 1), 256, 0, st>>>(t.g_ni, ngroups, Bi, t.item_off);
    cudaError_t e = launch_excl_scan(t.item_off, ngroups + 1, sort.sums, st);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(t.pairs, 0, sizeof(unsigned long long), st);
    k_tree_items<<<blocks_of(ngroups), 256, 0, st>>>(t.g_i0, t.g_ni, t.item_off, t.j_off, ngroups, Bi,
                                                    t.items, t.pairs);
    cudaMemcpyAsync(t.runs_dev + kLevels + 1, t.item_off + ngroups, sizeof(unsigned),
                    cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError();
}

}  // namespace pg
