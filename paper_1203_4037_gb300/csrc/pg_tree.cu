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
//    or the finest level) gives its particles, else N is opened;
//  - a list is breadth first: the entries of level 0's decisions, then
//    level 1's, ..., each level's in key order (the paper fixes the list as
//    a set; the order only changes the rounding of the sums).
// Every FP64 operation of the decisions uses an explicitly rounded
// intrinsic (no fused multiply-add), so the lists are reproducible bit for
// bit by any implementation that rounds the same operations the same way.
#include <algorithm>

#include "pg_device.cuh"

namespace pg {

namespace {

constexpr int kLevels = 11;      // levels 0 .. 10
constexpr int kBits = 10;        // key bits per axis

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
    // the block's extremes, then one atomic per value and block (a warp's
    // own atomics on the same six words serialised in L2)
    __shared__ unsigned long long part[32][6];
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            part[w][a] = lo[a];
            part[w][3 + a] = hi[a];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int v = threadIdx.x;
        unsigned long long r = part[0][v];
        for (int k = 1; k < nw; ++k) r = v < 3 ? min(r, part[k][v]) : max(r, part[k][v]);
        if (v < 3) atomicMin(&bb[v], r);
        else atomicMax(&bb[v], r);
    }
}

// geo = {lo_x, lo_y, lo_z, span, 1024 / span rounded}
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
    geo[4] = __ddiv_rn(1024.0, span);
}

__device__ __forceinline__ unsigned spread10(unsigned v)
{
    unsigned r = 0;
#pragma unroll
    for (int b = 0; b < kBits; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

// The cell index q = floor(RN(d / span) 1024) of d = RN(x - lo) >= 0 per
// axis. RN(d / span) 1024 is z = 1024 d / span rounded to nearest (the
// scaling is exact), so q = floor(z) except where z lies within half an
// ulp (at most 2^-43, z <= 1024) below an integer, which it rounds up to.
// t = RN(d RN(1024 / span)) is within 2^-41 of z (two roundings of
// relative 2^-53, z <= 1024); where t is more than 2^-40 from every
// integer, no integer lies between z and t and none within half an ulp
// above z, so q = floor(t). Nearer an integer (or t not finite, a span so
// small that 1024 / span overflows) the quotient is formed exactly. The
// keys are those of the correctly rounded division, bit for bit, with one
// FP64 multiply per axis instead of a division. The integer part of t and
// its distance to the integers on either side come from t's bits (FP64
// instructions issue at about two per SM-clock on this GPU, integer ones
// at 64): t = mant 2^(e - 52), and for 0 <= e <= 10 the low sh = 52 - e
// bits of mant are t's fraction in units of 2^-sh.
__device__ __forceinline__ unsigned cell_of(double x, double lo, double span, double c1024)
{
    const double d = __dsub_rn(x, lo);
    const double t = __dmul_rn(d, c1024);
    const unsigned long long u = (unsigned long long)__double_as_longlong(t);
    const int e = (int)((u >> 52) & 0x7ffu) - 1023;
    const unsigned long long f52 = u & ((1ull << 52) - 1);
    bool near;          // within 2^-40 of an integer, or outside [0, 2048)
    unsigned q = 0;
    if ((u >> 63) || e > 10) {
        near = true;                                    // negative, >= 2048, inf or NaN
    } else if (e < 0) {
        // q = 0; near 0: t <= 2^-40; near 1: t >= 1 - 2^-40 (e = -1 and
        // 1 + f52 2^-52 >= 2 - 2^-39)
        near = e < -40 || (e == -40 && f52 == 0) || (e == -1 && f52 >= (1ull << 52) - (1ull << 13));
    } else {
        const int sh = 52 - e;                          // 42 .. 52
        const unsigned long long mant = f52 | (1ull << 52);
        const unsigned long long fr = mant & ((1ull << sh) - 1), tol = 1ull << (sh - 40);
        q = (unsigned)(mant >> sh);
        near = fr <= tol || fr >= (1ull << sh) - tol;
    }
    if (near) {
        const double f = floor(__dmul_rn(__ddiv_rn(d, span), 1024.0));
        return f >= 1023.0 ? 1023u : (unsigned)f;
    }
    return q >= 1023u ? 1023u : q;
}

__global__ void k_tree_keys(const double4 *__restrict__ x, long long n, const double *geo,
                            unsigned *__restrict__ key, unsigned *__restrict__ idx)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 v = x[i];
    const double c[3] = {v.x, v.y, v.z};
    const double span = geo[3], c1024 = geo[4];
    unsigned k = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) k |= spread10(cell_of(c[a], geo[a], span, c1024)) << (2 - a);
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
// Level L's run flags sit in scan[L (n + 1) .. L (n + 1) + n] (a 1 at each
// run's first particle, 0 at position n), and one more 0 ends the array.
// One exclusive scan over the whole array numbers every node: the entry at a
// run's first particle is the runs of all lower levels plus the runs of its
// own level before it, its node index.
__global__ void k_tree_flags(const unsigned *__restrict__ key, long long n, unsigned *__restrict__ scan)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int L = blockIdx.y;
    if (i > n) return;
    const int sh = 3 * (kBits - L);
    unsigned *flag = scan + (long long)L * (n + 1);
    flag[i] = i == n ? 0u : (i == 0 || (key[i] >> sh) != (key[i - 1] >> sh)) ? 1u : 0u;
    if (L == kLevels - 1 && i == n) scan[(long long)kLevels * (n + 1)] = 0u;
}

// the level offsets and the node count, checked against the room the host
// gave the nodes and against the records' 27-bit index limit
__global__ void k_tree_level_meta(const unsigned *__restrict__ scan, long long n, int npseudo,
                                  long long cap_nodes, TreeMeta *m)
{
    if (threadIdx.x != 0) return;
    long long o = 0;
    for (int L = 0; L < kLevels; ++L) {
        m->lev_off[L] = o;
        o += scan[(long long)(L + 1) * (n + 1)] - scan[(long long)L * (n + 1)];
    }
    m->lev_off[kLevels] = o;
    m->nnodes = o;
    int f = 0;
    if (o > cap_nodes) f |= kTreeRoomNodes;
    if (n + npseudo * o >= (1LL << 27)) f |= kTreeTooLarge;
    m->flags |= f;
}

// each run's first particle, every level
__global__ void k_tree_starts(const TreeMeta *__restrict__ m, const unsigned *__restrict__ key,
                              const unsigned *__restrict__ scan, long long n, int *__restrict__ first)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int L = blockIdx.y;
    if (i >= n || m->flags) return;
    const int sh = 3 * (kBits - L);
    if (i == 0 || (key[i] >> sh) != (key[i - 1] >> sh)) first[scan[(long long)L * (n + 1) + i]] = (int)i;
}

// counts, levels and children, every level (blockIdx.y; level offsets read
// on the device, the grid strides over the level): the children of a node
// with particles [f, e) are the next level's runs from the one at f to the
// one at e
__global__ void k_tree_nodes(const TreeMeta *__restrict__ m, long long n, const unsigned *__restrict__ scan,
                             const int *__restrict__ first, int *__restrict__ count,
                             int *__restrict__ child0, int *__restrict__ childn,
                             unsigned char *__restrict__ lev)
{
    const int L = blockIdx.y;
    if (m->flags) return;
    const long long o = m->lev_off[L], runs = m->lev_off[L + 1] - o;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < runs;
         r += (long long)gridDim.x * blockDim.x) {
        const long long k = o + r;
        const int f = first[k];
        const int e = r + 1 < runs ? first[k + 1] : (int)n;
        count[k] = e - f;
        lev[k] = (unsigned char)L;
        if (L + 1 < kLevels) {
            const unsigned *next = scan + (long long)(L + 1) * (n + 1);
            child0[k] = (int)next[f];
            childn[k] = (int)(next[e] - next[f]);
        } else {
            child0[k] = 0;
            childn[k] = 0;
        }
    }
}

// Per node, once its mass M and first moment S are summed: the centre of
// mass (S / M, M), the walk's record, with monopoles the pseudo-particle
// itself, and with quadrupoles the second moment about the centre
struct NodeOut {
    double4 *com;        // centre of mass (S / M, M)
    double4 *mono;       // monopole j records, or nullptr
    TreeNodeW *nodew;    // the walk's records
    double *T;           // second moments {xx, xy, xz, yy, yz, zz}, or nullptr
};

__device__ __forceinline__ double4 node_finish(long long k, double m, double s0, double s1, double s2,
                                               const int *first, const int *count, const int *child0,
                                               const int *childn, const NodeOut &o)
{
    const double4 c = make_double4(__ddiv_rn(s0, m), __ddiv_rn(s1, m), __ddiv_rn(s2, m), m);
    o.com[k] = c;
    if (o.mono) o.mono[k] = c;
    TreeNodeW w;
    w.cx = __double2float_rn(c.x);
    w.cy = __double2float_rn(c.y);
    w.cz = __double2float_rn(c.z);
    w.pad = 0.f;
    w.first = first[k];
    w.count = count[k];
    w.child0 = child0[k];
    w.childn = childn[k];
    o.nodew[k] = w;
    return c;
}

// one node of the finest level
__device__ __forceinline__ void moments_leaf_one(long long k, const int *__restrict__ first,
                                                 const int *__restrict__ count, const int *__restrict__ child0,
                                                 const int *__restrict__ childn, const double4 *__restrict__ xs,
                                                 double *__restrict__ M, double *__restrict__ S, const NodeOut &o)
{
    double m = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const int f = first[k], e = f + count[k];
    for (int i = f; i < e; ++i) {
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
    const double4 c = node_finish(k, m, s0, s1, s2, first, count, child0, childn, o);
    if (!o.T) return;
    double t[6] = {0, 0, 0, 0, 0, 0};
    for (int i = f; i < e; ++i) {
        const double4 v = xs[i];
        const double y0 = v.x - c.x, y1 = v.y - c.y, y2 = v.z - c.z;
        t[0] += v.w * y0 * y0;
        t[1] += v.w * y0 * y1;
        t[2] += v.w * y0 * y2;
        t[3] += v.w * y1 * y1;
        t[4] += v.w * y1 * y2;
        t[5] += v.w * y2 * y2;
    }
    for (int q = 0; q < 6; ++q) o.T[6 * k + q] = t[q];
}

// the finest level from its particles, in key order; T = sum m (x - c)(x - c)^T
__global__ void k_tree_moments_leaf(const TreeMeta *__restrict__ tm, const int *__restrict__ first,
                                    const int *__restrict__ count, const int *__restrict__ child0,
                                    const int *__restrict__ childn, const double4 *__restrict__ xs,
                                    double *__restrict__ M, double *__restrict__ S, NodeOut o)
{
    if (tm->flags) return;
    const long long off = tm->lev_off[kLevels - 1], runs = tm->lev_off[kLevels] - off;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < runs;
         r += (long long)gridDim.x * blockDim.x)
        moments_leaf_one(off + r, first, count, child0, childn, xs, M, S, o);
}

// one node above the finest level
__device__ __forceinline__ void moments_up_one(long long k, const int *__restrict__ first,
                                               const int *__restrict__ count, const int *__restrict__ child0,
                                               const int *__restrict__ childn, double *__restrict__ M,
                                               double *__restrict__ S, const NodeOut &o)
{
    double m = 0.0, s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const int c0 = child0[k], c1 = c0 + childn[k];
    for (int ch = c0; ch < c1; ++ch) {
        m = __dadd_rn(m, M[ch]);
        s0 = __dadd_rn(s0, S[3 * ch]);
        s1 = __dadd_rn(s1, S[3 * ch + 1]);
        s2 = __dadd_rn(s2, S[3 * ch + 2]);
    }
    M[k] = m;
    S[3 * k] = s0;
    S[3 * k + 1] = s1;
    S[3 * k + 2] = s2;
    const double4 c = node_finish(k, m, s0, s1, s2, first, count, child0, childn, o);
    if (!o.T) return;
    double t[6] = {0, 0, 0, 0, 0, 0};
    for (int ch = c0; ch < c1; ++ch) {
        const double4 cc = o.com[ch];
        const double y0 = cc.x - c.x, y1 = cc.y - c.y, y2 = cc.z - c.z;
        const double *tc = o.T + 6 * (long long)ch;
        t[0] += tc[0] + cc.w * y0 * y0;
        t[1] += tc[1] + cc.w * y0 * y1;
        t[2] += tc[2] + cc.w * y0 * y2;
        t[3] += tc[3] + cc.w * y1 * y1;
        t[4] += tc[4] + cc.w * y1 * y2;
        t[5] += tc[5] + cc.w * y2 * y2;
    }
    for (int q = 0; q < 6; ++q) o.T[6 * k + q] = t[q];
}

// the levels above from their children in order; T moved to the parent's
// centre by the parallel-axis rule, T = sum T_ch + M_ch (c_ch - c)(c_ch - c)^T
__global__ void k_tree_moments_up(const TreeMeta *__restrict__ tm, int L, const int *__restrict__ first,
                                  const int *__restrict__ count, const int *__restrict__ child0,
                                  const int *__restrict__ childn, double *__restrict__ M,
                                  double *__restrict__ S, NodeOut o)
{
    if (tm->flags) return;
    const long long off = tm->lev_off[L], runs = tm->lev_off[L + 1] - off;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < runs;
         r += (long long)gridDim.x * blockDim.x)
        moments_up_one(off + r, first, count, child0, childn, M, S, o);
}

// The coarse levels L0, L0 - 1, ..., 0 in one block, level after level
// (the barrier makes a level's moments visible to the next): they hold few
// nodes, and a launch each was mostly launch and latency.
__global__ void __launch_bounds__(1024) k_tree_moments_top(const TreeMeta *__restrict__ tm, int L0,
                                                          const int *__restrict__ first,
                                                          const int *__restrict__ count,
                                                          const int *__restrict__ child0,
                                                          const int *__restrict__ childn, double *__restrict__ M,
                                                          double *__restrict__ S, NodeOut o)
{
    if (tm->flags) return;
    for (int L = L0; L >= 0; --L) {
        const long long off = tm->lev_off[L], runs = tm->lev_off[L + 1] - off;
        for (long long r = threadIdx.x; r < runs; r += blockDim.x)
            moments_up_one(off + r, first, count, child0, childn, M, S, o);
        __syncthreads();
    }
}

// group marks at their first particle: gat[i] = node, else -1 (set before)
// groups: nodes with at most ncrit particles whose parent (the previous
// level's node holding the first particle) has more, and finest-level nodes
// whose parent has more; marked at their first particle, every level
__global__ void k_tree_group_marks(const TreeMeta *__restrict__ m, long long n,
                                   const unsigned *__restrict__ scan, const int *__restrict__ first,
                                   const int *__restrict__ count, int ncrit, int *__restrict__ gat)
{
    const int L = blockIdx.y;
    if (m->flags) return;
    const long long o = m->lev_off[L], runs = m->lev_off[L + 1] - o;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < runs;
         r += (long long)gridDim.x * blockDim.x) {
        const long long k = o + r;
        long long pc = -1;
        if (L > 0) {
            const long long p = (long long)scan[(long long)(L - 1) * (n + 1) + first[k] + 1] - 1;
            pc = count[p];
        }
        const bool grp = (count[k] <= ncrit && (L == 0 || pc > ncrit)) ||
                         (L == kLevels - 1 && pc > ncrit);
        if (grp) gat[first[k]] = (int)k;
    }
}

__global__ void k_tree_group_flags(const int *__restrict__ gat, long long n, unsigned *__restrict__ f)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i > n) return;
    f[i] = i < n && gat[i] >= 0 ? 1u : 0u;
}

// groups in particle order; i_off[g] (ngroups + 1 entries); the group count
// (checked against the room the host gave the groups)
__global__ void k_tree_groups(TreeMeta *m, long long cap_groups, const int *__restrict__ gat,
                              const unsigned *__restrict__ gscan, long long n, const int *__restrict__ count,
                              int *__restrict__ g_i0, int *__restrict__ g_ni, long long *__restrict__ i_off)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long ng = gscan[n];
    if (ng > cap_groups) {
        if (i == 0) atomicOr(&m->flags, kTreeRoomGroups);
        return;
    }
    if (i == n) {
        i_off[ng] = n;
        m->ngroups = ng;
    }
    if (i >= n || gat[i] < 0) return;
    const unsigned g = gscan[i];
    g_i0[g] = (int)i;
    g_ni[g] = count[gat[i]];
    i_off[g] = i;
}

// a group's bounding box, one warp per group: FP64, and rounded to nearest
// FP32 for the walk's pre-test. Minima and maxima are taken on the
// order-preserving integer images of the coordinates (integer compares run
// at full rate; FP64 compares do not)
__global__ void k_tree_gbox(const int *__restrict__ g_i0, const int *__restrict__ g_ni,
                            const TreeMeta *__restrict__ m, const double4 *__restrict__ xs,
                            double *__restrict__ gbox, float4 *__restrict__ gboxf, double4 *__restrict__ ctr)
{
    const long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (m->flags || g >= m->ngroups) return;
    const int i0 = g_i0[g], ni = g_ni[g];
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    for (int k = i0 + lane; k < i0 + ni; k += 32) {
        const double4 v = xs[k];
        const unsigned long long c[3] = {ord_of(v.x), ord_of(v.y), ord_of(v.z)};
        for (int a = 0; a < 3; ++a) {
            lo[a] = c[a] < lo[a] ? c[a] : lo[a];
            hi[a] = c[a] > hi[a] ? c[a] : hi[a];
        }
    }
    for (int s = 16; s; s >>= 1)
        for (int a = 0; a < 3; ++a) {
            const unsigned long long l = __shfl_xor_sync(0xffffffffu, lo[a], s);
            const unsigned long long h = __shfl_xor_sync(0xffffffffu, hi[a], s);
            lo[a] = l < lo[a] ? l : lo[a];
            hi[a] = h > hi[a] ? h : hi[a];
        }
    if (lane == 0) {
        double dl[3], dh[3];
        for (int a = 0; a < 3; ++a) {
            dl[a] = val_of(lo[a]);
            dh[a] = val_of(hi[a]);
            gbox[6 * g + a] = dl[a];
            gbox[6 * g + 3 + a] = dh[a];
        }
        gboxf[2 * g] = make_float4(__double2float_rn(dl[0]), __double2float_rn(dl[1]),
                                   __double2float_rn(dl[2]), 0.f);
        gboxf[2 * g + 1] = make_float4(__double2float_rn(dh[0]), __double2float_rn(dh[1]),
                                       __double2float_rn(dh[2]), 0.f);
        // the centre the force kernel takes its FP32 offsets from: the box's
        // midpoint
        ctr[g] = make_double4(0.5 * (dl[0] + dh[0]), 0.5 * (dl[1] + dh[1]), 0.5 * (dl[2] + dh[2]), 0.0);
    }
}

// The walk runs level by level over all groups at once. The frontier of
// level L is a run of (group, node) pairs, sorted by group and then node,
// stored with every other level's frontier ("visits"); one thread decides
// one pair, a scan of the opened children places the next level's
// frontier, and the decisions' entries are placed afterwards. A group's
// list comes out breadth first: its level-0 entries, then level 1, ..., in
// key order within a level.
//
// The opening test is decided in FP32 where that is certain. With every
// coordinate (particles, centres of mass, box corners) at most R in
// magnitude and u = 2^-24, the FP32 distance per axis, from operands rounded
// to nearest, is within 4.1 u R of the exact one; e = 8 u R bounds it.
// Intervals for d^2 and theta^2 d^2 taken with round-down and round-up
// arithmetic (and a 2^-23 relative widening, far above the FP64 test's own
// rounding) then contain the FP64 test's theta^2 d^2. If side^2 lies
// outside the interval the answer is the FP64 test's; inside, the FP64 test
// runs. The bounds assume magnitudes where nothing overflows or falls below
// the normal range; elsewhere every test is FP64.
struct LevelArgs {
    long long n, ngroups;
    long long o, nf;           // this level's frontier: visits [o, o + nf)
    int L;
    const int *g_i0;
    const double *gbox;
    const float4 *gboxf;
    const TreeNodeW *nodew;
    const double4 *com;        // per node: centre of mass S / M, mass (FP64)
    const WalkFilter *filt;
    int nleaf;
    int npseudo;               // entries of an accepted node: 1 or 3
    const int *vg;             // visits: group
    int *vk;                   // visits: node, ~node once accepted
    unsigned *ve;              // visits: entries the decision emits
    unsigned *vc;              // this level: children the decision opens (nf + 1)
    unsigned *seg;             // per level and group: visits [first, end)
    unsigned long long *ent;   // 64-bit sum of the entries
    double theta2;
};

__global__ void k_walk_filter(const double *geo, double theta2, WalkFilter *f)
{
    if (threadIdx.x != 0) return;
    const double span = geo[3];
    double R = 0.0;
    for (int a = 0; a < 3; ++a) R = fmax(R, fabs(geo[a]) + span);
    R = R * (1.0 + 0x1p-20);
    for (int L = 0; L < kLevels; ++L) {
        const double side = ldexp(span, -L);
        const double s2 = __dmul_rn(side, side);
        f->s2[L] = s2;
        f->s2lo[L] = __double2float_rd(s2);
        f->s2hi[L] = __double2float_ru(s2);
    }
    f->e = __double2float_ru(R * 0x1p-21);
    f->t2lo = __double2float_rd(theta2);
    f->t2hi = __double2float_ru(theta2);
    f->on = R >= 0x1p-20 && R <= 0x1p60 && span >= R * 0x1p-30 &&
            (theta2 == 0.0 || (theta2 >= 0x1p-40 && theta2 <= 0x1p40));
}

// the level walk's start: every group at the root, the entry sum at zero
// (a group walk that ran out of queue before it counted some entries)
__global__ void k_walk_init(long long ngroups, int *vg, int *vk, TreeMeta *m)
{
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g < ngroups) {
        vg[g] = (int)g;
        vk[g] = 0;          // the root
    }
    if (g == 0) {
        m->ent = 0ull;
        m->flags &= ~kTreeWalkQueue;
    }
}

// the FP32 bounds of one axis' squared distance, added into [lo2, hi2]
__device__ __forceinline__ void axis_bounds(float c, float lo, float hi, float e, float &lo2,
                                            float &hi2)
{
    const float d = c < lo ? lo - c : c > hi ? c - hi : 0.f;
    const float dl = fmaxf(__fsub_rd(d, e), 0.f), dh = __fadd_ru(d, e);
    lo2 = __fadd_rd(lo2, __fmul_rd(dl, dl));
    hi2 = __fadd_ru(hi2, __fmul_ru(dh, dh));
}

// The opening decision for node k of level L (record nd) and a group whose
// first particle is i0, with its box in FP32 (gbf: low, high corner) and
// FP64 (bx: low x, y, z, high x, y, z): true where the node is taken as
// its pseudo-particles. Both walks decide with this one function.
__device__ __forceinline__ bool walk_accepts(const WalkFilter &F, int L, const TreeNodeW &nd, int k, int i0,
                                             const float4 *gbf, const double *bx, const double4 *com,
                                             double theta2)
{
    if (nd.first <= i0 && i0 < nd.first + nd.count) return false;     // it holds the group
    int verdict = 0;                   // 1 accept, -1 not, 0 undecided
    if (F.on) {
        const float4 bl = gbf[0], bh = gbf[1];
        float lo2 = 0.f, hi2 = 0.f;
        axis_bounds(nd.cx, bl.x, bh.x, F.e, lo2, hi2);
        axis_bounds(nd.cy, bl.y, bh.y, F.e, lo2, hi2);
        axis_bounds(nd.cz, bl.z, bh.z, F.e, lo2, hi2);
        const float limlo = __fmul_rd(__fmul_rd(F.t2lo, lo2), 0x1.fffffcp-1f);
        const float limhi = __fmul_ru(__fmul_ru(F.t2hi, hi2), 0x1.000002p+0f);
        if (F.s2hi[L] < limlo) verdict = 1;
        else if (F.s2lo[L] >= limhi) verdict = -1;
    }
    if (verdict == 0) {
        // the FP64 test, rounded operation by operation
        const double4 cm = com[k];
        double d2 = 0.0;
        for (int x = 0; x < 3; ++x) {
            const double c = x == 0 ? cm.x : x == 1 ? cm.y : cm.z;
            const double lo = bx[x], hi = bx[3 + x];
            double d = 0.0;
            if (c < lo) d = __dsub_rn(lo, c);
            else if (c > hi) d = __dsub_rn(c, hi);
            d2 = __dadd_rn(d2, __dmul_rn(d, d));
        }
        verdict = F.s2[L] < __dmul_rn(theta2, d2) ? 1 : -1;
    }
    return verdict > 0;
}

__global__ void k_walk_test(LevelArgs a)
{
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    unsigned long long e64 = 0;
    if (q < a.nf) {
        const long long v = a.o + q;
        const int g = a.vg[v], k = a.vk[v];
        const TreeNodeW nd = a.nodew[k];
        const bool accept = walk_accepts(*a.filt, a.L, nd, k, a.g_i0[g], a.gboxf + 2 * (long long)g,
                                         a.gbox + 6 * (long long)g, a.com, a.theta2);
        unsigned e = 0, c = 0;
        if (accept) {
            e = (unsigned)a.npseudo;
            a.vk[v] = ~k;
        } else if (a.L == kLevels - 1 || nd.count <= a.nleaf) {
            e = (unsigned)nd.count;
        } else {
            c = (unsigned)nd.childn;
        }
        a.ve[v] = e;
        a.vc[q] = c;
        e64 = e;
        // the group's run of visits in this level
        unsigned *sg = a.seg + (2 * (long long)a.L) * a.ngroups;
        if (q == 0 || a.vg[v - 1] != g) sg[g] = (unsigned)v;
        if (q + 1 == a.nf || a.vg[v + 1] != g) sg[a.ngroups + g] = (unsigned)(v + 1);
    } else if (q == a.nf) {
        a.vc[q] = 0u;
    }
    for (int s = 16; s; s >>= 1) e64 += __shfl_xor_sync(0xffffffffu, e64, s);
    if ((threadIdx.x & 31) == 0 && e64) atomicAdd(a.ent, e64);
}

// the opened nodes' children, in order, after this level's frontier
__global__ void k_walk_expand(const TreeNodeW *__restrict__ nodew, long long o, long long nf,
                              const unsigned *__restrict__ vc, int *vg, int *vk)
{
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= nf) return;
    const unsigned c = vc[q + 1] - vc[q];
    if (!c) return;
    const long long v = o + q, dst = o + nf + vc[q];
    const int g = vg[v], ch0 = nodew[vk[v]].child0;
    for (unsigned t = 0; t < c; ++t) {
        vg[dst + t] = g;
        vk[dst + t] = ch0 + (int)t;
    }
}

// entries per group: its visits' entries over all levels (ve scanned)
__global__ void k_walk_count(long long ngroups, int nlev, const unsigned *__restrict__ seg,
                             const unsigned *__restrict__ ve, unsigned *__restrict__ jcount)
{
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g > ngroups) return;
    unsigned s = 0;
    if (g < ngroups)
        for (int L = 0; L < nlev; ++L)
            s += ve[seg[(2 * L + 1) * ngroups + g]] - ve[seg[(2 * L) * ngroups + g]];
    jcount[g] = s;
}

// list offsets, and per group and level the shift from the scanned visit
// order to the list position
__global__ void k_walk_base(long long ngroups, int nlev, const unsigned *__restrict__ jscan,
                            const unsigned *__restrict__ seg, const unsigned *__restrict__ ve,
                            long long *__restrict__ j_off, long long *__restrict__ base,
                            TreeMeta *m)
{
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g > ngroups) return;
    long long off = jscan[g];
    j_off[g] = off;
    if (g == ngroups) {
        m->nlist = off;    // the list length, beside the entry sum
        return;
    }
    for (int L = 0; L < nlev; ++L) {
        const unsigned s0 = ve[seg[(2 * L) * ngroups + g]], s1 = ve[seg[(2 * L + 1) * ngroups + g]];
        base[L * ngroups + g] = off - (long long)s0;
        off += s1 - s0;
    }
}

// the entries of level L's visits [o, o + nf)
__global__ void k_walk_fill(int L, long long o, long long nf, long long n, long long ngroups,
                            int npseudo, const int *__restrict__ vg, const int *__restrict__ vk,
                            const unsigned *__restrict__ ve, const long long *__restrict__ base,
                            const long long *__restrict__ j_off, const TreeNodeW *__restrict__ nodew,
                            int *__restrict__ jlist, int *status)
{
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= nf) return;
    const long long v = o + q;
    const unsigned e = ve[v + 1] - ve[v];
    if (!e) return;
    const int g = vg[v], k = vk[v];
    const long long dst = base[L * ngroups + g] + ve[v];
    // the entries stay inside the group's list; anything else is reported
    if (dst < j_off[g] || dst + e > j_off[g + 1] || (k < 0 && e != (unsigned)npseudo)) {
        report(status, kStatusBadIndex, 10);
        return;
    }
    if (k < 0) {
        const int p0 = (int)(n + (long long)npseudo * ~k);
        for (int q = 0; q < npseudo; ++q) jlist[dst + q] = p0 + q;
    } else {
        const int f = nodew[k].first;
        for (unsigned t = 0; t < e; ++t) jlist[dst + t] = f + (int)t;
    }
}

// The group walk: one warp walks one group's tree at a time, breadth first,
// and needs neither the visit arrays nor a launch per level. The warp keeps
// the nodes its group opened at the level before, as (first child, number
// of children) packed in one word (child0 << 3 | childn - 1: child0 < 2^27,
// 1 <= childn <= 8), in a shared-memory queue. Per level it lays their
// children out in order (at most 256 per 32 opened nodes), decides 32 at a
// time with walk_accepts, appends the nodes it opens to the next queue in
// order (ballot), and gives the decisions' entries consecutive list
// positions (a warp scan). Children of nodes in key order come in key
// order, so the list is the level walk's: each level's entries in key
// order, level after level. A level that opens more than kGroupWalkQ nodes
// stops the pass (flag kTreeWalkQueue) and the call takes the level walk.
// The count pass gives each group's entries; the fill pass writes them.
constexpr int kGwWarps = 8;                       // warps per block
constexpr int kGwKids = 256;                      // children of 32 opened nodes
constexpr int kGwU = 2;                           // chunks of 32 children a step decides
constexpr int kGwWords = 2 * kGroupWalkQ + kGwKids;   // shared words per warp

struct GroupWalkArgs {
    long long n;
    TreeMeta *meta;
    const int *g_i0;
    const double *gbox;
    const float4 *gboxf;
    const TreeNodeW *nodew;
    const double4 *com;
    const WalkFilter *filt;
    int nleaf, npseudo;
    double theta2;
    unsigned *jcount;          // count pass: entries per group, 0 at ngroups
    const long long *j_off;    // fill pass: the list offsets
    int *jlist;                // fill pass: the lists
    int *status;               // fill pass: an entry outside its group's list
    // the count pass's record of each group's emitting nodes, in list order
    // (bit 31 set: accepted, its pseudo-particles; clear: a leaf, its
    // particles), which the fill pass expands instead of walking again;
    // emit == nullptr: not recorded
    unsigned *wscratch;        // kGroupWalkScratch per warp of the grid
    unsigned *emit;            // emit_cap: every group's emitters
    long long emit_cap;
    int2 *gemit;               // per group: first emitter and count (first -1: walk again)
};

__device__ __forceinline__ unsigned warp_incl_scan(unsigned v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// the end of a group's count pass: its nemit emitters (in the warp's
// scratch) get a slice of the emitter array, or first = -1 when they
// overflowed the scratch or the array's room (the fill pass then walks the
// group again)
__device__ __forceinline__ void place_emitters(const GroupWalkArgs &a, TreeMeta *m, const unsigned *scr,
                                               unsigned nemit, long long g, int lane)
{
    __syncwarp();                           // every lane's scratch writes visible
    long long first = -1;
    if (nemit <= (unsigned)kGroupWalkScratch) {
        unsigned long long f = 0;
        if (lane == 0) f = atomicAdd(&m->emit_next, nemit);
        f = __shfl_sync(0xffffffffu, f, 0);
        // the first emitter is kept as an int
        if (f + nemit <= (unsigned long long)min(a.emit_cap, 0x7fffffffLL)) first = (long long)f;
    }
    if (first >= 0)
        for (unsigned t = lane; t < nemit; t += 32) a.emit[first + t] = scr[t];
    if (lane == 0) a.gemit[g] = make_int2(first >= 0 ? (int)first : -1, (int)nemit);
    __syncwarp();
}

// the fill pass of a recorded group: its cnt emitters from emit[first]
// expanded into list entries from pos, in order
__device__ __forceinline__ void expand_emitters(const GroupWalkArgs &a, int first, int cnt, long long pos,
                                                long long hi, int lane)
{
    for (int b = 0; b < cnt; b += 32) {
        unsigned e = 0;
        int p0 = 0;
        if (b + lane < cnt) {
            const unsigned code = a.emit[first + b + lane];
            const int k = (int)(code & 0x7fffffffu);
            if (code >> 31) {
                e = (unsigned)a.npseudo;
                p0 = (int)(a.n + (long long)a.npseudo * k);
            } else {
                const TreeNodeW nd = a.nodew[k];
                e = (unsigned)nd.count;
                p0 = nd.first;
            }
        }
        const unsigned ei = warp_incl_scan(e, lane);
        if (e) {
            const long long d = pos + (ei - e);
            if (d + e > hi) report(a.status, kStatusBadIndex, 13);
            else
                for (unsigned t = 0; t < e; ++t) a.jlist[d + t] = p0 + (int)t;
        }
        pos += __shfl_sync(0xffffffffu, ei, 31);
    }
    if (pos != hi && lane == 0) report(a.status, kStatusBadIndex, 12);
}

template <bool FILL>
__global__ void __launch_bounds__(32 * kGwWarps) k_walk_groups(GroupWalkArgs a)
{
    __shared__ unsigned sq[kGwWarps * kGwWords];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    TreeMeta *m = a.meta;
    if (m->flags) return;
    const long long ng = m->ngroups;
    if (!FILL && blockIdx.x == 0 && threadIdx.x == 0) a.jcount[ng] = 0u;
    unsigned *qa = sq + w * kGwWords, *qb = qa + kGroupWalkQ, *kids = qb + kGroupWalkQ;
    const unsigned below = (1u << lane) - 1u;
    const WalkFilter &F = *a.filt;
    unsigned long long ent = 0;
    unsigned qmax = 0;
    bool over = false;
    unsigned *scr = !FILL && a.emit
                        ? a.wscratch + ((long long)blockIdx.x * kGwWarps + w) * kGroupWalkScratch
                        : nullptr;
    for (;;) {
        unsigned gq = 0;
        if (lane == 0) gq = *(volatile int *)&m->flags ? 0xffffffffu : atomicAdd(&m->next[FILL ? 1 : 0], 1u);
        const long long g = __shfl_sync(0xffffffffu, gq, 0);
        if (g >= ng) break;
        const int i0 = a.g_i0[g];
        const float4 *gbf = a.gboxf + 2 * g;
        const double *bx = a.gbox + 6 * g;
        const long long lo = FILL ? a.j_off[g] : 0, hi = FILL ? a.j_off[g + 1] : 0;
        long long pos = lo;
        if (FILL && a.emit) {
            // the count pass recorded this group's emitters: expand them
            const int2 ge = a.gemit[g];
            if (ge.x >= 0) {
                expand_emitters(a, ge.x, ge.y, pos, hi, lane);
                continue;
            }
        }
        unsigned nemit = 0;
        unsigned *cur = qa, *nxt = qb;
        unsigned ncur = 1;
        if (lane == 0) cur[0] = 0u;          // the root: one child, node 0
        __syncwarp();
        for (int L = 0; L < kLevels && ncur; ++L) {
            unsigned nnext = 0;
            for (unsigned pb = 0; pb < ncur; pb += 32) {
                unsigned c0 = 0, cn = 0;
                if (pb + lane < ncur) {
                    const unsigned e = cur[pb + lane];
                    c0 = e >> 3;
                    cn = (e & 7u) + 1u;
                }
                const unsigned incl = warp_incl_scan(cn, lane);
                const unsigned nk = __shfl_sync(0xffffffffu, incl, 31);
                for (unsigned t = 0, d = incl - cn; t < cn; ++t) kids[d + t] = c0 + t;
                __syncwarp();
                // kGwU chunks of 32 children per step: their records load
                // together, then each chunk's decisions go out in order
                for (unsigned kb = 0; kb < nk; kb += 32 * kGwU) {
                    unsigned e[kGwU];
                    bool acc[kGwU], open[kGwU];
                    int k[kGwU];
                    TreeNodeW nd[kGwU];
#pragma unroll
                    for (int u = 0; u < kGwU; ++u) {
                        k[u] = -1;
                        if (kb + 32 * u + lane < nk) {
                            k[u] = (int)kids[kb + 32 * u + lane];
                            nd[u] = a.nodew[k[u]];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kGwU; ++u) {
                        e[u] = 0;
                        acc[u] = open[u] = false;
                        if (k[u] >= 0) {
                            acc[u] = walk_accepts(F, L, nd[u], k[u], i0, gbf, bx, a.com, a.theta2);
                            if (acc[u]) e[u] = (unsigned)a.npseudo;
                            else if (L == kLevels - 1 || nd[u].count <= a.nleaf) e[u] = (unsigned)nd[u].count;
                            else open[u] = true;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kGwU; ++u) {
                        const unsigned om = __ballot_sync(0xffffffffu, open[u]);
                        if (open[u]) {
                            const unsigned slot = nnext + __popc(om & below);
                            if (slot < (unsigned)kGroupWalkQ)
                                nxt[slot] = ((unsigned)nd[u].child0 << 3) | (unsigned)(nd[u].childn - 1);
                        }
                        nnext += __popc(om);
                        if (!FILL && scr) {      // record the chunk's emitters in order
                            const unsigned em = __ballot_sync(0xffffffffu, e[u] != 0u);
                            const unsigned slot = nemit + __popc(em & below);
                            if (e[u] && slot < (unsigned)kGroupWalkScratch)
                                scr[slot] = acc[u] ? (0x80000000u | (unsigned)k[u]) : (unsigned)k[u];
                            nemit += __popc(em);
                        }
                        const unsigned ei = warp_incl_scan(e[u], lane);
                        if (FILL && e[u]) {
                            const long long d = pos + (ei - e[u]);
                            if (d + e[u] > hi) {
                                report(a.status, kStatusBadIndex, 11);
                            } else if (acc[u]) {
                                const int p0 = (int)(a.n + (long long)a.npseudo * k[u]);
                                for (int q = 0; q < a.npseudo; ++q) a.jlist[d + q] = p0 + q;
                            } else {
                                for (unsigned t = 0; t < e[u]; ++t) a.jlist[d + t] = nd[u].first + (int)t;
                            }
                        }
                        pos += __shfl_sync(0xffffffffu, ei, 31);
                    }
                }
                __syncwarp();
            }
            qmax = nnext > qmax ? nnext : qmax;
            if (nnext > (unsigned)kGroupWalkQ) {
                over = true;
                break;
            }
            unsigned *tq = cur;
            cur = nxt;
            nxt = tq;
            ncur = nnext;
            __syncwarp();
        }
        if (over) break;
        if (FILL) {
            if (pos != hi && lane == 0) report(a.status, kStatusBadIndex, 12);
        } else {
            if (lane == 0) a.jcount[g] = (unsigned)pos;
            ent += (unsigned long long)pos;
            if (scr) place_emitters(a, m, scr, nemit, g, lane);
        }
    }
    if (lane == 0) {
        if (over) atomicOr(&m->flags, kTreeWalkQueue);
        if (!FILL) {
            if (ent) atomicAdd(&m->ent, ent);
            atomicMax(&m->qmax, qmax);
        }
    }
}

// the list offsets from the scanned entry counts, the list length, and its
// checks (2^32 entries; the room the host gave the list)
__global__ void k_walk_offsets(TreeMeta *m, const unsigned *__restrict__ jscan, long long *__restrict__ j_off,
                               long long cap_list)
{
    if (m->flags) return;
    const long long ng = m->ngroups;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g <= ng;
         g += (long long)gridDim.x * blockDim.x)
        j_off[g] = jscan[g];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long len = jscan[ng];
        m->nlist = (long long)len;
        if (m->ent >= (1ull << 32) || m->ent != len) atomicOr(&m->flags, kTreeListLong);
        else if ((long long)len > cap_list) atomicOr(&m->flags, kTreeRoomList);
    }
}

// Jacobi rotation zeroing a[p][q] of the symmetric 3x3 a (r the third
// index), with the update written element by element; v accumulates the
// rotations in its columns
__device__ __forceinline__ void jacobi_rotate(double (&a)[3][3], double (&v)[3][3], int p, int q, int r)
{
    const double apq = a[p][q];
    if (apq == 0.0) return;
    const double h = 0.5 * (a[q][q] - a[p][p]) / apq;
    const double t = copysign(1.0, h) / (fabs(h) + sqrt(fma(h, h, 1.0)));
    const double c = rsqrt(fma(t, t, 1.0)), s = t * c;
    a[p][p] -= t * apq;
    a[q][q] += t * apq;
    a[p][q] = a[q][p] = 0.0;
    const double arp = a[r][p], arq = a[r][q];
    a[r][p] = a[p][r] = c * arp - s * arq;
    a[r][q] = a[q][r] = s * arp + c * arq;
    for (int k = 0; k < 3; ++k) {
        const double vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq;
        v[k][q] = s * vkp + c * vkq;
    }
}

// the three pseudo-particles of node k from its centre c, the spreads a, b
// along the unit principal axes e1, e2 (e1's sign set here: its largest
// component positive), mass M / 3 each
__device__ __forceinline__ void write_quad(double4 *out, long long k, double4 c, double al, double be,
                                           double e1x, double e1y, double e1z, double e2x, double e2y,
                                           double e2z)
{
    double big = e1x;
    if (fabs(e1y) > fabs(big)) big = e1y;
    if (fabs(e1z) > fabs(big)) big = e1z;
    if (big < 0.0) {
        e1x = -e1x;
        e1y = -e1y;
        e1z = -e1z;
    }
    const double hb = 0.8660254037844386 * be;      // sqrt(3) / 2, rounded
    const double m3 = c.w / 3.0;
    const double ax = al * e1x, ay = al * e1y, az = al * e1z;
    const double bx = hb * e2x, by = hb * e2y, bz = hb * e2z;
    out[3 * k] = make_double4(c.x + ax, c.y + ay, c.z + az, m3);
    out[3 * k + 1] = make_double4(c.x - 0.5 * ax + bx, c.y - 0.5 * ay + by, c.z - 0.5 * az + bz, m3);
    out[3 * k + 2] = make_double4(c.x - 0.5 * ax - bx, c.y - 0.5 * ay - by, c.z - 0.5 * az - bz, m3);
}

// The quadrupole pseudo-particles (Kawai and Makino's three): with T's
// eigenvalues l1 >= l2 >= l3 and unit eigenvectors e1, e2, mass M / 3 at
// c + a e1 and c - a/2 e1 +- (sqrt 3 / 2) b e2, a = sqrt(2 (l1 - l3) / M),
// b = sqrt(2 (l2 - l3) / M); they carry M, a zero dipole and T - l3 I (the
// trace-free quadrupole of T). Nodes of one or two particles have them in
// closed form (one: T = 0, all three at c; two: T = (m1 m2 / M) d d^T with
// d = x2 - x1, so e1 = d / |d|, a = |d| sqrt(2 m1 m2) / M, b = 0); the others
// go to a list for the eigen-solver.
__device__ __forceinline__ void quad_small_one(long long k, long long nnodes, const double4 *__restrict__ com,
                                               const int *__restrict__ first, const int *__restrict__ count,
                                               const double4 *__restrict__ xs, double4 *__restrict__ out,
                                               int *__restrict__ big_list, unsigned *__restrict__ nbig)
{
    bool big = false;
    if (k < nnodes) {
        const double4 c = com[k];
        const int cnt = count[k];
        if (cnt == 1) {
            write_quad(out, k, c, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0);
        } else if (cnt == 2) {
            const double4 p = xs[first[k]], q = xs[first[k] + 1];
            const double dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
            const double dn = sqrt(dx * dx + dy * dy + dz * dz);
            if (dn > 0.0) {
                const double al = dn * sqrt(2.0 * p.w * q.w) / c.w;
                write_quad(out, k, c, al, 0.0, dx / dn, dy / dn, dz / dn, 0.0, 0.0, 0.0);
            } else {
                write_quad(out, k, c, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0);
            }
        } else {
            big = true;
        }
    }
    // append the other nodes to the list, one atomic per warp
    const unsigned mask = __ballot_sync(0xffffffffu, big);
    if (!mask) return;
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(nbig, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (big) big_list[base + __popc(mask & ((1u << lane) - 1u))] = (int)k;
}

__global__ void k_tree_quad_small(const TreeMeta *__restrict__ m, const double4 *__restrict__ com,
                                  const int *__restrict__ first, const int *__restrict__ count,
                                  const double4 *__restrict__ xs, double4 *__restrict__ out,
                                  int *__restrict__ big_list, unsigned *__restrict__ nbig)
{
    if (m->flags) return;
    const long long nnodes = m->nnodes;
    // the loop is uniform over each warp (its ballot takes every lane)
    for (long long k0 = blockIdx.x * (long long)blockDim.x; k0 < nnodes; k0 += (long long)gridDim.x * blockDim.x)
        quad_small_one(k0 + threadIdx.x, nnodes, com, first, count, xs, out, big_list, nbig);
}

// the listed nodes: T's eigen-decomposition by cyclic Jacobi rotations
// (grid-stride over the list, whose length is read on the device)
__global__ void k_tree_quad_big(const int *__restrict__ big_list, const unsigned *__restrict__ nbig,
                                const double4 *__restrict__ com, const double *__restrict__ T,
                                double4 *__restrict__ out)
{
    const long long nb = *nbig;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < nb;
         w += (long long)gridDim.x * blockDim.x) {
        const long long k = big_list[w];
        const double4 c = com[k];
        const double *t = T + 6 * k;
        double a[3][3] = {{t[0], t[1], t[2]}, {t[1], t[3], t[4]}, {t[2], t[4], t[5]}};
        double v[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int sweep = 0; sweep < 12; ++sweep) {
            const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
            if (!(off > 1e-18 * (fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2])))) break;
            jacobi_rotate(a, v, 0, 1, 2);
            jacobi_rotate(a, v, 0, 2, 1);
            jacobi_rotate(a, v, 1, 2, 0);
        }
        // selects instead of indexing keep the arrays in registers
        const double lam0 = a[0][0], lam1 = a[1][1], lam2 = a[2][2];
        int i1 = 0, i3 = 0;
        if (lam1 > lam0) i1 = 1;
        if (lam2 > (i1 ? lam1 : lam0)) i1 = 2;
        if (lam1 < lam0) i3 = 1;
        if (lam2 < (i3 ? lam1 : lam0)) i3 = 2;
        if (i1 == i3) i3 = i1 == 2 ? 0 : i1 + 1;
        const int i2 = 3 - i1 - i3;
        auto pick = [](int i, double x0, double x1, double x2) { return i == 0 ? x0 : i == 1 ? x1 : x2; };
        const double l1 = pick(i1, lam0, lam1, lam2), l2 = pick(i2, lam0, lam1, lam2),
                     l3 = pick(i3, lam0, lam1, lam2);
        const double al = sqrt(2.0 * fmax(l1 - l3, 0.0) / c.w);
        const double be = sqrt(2.0 * fmax(l2 - l3, 0.0) / c.w);
        write_quad(out, k, c, al, be, pick(i1, v[0][0], v[0][1], v[0][2]), pick(i1, v[1][0], v[1][1], v[1][2]),
                   pick(i1, v[2][0], v[2][1], v[2][2]), pick(i2, v[0][0], v[0][1], v[0][2]),
                   pick(i2, v[1][0], v[1][1], v[1][2]), pick(i2, v[2][0], v[2][1], v[2][2]));
    }
}

// items: the groups cut into chunks of at most Bi particles; pairs = sum ni nj
__device__ __forceinline__ void items_one(long long g, long long ngroups, const int *__restrict__ g_i0,
                                          const int *__restrict__ g_ni, const unsigned *__restrict__ item_off,
                                          const long long *__restrict__ j_off, int Bi,
                                          GroupItem *__restrict__ items, unsigned long long *pairs)
{
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

__global__ void k_tree_items(TreeMeta *m, const int *__restrict__ g_i0, const int *__restrict__ g_ni,
                             const unsigned *__restrict__ item_off, const long long *__restrict__ j_off,
                             int Bi, GroupItem *__restrict__ items)
{
    if (m->flags) return;           // the item count stays zero: the force kernel does nothing
    const long long ngroups = m->ngroups;
    if (blockIdx.x == 0 && threadIdx.x == 0) m->nitems = item_off[ngroups];
    // the loop is uniform over each warp (its reduction takes every lane)
    for (long long g0 = blockIdx.x * (long long)blockDim.x; g0 < ngroups; g0 += (long long)gridDim.x * blockDim.x)
        items_one(g0 + threadIdx.x, ngroups, g_i0, g_ni, item_off, j_off, Bi, items, &m->pairs);
}

// items per group, and zero from the group count up to the room (cap + 1
// entries, the length the host scans)
__global__ void k_tree_item_counts(const TreeMeta *__restrict__ m, const int *__restrict__ g_ni, long long cap,
                                   int Bi, unsigned *__restrict__ c)
{
    const long long ngroups = m->flags ? 0 : m->ngroups;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g <= cap;
         g += (long long)gridDim.x * blockDim.x)
        c[g] = g < ngroups ? (unsigned)((g_ni[g] + Bi - 1) / Bi) : 0u;
}

unsigned blocks_of(long long n) { return (unsigned)((std::max(n, 1LL) + 255) / 256); }

// an exclusive scan in place, counted in the stage's launches (three kernels)
cudaError_t scan(TreeScratch &t, unsigned *a, long long n, unsigned *sums, cudaStream_t st)
{
    if (n > 0) t.launches += 3;
    return launch_excl_scan(a, n, sums, st);
}

// the widest level of the last call's tree: the grid of the per-level
// kernels (they stride over the level, so any grid is correct)
long long widest_hint(const TreeScratch &t)
{
    long long w = 1;
    for (int L = 0; L < kLevels; ++L) w = std::max(w, t.hint_runs[L]);
    return w;
}

// blocks of the group walk per SM, once per device
int gw_blocks_per_sm()
{
    static int per[kMaxDevices];
    static bool done[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return 1;
    }
    once_per_device(done, [&]() {
        int b = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_walk_groups<false>, 32 * kGwWarps, 0);
        per[dev] = e == cudaSuccess && b > 0 ? b : 1;
        return e;
    });
    (void)cudaGetLastError();
    return per[dev] > 0 ? per[dev] : 1;
}

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
    t.launches += 4 + (n > 0 ? (3 * kBits + 7) / 8 * 5 : 0) + 3;   // with the gather, flags, offsets
    cudaMemcpyAsync(t.key, ko, n * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(t.perm, perm, n * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    k_tree_gather<<<blocks_of(n), 256, 0, st>>>(jrec, t.perm, n, t.xs, t.xi0);
    // every level's run flags, one scan numbering all nodes
    k_tree_flags<<<dim3(blocks_of(n + 1), kLevels), 256, 0, st>>>(t.key, n, t.scan);
    if ((e = scan(t, t.scan, (long long)kLevels * (n + 1) + 1, t.tsums, st)) != cudaSuccess) return e;
    k_tree_level_meta<<<1, 32, 0, st>>>(t.scan, n, t.npseudo, t.cap_nodes, t.meta);
    return cudaGetLastError();
}

// node starts, counts and children (every level)
cudaError_t tree_stage_links(long long n, TreeScratch &t, cudaStream_t st)
{
    const unsigned wide = blocks_of(widest_hint(t));
    k_tree_starts<<<dim3(blocks_of(n), kLevels), 256, 0, st>>>(t.meta, t.key, t.scan, n, t.first);
    k_tree_nodes<<<dim3(wide, kLevels), 256, 0, st>>>(t.meta, n, t.scan, t.first, t.count, t.child0, t.childn,
                                                      t.lev);
    t.launches += 2;
    return cudaGetLastError();
}

// moments bottom-up, with each node's centre, walk record and (quadrupole)
// second moment
cudaError_t tree_stage_moments(long long n, TreeScratch &t, cudaStream_t st)
{
    NodeOut no{t.com, t.npseudo == 1 ? t.jrec2 + n : nullptr, t.nodew, t.npseudo == 3 ? t.T : nullptr};
    k_tree_moments_leaf<<<blocks_of(t.hint_runs[kLevels - 1]), 256, 0, st>>>(t.meta, t.first, t.count, t.child0,
                                                                             t.childn, t.xs, t.M, t.S, no);
    // levels of at most kTopNodes nodes in the last call (their counts grow
    // with the level) go to the one-block kernel
    constexpr long long kTopNodes = 2048;
    int L0 = -1;
    while (L0 + 1 < kLevels - 1 && t.hint_runs[L0 + 1] <= kTopNodes) ++L0;
    for (int L = kLevels - 2; L > L0; --L)
        k_tree_moments_up<<<blocks_of(t.hint_runs[L]), 256, 0, st>>>(t.meta, L, t.first, t.count, t.child0,
                                                                     t.childn, t.M, t.S, no);
    if (L0 >= 0)
        k_tree_moments_top<<<1, 1024, 0, st>>>(t.meta, L0, t.first, t.count, t.child0, t.childn, t.M, t.S, no);
    t.launches += 1 + (kLevels - 2 - L0) + (L0 >= 0 ? 1 : 0);
    return cudaGetLastError();
}

// the groups: marks at their first particle, numbered by a scan
cudaError_t tree_stage_groups(long long n, int ncrit, TreeScratch &t, SortScratch &sort, cudaStream_t st)
{
    const unsigned wide = blocks_of(widest_hint(t));
    cudaMemsetAsync(t.gat, 0xff, n * sizeof(int), st);
    k_tree_group_marks<<<dim3(wide, kLevels), 256, 0, st>>>(t.meta, n, t.scan, t.first, t.count, ncrit, t.gat);
    k_tree_group_flags<<<blocks_of(n + 1), 256, 0, st>>>(t.gat, n, t.gscan);
    t.launches += 3;         // marks, flags, groups
    cudaError_t e = scan(t, t.gscan, n + 1, sort.sums, st);
    if (e != cudaSuccess) return e;
    k_tree_groups<<<blocks_of(n + 1), 256, 0, st>>>(t.meta, t.cap_groups, t.gat, t.gscan, n, t.count, t.g_i0,
                                                    t.g_ni, t.i_off);
    return cudaGetLastError();
}

cudaError_t tree_walk_prep(double theta, TreeScratch &t, cudaStream_t st)
{
    k_tree_gbox<<<(unsigned)((t.cap_groups + 7) / 8), 256, 0, st>>>(t.g_i0, t.g_ni, t.meta, t.xs, t.gbox,
                                                                    t.gboxf, t.gctr);
    k_walk_filter<<<1, 32, 0, st>>>(t.geo, theta * theta, t.filt);
    t.launches += 2;
    return cudaGetLastError();
}

cudaError_t tree_group_walk(bool fill, long long n, double theta, int nleaf, int sms, TreeScratch &t,
                            SortScratch &sort, int *status, cudaStream_t st)
{
    GroupWalkArgs a{};
    a.n = n;
    a.meta = t.meta;
    a.g_i0 = t.g_i0;
    a.gbox = t.gbox;
    a.gboxf = t.gboxf;
    a.nodew = t.nodew;
    a.com = t.com;
    a.filt = t.filt;
    a.nleaf = nleaf;
    a.npseudo = t.npseudo;
    a.theta2 = theta * theta;
    a.jcount = t.jcount;
    a.j_off = t.j_off;
    a.jlist = t.jlist;
    a.status = status;
    a.wscratch = t.wscratch;
    a.emit = t.emit;
    a.emit_cap = t.emit_cap;
    a.gemit = t.gemit;
    const unsigned grid = (unsigned)std::max(1, sms * gw_blocks_per_sm());
    if (fill) {
        k_walk_groups<true><<<grid, 32 * kGwWarps, 0, st>>>(a);
        ++t.launches;
        return cudaGetLastError();
    }
    k_walk_groups<false><<<grid, 32 * kGwWarps, 0, st>>>(a);
    cudaError_t e = scan(t, t.jcount, t.cap_groups + 1, sort.sums, st);
    if (e != cudaSuccess) return e;
    k_walk_offsets<<<std::min(blocks_of(t.cap_groups + 1), 4096u), 256, 0, st>>>(t.meta, t.jcount, t.j_off,
                                                                                  t.cap_list);
    t.launches += 2;
    return cudaGetLastError();
}

long long group_walk_warps(int sms) { return (long long)std::max(1, sms * gw_blocks_per_sm()) * kGwWarps; }

cudaError_t tree_walk_init(long long ngroups, TreeScratch &t, cudaStream_t st)
{
    cudaMemsetAsync(t.seg, 0, 2 * (size_t)kLevels * ngroups * sizeof(unsigned), st);
    k_walk_init<<<blocks_of(ngroups), 256, 0, st>>>(ngroups, t.vg, t.vk, t.meta);
    ++t.launches;
    return cudaGetLastError();
}

cudaError_t tree_walk_level(long long n, long long ngroups, int L, long long o, long long nf,
                            double theta, int nleaf, TreeScratch &t, cudaStream_t st)
{
    LevelArgs a{};
    a.n = n;
    a.ngroups = ngroups;
    a.o = o;
    a.nf = nf;
    a.L = L;
    a.g_i0 = t.g_i0;
    a.gbox = t.gbox;
    a.gboxf = t.gboxf;
    a.nodew = t.nodew;
    a.com = t.com;
    a.filt = t.filt;
    a.nleaf = nleaf;
    a.npseudo = t.npseudo;
    a.vg = t.vg;
    a.vk = t.vk;
    a.ve = t.ve;
    a.vc = t.vc;
    a.seg = t.seg;
    a.ent = &t.meta->ent;
    a.theta2 = theta * theta;
    k_walk_test<<<blocks_of(nf + 1), 256, 0, st>>>(a);
    ++t.launches;
    return scan(t, t.vc, nf + 1, t.vsums, st);
}

cudaError_t tree_walk_expand(long long o, long long nf, TreeScratch &t, cudaStream_t st)
{
    k_walk_expand<<<blocks_of(nf), 256, 0, st>>>(t.nodew, o, nf, t.vc, t.vg, t.vk);
    ++t.launches;
    return cudaGetLastError();
}

cudaError_t tree_walk_lists(long long ngroups, const long long *lev_v, int nlev, TreeScratch &t,
                            SortScratch &sort, cudaStream_t st)
{
    const long long nv = lev_v[nlev];
    cudaMemsetAsync(t.ve + nv, 0, sizeof(unsigned), st);
    cudaError_t e = scan(t, t.ve, nv + 1, t.vsums, st);
    if (e != cudaSuccess) return e;
    k_walk_count<<<blocks_of(ngroups + 1), 256, 0, st>>>(ngroups, nlev, t.seg, t.ve, t.jcount);
    if ((e = scan(t, t.jcount, ngroups + 1, sort.sums, st)) != cudaSuccess) return e;
    k_walk_base<<<blocks_of(ngroups + 1), 256, 0, st>>>(ngroups, nlev, t.jcount, t.seg, t.ve, t.j_off,
                                                        t.base, t.meta);
    t.launches += 2;
    return cudaGetLastError();
}

cudaError_t tree_walk_fill(long long n, long long ngroups, const long long *lev_v, int nlev,
                           TreeScratch &t, int *status, cudaStream_t st)
{
    for (int L = 0; L < nlev; ++L) {
        const long long o = lev_v[L], nf = lev_v[L + 1] - o;
        k_walk_fill<<<blocks_of(nf), 256, 0, st>>>(L, o, nf, n, ngroups, t.npseudo, t.vg, t.vk, t.ve,
                                                   t.base, t.j_off, t.nodew, t.jlist, status);
        ++t.launches;
    }
    return cudaGetLastError();
}

// the j records: particles in key order, then P pseudo-particles per node
// (monopoles: written with the moments; quadrupoles: three from the second
// moments)
cudaError_t tree_stage_jrec(long long n, int sms, TreeScratch &t, cudaStream_t st)
{
    cudaMemcpyAsync(t.jrec2, t.xs, n * sizeof(double4), cudaMemcpyDeviceToDevice, st);
    if (t.npseudo == 3) {
        cudaMemsetAsync(t.nbig, 0, sizeof(unsigned), st);
        long long hint = 0;
        for (int L = 0; L < kLevels; ++L) hint += t.hint_runs[L];
        k_tree_quad_small<<<blocks_of(hint), 256, 0, st>>>(t.meta, t.com, t.first, t.count, t.xs, t.jrec2 + n,
                                                           t.big_list, t.nbig);
        k_tree_quad_big<<<(unsigned)std::max(1, 4 * sms), 128, 0, st>>>(t.big_list, t.nbig, t.com, t.T,
                                                                       t.jrec2 + n);
        t.launches += 2;
    }
    return cudaGetLastError();
}

cudaError_t tree_stage_records(int Bi, TreeScratch &t, SortScratch &sort, cudaStream_t st)
{
    k_tree_item_counts<<<std::min(blocks_of(t.cap_groups + 1), 4096u), 256, 0, st>>>(t.meta, t.g_ni, t.cap_groups,
                                                                                      Bi, t.item_off);
    t.launches += 2;      // with the items below
    cudaError_t e = scan(t, t.item_off, t.cap_groups + 1, sort.sums, st);
    if (e != cudaSuccess) return e;
    k_tree_items<<<blocks_of(t.cap_groups), 256, 0, st>>>(t.meta, t.g_i0, t.g_ni, t.item_off, t.j_off, Bi,
                                                          t.items);
    return cudaGetLastError();
}

}  // namespace pg
