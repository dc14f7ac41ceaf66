// pg_groups.cu -- batched i-groups, each with its own j-list (the tree usage
// of Section 5.1: a group of nearby i-particles shares one interaction list
// of particles and pseudo-particles), and the periodic cell list that turns
// the cutoff force into the same shape of work.
//
// One persistent launch: every CTA takes work items (group, i-chunk) from an
// atomic queue ordered longest-first, gathers the group's j records into
// shared memory (converted once per record to FP32 offsets in the group's
// frame), and evaluates the Newton or tabulated pair term with the
// i-particles in registers. A small group splits each set of i-particles
// across L lanes, each taking every L-th j, and combines the lanes with warp
// shuffles. The smallest items (few i-particles and short lists) come last
// and run one per warp instead of one per CTA: inside the same launch for the
// caller's groups, in a second kernel (k_groups_warp) for the cell list and
// the narrow all-pairs path.
#include <algorithm>

#include "pg_device.cuh"

namespace pg {

constexpr int kTJG = 512;          // j entries staged per step

// unroll depth of a CTA-mode item's j loop (measured on GB300: 8 for the
// table lookups, whose latency wants more terms in flight; 2 for Newton)
template <bool TABLE> struct GroupsUnrollJ { static constexpr int value = TABLE ? 8 : 2; };

// Records come in two forms.
//  CELL = false: any particle as a double-float pair, hi = (x, y, z, m) in
//    FP32 and lo = the FP32 residual of x - hi (built once per run from the
//    FP64 record). The group's FP64 centre is split the same way and the
//    offset formed as (hi_j - c_hi) + (lo_j - c_lo) in FP32: the same
//    rounding as differencing in FP64 and rounding once, without FP64
//    instructions (GB300 runs FP64 at about two operations per SM-clock).
//  CELL = true: the periodic cell list's FP32 record (o, m), o = the
//    particle's offset from its cell's corner in scaled units. The j-list of
//    a cell is the 27 neighbour cells' runs of the cell-sorted records, each
//    with its direction (dx, dy, dz) in {-1, 0, 1}^3 from the i-cell, so the
//    j offset in the i-cell's frame is o_j + (dx, dy, dz) h~ -- FP32 only,
//    with the periodic wrap already in the direction.
//
// DF (narrow all-pairs, whose i chunks can be spread over the whole system):
// no FP32 offsets at all; a pair's difference is formed from the
// double-float records as (hi_j - hi_i) + (lo_j - lo_i). The first
// subtraction is rounded relative to |d| itself (exact when the two are
// within a factor of two), the second is tiny, so d keeps FP32 precision
// relative to |d| however far the chunk's i-particles are from each other.
// Table mode scales d afterwards (one multiply, relative error 2^-24).
//
// Thread layout of an item: nsets sets of 2*NP i-particles; each set owns L
// consecutive lanes of one warp (any L from 1 to 32, sets never straddle a
// warp), lane l of a set takes the j with index = l (mod L), and the set's
// lanes are combined by a segmented shuffle reduction at the end. NP (i-pairs
// per thread) is chosen per item, 2 or 4, for the better thread use.

// floor(a / b) for 0 <= a < 2^16 and 1 <= b <= 128 as one high multiply by
// ceil(2^32 / b) (exact in that range), not the generic division sequence
__constant__ unsigned kRecip[129] = {
    0u, 0u, 2147483648u, 1431655766u, 1073741824u, 858993460u, 715827883u,
    613566757u, 536870912u, 477218589u, 429496730u, 390451573u, 357913942u, 330382100u,
    306783379u, 286331154u, 268435456u, 252645136u, 238609295u, 226050911u, 214748365u,
    204522253u, 195225787u, 186737709u, 178956971u, 171798692u, 165191050u, 159072863u,
    153391690u, 148102321u, 143165577u, 138547333u, 134217728u, 130150525u, 126322568u,
    122713352u, 119304648u, 116080198u, 113025456u, 110127367u, 107374183u, 104755300u,
    102261127u, 99882961u, 97612894u, 95443718u, 93368855u, 91382283u, 89478486u,
    87652394u, 85899346u, 84215046u, 82595525u, 81037119u, 79536432u, 78090315u,
    76695845u, 75350304u, 74051161u, 72796056u, 71582789u, 70409300u, 69273667u,
    68174085u, 67108864u, 66076420u, 65075263u, 64103990u, 63161284u, 62245903u,
    61356676u, 60492498u, 59652324u, 58835169u, 58040099u, 57266231u, 56512728u,
    55778797u, 55063684u, 54366675u, 53687092u, 53024288u, 52377650u, 51746594u,
    51130564u, 50529028u, 49941481u, 49367441u, 48806447u, 48258060u, 47721859u,
    47197443u, 46684428u, 46182445u, 45691142u, 45210183u, 44739243u, 44278014u,
    43826197u, 43383509u, 42949673u, 42524429u, 42107523u, 41698712u, 41297763u,
    40904451u, 40518560u, 40139882u, 39768216u, 39403370u, 39045158u, 38693400u,
    38347923u, 38008561u, 37675152u, 37347542u, 37025581u, 36709123u, 36398028u,
    36092163u, 35791395u, 35495598u, 35204650u, 34918434u, 34636834u, 34359739u,
    34087043u, 33818641u, 33554432u};

__device__ __forceinline__ int div_small(int a, int b)
{
    return b == 1 ? a : (int)__umulhi((unsigned)a, kRecip[b]);
}

struct ItemShape {
    int nsets, L, spw;
};

template <int NT = kNT>
__device__ __forceinline__ ItemShape item_shape(int ni, int np)
{
    ItemShape s;
    s.nsets = (ni + 2 * np - 1) / (2 * np);
    int L = div_small(NT, s.nsets > 0 ? s.nsets : 1);
    L = L > 32 ? 32 : L < 1 ? 1 : L;
    while (L > 1 && (NT / 32) * div_small(32, L) < s.nsets) --L;
    s.L = L;
    s.spw = div_small(32, L);
    return s;
}

// Cell mode. The j-list of cell g is the particles of its 27 neighbour cells
// (itself included), direction d = 9 (dx + 1) + 3 (dy + 1) + (dz + 1), each a
// contiguous run of the cell-sorted arrays. One warp writes the runs as a
// prefix table cr[0..63]: cr[d] = entries before run d (cr[27..31] = the
// total), cr[32 + d] = first particle of run d minus cr[d], so that list
// position p of run d is particle cr[32 + d] + p.
constexpr int kCellTab = 64;

__device__ __forceinline__ void cell_ranges(const GroupArgs &a, int g, int lane32, int *cr)
{
    int first = 0, cnt = 0;
    if (lane32 < 27) {
        const int nc = a.nc;
        const int cz = g % nc, cxy = g / nc;
        const int cy = cxy % nc, cx = cxy / nc;
        int x = cx + lane32 / 9 - 1, y = cy + (lane32 / 3) % 3 - 1, z = cz + lane32 % 3 - 1;
        x = x < 0 ? x + nc : x >= nc ? x - nc : x;
        y = y < 0 ? y + nc : y >= nc ? y - nc : y;
        z = z < 0 ? z + nc : z >= nc ? z - nc : z;
        const long long nb = ((long long)x * nc + y) * nc + z;
        first = (int)a.cstart[nb];
        cnt = (int)(a.cstart[nb + 1] - (unsigned)first);
    }
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane32 >= o) inc += v;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 26);
    const int exc = inc - cnt;
    cr[lane32] = lane32 < 27 ? exc : total;
    if (lane32 < 27) cr[32 + lane32] = first - exc;
}

// run holding list position p (0 <= p < total): the largest d with cr[d] <= p
__device__ __forceinline__ int cell_find(const int *cr, int p)
{
    int d = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
        if (cr[d + step] <= p) d += step;
    return d;
}

// item k of the queue: stored, or for narrow all-pairs the (i chunk, j chunk)
// pair k / nchunks, k mod nchunks
__device__ __forceinline__ GroupItem item_at(const GroupArgs &a, int k)
{
    if (a.jchunk == 0) return a.items[k];
    GroupItem it;
    const int ic = k / a.nchunks;
    it.group = ic;
    it.i0 = ic * a.ichunk;
    it.ni = (int)min((long long)a.ichunk, a.ni - it.i0);
    it.pad = k - ic * a.nchunks;
    return it;
}

// A list that holds i itself (the tree): the loop added -m_i rsqrt(eps^2)
// for the own pair (d = 0); nothing at eps = 0 (the zero guard)
__device__ __forceinline__ double list_self_pot(const GroupArgs &a, long long i)
{
    return a.eps2 > 0.0f ? -(double)__fmul_rn(a.jhl[2 * i].w, rsq(a.eps2)) : 0.0;
}

// Cell mode with a potential: particle i (cell order) is in its own cell's
// list, so the sum holds its own pair at s = 2 (d = 0): m_i psi~(2), the
// value of knot 0. Subtracted in FP64 from the computed FP32 product.
__device__ __forceinline__ double cell_self_pot(const GroupArgs &a, const float2 *tab, long long i)
{
    const float4 t0 = reinterpret_cast<const float4 *>(tab)[0];
    return (double)__fmul_rn(a.xo[i].w, __fmaf_rn(2.0f, t0.w, t0.z));
}

// One packed pair term (two interactions) from r2 = (ra, rb): Newton with
// the MUFU rsqrt (EXT: zero for a coincident pair at eps = 0), or the
// table's interpolant at s = min(r2, s_max) (EXT: with the potential half).
template <bool TABLE, bool EXT>
__device__ __forceinline__ void pair_term(float ra, float rb, u64 dx, u64 dy, u64 dz, u64 m,
                                          unsigned tb0, int sh3, unsigned smax_bits, u64 &ax,
                                          u64 &ay, u64 &az, u64 &ph)
{
    if (!TABLE) {
        float qa = rsq(ra), qb = rsq(rb);
        if (EXT) {
            qa = ra > 0.0f ? qa : 0.0f;
            qb = rb > 0.0f ? qb : 0.0f;
        }
        const u64 q = pk2(qa, qb);
        const u64 mq = f2mul(m, q);
        const u64 mq3 = f2mul(mq, f2mul(q, q));
        ph = f2sub(ph, mq);
        ax = f2fma(mq3, dx, ax);
        ay = f2fma(mq3, dy, ay);
        az = f2fma(mq3, dz, az);
    } else {
        ra = clamp_pos(ra, smax_bits);
        rb = clamp_pos(rb, smax_bits);
        u64 g;
        if (EXT) {
            const float4 ta = tab4_at(tb0, __float_as_uint(ra), sh3);
            const float4 tb = tab4_at(tb0, __float_as_uint(rb), sh3);
            g = pk2(__fmaf_rn(ra, ta.y, ta.x), __fmaf_rn(rb, tb.y, tb.x));
            ph = f2fma(m, pk2(__fmaf_rn(ra, ta.w, ta.z), __fmaf_rn(rb, tb.w, tb.z)), ph);
        } else {
            const float2 ta = tab_at(tb0, __float_as_uint(ra), sh3);
            const float2 tb = tab_at(tb0, __float_as_uint(rb), sh3);
            g = pk2(__fmaf_rn(ra, ta.y, ta.x), __fmaf_rn(rb, tb.y, tb.x));
        }
        const u64 mg = f2mul(m, g);
        ax = f2fma(mg, dx, ax);
        ay = f2fma(mg, dy, ay);
        az = f2fma(mg, dz, az);
    }
}

template <int NP, bool TABLE, bool CELL, bool EXT, bool HL = false, bool DF = false, int TJ = kTJG,
          int NT = kNT>
__device__ __forceinline__ void group_item(const GroupArgs &a, const GroupItem &it, const ItemShape sh,
                                           u64 *cvt, u64 *run, int *cr, const float2 *tab,
                                           const float4 *dirt, int tid)
{
    constexpr int kPT = TJ / NT;       // j records each thread stages per tile
    static_assert(!(DF && CELL), "double-float differencing is for particle records");
    long long jb = 0, je = 0;
    if (CELL) {
        if (tid < 32) cell_ranges(a, it.group, tid, cr);
        __syncthreads();
        je = cr[27];
    } else if (a.jchunk > 0) {
        jb = (long long)it.pad * a.jchunk;
        je = min(jb + a.jchunk, a.nj);
    } else {
        jb = a.j_off[it.group];
        je = a.j_off[it.group + 1];
    }
    double4 c = make_double4(0, 0, 0, 0);
    float chx = 0, chy = 0, chz = 0, clx = 0, cly = 0, clz = 0;   // centre as hi + lo
    if (!CELL) {
        c = a.gctr[it.group];
        chx = (float)c.x; clx = (float)(c.x - (double)chx);
        chy = (float)c.y; cly = (float)(c.y - (double)chy);
        chz = (float)c.z; clz = (float)(c.z - (double)chz);
    }
    const float c0 = TABLE ? 2.0f : a.eps2;
    const u64 c0v = pk2(c0, c0);
    const float scf = TABLE && !CELL ? (float)a.tab.scale : 1.0f;
    const int sh3 = a.tab.shift - (EXT ? 4 : 3);
    const unsigned tb0 = smem_u32(tab) - (a.tab.base << (EXT ? 4 : 3));
    const unsigned smax_bits = __float_as_uint(a.tab.s_max);
    auto RH = [&](int p, int k) -> u64 & { return run[(8 * p + k) * NT + tid]; };
    auto RL = [&](int p, int k) -> u64 & { return run[(8 * p + 4 + k) * NT + tid]; };

    const int L = sh.L;
    const int wl = tid & 31;
    const int wq = div_small(wl, L);
    const int set = (tid >> 5) * sh.spw + wq, lane = wl - wq * L;
    const bool active = wl < sh.spw * L && set < sh.nsets;

    u64 xi[NP], yi[NP], zi[NP];
    u64 lxi[DF ? NP : 1], lyi[DF ? NP : 1], lzi[DF ? NP : 1];   // DF: the records' lo parts
    u64 e2i[NP];                       // Newton EXT: each i-pair's own eps^2
    u64 ax[NP], ay[NP], az[NP], ph[NP];
    const u64 scf2 = pk2(scf, scf);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float fx[2] = {0, 0}, fy[2] = {0, 0}, fz[2] = {0, 0}, fe[2] = {0, 0};
        float gx[2] = {0, 0}, gy[2] = {0, 0}, gz[2] = {0, 0};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            int k = set * 2 * NP + 2 * p + q;
            if (active && k < it.ni) {
                if (CELL) {
                    float4 o = a.xo[it.i0 + k];
                    fx[q] = o.x; fy[q] = o.y; fz[q] = o.z;
                } else if (DF) {
                    const float4 h = a.ihl[2 * (it.i0 + k)], l = a.ihl[2 * (it.i0 + k) + 1];
                    fx[q] = h.x; fy[q] = h.y; fz[q] = h.z;
                    gx[q] = l.x; gy[q] = l.y; gz[q] = l.z;
                    fe[q] = l.w;
                } else {
                    const float4 h = a.ihl[2 * (it.i0 + k)], l = a.ihl[2 * (it.i0 + k) + 1];
                    fx[q] = ((h.x - chx) + (l.x - clx)) * scf;
                    fy[q] = ((h.y - chy) + (l.y - cly)) * scf;
                    fz[q] = ((h.z - chz) + (l.z - clz)) * scf;
                    fe[q] = l.w;
                }
            }
        }
        xi[p] = pk2(fx[0], fx[1]);
        yi[p] = pk2(fy[0], fy[1]);
        zi[p] = pk2(fz[0], fz[1]);
        if (DF) {
            lxi[p] = pk2(gx[0], gx[1]);
            lyi[p] = pk2(gy[0], gy[1]);
            lzi[p] = pk2(gz[0], gz[1]);
        }
        e2i[p] = pk2(fe[0], fe[1]);
#pragma unroll
        for (int k = 0; k < 4; ++k) RH(p, k) = RL(p, k) = 0ull;
    }

    // register prefetch of one tile of records. With a j-list (single-form
    // variants: the tree and group lists) the list indices run one tile
    // further ahead (jidx holds the next tile's), so a record gather never
    // waits on the index load issued just before it; the double-float
    // variants serve the list-free narrow path and keep one stage (their
    // registers are at the three-CTA limit)
    constexpr bool kIdxAhead = !CELL && !DF;
    float4 rc32[kPT];
    float4 rlo[CELL ? 1 : kPT];
    int code[CELL ? kPT : 1];
    int jidx[kIdxAhead ? kPT : 1];
    auto fetch_idx = [&](long long t0) {
        if constexpr (kIdxAhead) {
#pragma unroll
            for (int r = 0; r < kPT; ++r) {
                const long long e = t0 + r * NT + tid;
                jidx[r] = a.jlist ? (e < je ? a.jlist[e] : 0) & 0x07ffffff : 0;
            }
        }
    };
    auto fetch = [&](long long t0) {
#pragma unroll
        for (int r = 0; r < kPT; ++r) {
            long long e = t0 + r * NT + tid;
            bool ok = e < je;
            long long j;
            if (CELL) {
                code[r] = cell_find(cr, (int)e);
                j = (long long)cr[32 + code[r]] + e;
            } else if constexpr (kIdxAhead) {
                j = a.jlist ? (long long)jidx[r] : e;
            } else {
                j = a.jlist ? (ok ? a.jlist[e] : 0) & 0x07ffffff : e;
            }
            if (ok && (j < 0 || j >= a.nj)) {   // bad index: record it, contribute nothing
                report(a.status, kStatusBadIndex, 2);
                ok = false;
            }
            if (CELL) {
                rc32[r] = ok ? __ldg(a.xo + j) : make_float4(0, 0, 0, -1.0f);
            } else {
                rc32[r] = ok ? __ldg(a.jhl + 2 * j) : make_float4(0, 0, 0, -1.0f);
                rlo[r] = ok ? __ldg(a.jhl + 2 * j + 1) : make_float4(0, 0, 0, 0);
            }
        }
    };
    fetch_idx(jb);
    fetch(jb);
    fetch_idx(jb + TJ);
    for (long long t0 = jb; t0 < je; t0 += TJ) {
        // publish the prefetched tile as FP32 offsets in the i frame
#pragma unroll
        for (int r = 0; r < kPT; ++r) {
            const int e = r * NT + tid;
            float x, y, z, m, lx = 0.0f, ly = 0.0f, lz = 0.0f;
            const bool real = rc32[r].w >= 0.0f;
            if (real && DF) {
                x = rc32[r].x; y = rc32[r].y; z = rc32[r].z;
                lx = rlo[r].x; ly = rlo[r].y; lz = rlo[r].z;
                m = rc32[r].w;
            } else if (real && CELL) {
                const float4 dv = dirt[code[r]];     // direction x cell side, scaled
                x = rc32[r].x + dv.x;
                y = rc32[r].y + dv.y;
                z = rc32[r].z + dv.z;
                m = rc32[r].w;
            } else if (real) {
                x = ((rc32[r].x - chx) + (rlo[r].x - clx)) * scf;
                y = ((rc32[r].y - chy) + (rlo[r].y - cly)) * scf;
                z = ((rc32[r].z - chz) + (rlo[r].z - clz)) * scf;
                m = rc32[r].w;
            } else {   // padding: zero mass far away contributes exactly 0
                x = y = z = 1.0e4f;
                m = 0.0f;
            }
            if (CELL && !EXT) {
                // one 16-byte word per j (the cell list's kernel is bound by
                // the shared-memory pipe: one wavefront per j step instead
                // of two; the pairs are formed in registers; with the
                // potential's table the registers would spill)
                reinterpret_cast<float4 *>(cvt)[e] = make_float4(x, y, z, m);
            } else {
                // separate {x, y} and {z, m} arrays: lanes of a set that read
                // consecutive j then read consecutive 16-byte words
                cvt[2 * e + 0] = pk2(x, x);
                cvt[2 * e + 1] = pk2(y, y);
                cvt[2 * TJ + 2 * e + 0] = pk2(z, z);
                cvt[2 * TJ + 2 * e + 1] = pk2(m, m);
            }
            if (DF) {
                cvt[4 * TJ + 2 * e + 0] = pk2(lx, lx);
                cvt[4 * TJ + 2 * e + 1] = pk2(ly, ly);
                cvt[6 * TJ + 2 * e + 0] = pk2(lz, lz);
                cvt[6 * TJ + 2 * e + 1] = 0ull;
            }
        }
        __syncthreads();
        if (t0 + TJ < je) {                  // loads in flight during the compute
            fetch(t0 + TJ);
            fetch_idx(t0 + 2 * TJ);
        }
        long long nv = je - t0;
        if (nv > TJ) nv = TJ;
        if (active) {
#pragma unroll
            for (int p = 0; p < NP; ++p) ax[p] = ay[p] = az[p] = ph[p] = 0ull;
            const int nv_lane = (int)nv;
#pragma unroll(GroupsUnrollJ<TABLE>::value)
            for (int e = lane; e < nv_lane; e += L) {
                ulonglong2 xy, zm;
                if (CELL && !EXT) {
                    const float4 v = reinterpret_cast<const float4 *>(cvt)[e];
                    xy = make_ulonglong2(pk2(v.x, v.x), pk2(v.y, v.y));
                    zm = make_ulonglong2(pk2(v.z, v.z), pk2(v.w, v.w));
                } else {
                    xy = reinterpret_cast<const ulonglong2 *>(cvt)[e];
                    zm = reinterpret_cast<const ulonglong2 *>(cvt)[TJ + e];
                }
                ulonglong2 lxy = make_ulonglong2(0ull, 0ull), lz0 = lxy;
                if (DF) {
                    lxy = reinterpret_cast<const ulonglong2 *>(cvt)[2 * TJ + e];
                    lz0 = reinterpret_cast<const ulonglong2 *>(cvt)[3 * TJ + e];
                }
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    u64 dx = f2sub(xy.x, xi[p]);
                    u64 dy = f2sub(xy.y, yi[p]);
                    u64 dz = f2sub(zm.x, zi[p]);
                    if (DF) {
                        dx = f2add(dx, f2sub(lxy.x, lxi[p]));
                        dy = f2add(dy, f2sub(lxy.y, lyi[p]));
                        dz = f2add(dz, f2sub(lz0.x, lzi[p]));
                        if (TABLE) {
                            dx = f2mul(dx, scf2);
                            dy = f2mul(dy, scf2);
                            dz = f2mul(dz, scf2);
                        }
                    }
                    u64 r2 = f2fma(dx, dx, !TABLE && EXT ? e2i[p] : c0v);
                    r2 = f2fma(dy, dy, r2);
                    r2 = f2fma(dz, dz, r2);
                    float ra, rb;
                    up2(r2, ra, rb);
                    pair_term<TABLE, EXT>(ra, rb, dx, dy, dz, zm.y, tb0, sh3, smax_bits,
                                          ax[p], ay[p], az[p], ph[p]);
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
        __syncthreads();   // everyone done with this tile before it is overwritten
    }

    // combine the L lanes of each set: segmented shuffle reduction of the
    // (hi, lo) FP32 pairs with TwoSum (FP64 would dominate small items on
    // GB300), one conversion to FP64 on the set's first lane
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float h[8], l[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            up2(RH(p, k), h[2 * k], h[2 * k + 1]);
            up2(RL(p, k), l[2 * k], l[2 * k + 1]);
        }
        for (int off = 1; off < L; off <<= 1) {
            const bool take = lane + off < L;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (TABLE && !EXT && (k == 6 || k == 7)) continue;   // no potential
                const float oh = __shfl_down_sync(0xffffffffu, h[k], off);
                const float ol = __shfl_down_sync(0xffffffffu, l[k], off);
                if (take) {
                    float sm, er;
                    two_sum(h[k], oh, sm, er);
                    h[k] = sm;
                    l[k] = __fadd_rn(l[k], __fadd_rn(ol, er));
                }
            }
        }
        if constexpr (HL) {
            // FP32 (hi, lo) sums out; the finish kernel converts them on full warps
            if (active && lane == 0) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int k_i = set * 2 * NP + 2 * p + q;
                    if (k_i < it.ni) {
                        const long long i = it.i0 + k_i;
                        a.hl[2 * i] = make_float4(h[0 + q], h[2 + q], h[4 + q], h[6 + q]);
                        a.hl[2 * i + 1] = make_float4(l[0 + q], l[2 + q], l[4 + q], l[6 + q]);
                    }
                }
            }
            continue;
        }
        if (active && lane == 0) {
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = (double)h[k] + (double)l[k];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                int k = set * 2 * NP + 2 * p + q;
                if (k < it.ni) {
                    long long i = it.i0 + k;
                    const double phi = TABLE && !EXT ? 0.0 : v[6 + q];
                    if (a.part) {          // one partial of a narrow all-pairs sum
                        a.part[(long long)it.pad * a.part_stride + i] =
                            make_double4(v[0 + q], v[2 + q], v[4 + q], phi);
                        continue;
                    }
                    long long o = a.perm ? (long long)a.perm[i] : i;
                    a.acc[3 * o] = v[0 + q] * a.accscale;
                    a.acc[3 * o + 1] = v[2 + q] * a.accscale;
                    a.acc[3 * o + 2] = v[4 + q] * a.accscale;
                    if (a.pot)
                        a.pot[o] = CELL && EXT ? phi - cell_self_pot(a, tab, i)
                                 : !TABLE && a.list_self ? phi - list_self_pot(a, i) : phi;
                }
            }
        }
    }
}

// Warp mode: one warp evaluates one small item at a time (at most 64
// i-particles per pass, one i-pair per lane) with its own 4 KB slice of the
// staging buffer and warp-level synchronisation only, so the warps of a CTA
// work through small items independently instead of meeting at CTA barriers.
// Small items are short, so the warp pipelines across them: the queue claim
// for the item after next, the next item's record, its j range, its
// i-particles and its first j tile are all in flight while the current
// item's last tile is evaluated.
constexpr int kWarpTJ = 128;        // j entries per warp-staged tile
// in the CTA-mode kernel the warps' staging slices (kW kWarpTJ words each)
// share the CTA staging buffer's space (kW TJ words), which is sized for
// the larger of the two
constexpr int kWarpItemNi = 32;     // items up to this size (i-particles)
constexpr long long kWarpItemPairs = 32768;   // and this many pairs go to warp mode

// Claims come from counter q: item qbase + (q's previous value); nwarps is
// the number of warps of the launch claiming from it.
template <bool TABLE, bool CELL, bool EXT, bool HL = false, bool DF = false>
__device__ __forceinline__ void warp_loop(const GroupArgs &a, int nitems, int cur, int held,
                                          u64 *wcvt, int *wcr, const float2 *tab,
                                          const float4 *dirt, int lane32, int *q, int qbase,
                                          int nwarps)
{
    static_assert(!(DF && CELL), "double-float differencing is for particle records");
    constexpr unsigned kFull = 0xffffffffu;
    int pend = -1;                      // lane 0: a claimed item not yet started
    if (lane32 == 0) pend = held;
    if (cur < 0) {
        int c2 = 0;
        if (lane32 == 0) {
            c2 = pend >= 0 ? pend : qbase + atomicAdd(q, 1);
            pend = -1;
        }
        cur = __shfl_sync(kFull, c2, 0);
    }
    if (cur >= nitems) return;
    // claims run one item ahead while more than one item per warp is left
    const int ahead_limit = nitems - nwarps;

    const float c0 = TABLE ? 2.0f : a.eps2;
    const u64 c0v = pk2(c0, c0);
    const float scf = TABLE && !CELL ? (float)a.tab.scale : 1.0f;
    const int sh3 = a.tab.shift - (EXT ? 4 : 3);
    const unsigned tb0 = smem_u32(tab) - (a.tab.base << (EXT ? 4 : 3));
    const unsigned smax_bits = __float_as_uint(a.tab.s_max);
    ulonglong2 *sxy = reinterpret_cast<ulonglong2 *>(wcvt);            // [kWarpTJ]
    ulonglong2 *szm = sxy + kWarpTJ;                                   // [kWarpTJ]
    ulonglong2 *slxy = szm + kWarpTJ;                                  // DF: [kWarpTJ] lo x, y
    ulonglong2 *slz = slxy + kWarpTJ;                                  // DF: [kWarpTJ] lo z
    const u64 scf2 = pk2(scf, scf);

    // j range of an item (cell mode: its run table, written to cr)
    auto setup = [&](const GroupItem &it, int *cr, long long &jb, long long &je) {
        if (CELL) {
            cell_ranges(a, it.group, lane32, cr);
            __syncwarp();
            jb = 0;
            je = cr[27];
        } else if (a.jchunk > 0) {
            jb = (long long)it.pad * a.jchunk;
            je = min(jb + a.jchunk, a.nj);
        } else {
            jb = a.j_off[it.group];
            je = a.j_off[it.group + 1];
        }
    };

    // register prefetch of one j tile (kR records per lane)
    constexpr int kR = kWarpTJ / 32;
    float4 rc32[kR];
    float4 rlo[CELL ? 1 : kR];
    int code[CELL ? kR : 1];
    auto fetch = [&](long long t0, long long je, const int *cr) {
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const long long e = t0 + r * 32 + lane32;
            bool ok = e < je;
            long long j;
            if (CELL) {
                code[r] = cell_find(cr, (int)e);
                j = (long long)cr[32 + code[r]] + e;
            } else {
                j = a.jlist ? (ok ? a.jlist[e] : 0) & 0x07ffffff : e;
            }
            if (ok && (j < 0 || j >= a.nj)) {
                report(a.status, kStatusBadIndex, 4);
                ok = false;
            }
            if (CELL) {
                rc32[r] = ok ? __ldg(a.xo + j) : make_float4(0, 0, 0, -1.0f);
            } else {
                rc32[r] = ok ? __ldg(a.jhl + 2 * j) : make_float4(0, 0, 0, -1.0f);
                rlo[r] = ok ? __ldg(a.jhl + 2 * j + 1) : make_float4(0, 0, 0, 0);
            }
        }
    };

    // lane layout of a pass over ni i-particles: sets of L lanes, one i-pair
    // per set
    struct Shape {
        int L, set, lane;
        bool active;
    };
    auto shape_of = [&](int ni) {
        Shape sp;
        const int nsets = (ni + 1) / 2;
        int L = div_small(32, nsets);
        sp.L = L < 1 ? 1 : L;
        const int spw = div_small(32, sp.L);
        sp.set = div_small(lane32, sp.L);
        sp.lane = lane32 - sp.set * sp.L;
        sp.active = lane32 < spw * sp.L && sp.set < nsets;
        return sp;
    };
    // raw i records of a pass (converted once the item starts)
    float4 ih[2], il[CELL ? 1 : 2];
    auto load_i = [&](const GroupItem &it, int i0, const Shape &sp) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k = i0 + 2 * sp.set + q;
            const bool ok = sp.active && k < it.ni;
            if (CELL) {
                ih[q] = ok ? a.xo[it.i0 + k] : make_float4(0, 0, 0, 0);
            } else {
                ih[q] = ok ? a.ihl[2 * (it.i0 + k)] : make_float4(0, 0, 0, 0);
                il[q] = ok ? a.ihl[2 * (it.i0 + k) + 1] : make_float4(0, 0, 0, 0);
            }
        }
    };

    GroupItem it = item_at(a, cur);
    int slot = 0;
    long long jb, je;
    setup(it, wcr, jb, je);
    fetch(jb, je, wcr);
    Shape sp = shape_of(min(64, it.ni));
    load_i(it, 0, sp);
    for (;;) {
        // claim the next item now (its latency hides behind this one) while
        // the queue is long; in its last stretch only once this one is done
        if (lane32 == 0 && pend < 0 && cur < ahead_limit) pend = qbase + atomicAdd(q, 1);
        int nxt = nitems;
        GroupItem itn = it;
        const int *crc = wcr + slot * kCellTab;
        int *crn = wcr + (slot ^ 1) * kCellTab;
        long long jbn = 0, jen = 0;
        Shape spn = sp;
        bool staged = false;

        float chx = 0, chy = 0, chz = 0, clx = 0, cly = 0, clz = 0;
        if (!CELL) {
            const double4 c = a.gctr[it.group];
            chx = (float)c.x; clx = (float)(c.x - (double)chx);
            chy = (float)c.y; cly = (float)(c.y - (double)chy);
            chz = (float)c.z; clz = (float)(c.z - (double)chz);
        }
        for (int i0 = 0; i0 < it.ni; i0 += 64) {
            const bool last_pass = i0 + 64 >= it.ni;
            if (i0 > 0) {          // a further pass restarts the j-list
                sp = shape_of(min(64, it.ni - i0));
                load_i(it, i0, sp);
                fetch(jb, je, crc);
            }
            float fx[2], fy[2], fz[2], fe[2] = {0.0f, 0.0f};
            float gx[2] = {0.0f, 0.0f}, gy[2] = {0.0f, 0.0f}, gz[2] = {0.0f, 0.0f};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (CELL) {
                    fx[q] = ih[q].x; fy[q] = ih[q].y; fz[q] = ih[q].z;
                } else if (DF) {
                    fx[q] = ih[q].x; fy[q] = ih[q].y; fz[q] = ih[q].z;
                    gx[q] = il[q].x; gy[q] = il[q].y; gz[q] = il[q].z;
                    fe[q] = il[q].w;
                } else {
                    fx[q] = ((ih[q].x - chx) + (il[q].x - clx)) * scf;
                    fy[q] = ((ih[q].y - chy) + (il[q].y - cly)) * scf;
                    fz[q] = ((ih[q].z - chz) + (il[q].z - clz)) * scf;
                    fe[q] = il[q].w;
                }
            }
            const u64 xi = pk2(fx[0], fx[1]), yi = pk2(fy[0], fy[1]), zi = pk2(fz[0], fz[1]);
            const u64 lxi = pk2(gx[0], gx[1]), lyi = pk2(gy[0], gy[1]), lzi = pk2(gz[0], gz[1]);
            const u64 r0 = !TABLE && EXT ? pk2(fe[0], fe[1]) : c0v;   // eps^2 (or 2 in table units)
            const int L = sp.L, lane = sp.lane;
            const bool active = sp.active;
            u64 hx = 0, hy = 0, hz = 0, hp = 0, lx = 0, ly = 0, lz = 0, lp = 0;

            for (long long t0 = jb; t0 < je; t0 += kWarpTJ) {
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const int e = r * 32 + lane32;
                    float x, y, z, m, lx = 0.0f, ly = 0.0f, lz = 0.0f;
                    if (rc32[r].w >= 0.0f && DF) {
                        x = rc32[r].x; y = rc32[r].y; z = rc32[r].z;
                        lx = rlo[r].x; ly = rlo[r].y; lz = rlo[r].z;
                        m = rc32[r].w;
                    } else if (rc32[r].w >= 0.0f && CELL) {
                        const float4 dv = dirt[code[r]];
                        x = rc32[r].x + dv.x; y = rc32[r].y + dv.y; z = rc32[r].z + dv.z;
                        m = rc32[r].w;
                    } else if (rc32[r].w >= 0.0f) {
                        x = ((rc32[r].x - chx) + (rlo[r].x - clx)) * scf;
                        y = ((rc32[r].y - chy) + (rlo[r].y - cly)) * scf;
                        z = ((rc32[r].z - chz) + (rlo[r].z - clz)) * scf;
                        m = rc32[r].w;
                    } else {   // padding adds exactly 0
                        x = y = z = 1.0e4f;
                        m = 0.0f;
                    }
                    sxy[e] = make_ulonglong2(pk2(x, x), pk2(y, y));
                    szm[e] = make_ulonglong2(pk2(z, z), pk2(m, m));
                    if (DF) {
                        slxy[e] = make_ulonglong2(pk2(lx, lx), pk2(ly, ly));
                        slz[e] = make_ulonglong2(pk2(lz, lz), 0ull);
                    }
                }
                __syncwarp();
                // loads in flight during the compute: this item's next tile,
                // or the next item's range, i-particles and first tile
                if (t0 + kWarpTJ < je) {
                    fetch(t0 + kWarpTJ, je, crc);
                } else if (last_pass) {
                    const int claimed = __shfl_sync(kFull, pend, 0);
                    if (claimed >= 0 && claimed < nitems) {
                        nxt = claimed;
                        itn = item_at(a, nxt);
                        setup(itn, crn, jbn, jen);
                        fetch(jbn, jen, crn);
                        spn = shape_of(min(64, itn.ni));
                        load_i(itn, 0, spn);
                        staged = true;
                    }
                }
                if (active) {
                    u64 ax = 0, ay = 0, az = 0, ph = 0;
                    const int nvl = (int)min((long long)kWarpTJ, je - t0);
#pragma unroll 4
                    for (int e = lane; e < nvl; e += L) {
                        const ulonglong2 xy = sxy[e], zm = szm[e];
                        u64 dx = f2sub(xy.x, xi), dy = f2sub(xy.y, yi), dz = f2sub(zm.x, zi);
                        if (DF) {
                            const ulonglong2 lxy = slxy[e], lz0 = slz[e];
                            dx = f2add(dx, f2sub(lxy.x, lxi));
                            dy = f2add(dy, f2sub(lxy.y, lyi));
                            dz = f2add(dz, f2sub(lz0.x, lzi));
                            if (TABLE) {
                                dx = f2mul(dx, scf2);
                                dy = f2mul(dy, scf2);
                                dz = f2mul(dz, scf2);
                            }
                        }
                        u64 r2 = f2fma(dx, dx, r0);
                        r2 = f2fma(dy, dy, r2);
                        r2 = f2fma(dz, dz, r2);
                        float ra, rb;
                        up2(r2, ra, rb);
                        pair_term<TABLE, EXT>(ra, rb, dx, dy, dz, zm.y, tb0, sh3, smax_bits, ax, ay,
                                              az, ph);
                    }
                    fold2(hx, lx, ax);
                    fold2(hy, ly, ay);
                    fold2(hz, lz, az);
                    if (!TABLE || EXT) fold2(hp, lp, ph);
                }
                __syncwarp();
            }

            // segmented reduction of the set's lanes, first lane writes
            float h[8], l[8];
            up2(hx, h[0], h[1]); up2(hy, h[2], h[3]); up2(hz, h[4], h[5]); up2(hp, h[6], h[7]);
            up2(lx, l[0], l[1]); up2(ly, l[2], l[3]); up2(lz, l[4], l[5]); up2(lp, l[6], l[7]);
            for (int off = 1; off < L; off <<= 1) {
                const bool take = lane + off < L;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (TABLE && !EXT && (k == 6 || k == 7)) continue;
                    const float oh = __shfl_down_sync(kFull, h[k], off);
                    const float ol = __shfl_down_sync(kFull, l[k], off);
                    if (take) {
                        float sm, er;
                        two_sum(h[k], oh, sm, er);
                        h[k] = sm;
                        l[k] = __fadd_rn(l[k], __fadd_rn(ol, er));
                    }
                }
            }
            // spread the results over the lanes, one (i, component) each,
            // so that the FP64 conversion runs on every lane of the warp
            const int nout = min(64, it.ni - i0) * 4;        // x, y, z, potential
            for (int o0 = 0; o0 < nout; o0 += 32) {
                const int oi = o0 + lane32;
                const int ip = oi >> 2, comp = oi & 3, src = (ip >> 1) * L, want = 2 * comp + (ip & 1);
                float vh = 0.0f, vl = 0.0f;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (TABLE && !EXT && (k == 6 || k == 7)) continue;
                    const float th = __shfl_sync(kFull, h[k], src & 31);
                    const float tl = __shfl_sync(kFull, l[k], src & 31);
                    if (k == want) {
                        vh = th;
                        vl = tl;
                    }
                }
                if (HL && oi < nout) {
                    float *hlf = reinterpret_cast<float *>(a.hl);
                    const long long i = it.i0 + i0 + ip;
                    hlf[8 * i + comp] = vh;
                    hlf[8 * i + 4 + comp] = vl;
                } else if (oi < nout) {
                    const long long i = it.i0 + i0 + ip;
                    const double v = (double)vh + (double)vl;
                    if (a.part) {          // one partial of a narrow all-pairs sum
                        reinterpret_cast<double *>(a.part + (long long)it.pad * a.part_stride + i)[comp] = v;
                    } else {
                        const long long o = a.perm ? (long long)a.perm[i] : i;
                        if (comp < 3)
                            a.acc[3 * o + comp] = v * a.accscale;
                        else if (a.pot)       // zero in table mode without a potential
                            a.pot[o] = CELL && EXT ? v - cell_self_pot(a, tab, i)
                                     : !TABLE && a.list_self ? v - list_self_pot(a, i) : v;
                    }
                }
            }
        }
        if (!staged) {             // nothing claimed ahead, or no j tile to overlap with
            int c2 = 0;
            if (lane32 == 0) c2 = pend >= 0 ? pend : qbase + atomicAdd(q, 1);
            nxt = __shfl_sync(kFull, c2, 0);
            if (nxt >= nitems) return;
            itn = item_at(a, nxt);
            setup(itn, crn, jbn, jen);
            fetch(jbn, jen, crn);
            spn = shape_of(min(64, itn.ni));
            load_i(itn, 0, spn);
        }
        if (lane32 == 0) pend = -1;
        cur = nxt;
        it = itn;
        jb = jbn;
        je = jen;
        sp = spn;
        slot ^= 1;
    }
}

// NPMAX: the largest i-pair count per thread; items whose shape uses the
// threads better with half of it run with NPMAX / 2
// staging words per j entry: {x, y} and {z, m} in both lanes, with DF also
// the lo parts {lx, ly} and {lz, 0}
template <bool DF> struct GroupWords { static constexpr int value = DF ? 8 : 4; };

// the staging area of a CTA: the CTA-mode tile or, after it, the warps'
// warp-mode slices, whichever is larger (u64 words)
template <bool DF, int TJ, int NT>
struct StageWords {
    static constexpr int kW = GroupWords<DF>::value;
    static constexpr int a = kW * TJ, b = (NT / 32) * kW * kWarpTJ;
    static constexpr int value = a > b ? a : b;
};

template <int NPMAX, bool TABLE, bool CELL, bool EXT, bool HL = false, bool DF = false, int TJ = kTJG,
          int NT = kNT>
__global__ void __launch_bounds__(NT) k_groups(GroupArgs a)
{
    constexpr int kW = GroupWords<DF>::value;
    static_assert(TJ % NT == 0 && NT % 32 == 0, "j tile and block size");
    extern __shared__ __align__(128) unsigned char smem[];
    u64 *cvt = reinterpret_cast<u64 *>(smem);                            // [kW][TJ], or warp slices
    u64 *run = cvt + StageWords<DF, TJ, NT>::value;                      // [8 NPMAX][NT]
    float4 *dirt = reinterpret_cast<float4 *>(run + 8 * NPMAX * NT);     // [27] cell mode
    int *sh = reinterpret_cast<int *>(dirt + 28);                        // item slot
    int *cr = sh + 4;                                                    // [warps][2][kCellTab] cell mode
    float2 *tab = reinterpret_cast<float2 *>(cr + (NT / 32) * 2 * kCellTab);

    const int tid = threadIdx.x;
    // a cell-list launch lets its warp-mode kernel start as CTAs drain
    if (CELL) asm volatile("griddepcontrol.launch_dependents;");
    if (TABLE && !EXT)
        for (int k = tid; k < a.tab.n; k += NT) tab[k] = a.tab.AG1[k];
    if (TABLE && EXT)
        for (int k = tid; k < a.tab.n; k += NT) reinterpret_cast<float4 *>(tab)[k] = a.tab.AGP[k];
    if (CELL && tid < 27)
        dirt[tid] = make_float4((float)(tid / 9 - 1) * a.cell_h, (float)((tid / 3) % 3 - 1) * a.cell_h,
                                (float)(tid % 3 - 1) * a.cell_h, 0.0f);
    const int nitems = a.nitems >= 0 ? a.nitems : (int)*a.nitems_dev;

    const int warp_from = a.warp_from >= 0 ? a.warp_from : (int)*a.warp_from_dev;

    // Thread 0 claims the next item while the current one runs (kept in a
    // register), so the queue's atomic latency overlaps work, as long as more
    // than one item per CTA is left; in that last stretch it claims only once
    // the current item is done, so that no CTA holds an item another could
    // start.
    int next = -1;
    const int ahead_limit = nitems - (int)gridDim.x;
    int first_small = -1;
    for (;;) {
        __syncthreads();   // previous item fully done with shared memory
        if (tid == 0) {
            const int cur = next >= 0 ? next : atomicAdd(a.queue, 1);
            sh[0] = cur;
            next = cur < ahead_limit ? atomicAdd(a.queue, 1) : -1;
        }
        __syncthreads();
        const int item = sh[0];
        if (item >= nitems) return;
        if (item >= warp_from) {   // the small items: continue in warp mode
            if (a.queue_w) return;  // or leave them to the warp-mode kernel
            first_small = item;
            break;
        }
        const GroupItem it = item_at(a, item);
        if (NPMAX > 1 && it.ni <= NT * NPMAX) {
            const ItemShape big = item_shape<NT>(it.ni, NPMAX);
            const ItemShape small = item_shape<NT>(it.ni, NPMAX / 2);
            if (small.nsets <= 4 * small.spw && small.nsets * small.L > big.nsets * big.L) {
                group_item<(NPMAX > 1 ? NPMAX / 2 : 1), TABLE, CELL, EXT, HL, DF, TJ, NT>(a, it, small, cvt, run,
                                                                                 cr, tab, dirt, tid);
                continue;
            }
        }
        group_item<NPMAX, TABLE, CELL, EXT, HL, DF, TJ, NT>(a, it, item_shape<NT>(it.ni, NPMAX), cvt, run, cr, tab,
                                                  dirt, tid);
    }

    // warp mode: warp 0 takes the item that ended CTA mode and thread 0's
    // prefetched claim; every warp then claims its own items
    __syncthreads();   // no warp still reads the CTA-wide staging buffer
    const int w = tid >> 5, lane32 = tid & 31;
    warp_loop<TABLE, CELL, EXT, HL, DF>(a, nitems, w == 0 ? first_small : -1,
                                      (w == 0 && lane32 == 0) ? next : -1,
                                      cvt + w * (kW * kWarpTJ), cr + w * 2 * kCellTab, tab, dirt,
                                      lane32, a.queue, 0, (int)gridDim.x * (NT / 32));
}

// The warp-mode items alone, in a launch of their own: the cell list's small
// cells (after the CTA-mode kernel, by programmatic dependent launch) and
// every item of a narrow all-pairs run whose i chunks fit one warp pass.
// Without the CTA-mode item's registers and staging buffers, more warps fit
// on an SM, which the short, latency-bound small items need. Every warp
// claims items warp_from, warp_from + 1, ... from counter queue_w.
// Two blocks of 256 threads per SM (16 warps, against 12 in the CTA-mode
// kernel) at up to 128 registers a thread; three blocks (24 warps) cap the
// registers at 80, and the spills made the uniform-cell half slower.
constexpr int kWNT = 256;          // threads per block
constexpr int kWMinBlocks = 2;     // resident blocks per SM wanted (register cap)

template <bool TABLE, bool CELL, bool EXT, bool HL = false, bool DF = false>
__global__ void __launch_bounds__(kWNT, kWMinBlocks) k_groups_warp(GroupArgs a)
{
    constexpr int kW = GroupWords<DF>::value;
    extern __shared__ __align__(128) unsigned char smem[];
    u64 *wcvt = reinterpret_cast<u64 *>(smem);                             // [warps][kW kWarpTJ]
    float4 *dirt = reinterpret_cast<float4 *>(wcvt + (kWNT / 32) * kW * kWarpTJ);  // [28]
    int *cr = reinterpret_cast<int *>(dirt + 28);                          // [warps][2][kCellTab]
    float2 *tab = reinterpret_cast<float2 *>(cr + (kWNT / 32) * 2 * kCellTab);

    const int tid = threadIdx.x;
    if (TABLE && !EXT)
        for (int k = tid; k < a.tab.n; k += kWNT) tab[k] = a.tab.AG1[k];
    if (TABLE && EXT)
        for (int k = tid; k < a.tab.n; k += kWNT) reinterpret_cast<float4 *>(tab)[k] = a.tab.AGP[k];
    if (CELL && tid < 27)
        dirt[tid] = make_float4((float)(tid / 9 - 1) * a.cell_h, (float)((tid / 3) % 3 - 1) * a.cell_h,
                                (float)(tid % 3 - 1) * a.cell_h, 0.0f);
    __syncthreads();
    const int nitems = a.nitems >= 0 ? a.nitems : (int)*a.nitems_dev;
    const int warp_from = a.warp_from >= 0 ? a.warp_from : (int)*a.warp_from_dev;
    const int w = tid >> 5, lane32 = tid & 31;
    warp_loop<TABLE, CELL, EXT, HL, DF>(a, nitems, -1, -1, wcvt + w * (kW * kWarpTJ),
                                      cr + w * 2 * kCellTab, tab, dirt, lane32, a.queue_w, warp_from,
                                      (int)gridDim.x * (kWNT / 32));
    // when launched while the CTA-mode kernel may still run (programmatic
    // dependent launch): its items are disjoint from this kernel's, and this
    // kernel ends only after that one has, so later work sees both (a no-op
    // after an ordinary launch)
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------------ host
size_t groups_smem(int np, bool table, int ntab, bool df, int tj, int nt)
{
    const size_t kw = df ? 8 : 4;
    const size_t stage = std::max<size_t>((size_t)tj * kw, (size_t)(nt / 32) * kw * kWarpTJ);
    size_t s = stage * sizeof(u64) + 8 * (size_t)np * nt * sizeof(u64) + 28 * 16 + 16 +
               (size_t)(nt / 32) * 2 * kCellTab * sizeof(int);
    if (table) s += (size_t)ntab * sizeof(float2);
    return s;
}

int groups_bi(int np, int nt) { return nt * 2 * np; }

// the compiled (j-tile depth, threads per CTA) shapes of the batched kernel:
// every path has the first; the plain Newton lists (no table, cells, per-i
// softening or double-float records) also the others, for the autotuner
bool groups_tile_ok(int tj, int nt, bool plain)
{
    if (tj == kTJG && nt == kNT) return true;
    if (!plain) return false;
    return (tj == 256 && nt == 128) || (tj == 1024 && nt == 256) || (tj == 512 && nt == 256);
}

template <int NP, bool TABLE, bool CELL, bool EXT, bool HL = false, bool DF = false, int TJ = kTJG,
          int NT = kNT>
static cudaError_t configure_g()
{
    static bool done[kMaxDevices] = {};
    return once_per_device(done, [] {
        return cudaFuncSetAttribute(k_groups<NP, TABLE, CELL, EXT, HL, DF, TJ, NT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)groups_smem(NP, TABLE, 2 << 13, DF, TJ, NT));
    });
}

template <int NP, bool TABLE, bool CELL, bool EXT, bool DF = false, int TJ = kTJG, int NT = kNT>
static int occ_g(size_t smem)
{
    if (configure_g<NP, TABLE, CELL, EXT, false, DF, TJ, NT>() != cudaSuccess) return 1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_groups<NP, TABLE, CELL, EXT, false, DF, TJ, NT>,
                                                      NT, smem) != cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

template <int NP>
static int occ_plain(int tj, int nt, size_t smem)
{
    if (tj == 256 && nt == 128) return occ_g<NP, false, false, false, false, 256, 128>(smem);
    if (tj == 1024 && nt == 256) return occ_g<NP, false, false, false, false, 1024, 256>(smem);
    if (tj == 512 && nt == 256) return occ_g<NP, false, false, false, false, 512, 256>(smem);
    return occ_g<NP, false, false, false>(smem);
}

template <int NP>
static int occ_np(bool table, bool cell, bool ext, bool df, int tj, int nt, size_t smem)
{
    if (!table && !cell && !ext && !df) return occ_plain<NP>(tj, nt, smem);
    if (df && !cell) {
        if (!table) return ext ? occ_g<NP, false, false, true, true>(smem) : occ_g<NP, false, false, false, true>(smem);
        return ext ? occ_g<NP, true, false, true, true>(smem) : occ_g<NP, true, false, false, true>(smem);
    }
    if (!table) return ext ? occ_g<NP, false, false, true>(smem) : occ_g<NP, false, false, false>(smem);
    if (cell) return ext ? occ_g<NP, true, true, true>(smem) : occ_g<NP, true, true, false>(smem);
    return ext ? occ_g<NP, true, false, true>(smem) : occ_g<NP, true, false, false>(smem);
}

int groups_max_blocks_per_sm(int np, bool table, int ntab, bool cell, bool ext, bool df, int tj, int nt)
{
    size_t smem = groups_smem(np, table, ntab, df && !cell, tj, nt);
    return np == 1 ? occ_np<1>(table, cell, ext, df, tj, nt, smem)
         : np == 4 ? occ_np<4>(table, cell, ext, df, tj, nt, smem)
                   : occ_np<2>(table, cell, ext, df, tj, nt, smem);
}

template <int NP, bool TABLE, bool CELL, bool EXT, bool HL = false, bool DF = false, int TJ = kTJG,
          int NT = kNT>
static cudaError_t launch_g(const GroupArgs &g, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = configure_g<NP, TABLE, CELL, EXT, HL, DF, TJ, NT>();
    if (e != cudaSuccess) return e;
    k_groups<NP, TABLE, CELL, EXT, HL, DF, TJ, NT><<<grid, NT, smem, st>>>(g);
    return cudaGetLastError();
}

template <int NP>
static cudaError_t launch_gnp(const GroupArgs &g, int grid, bool table, bool cell, bool ext, bool df,
                              int tj, int nt, size_t smem, cudaStream_t st)
{
    if (g.hl) {   // FP32 outputs: Newton lists only
        if (table || cell || df) return cudaErrorInvalidValue;
        return ext ? launch_g<NP, false, false, true, true>(g, grid, smem, st)
                   : launch_g<NP, false, false, false, true>(g, grid, smem, st);
    }
    if (!table && !cell && !ext && !df) {   // the plain Newton lists: every compiled tile shape
        if (tj == 256 && nt == 128) return launch_g<NP, false, false, false, false, false, 256, 128>(g, grid, smem, st);
        if (tj == 1024 && nt == 256) return launch_g<NP, false, false, false, false, false, 1024, 256>(g, grid, smem, st);
        if (tj == 512 && nt == 256) return launch_g<NP, false, false, false, false, false, 512, 256>(g, grid, smem, st);
        return launch_g<NP, false, false, false>(g, grid, smem, st);
    }
    if (df) {     // double-float differencing: particle records (no cells)
        if (cell) return cudaErrorInvalidValue;
        if (!table) return ext ? launch_g<NP, false, false, true, false, true>(g, grid, smem, st)
                               : launch_g<NP, false, false, false, false, true>(g, grid, smem, st);
        return ext ? launch_g<NP, true, false, true, false, true>(g, grid, smem, st)
                   : launch_g<NP, true, false, false, false, true>(g, grid, smem, st);
    }
    if (!table) return launch_g<NP, false, false, true>(g, grid, smem, st);
    if (cell) return ext ? launch_g<NP, true, true, true>(g, grid, smem, st)
                         : launch_g<NP, true, true, false>(g, grid, smem, st);
    return ext ? launch_g<NP, true, false, true>(g, grid, smem, st)
               : launch_g<NP, true, false, false>(g, grid, smem, st);
}

size_t groups_warp_smem(bool table, int ntab, bool df)
{
    size_t s = (kWNT / 32) * (df ? 8 : 4) * kWarpTJ * sizeof(u64) + 28 * 16 +
               (kWNT / 32) * 2 * kCellTab * sizeof(int);
    if (table) s += (size_t)ntab * sizeof(float2);
    return s;
}

template <bool TABLE, bool CELL, bool EXT, bool DF = false>
static cudaError_t configure_gw()
{
    static bool done[kMaxDevices] = {};
    return once_per_device(done, [] {
        cudaError_t e = cudaFuncSetAttribute(k_groups_warp<TABLE, CELL, EXT, false, DF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)groups_warp_smem(TABLE, 2 << 13, DF));
        // the same shared-memory carveout as the CTA-mode kernel, so that its
        // blocks can join an SM on which that kernel still runs
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_groups_warp<TABLE, CELL, EXT, false, DF>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        return e;
    });
}

template <bool TABLE, bool CELL, bool EXT, bool DF = false>
static int occ_gw(size_t smem)
{
    int nb = 0;
    if (configure_gw<TABLE, CELL, EXT, DF>() != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_groups_warp<TABLE, CELL, EXT, false, DF>, kWNT,
                                                      smem) != cudaSuccess)
        return 0;
    return nb;
}

// blocks per SM of the warp-mode kernel for a table of ntab float2 units
// (0 if the kernel cannot be configured; cell mode needs the table)
int groups_warp_blocks_per_sm(bool table, bool cell, bool ext, int ntab, bool df)
{
    if (cell && (!table || df)) return 0;
    const size_t smem = groups_warp_smem(table, ntab, df);
    if (cell) return ext ? occ_gw<true, true, true>(smem) : occ_gw<true, true, false>(smem);
    if (df) {
        if (table) return ext ? occ_gw<true, false, true, true>(smem) : occ_gw<true, false, false, true>(smem);
        return ext ? occ_gw<false, false, true, true>(smem) : occ_gw<false, false, false, true>(smem);
    }
    if (table) return ext ? occ_gw<true, false, true>(smem) : occ_gw<true, false, false>(smem);
    return ext ? occ_gw<false, false, true>(smem) : occ_gw<false, false, false>(smem);
}

int groups_warp_warps_per_block() { return kWNT / 32; }

template <bool TABLE, bool CELL, bool EXT, bool DF = false>
static cudaError_t launch_gw(const GroupArgs &g, int grid, size_t smem, bool pdl, cudaStream_t st)
{
    cudaError_t e = configure_gw<TABLE, CELL, EXT, DF>();
    if (e != cudaSuccess) return e;
    if (!pdl) {
        k_groups_warp<TABLE, CELL, EXT, false, DF><<<grid, kWNT, smem, st>>>(g);
        return cudaGetLastError();
    }
    // programmatic stream serialisation: the blocks may start once every
    // block of the kernel before it has started
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kWNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_groups_warp<TABLE, CELL, EXT, false, DF>, g);
}

cudaError_t launch_groups_warp(const GroupArgs &g, int grid, bool table, bool cell, bool ext, int ntab,
                               bool pdl, bool df, cudaStream_t st)
{
    if (grid <= 0 || !g.queue_w || (cell && (!table || df)) || g.hl) return cudaErrorInvalidValue;
    const size_t smem = groups_warp_smem(table, ntab, df);
    if (cell) return ext ? launch_gw<true, true, true>(g, grid, smem, pdl, st)
                         : launch_gw<true, true, false>(g, grid, smem, pdl, st);
    if (df) {
        if (table) return ext ? launch_gw<true, false, true, true>(g, grid, smem, pdl, st)
                              : launch_gw<true, false, false, true>(g, grid, smem, pdl, st);
        return ext ? launch_gw<false, false, true, true>(g, grid, smem, pdl, st)
                   : launch_gw<false, false, false, true>(g, grid, smem, pdl, st);
    }
    if (table) return ext ? launch_gw<true, false, true>(g, grid, smem, pdl, st)
                          : launch_gw<true, false, false>(g, grid, smem, pdl, st);
    return ext ? launch_gw<false, false, true>(g, grid, smem, pdl, st)
               : launch_gw<false, false, false>(g, grid, smem, pdl, st);
}

cudaError_t launch_groups(const GroupArgs &g, int grid, int np, bool table, bool cell, bool ext, bool df,
                          int tj, int nt, size_t smem, cudaStream_t st)
{
    if (grid <= 0) return cudaSuccess;
    if (cell && !table) return cudaErrorInvalidValue;
    if (!groups_tile_ok(tj, nt, !table && !cell && !ext && !df && !g.hl)) return cudaErrorInvalidValue;
    if (np == 1) return launch_gnp<1>(g, grid, table, cell, ext, df, tj, nt, smem, st);
    if (np == 2) return launch_gnp<2>(g, grid, table, cell, ext, df, tj, nt, smem, st);
    if (np == 4) return launch_gnp<4>(g, grid, table, cell, ext, df, tj, nt, smem, st);
    return cudaErrorInvalidValue;
}

// the FP64 outputs of a run with FP32 (hi, lo) sums: one thread per i, so
// the conversions, the permutation and the stores run on full warps
__global__ void k_groups_finish(GroupArgs a)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= a.ni) return;
    const float4 h = a.hl[2 * i], l = a.hl[2 * i + 1];
    const long long o = a.perm ? (long long)a.perm[i] : i;
    a.acc[3 * o] = ((double)h.x + (double)l.x) * a.accscale;
    a.acc[3 * o + 1] = ((double)h.y + (double)l.y) * a.accscale;
    a.acc[3 * o + 2] = ((double)h.z + (double)l.z) * a.accscale;
    if (a.pot) {
        const double phi = (double)h.w + (double)l.w;
        a.pot[o] = a.list_self ? phi - list_self_pot(a, i) : phi;
    }
}

cudaError_t launch_groups_finish(const GroupArgs &g, cudaStream_t st)
{
    if (g.ni <= 0) return cudaSuccess;
    k_groups_finish<<<(unsigned)((g.ni + 255) / 256), 256, 0, st>>>(g);
    return cudaGetLastError();
}

// Narrow all-pairs: the sum over j chunks of each i's FP64 partials in a
// fixed order (so the result does not depend on which CTA ran which item),
// then the same self-pair correction and scaling as the tiled path.
// One 128-thread block per i: thread t adds chunks t, t + 128, ..., a fixed
// butterfly adds each warp's lanes and thread 0 the four warps in order
// (hundreds of chunks would be a long chain of dependent loads for one
// thread).
constexpr int kCombineThreads = 128;

__global__ void __launch_bounds__(kCombineThreads)
k_group_partials_combine(CombineArgs c, int nchunks)
{
    __shared__ double4 wsum[kCombineThreads / 32];
    const long long i = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31;
    double ax = 0, ay = 0, az = 0, ph = 0;
    for (int k = t; k < nchunks; k += kCombineThreads) {
        const double4 v = c.part[(long long)k * c.ni + i];
        ax += v.x; ay += v.y; az += v.z; ph += v.w;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
        ph += __shfl_xor_sync(0xffffffffu, ph, o);
    }
    if (lane == 0) wsum[t >> 5] = make_double4(ax, ay, az, ph);
    __syncthreads();
    if (t != 0) return;
    ax = ay = az = ph = 0;
    for (int w = 0; w < kCombineThreads / 32; ++w) {
        ax += wsum[w].x; ay += wsum[w].y; az += wsum[w].z; ph += wsum[w].w;
    }
    if (c.self) ph -= self_potential(c, i);   // the list held i's own pair (d = 0)
    c.acc[3 * i] = ax * c.accscale;
    c.acc[3 * i + 1] = ay * c.accscale;
    c.acc[3 * i + 2] = az * c.accscale;
    if (c.pot) c.pot[i] = c.newton || c.tabpot ? ph : 0.0;
}

cudaError_t launch_group_partials_combine(const CombineArgs &c, int nchunks, cudaStream_t st)
{
    if (c.ni <= 0) return cudaSuccess;
    k_group_partials_combine<<<(unsigned)c.ni, kCombineThreads, 0, st>>>(c, nchunks);
    return cudaGetLastError();
}

// double-float records: (hi, w) then (lo, w) per particle, lo = x - hi, w
// the record's fourth value (the mass of a j record; eps^2 of an i record
// with per-i softening, else 0)
__device__ __forceinline__ void pack_hilo_one(const double4 *__restrict__ in, long long i,
                                              float4 *__restrict__ out)
{
    double4 v = in[i];
    float hx = (float)v.x, hy = (float)v.y, hz = (float)v.z;
    out[2 * i] = make_float4(hx, hy, hz, (float)v.w);
    out[2 * i + 1] = make_float4((float)(v.x - (double)hx), (float)(v.y - (double)hy),
                                 (float)(v.z - (double)hz), (float)v.w);
}

__global__ void k_pack_hilo(const double4 *__restrict__ in, long long n, float4 *__restrict__ out)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    pack_hilo_one(in, i, out);
}

cudaError_t launch_pack_hilo(const double4 *in, long long n, float4 *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_pack_hilo<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, n, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ prep
// FP64 centre of each group: midpoint of its i-particles' bounding box
// group g holds i_off[g] .. i_off[g + 1], or without offsets the chunk
// g chunk .. min((g + 1) chunk, ni)
__device__ __forceinline__ void group_ctr_warp(const double4 *__restrict__ xi,
                                               const long long *__restrict__ i_off, long long g,
                                               long long chunk, long long ni, int lane,
                                               double4 *__restrict__ ctr)
{
    const long long ib = i_off ? i_off[g] : g * chunk;
    const long long ie = i_off ? i_off[g + 1] : min((g + 1) * chunk, ni);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (long long i = ib + lane; i < ie; i += 32) {
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

__global__ void k_group_ctr(const double4 *__restrict__ xi, const long long *__restrict__ i_off,
                            long long ngroups, const long long *__restrict__ ngroups_dev, long long chunk,
                            long long ni, double4 *__restrict__ ctr)
{
    long long g = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= ngroups || (ngroups_dev && g >= *ngroups_dev)) return;
    group_ctr_warp(xi, i_off, g, chunk, ni, threadIdx.x & 31, ctr);
}

// The narrow path's preparation in one launch: the FP64 centre of each of
// the nic i chunks (one warp each, blocks [0, cb)), the double-float i
// records (blocks cb onwards, one thread each), and the two work counters
// set to zero.
__global__ void k_narrow_prep(const double4 *__restrict__ xi, long long ni, long long chunk, long long nic,
                              long long cb, double4 *__restrict__ ctr, float4 *__restrict__ ihl,
                              int *__restrict__ queue)
{
    if (blockIdx.x == 0 && threadIdx.x < 2) queue[threadIdx.x] = 0;
    if (blockIdx.x < cb) {
        const long long g = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
        if (g < nic) group_ctr_warp(xi, nullptr, g, chunk, ni, threadIdx.x & 31, ctr);
        return;
    }
    const long long i = (blockIdx.x - cb) * (long long)blockDim.x + threadIdx.x;
    if (i < ni) pack_hilo_one(xi, i, ihl);
}

cudaError_t launch_narrow_prep(const double4 *xi, long long ni, long long chunk, long long nic,
                              double4 *ctr, float4 *ihl, int *queue, cudaStream_t st)
{
    if (ni <= 0 || nic <= 0) return cudaErrorInvalidValue;
    const long long cb = (nic + 3) / 4;                  // 4 warps of 128 threads
    const long long pb = (ni + 127) / 128;
    k_narrow_prep<<<(unsigned)(cb + pb), 128, 0, st>>>(xi, ni, chunk, nic, cb, ctr, ihl, queue);
    return cudaGetLastError();
}

cudaError_t launch_group_ctr(const double4 *xi, const long long *i_off, long long ngroups,
                             long long chunk, long long ni, double4 *ctr, cudaStream_t st,
                             const long long *ngroups_dev)
{
    if (ngroups <= 0) return cudaSuccess;
    k_group_ctr<<<(unsigned)((ngroups + 3) / 4), 128, 0, st>>>(xi, i_off, ngroups, ngroups_dev, chunk, ni, ctr);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ cell list
// Periodic cube of side box, nc cells per axis (side box/nc >= r_cut). The
// FP64 pipe is narrow, so the per-particle work uses multiplies by the
// host's 1/box and nc/box instead of divisions.
__device__ __forceinline__ double wrap_box(double x, double box, double inv_box)
{
    if (x >= 0.0 && x < box) return x;            // already inside: unchanged
    double w = x - box * floor(x * inv_box);
    if (w >= box) w -= box;                       // rounding can land on box
    if (w < 0.0) w += box;                        // or just below 0
    return w;
}

__device__ __forceinline__ int cell_axis(double w, double per_len, int nc)
{
    const int c = (int)(w * per_len);             // w >= 0: truncation is floor
    return c >= nc ? nc - 1 : c;
}

// wrapped positions (x, y, z, m) and the cell key of every particle
__global__ void k_cell_key(const double4 *__restrict__ jrec, long long n, double box,
                           double inv_box, double per_len, int nc, unsigned *__restrict__ key,
                           unsigned *__restrict__ idx, double4 *__restrict__ wrapped)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 v = jrec[i];
    const double wx = wrap_box(v.x, box, inv_box), wy = wrap_box(v.y, box, inv_box),
                 wz = wrap_box(v.z, box, inv_box);
    wrapped[i] = make_double4(wx, wy, wz, v.w);
    const int cx = cell_axis(wx, per_len, nc), cy = cell_axis(wy, per_len, nc),
              cz = cell_axis(wz, per_len, nc);
    key[i] = (unsigned)((cx * nc + cy) * nc + cz);
    idx[i] = (unsigned)i;
}

__global__ void k_cell_count(const unsigned *__restrict__ key, long long n, unsigned *__restrict__ cnt)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[key[i]], 1u);
}

// particles in cell order, as FP32 offsets from their cell's corner in the
// table's scaled units (the FP64 corner is implicit in the cell index)
__global__ void k_cell_gather(const double4 *__restrict__ wrapped, const unsigned *__restrict__ perm,
                              const unsigned *__restrict__ key, long long n, int nc, double h,
                              double scale, double4 *__restrict__ xs, float4 *__restrict__ xo)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= n) return;
    double4 w = wrapped[perm[p]];
    xs[p] = w;
    unsigned c = key[p];
    int cx = (int)(c / ((unsigned)nc * nc)), cy = (int)((c / nc) % nc), cz = (int)(c % nc);
    xo[p] = make_float4((float)(fma(-(double)cx, h, w.x) * scale),
                        (float)(fma(-(double)cy, h, w.y) * scale),
                        (float)(fma(-(double)cz, h, w.z) * scale), (float)w.w);
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

// one item per (cell, chunk of <= Bi i-particles), keyed longest-first
__global__ void k_cell_items(const unsigned *__restrict__ start, long long ncell, int Bi,
                             const unsigned *__restrict__ ioff, const unsigned *__restrict__ jcount,
                             GroupItem *__restrict__ items, unsigned *__restrict__ keys,
                             unsigned *__restrict__ vals, unsigned *__restrict__ ncta)
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
        // CTA-sized items first, longest first (by cost classes a quarter
        // of a binade wide: q = 4 floor(log2 c) + the next two bits of c);
        // then the warp-sized ones. One 8-bit radix pass; 255 is left for the
        // unused slots, which sort last. The order only balances the queue:
        // each item's sums do not depend on it.
        const unsigned long long cost = (unsigned long long)it.ni * jcount[g];
        const int e = 63 - __clzll(cost | 1ull);
        const unsigned q = 4u * (unsigned)e + (unsigned)(e >= 2 ? (cost >> (e - 2)) & 3ull : (cost << (2 - e)) & 3ull);
        const unsigned cq = q > 126u ? 126u : q;
        const bool small = it.ni <= kWarpItemNi && (long long)it.ni * jcount[g] <= kWarpItemPairs;
        keys[o + k] = ((small ? 1u : 0u) << 7) | (126u - cq);
        vals[o + k] = o + k;
        if (!small) atomicAdd(ncta, 1u);
    }
}

__global__ void k_items_permute(const GroupItem *__restrict__ in, const unsigned *__restrict__ order,
                                const unsigned *__restrict__ nitems, GroupItem *__restrict__ out)
{
    long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < (long long)*nitems) out[k] = in[order[k]];
}

cudaError_t launch_cell_build(const double4 *jrec, long long n, double box, int nc, int Bi,
                              double scale, CellScratch &s, SortScratch &sort, cudaStream_t st)
{
    long long ncell = (long long)nc * nc * nc;
    unsigned gb = (unsigned)((n + 255) / 256);
    unsigned gc = (unsigned)((ncell + 255) / 256);
    k_cell_key<<<gb, 256, 0, st>>>(jrec, n, box, 1.0 / box, nc / box, nc, sort.keys[0], sort.vals[0],
                                   s.wrapped);
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
    k_cell_gather<<<gb, 256, 0, st>>>(s.wrapped, perm, ko, n, nc, box / nc, scale, s.xs, s.xo);
    k_cell_sizes<<<gc, 256, 0, st>>>(s.start, nc, Bi, s.jcount, s.icount);
    cudaMemsetAsync(s.pairs, 0, sizeof(unsigned long long), st);
    k_cell_pairs<<<gc < 1024 ? gc : 1024, 256, 0, st>>>(s.start, s.jcount, ncell, s.pairs);
    // items
    cudaMemcpyAsync(s.ioff, s.icount, ncell * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(s.ioff + ncell, 0, sizeof(unsigned), st);
    if ((e = launch_excl_scan(s.ioff, ncell + 1, sort.sums, st)) != cudaSuccess) return e;
    // unused item slots sort last
    cudaMemsetAsync(sort.keys[0], 0xff, s.item_cap * sizeof(unsigned), st);
    k_fill_iota<<<(unsigned)((s.item_cap + 255) / 256), 256, 0, st>>>(sort.vals[0], s.item_cap);
    cudaMemsetAsync(s.ncta, 0, sizeof(unsigned), st);
    k_cell_items<<<gc, 256, 0, st>>>(s.start, ncell, Bi, s.ioff, s.jcount, s.items_raw,
                                     sort.keys[0], sort.vals[0], s.ncta);
    unsigned *order;
    if ((e = launch_radix_sort(sort.keys[0], sort.vals[0], s.item_cap, 8, sort, &ko, &order, st)) !=
        cudaSuccess)
        return e;
    k_items_permute<<<(unsigned)((s.item_cap + 255) / 256), 256, 0, st>>>(s.items_raw, order,
                                                                          s.ioff + ncell, s.items);
    return cudaGetLastError();
}

}  // namespace pg
