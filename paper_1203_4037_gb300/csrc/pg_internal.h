// pg_internal.h -- launch arguments and launcher declarations shared by the
// host side of the pg library (pg_api.cu) and its kernel files. Not part of
// the public C ABI (that is include/pg.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

namespace pg {

// j sub-tile depth of the all-pairs kernel (j records staged per step)
constexpr int kTJ = 256;
// threads per CTA of the all-pairs and group kernels
constexpr int kNT = 128;
// devices a process may use (per-device set-up flags)
constexpr int kMaxDevices = 256;
// time limit of any device-side wait, in nanoseconds
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// device status word codes (status[0] = code, status[1] = where)
constexpr int kStatusTimeout = 1;
constexpr int kStatusBadIndex = 2;

// Interpolation constants of the bit-pattern table, as the kernels use them.
struct TableDev {
    const float2 *AG1;     // per knot {A_k = G0_k - s_k G1_k, G1_k}, 2^(E+F) entries
    const float4 *AGP;     // with a potential table: {A_k, G1_k, A_p,k, P1_k}, else nullptr
    int n;                 // 2^(E+F)
    int shift;             // 23 - F
    unsigned base;         // bit pattern of 2.0f >> shift (index of s = 2)
    float s_max;           // 2^(2^E) (2 - 2^-F)
    double scale;          // sqrt(s_max - 2) / r_cut: positions -> scaled units
};

// all-pairs force launch (stream-K split of (i-tile, j-sub-tile) units)
struct AllPairsArgs {
    const double4 *xi;     // i positions (x, y, z, -) in tile order
    const double4 *ctr;    // FP64 centre of each i-tile
    const double4 *jrec;   // j records (x, y, z, m), FP64
    const float4 *jhl;     // Newton, single form: the j records as double-float pairs
                           // (hi, m), (lo, m), staged instead of jrec
    long long ni, nj;
    int ntiles;            // ceil(ni / Bi)
    int njsub;             // ceil(nj / kTJ)
    long long W;           // ntiles * njsub work units
    int smax_slots;        // partial slots per tile
    float eps2;
    TableDev tab;
    double4 *part;         // partial sums [ntiles][smax_slots][Bi]
    int *status;
};

// combine partials into the outputs (fixed slot order) and scatter
struct CombineArgs {
    const double4 *part;
    const unsigned *perm;  // tile order -> caller's i index (nullptr: identity)
    const double4 *jrec;   // for the self term (mass of j = caller's i index)
    long long ni;
    int Bi, njsub, smax_slots, grid;
    long long W;
    int self;              // leave out i's own pair (i index k == j index k + self_off)
    long long self_off;    // j index of i-particle 0 in self mode
    int newton;            // 1: Newton (has potential), 0: table
    int tabpot;            // table mode with a potential table (agp set)
    const float4 *agp;     // the {A, G1, A_p, P1} table (its knot 0 gives the self term)
    int epsi;              // per-i softening: eps_k^2 in xi[k].w
    const double4 *xi;     // caller-order i records (for the per-i self term)
    float eps2;
    double accscale;       // table: r_cut / sqrt(s_max - 2); Newton: 1
    double *acc;           // out: (ni, 3)
    double *pot;           // out: (ni), may be null
    const int *fail_nan = nullptr;   // set: a nonzero word here (a force kernel's failure
                                     // status) makes every output NaN
};

// the all-pairs Newton loop of a small i-set in one launch (pg_small.cu):
// tiles of small_bi() i in caller order times nchunk chunks of jchunk j
// records (nchunk a multiple of small_cluster()), pair differences in
// double-float; each cluster sums its chunks in distributed shared memory,
// the last block of each tile adds the clusters' sums
constexpr int kSmallMaxChunk = 1024;   // j records per chunk (staged in shared memory)
struct SmallArgs {
    const float4 *ihl;     // i positions as double-float pairs (hi, -), (lo, -), caller order
    const double4 *xi;     // i records (w: eps_i^2 with per-i softening)
    const float4 *jhl;     // j records as double-float pairs (hi, m), (lo, m)
    long long ni, nj;
    int nchunk, jchunk;
    float eps2;
    int epsi;              // per-i softening: eps_i^2 in xi[i].w
    int self;              // leave out i's own pair, j index i + self_off
    long long self_off;
    float *part;           // [ntiles][nchunk / small_cluster()][8][small_bi()]: each cluster's
                           // FP32 sums, hi of x, y, z, phi then lo
    unsigned *ticket;      // [ntiles], zero between calls
    double *acc, *pot;     // out: caller order; pot may be null
};
int small_bi();
int small_cluster();                   // blocks per thread-block cluster (chunks of one tile)
int small_max_clusters(bool ext);      // clusters resident at once on the current device
int small_blocks_per_sm();
size_t small_smem(int jchunk);
cudaError_t launch_small(const SmallArgs &a, bool ext, cudaStream_t st);

// batched groups: one work item = (group, i-range of at most Bi)
struct GroupItem {
    int group;
    int i0;                // first i (index into the i array)
    int ni;                // i count in this item
    int pad;
};

struct GroupArgs {
    const double4 *xi;     // i positions (x, y, z, -)
    const double4 *jrec;   // j records (x, y, z, m)
    const long long *j_off;        // group mode: CSR offsets into jlist, ngroups + 1
    const int *jlist;      // group mode: j indices (low 27 bits)
    const GroupItem *items;
    const double4 *gctr;   // FP64 centre of each group
    int nitems;            // item count, or -1: read *nitems_dev
    const unsigned *nitems_dev;
    int warp_from;         // first warp-mode item (items after are small), -1: *warp_from_dev
    const unsigned *warp_from_dev;
    int *queue;            // work counter (reset to 0 before each launch)
    int *queue_w = nullptr;   // set: the warp-mode items run in their own launch, claimed from this counter
    long long nj;          // number of j records (bounds check)
    float eps2;
    TableDev tab;
    const float4 *jhl;     // FP64 mode: j records as (hi, m), (lo, 0) FP32 pairs
    const float4 *ihl;     // FP64 mode: i positions as (hi, -), (lo, -) FP32 pairs
    const float4 *xo;      // cell mode: FP32 offset records (o, m) in scaled units
    float cell_h;          // cell mode: cell side in scaled units
    const unsigned *cstart;        // cell mode: first particle of each cell, ncell + 1
    int nc;                // cell mode: cells per box side (>= 3)
    int jchunk;            // narrow all-pairs: item k is i chunk k / nchunks (ichunk
                           // particles from (k / nchunks) ichunk, up to ni) against the
                           // j records [pad jchunk, (pad + 1) jchunk), pad = k mod
                           // nchunks; items are not stored. 0: stored items, lists
    int nchunks, ichunk;
    long long ni;
    double4 *part;         // narrow all-pairs: raw FP64 sums (a, phi) per item,
    long long part_stride; //   at part[pad * part_stride + i]; nullptr: write acc
    int list_self;         // Newton lists that hold each i itself as j record i
                           // (the tree): its own pair is removed at the output
    const unsigned *perm;  // i index -> output index (nullptr: identity)
    double accscale;
    double *acc, *pot;
    int *status;
    float4 *hl = nullptr;  // Newton lists: the sums as FP32 (hi, lo) pairs, two float4 per i
                           // (x, y, z, phi), converted by the finish kernel (nullptr: FP64 out)
};

// backward (all-pairs, self mode)
struct BackwardArgs {
    const double4 *xi;     // i positions + mass (x, y, z, m) in tile order
    const double4 *wv;     // i loss weights (wx, wy, wz, -) in tile order
    const double4 *ctr;    // tile centres
    const double4 *jx;     // j positions + mass (record order; tile order for the Newton kernel)
    const double4 *jwv;    // j loss weights, in the order of jx
    long long n;
    int ntiles, njsub;
    long long W;
    int smax_slots;
    float eps2;
    TableDev tab;
    double4 *part;         // partials [ntiles][slots][Bi] {gx, gy, gz, gm}
    double *dv;            // knot-gradient accumulators (FP64, 2^(E+F)), may be null
    const unsigned *perm;  // tile order -> particle index (nullptr: identity): the own pair
    int *status;
};

// Run a kernel's one-time set-up f (a function attribute) once on each
// device: attributes belong to the device's context, so a process that uses
// a second GPU sets them there too. `done` is the caller's per-kernel flags.
template <typename F>
inline cudaError_t once_per_device(bool (&done)[kMaxDevices], F f)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool slot = dev >= 0 && dev < kMaxDevices;
    if (slot && done[dev]) return cudaSuccess;
    e = f();
    if (e == cudaSuccess && slot) done[dev] = true;
    return e;
}

// ---------------------------------------------------------------- launchers
// all return cudaError_t of the launch

cudaError_t launch_pack_j(const double *x, const double *m, double4 *jrec, long long n,
                          cudaStream_t st);
// i records, and with ihl set also their double-float pairs (hi, 0), (lo, 0)
cudaError_t launch_pack_i(const double *x, double4 *xi, long long n, cudaStream_t st,
                          float4 *ihl = nullptr);

// spatial ordering of i: Morton keys in the bounding box, LSD radix sort
struct SortScratch {
    unsigned *keys[2];
    unsigned *vals[2];
    unsigned *hist;        // 256 * nchunks (+ block sums)
    unsigned *sums;
    unsigned long long *bbox;  // 6 ordered-int words
    size_t cap;            // elements
    size_t hist_cap;
};
size_t sort_hist_entries(long long n);
cudaError_t launch_morton_sort(const double4 *xi, long long n, SortScratch &s, unsigned **perm_out,
                               cudaStream_t st);
cudaError_t launch_radix_sort(unsigned *keys, unsigned *vals, long long n, int key_bits,
                              SortScratch &s, unsigned **keys_out, unsigned **vals_out,
                              cudaStream_t st);

// ---------------------------------------------------------------- PM
// The particle-mesh long-range force (pg_pm.cu): mesh, plans and tables,
// kept between calls. pm_run assigns the ns source records (x, y, z, m) to
// an N^3 mesh over the periodic cube of side L, solves with the split
// (0: Gaussian exp(-k^2 scale^2), 1: S2 clouds of diameter scale), and
// writes (or adds) the acceleration (3 per target) and potential (may be
// null) at the nt target records. Returns a PG_* code, err says what failed.
struct PmState;
PmState *pm_create();
void pm_destroy(PmState *s);
// 0: the hand-written FFTs for a power-of-two mesh from 8 to 512 (cuFFT
// for other sizes), 1: cuFFT always; the last solve's FFT (1 hand-written,
// 2 cuFFT, 0 none yet)
void pm_set_fft(PmState *s, int mode);
int pm_last_fft(const PmState *s);
// the hand-written mesh solve (pg_fft.cu): rho (N^3) to the four fields
// (4 N^3: -dphi/dx, -dphi/dy, -dphi/dz, phi) with the Green's table gtab
// (by n^2) and the window table wtab (by index), kf = 2 pi / L; scratch S
// (N^2 N/2 complex) and W (3 N^2 N/2 complex); tw from fft_twiddles
bool fft_mesh_ok(int N);
void fft_twiddles(int N, float2 *host);
cudaError_t fft_solve(const float *rho, float *field, float2 *S, float2 *W, const float2 *tw, const float *gtab,
                      const float *wtab, float kf, int N, cudaStream_t st);
// tgt_order: an interpolation order of the targets to use instead of sorting
// them into mesh order (a permutation of 0 .. nt-1 that keeps neighbours
// together; the cell list's cell order), or nullptr
int pm_run(PmState *s, const double4 *src, long long ns, const double4 *tgt, long long nt, double L, int N,
           int split, double scale, double *acc, double *pot, bool add, SortScratch &sort, cudaStream_t st,
           int *launches, std::string &err, const unsigned *tgt_order = nullptr);
// the same in two steps, for sources split across ranks: pm_deposit writes
// the density mesh of its sources into rho (N^3 FP32, row-major, z fastest;
// mass per cell volume), which the ranks sum; pm_solve computes the fields
// from a (summed) mesh and interpolates them at its targets
int pm_deposit(PmState *s, const double4 *src, long long ns, double L, int N, int split, double scale,
               float *rho, SortScratch &sort, cudaStream_t st, int *launches, std::string &err);
int pm_solve(PmState *s, const float *rho, const double4 *tgt, long long nt, double L, int N, int split,
             double scale, double *acc, double *pot, bool add, SortScratch &sort, cudaStream_t st,
             int *launches, std::string &err);


// gather i into tile order and compute tile centres
cudaError_t launch_tile_prep(const double4 *xi, const unsigned *perm, long long n, int Bi,
                             double4 *xi_tiled, double4 *ctr, cudaStream_t st);

// df: double-float differencing (i-tiles that are not compact; packed
// arithmetic whatever `packed` says)
cudaError_t launch_allpairs(const AllPairsArgs &a, int grid, int np, bool table, bool ext,
                            bool packed, bool df, size_t smem, cudaStream_t st);
int allpairs_bi(int np);
// ntab: the table's size in float2 units (twice the knot count with a
// potential table)
size_t allpairs_smem(int np, bool table, int ntab, bool ext, bool df);
int allpairs_max_blocks_per_sm(int np, bool table, int ntab, bool packed, bool ext, bool df);
cudaError_t launch_combine(const CombineArgs &c, cudaStream_t st);
long long stream_k_first(long long u, int grid, long long W);

cudaError_t launch_table_prep(const float *G0, const float *G1, float2 *AG1, int E, int F,
                              cudaStream_t st);
cudaError_t launch_table_from_values(const float *v, float *G0, float *G1, int E, int F,
                                     cudaStream_t st);

// df: double-float differencing of particle records (narrow all-pairs)
// tj, nt: the kernel's j-tile depth and threads per CTA (groups_tile_ok)
cudaError_t launch_groups(const GroupArgs &g, int grid, int np, bool table, bool cell, bool ext, bool df,
                          int tj, int nt, size_t smem, cudaStream_t st);
// the FP64 outputs of a groups run made with g.hl set: one thread per i
cudaError_t launch_groups_finish(const GroupArgs &g, cudaStream_t st);
// one device-side bounded wait that nothing ends (the timeout path's self-test)
cudaError_t launch_wait_selftest(int *status, unsigned long long limit_ns, cudaStream_t st);
cudaError_t launch_pack_hilo(const double4 *in, long long n, float4 *out, cudaStream_t st);
// narrow path: chunk centres (chunks of `chunk` i, nic of them), double-float
// i records and the two work counters zeroed, in one launch
cudaError_t launch_narrow_prep(const double4 *xi, long long ni, long long chunk, long long nic,
                              double4 *ctr, float4 *ihl, int *queue, cudaStream_t st);
// the batched kernel's j-tile depth and threads per CTA by default, and
// whether (tj, nt) is compiled (every path: the default; plain Newton lists:
// also 256 x 128, 1024 x 256 and 512 x 256)
constexpr int kGroupsTJ = 512, kGroupsNT = 128;
bool groups_tile_ok(int tj, int nt, bool plain);
size_t groups_smem(int np, bool table, int ntab, bool df, int tj = kGroupsTJ,
                   int nt = kGroupsNT);   // ntab in float2 units, as above
int groups_bi(int np, int nt = kGroupsNT);
int groups_max_blocks_per_sm(int np, bool table, int ntab, bool cell, bool ext, bool df,
                             int tj = kGroupsTJ, int nt = kGroupsNT);
// warp-mode items in a launch of their own (k_groups_warp): the cell list's
// small cells after the CTA-mode kernel (pdl: programmatic dependent launch,
// for a kernel whose inputs were complete before the CTA-mode kernel
// started), and narrow all-pairs items (ordinary launch); g.queue_w set
size_t groups_warp_smem(bool table, int ntab, bool df);
int groups_warp_blocks_per_sm(bool table, bool cell, bool ext, int ntab, bool df);
int groups_warp_warps_per_block();
cudaError_t launch_groups_warp(const GroupArgs &g, int grid, bool table, bool cell, bool ext, int ntab,
                               bool pdl, bool df, cudaStream_t st);
cudaError_t launch_table_merge(const float2 *AG1, const float *P0, const float *P1, float4 *AGP,
                               int E, int F, cudaStream_t st);
cudaError_t launch_set_w(double4 *x, const double *eps, long long n, cudaStream_t st);
// ngroups_dev set: the group count is read on the device (ngroups bounds it)
cudaError_t launch_group_ctr(const double4 *xi, const long long *i_off, long long ngroups,
                             long long chunk, long long ni, double4 *ctr, cudaStream_t st,
                             const long long *ngroups_dev = nullptr);

// periodic cell list: particles binned and sorted by cell, one group per
// cell whose j-list is the 27 neighbour cells with image shift codes
struct CellScratch {
    double4 *wrapped;      // n: positions wrapped into the box (input order)
    double4 *xs;           // n: wrapped positions + mass in cell order
    float4 *xo;            // n: FP32 offsets from the cell corner (scaled) + mass, cell order
    unsigned *perm;        // n: cell order -> input index (own copy)
    unsigned *start;       // ncell + 1: first particle of each cell
    unsigned *jcount;      // ncell: particles in the 27 neighbour cells
    unsigned *icount;      // ncell: items of each cell
    unsigned *ioff;        // ncell + 1 (ioff[ncell] = number of items)
    GroupItem *items_raw;  // item_cap
    GroupItem *items;      // item_cap, longest first
    long long item_cap;
    unsigned long long *pairs;   // evaluated pairs of the build (device)
    unsigned *ncta;        // number of CTA-mode items (they sort first)
};
// the tree front end (device buffers; sizes in the comments)
// a node as the walk reads it: centre of mass rounded to FP32, and its
// particles and children
struct alignas(16) TreeNodeW {
    float cx, cy, cz, pad;
    int first, count, child0, childn;
};

// the walk's FP32 pre-test of the opening criterion: bounds that decide it
// for certain, else the FP64 test decides (see the walk kernel)
struct WalkFilter {
    double s2[11];              // side^2 per level, as the FP64 test rounds it
    float s2lo[11], s2hi[11];   // s2 rounded down and up to FP32
    float e;                    // bound on the FP32 per-axis distance error
    float t2lo, t2hi;           // theta^2 rounded down and up
    int on;                     // magnitudes in the range the bounds assume
};

// The tree call's counts, kept on the device: every stage after the one
// that produces a count reads it here, so a call needs no read-back before
// its end. flags records a count that exceeded the room the host gave it
// (the call's results are then void and it runs again with exact sizes) or
// a limit of the method.
struct TreeMeta {
    long long lev_off[12];      // nodes of level L: [lev_off[L], lev_off[L + 1])
    long long nnodes, ngroups, nlist;
    unsigned long long ent;     // list entries, 64-bit sum over the groups
    unsigned long long pairs;   // pairs the force kernel evaluates
    unsigned nitems;            // its work items
    unsigned next[2];           // group walk: claim counters (count, fill pass)
    unsigned qmax;              // group walk: most opened nodes one level held
    unsigned emit_next;         // group walk: emitters placed so far
    int flags;                  // kTree* bits
};
constexpr int kTreeRoomNodes = 1;    // nodes beyond the room
constexpr int kTreeRoomGroups = 2;   // groups beyond the room
constexpr int kTreeRoomList = 4;     // list entries beyond the room
constexpr int kTreeWalkQueue = 8;    // a group's walk opened more nodes than its queue holds
constexpr int kTreeTooLarge = 16;    // particles + pseudo-particles reach 2^27
constexpr int kTreeListLong = 32;    // list entries reach 2^32
constexpr int kTreeRoomMask = kTreeRoomNodes | kTreeRoomGroups | kTreeRoomList;
// opened nodes one warp's walk holds per level (the 2^20-particle Plummer
// and King W0 = 9 trees at theta = 0.75 open at most 66)
constexpr int kGroupWalkQ = 512;
// emitters (accepted nodes, leaves) one warp records for its group
constexpr int kGroupWalkScratch = 4096;

struct TreeScratch {
    unsigned long long *bbox;   // 6: ordered-int min and max per axis
    double *geo;                // 5: root corner, span, 1024 / span
    unsigned *key, *perm;       // n: keys in key order, key order -> input index
    double4 *xs, *xi0;          // n: particles in key order (x, m), (x, 0)
    unsigned *scan;             // 11 (n + 1) + 1: run flags of every level, scanned into node indices
    unsigned *tsums;            // scan sums for it
    TreeMeta *meta;             // the call's counts
    long long cap_nodes, cap_groups, cap_list;   // the room given to nodes, groups, list entries
    long long hint_runs[11];    // nodes per level of the last call: grid sizes only
    // the group walk's recorded decisions (nullptr: not recorded): per warp a
    // scratch of kGroupWalkScratch emitters, the emitters of every group
    // (emit_cap room), and per group its (first emitter, count), first = -1
    // where the fill pass walks again
    unsigned *wscratch, *emit;
    long long emit_cap;
    int2 *gemit;
    int *first, *count, *child0, *childn;   // nnodes
    unsigned char *lev;         // nnodes
    double *M, *S;              // nnodes, 3 nnodes
    int *gat;                   // n: group node at its first particle, else -1
    unsigned *gscan;            // n + 1
    int *g_i0, *g_ni;           // groups
    double *gbox;               // 6 per group
    double4 *gctr;              // per group: its box's midpoint (the force kernel's origin)
    float4 *gboxf;              // 2 per group: the box rounded to FP32
    TreeNodeW *nodew;           // nnodes
    double4 *com;               // nnodes: centre of mass (S / M, M)
    double *T;                  // 6 nnodes: second moments (quadrupole pseudo-particles)
    int *big_list;              // nnodes: nodes of three or more particles (quadrupole)
    unsigned *nbig;             // 1: their count
    int npseudo;                // pseudo-particles per node: 1 or 3
    WalkFilter *filt;           // 1
    long long *i_off;           // groups + 1
    unsigned *jcount;           // groups + 1
    long long *j_off;           // groups + 1
    int *jlist;                 // list entries
    double4 *jrec2;             // n + P nnodes: particles, then pseudo-particles
    unsigned *item_off;         // groups + 1
    GroupItem *items;
    unsigned long long *pairs;  // 2: pairs, work items
    // the walk: one (group, node) pair per visit, all levels
    int *vg, *vk;               // visits: group, node (~node once accepted)
    unsigned *ve;               // visits + 1: entries per decision, then scanned
    unsigned *vc;               // one level + 1: children opened, then scanned
    unsigned *vsums;            // scan sums for the visit arrays
    unsigned *seg;              // 2 * 11 * groups: visit span [first, end) per level and group
    long long *base;            // 11 * groups: list position shift per group and level
    unsigned long long *etot;   // 2: 64-bit total of the entries, list length
    int launches;               // kernels the stages launched
};
// The tree call's stages. Every stage reads the counts of the stages
// before it from t.meta and checks the room it writes into against t.cap_*;
// a count beyond its room sets a flag and the kernels after it do nothing.
// keys: sort, every level's runs, level offsets and node count
cudaError_t tree_stage_keys(const double4 *jrec, long long n, TreeScratch &t, SortScratch &sort,
                            cudaStream_t st);
// node starts, counts and children; then, independent of each other, the
// moments (with the monopole records and second moments) and the groups
cudaError_t tree_stage_links(long long n, TreeScratch &t, cudaStream_t st);
cudaError_t tree_stage_moments(long long n, TreeScratch &t, cudaStream_t st);
cudaError_t tree_stage_groups(long long n, int ncrit, TreeScratch &t, SortScratch &sort, cudaStream_t st);
// the j records: particles in key order, pseudo-particles
cudaError_t tree_stage_jrec(long long n, int sms, TreeScratch &t, cudaStream_t st);
// the groups' boxes and the walk's FP32 pre-test bounds (both walks)
cudaError_t tree_walk_prep(double theta, TreeScratch &t, cudaStream_t st);
// the group walk (one warp per group): the count pass with the list offsets
// (fill = false), then the fill pass writing jlist
cudaError_t tree_group_walk(bool fill, long long n, double theta, int nleaf, int sms, TreeScratch &t,
                            SortScratch &sort, int *status, cudaStream_t st);
// warps of the group walk's grid (the emitter scratch holds one slice each)
long long group_walk_warps(int sms);
// the level walk (all groups level by level; sizes from the host): init
// puts every group at the root; level L decides its frontier (visits
// [o, o + nf)) and scans the opened children, whose count is vc[nf]; expand
// writes them after the frontier; lists places every entry (offsets j_off),
// fill writes jlist
cudaError_t tree_walk_init(long long ngroups, TreeScratch &t, cudaStream_t st);
cudaError_t tree_walk_level(long long n, long long ngroups, int L, long long o, long long nf,
                            double theta, int nleaf, TreeScratch &t, cudaStream_t st);
cudaError_t tree_walk_expand(long long o, long long nf, TreeScratch &t, cudaStream_t st);
cudaError_t tree_walk_lists(long long ngroups, const long long *lev_v, int nlev, TreeScratch &t,
                            SortScratch &sort, cudaStream_t st);
cudaError_t tree_walk_fill(long long n, long long ngroups, const long long *lev_v, int nlev,
                           TreeScratch &t, int *status, cudaStream_t st);
// the force kernel's work items (groups cut into chunks of Bi), their count
// and the pairs
cudaError_t tree_stage_records(int Bi, TreeScratch &t, SortScratch &sort, cudaStream_t st);

// narrow all-pairs: part[k ni + i] for j chunks k = 0 .. nchunks - 1 (the
// tile fields of c are unused)
cudaError_t launch_group_partials_combine(const CombineArgs &c, int nchunks, cudaStream_t st);
cudaError_t launch_cell_build(const double4 *jrec, long long n, double box, int nc, int Bi,
                              double scale, CellScratch &s, SortScratch &sort, cudaStream_t st);
cudaError_t launch_excl_scan(unsigned *a, long long n, unsigned *sums, cudaStream_t st);

// backward
cudaError_t launch_backward(const BackwardArgs &a, int grid, bool table, size_t smem,
                            cudaStream_t st);
size_t backward_smem(bool table, int ntab);
int backward_bi();
int backward_max_blocks_per_sm(bool table, int ntab);
cudaError_t launch_pack_w(const double *w, const unsigned *perm, long long n, double4 *wj,
                          double4 *wt, cudaStream_t st);
cudaError_t launch_backward_combine(const double4 *part, const unsigned *perm, long long n,
                                    int njsub, int slots, int grid, long long W, double mscale,
                                    double *dx, double *dm, cudaStream_t st);
cudaError_t launch_dv_out(const double *acc, int n, double scale, float *dv, cudaStream_t st);

}  // namespace pg
