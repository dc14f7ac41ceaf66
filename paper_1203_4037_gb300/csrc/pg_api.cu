// pg_api.cu -- the C ABI of include/pg.h: context state, argument checks,
// host-side table construction (Section 3.4.1), staging copies, and the
// launch sequences of the force paths, optionally captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pg.h"
#include "pg_internal.h"

static_assert(pg::kGroupWalkQ == PG_TREE_WALK_QUEUE, "the group walk's queue is the documented one");

using namespace pg;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct PinBuf {
    void *p = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;   // last copy out of / into this buffer
};

}  // namespace

struct pg_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    // the tree call's second stream (the moments chain and the record
    // packing beside the groups and the walk) and its events: links built,
    // moments done, j records packed
    cudaStream_t side_stream = nullptr;
    cudaEvent_t tree_ev[3] = {nullptr, nullptr, nullptr};
    cudaStream_t stream = nullptr;
    int sms = 0;

    double eps = 0.0;
    int mode = PG_NEWTON;
    int self = 0;
    double box = 0.0;

    // table
    bool have_table = false;
    // table-mode potential: P0/P1 from psi's knot values, interleaved with
    // the force table as {A, G1, A_p, P1} (pot_* = the geometry it was built on)
    bool have_pot = false;
    int pot_E = -1, pot_F = -1;
    double pot_rcut = 0.0;
    // per-i softening (device eps per i; written into the i records' w)
    bool have_epsi = false, epsi_applied = false, w_dirty = false;
    long long n_epsi = 0;
    int E = 0, F = 0, ntab = 0;
    double r_cut = 0.0, scale = 1.0, s_max = 0.0;
    DevBuf G0, G1, AG1, P0, P1, AGP, epsi;

    // j
    long long nj_n = -1;          // pg_set_n, -1: unset
    long long nj_hw = 0;          // high-water mark of set_j
    DevBuf jrec;                  // double4 records
    DevBuf stage;                 // raw FP64 staging for host copies

    // i
    long long ni = -1;
    DevBuf xi;                    // double4
    bool i_dirty = true;

    // tiles and ordering
    DevBuf xt, ctr;
    SortScratch sort{};
    DevBuf skeys0, skeys1, svals0, svals1, shist, ssums, sbbox;
    unsigned *perm = nullptr;     // tile order -> i index (nullptr: identity)
    int sort_mode = -1;           // -1 auto, 0 never, 1 always
    int tiled_np = 0;

    // outputs and partials
    DevBuf acc, pot, part;
    DevBuf tickets;               // the small path's per-tile tickets (kept at zero between runs)
    int small_clusters[2] = {-1, -1};   // its resident clusters (without, with EXT; -1: not asked)
    size_t tickets_zeroed = 0;    // bytes of it known to be zero
    DevBuf status;                // 2 ints

    // host staging
    PinBuf pin_j, pin_i, pin_o;

    // groups (host copies of the CSR offsets rebuild the items when the
    // launch shape changes)
    bool have_groups = false;

    // tree front end (theta >= 0: on); device buffers by role, sizes of the
    // last build {n, nodes, groups, list entries, items, pseudo-particles per
    // node}
    // particle-mesh long-range force (pm_n > 0: on): mesh size, split
    // (0 Gaussian, 1 S2) and its scale; records and buffers of the
    // stand-alone entry points
    PmState *pm = nullptr;
    int pm_fft = PG_FFT_AUTO;
    int pm_n = 0, pm_split = 0;
    double pm_scale = 0.0;
    DevBuf pm_rec, pm_x, pm_m, pm_acc, pm_pot;

    bool tree_on = false;
    bool tree_quad = false;
    double tree_theta = 0.75;
    int tree_ncrit = 64, tree_nleaf = 8;
    int tree_walk_mode = PG_TREE_WALK_AUTO;
    enum { TB_BBOX, TB_GEO, TB_KEY, TB_PERM, TB_XS, TB_XI0, TB_SCAN, TB_META, TB_FIRST, TB_COUNT,
           TB_CHILD0, TB_CHILDN, TB_LEV, TB_M, TB_S, TB_GAT, TB_GSCAN, TB_GI0, TB_GNI, TB_GBOX,
           TB_IOFF, TB_JCOUNT, TB_JOFF, TB_JLIST, TB_JREC2, TB_ITEMOFF, TB_ITEMS,
           TB_VG, TB_VK, TB_VE, TB_VC, TB_VSUMS, TB_SEG, TB_BASE, TB_GBOXF, TB_NODEW,
           TB_FILT, TB_COM, TB_T, TB_BIG, TB_NBIG, TB_TSUMS, TB_HL, TB_WSCR, TB_EMIT, TB_GEMIT, TB_N };
    DevBuf tb[TB_N];
    long long tree_sizes[6] = {0, 0, 0, 0, 0, 0};
    // the room the last exact tree call left (nodes, groups, list entries),
    // for the n and pseudo-particle count it ran with, and its nodes per
    // level; a later call with the same n and P runs from these without
    // reading counts back (tree_fast)
    long long tree_cap[3] = {0, 0, 0};
    long long tree_cap_n = -1;
    int tree_cap_p = 0;
    long long tree_hint[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    bool tree_fast = false;
    long long tree_stats[4] = {0, 0, 0, 0};   // walk (1 group, 2 level), exact, queue peak, read-backs
    long long ngroups = 0;
    std::vector<long long> h_ioff, h_joff;
    DevBuf g_ioff, g_joff, g_jlist, g_items, g_ctr, g_queue, g_jhl, g_ihl;
    int g_nitems = 0;
    int g_warp_from = 0;
    int g_items_np = 0, g_items_nt = 0;   // the shape the stored items were cut for
    int g_tj = 0, g_nt = 0;       // batched kernel's j-tile depth and threads per CTA (0: default)
    int last_tj = 0, last_nt = 0; // those of the last batched launch
    long long g_pairs = 0;
    long long g_maxj = -1;       // largest j index listed

    // periodic cell list
    CellScratch cells{};
    DevBuf c_wrapped, c_xs, c_xo, c_perm, c_start, c_jcount, c_icount, c_ioff, c_items_raw,
        c_items, c_pairs;
    bool pairs_on_device = false;

    // narrow all-pairs (few i against many j): items (i chunk, j chunk) of
    // the groups kernel, FP64 partials per j chunk
    int path = PG_PATH_AUTO;
    DevBuf n_part;
    long long jhl_n = -1;         // j records in g_jhl as double-float pairs (-1: stale)
    long long ihl_n = -1;         // i-particles in g_ihl as double-float pairs, caller order (-1: stale)

    // backward
    DevBuf bw_wj, bw_wt, bw_dv;

    // launch shape (np = 0: chosen by problem size)
    int np = 0;
    int ctas_per_sm = 0;
    int packed = 1;             // f32x2 pair arithmetic (0: scalar FP32)
    int split = 0;              // narrow path: items per warp of the launch (0: one)

    // graph
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;
    std::string gkey;
    bool graph_jhl = false;     // the captured run reads the double-float j records

    // force-kernel timing (events recorded as graph nodes while capturing)
    bool capturing = false;
    bool timing = false;
    cudaEvent_t tk0 = nullptr, tk1 = nullptr;
    bool timed = false;

    // stats of the last run
    int last_np = 2;
    int diff_mode = 0;            // PG_DIFF_AUTO / SINGLE / DOUBLE (all-pairs paths)
    long long self_off = 0;       // self mode: i-particle k is j-particle self_off + k
    bool last_df = false;         // the last force kernel differenced in double-float
    long long last_pairs = 0, last_launches = 0, last_grid = 0, last_slots = 0, last_split = 0;

    std::string err;
};

static std::string g_create_err;

namespace {

int fail(pg_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(pg_ctx *c, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return fail(c, PG_ECUDA, m);
}

#define PG_CUDA(c, call)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

// a force-kernel timing event: while a graph is being captured the record
// becomes a graph node that records on every replay
cudaError_t record_timing(pg_ctx *c, cudaEvent_t ev)
{
    return c->capturing ? cudaEventRecordWithFlags(ev, c->stream, cudaEventRecordExternal)
                        : cudaEventRecord(ev, c->stream);
}

void drop_graph(pg_ctx *c);

// grows device buffer b to hold bytes; a captured graph holds the old
// address, so a reallocation also drops it
int ensure(pg_ctx *c, DevBuf &b, size_t bytes)
{
    if (bytes <= b.cap) return PG_OK;
    if (b.p) {
        drop_graph(c);
        // a fault of earlier work surfaces here, not at a later call
        const cudaError_t se = cudaStreamSynchronize(c->stream);
        cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
        if (se != cudaSuccess) return cuda_fail(c, se, "synchronisation before a buffer reallocation");
    }
    size_t want = std::max<size_t>(bytes, 256);
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(c, PG_ENOMEM, "device allocation of " + std::to_string(want) + " bytes failed");
    }
    b.cap = want;
    return PG_OK;
}

int ensure_pin(pg_ctx *c, PinBuf &b, size_t bytes);

// host memory the device can reach by DMA (page-locked or registered)
bool host_pinned(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

// a copy from the caller's page-locked memory, in stream order, finished
// before the call returns (the caller may then reuse the memory)
int copy_pinned_in(pg_ctx *c, void *dst, const void *src, size_t bytes, PinBuf &b)
{
    int rc;
    if ((rc = ensure_pin(c, b, 0))) return rc;      // the event; earlier copies through b done
    PG_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    PG_CUDA(c, cudaEventRecord(b.done, c->stream));
    PG_CUDA(c, cudaEventSynchronize(b.done));
    return PG_OK;
}

int ensure_pin(pg_ctx *c, PinBuf &b, size_t bytes)
{
    if (!b.done) {
        if (cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "cudaEventCreate");
    }
    // the previous copy through this buffer must have finished
    if (b.p) PG_CUDA(c, cudaEventSynchronize(b.done));
    if (bytes <= b.cap) return PG_OK;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t want = std::max<size_t>(bytes, 4096);
    if (cudaHostAlloc(&b.p, want, cudaHostAllocDefault) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(c, PG_ENOMEM, "pinned allocation of " + std::to_string(want) + " bytes failed");
    }
    b.cap = want;
    return PG_OK;
}

void free_dev(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

void free_pin(PinBuf &b)
{
    if (b.p) cudaFreeHost(b.p);
    if (b.done) cudaEventDestroy(b.done);
    b = PinBuf();
}

void drop_graph(pg_ctx *c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gkey.clear();
    c->graph_jhl = false;
}

long long nj_of(const pg_ctx *c) { return c->nj_n >= 0 ? c->nj_n : c->nj_hw; }

// FP32 bit pattern of knot k (Section 3.4.1: 2.0f plus k ticks of 2^(23-F))
float knot_s(int k, int F)
{
    unsigned u = 0x40000000u + ((unsigned)k << (23 - F));
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

int check_EF(pg_ctx *c, double r_cut, int E, int F)
{
    if (!(r_cut > 0.0) || !std::isfinite(r_cut))
        return fail(c, PG_EINVAL, "r_cut must be positive and finite");
    if (E < 0 || F < 0 || E > 7 || F > 20 || E + F < 1 || E + F > 13)
        return fail(c, PG_EINVAL, "need E, F >= 0, E <= 7, F <= 20, 1 <= E+F <= 13");
    return PG_OK;
}

// geometry shared by every table setter
void set_geometry(pg_ctx *c, double r_cut, int E, int F)
{
    c->E = E;
    c->F = F;
    c->ntab = 1 << (E + F);
    c->r_cut = r_cut;
    c->s_max = (double)knot_s(c->ntab - 1, F);   // = 2^(2^E) (2 - 2^-F)
    c->scale = std::sqrt(c->s_max - 2.0) / r_cut;
}

// after the force table changed: rebuild the interleaved table with the
// potential on the same knots, or drop the potential if the knots moved
int remerge_pot(pg_ctx *c)
{
    if (!c->have_pot) return PG_OK;
    if (c->pot_E != c->E || c->pot_F != c->F || c->pot_rcut != c->r_cut) {
        c->have_pot = false;
        return PG_OK;
    }
    PG_CUDA(c, launch_table_merge((const float2 *)c->AG1.p, (const float *)c->P0.p,
                                  (const float *)c->P1.p, (float4 *)c->AGP.p, c->E, c->F, c->stream));
    return PG_OK;
}

// G0/G1 from host knot values; then the device copies and the {A, G1} form
int upload_table(pg_ctx *c, const std::vector<float> &v)
{
    int n = c->ntab;
    std::vector<float> g0(n), g1(n);
    for (int k = 0; k < n; ++k) {
        if (k < n - 1) {
            double ds = (double)knot_s(k + 1, c->F) - (double)knot_s(k, c->F);
            g0[k] = v[k];
            g1[k] = (float)(((double)v[k + 1] - (double)v[k]) / ds);
        } else {
            g0[k] = 0.0f;
            g1[k] = 0.0f;
        }
    }
    int rc;
    if ((rc = ensure(c, c->G0, n * 4)) || (rc = ensure(c, c->G1, n * 4)) ||
        (rc = ensure(c, c->AG1, n * 8)))
        return rc;
    PG_CUDA(c, cudaMemcpyAsync(c->G0.p, g0.data(), n * 4, cudaMemcpyHostToDevice, c->stream));
    PG_CUDA(c, cudaMemcpyAsync(c->G1.p, g1.data(), n * 4, cudaMemcpyHostToDevice, c->stream));
    PG_CUDA(c, launch_table_prep((float *)c->G0.p, (float *)c->G1.p, (float2 *)c->AG1.p, c->E,
                                 c->F, c->stream));
    if ((rc = remerge_pot(c))) return rc;
    // the host vectors go out of scope: wait for the copies
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_table = true;
    drop_graph(c);
    return PG_OK;
}

// P0/P1 of a potential shape from host knot values (the same construction
// and cutoff reading as the force table), then the interleaved table
int upload_pot(pg_ctx *c, const std::vector<float> &v)
{
    int n = c->ntab;
    std::vector<float> p0(n), p1(n);
    for (int k = 0; k < n; ++k) {
        if (k < n - 1) {
            double ds = (double)knot_s(k + 1, c->F) - (double)knot_s(k, c->F);
            p0[k] = v[k];
            p1[k] = (float)(((double)v[k + 1] - (double)v[k]) / ds);
        } else {
            p0[k] = 0.0f;
            p1[k] = 0.0f;
        }
    }
    int rc;
    if ((rc = ensure(c, c->P0, n * 4)) || (rc = ensure(c, c->P1, n * 4)) ||
        (rc = ensure(c, c->AGP, (size_t)n * 16)))
        return rc;
    PG_CUDA(c, cudaMemcpyAsync(c->P0.p, p0.data(), n * 4, cudaMemcpyHostToDevice, c->stream));
    PG_CUDA(c, cudaMemcpyAsync(c->P1.p, p1.data(), n * 4, cudaMemcpyHostToDevice, c->stream));
    PG_CUDA(c, launch_table_merge((const float2 *)c->AG1.p, (const float *)c->P0.p,
                                  (const float *)c->P1.p, (float4 *)c->AGP.p, c->E, c->F, c->stream));
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_pot = true;
    c->pot_E = c->E;
    c->pot_F = c->F;
    c->pot_rcut = c->r_cut;
    drop_graph(c);
    return PG_OK;
}

TableDev table_dev(const pg_ctx *c)
{
    TableDev t{};
    t.AG1 = (const float2 *)c->AG1.p;
    t.AGP = c->have_pot ? (const float4 *)c->AGP.p : nullptr;
    t.n = c->ntab;
    t.shift = 23 - c->F;
    t.base = 0x40000000u >> (23 - c->F);
    t.s_max = (float)c->s_max;
    t.scale = c->scale;
    return t;
}

int read_status(pg_ctx *c)
{
    if (!c->status.p) return PG_OK;
    int st[2] = {0, 0};
    PG_CUDA(c, cudaMemcpyAsync(st, c->status.p, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (st[0] != 0) {
        PG_CUDA(c, cudaMemsetAsync(c->status.p, 0, 2 * sizeof(int), c->stream));
        char buf[128];
        snprintf(buf, sizeof buf, "device-side wait gave up (code %d, site %d)", st[0], st[1]);
        return fail(c, st[0] == kStatusTimeout ? PG_ETIMEOUT : PG_ECUDA, buf);
    }
    return PG_OK;
}

int prep_sort(pg_ctx *c, long long n);   // below, with the tree
int pack_j_hilo(pg_ctx *c, long long nj); // below, with the groups

}  // namespace

// ====================================================================== API

extern "C" {

const char *pg_version(void) { return "pg 0.1 (sm_103a)"; }

const char *pg_last_error(pg_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int pg_create(pg_ctx **out, int device)
{
    if (!out) return PG_EINVAL;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        (void)cudaGetLastError();
        g_create_err = e != cudaSuccess ? std::string("no CUDA device: ") + cudaGetErrorString(e)
                                        : "device index out of range";
        return e != cudaSuccess ? PG_ECUDA : PG_EINVAL;
    }
    if ((e = cudaSetDevice(device)) != cudaSuccess) {
        g_create_err = cudaGetErrorString(e);
        return PG_ECUDA;
    }
    pg_ctx *c = new pg_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if ((e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        g_create_err = cudaGetErrorString(e);
        delete c;
        return PG_ECUDA;
    }
    c->stream = c->own_stream;
    if (ensure(c, c->status, 2 * sizeof(int)) != PG_OK ||
        cudaMemsetAsync(c->status.p, 0, 2 * sizeof(int), c->stream) != cudaSuccess) {
        g_create_err = c->err;
        pg_destroy(c);
        return PG_ENOMEM;
    }
    *out = c;
    return PG_OK;
}

void pg_destroy(pg_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graph(c);
    DevBuf *bufs[] = {&c->G0, &c->G1, &c->AG1, &c->P0, &c->P1, &c->AGP, &c->epsi, &c->jrec, &c->stage, &c->xi, &c->xt, &c->ctr,
                      &c->skeys0, &c->skeys1, &c->svals0, &c->svals1, &c->shist, &c->ssums,
                      &c->sbbox, &c->acc, &c->pot, &c->part, &c->status, &c->g_ioff,
                      &c->g_joff, &c->g_jlist, &c->g_items, &c->g_ctr, &c->g_queue, &c->g_jhl,
                      &c->g_ihl,
                      &c->c_wrapped, &c->c_xs, &c->c_xo, &c->c_perm, &c->c_start, &c->c_jcount,
                      &c->c_icount, &c->c_ioff,
                      &c->c_items_raw, &c->c_items, &c->c_pairs, &c->n_part, &c->bw_wj,
                      &c->bw_wt, &c->bw_dv, &c->tickets};
    for (DevBuf *b : bufs) free_dev(*b);
    for (DevBuf &b : c->tb) free_dev(b);
    for (DevBuf *b : {&c->pm_rec, &c->pm_x, &c->pm_m, &c->pm_acc, &c->pm_pot}) free_dev(*b);
    pm_destroy(c->pm);
    free_pin(c->pin_j);
    free_pin(c->pin_i);
    free_pin(c->pin_o);
    if (c->tk0) cudaEventDestroy(c->tk0);
    if (c->tk1) cudaEventDestroy(c->tk1);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    if (c->side_stream) cudaStreamDestroy(c->side_stream);
    for (cudaEvent_t e : c->tree_ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

int pg_set_stream(pg_ctx *c, void *s)
{
    if (!c) return PG_EINVAL;
    cudaStream_t ns = (cudaStream_t)s;   // NULL: the CUDA legacy default stream
    if (ns != c->stream) {
        // keep ordering: the new stream waits for work already enqueued
        cudaEvent_t ev;
        PG_CUDA(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        PG_CUDA(c, cudaEventRecord(ev, c->stream));
        PG_CUDA(c, cudaStreamWaitEvent(ns, ev, 0));
        cudaEventDestroy(ev);
        c->stream = ns;
        drop_graph(c);
    }
    return PG_OK;
}

int pg_set_eps(pg_ctx *c, double eps)
{
    if (!c) return PG_EINVAL;
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(c, PG_EINVAL, "eps must be >= 0");
    if (eps != c->eps) drop_graph(c);
    c->eps = eps;
    return PG_OK;
}

int pg_set_mode(pg_ctx *c, int mode)
{
    if (!c) return PG_EINVAL;
    if (mode != PG_NEWTON && mode != PG_TABLE) return fail(c, PG_EINVAL, "unknown mode");
    if (mode != c->mode) drop_graph(c);
    c->mode = mode;
    return PG_OK;
}

int pg_set_table(pg_ctx *c, double (*g)(double, void *), void *user, double r_cut, int E, int F)
{
    if (!c) return PG_EINVAL;
    if (!g) return fail(c, PG_EINVAL, "g is NULL");
    int rc = check_EF(c, r_cut, E, F);
    if (rc) return rc;
    set_geometry(c, r_cut, E, F);
    double sc2 = (c->s_max - 2.0) / (r_cut * r_cut);
    std::vector<float> v(c->ntab);
    for (int k = 0; k < c->ntab; ++k) {
        double r = std::sqrt(((double)knot_s(k, F) - 2.0) / sc2);
        double gv = g(r, user);
        if (!std::isfinite(gv)) return fail(c, PG_EINVAL, "g(r) is not finite at a knot");
        v[k] = (float)gv;
    }
    return upload_table(c, v);
}

int pg_set_table_values(pg_ctx *c, const float *v, long long n, double r_cut, int E, int F)
{
    if (!c) return PG_EINVAL;
    if (!v) return fail(c, PG_EINVAL, "v is NULL");
    int rc = check_EF(c, r_cut, E, F);
    if (rc) return rc;
    if (n != (1LL << (E + F))) return fail(c, PG_EINVAL, "n must be 2^(E+F)");
    set_geometry(c, r_cut, E, F);
    return upload_table(c, std::vector<float>(v, v + n));
}

int pg_set_table_values_dev(pg_ctx *c, const float *v, long long n, double r_cut, int E, int F)
{
    if (!c) return PG_EINVAL;
    if (!v) return fail(c, PG_EINVAL, "v is NULL");
    int rc = check_EF(c, r_cut, E, F);
    if (rc) return rc;
    if (n != (1LL << (E + F))) return fail(c, PG_EINVAL, "n must be 2^(E+F)");
    bool same = c->have_table && c->E == E && c->F == F && c->r_cut == r_cut;
    set_geometry(c, r_cut, E, F);
    if ((rc = ensure(c, c->G0, n * 4)) || (rc = ensure(c, c->G1, n * 4)) ||
        (rc = ensure(c, c->AG1, n * 8)))
        return rc;
    PG_CUDA(c, launch_table_from_values(v, (float *)c->G0.p, (float *)c->G1.p, E, F, c->stream));
    PG_CUDA(c, launch_table_prep((float *)c->G0.p, (float *)c->G1.p, (float2 *)c->AG1.p, E, F,
                                 c->stream));
    if ((rc = remerge_pot(c))) return rc;
    c->have_table = true;
    if (!same) drop_graph(c);
    return PG_OK;
}

int pg_get_table(pg_ctx *c, float *G0, float *G1, long long n)
{
    if (!c) return PG_EINVAL;
    if (!c->have_table) return fail(c, PG_ESTATE, "no table set");
    if (n != c->ntab || !G0 || !G1) return fail(c, PG_EINVAL, "n must be 2^(E+F), arrays non-NULL");
    PG_CUDA(c, cudaMemcpyAsync(G0, c->G0.p, n * 4, cudaMemcpyDeviceToHost, c->stream));
    PG_CUDA(c, cudaMemcpyAsync(G1, c->G1.p, n * 4, cudaMemcpyDeviceToHost, c->stream));
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    return PG_OK;
}

int pg_set_tree(pg_ctx *c, double theta, int ncrit, int nleaf)
{
    if (!c) return PG_EINVAL;
    if (!(theta >= 0.0)) {
        c->tree_on = false;
        return PG_OK;
    }
    if (!std::isfinite(theta) || ncrit < 1 || nleaf < 1 || ncrit > (1 << 20))
        return fail(c, PG_EINVAL, "need finite theta >= 0, 1 <= ncrit <= 2^20, nleaf >= 1");
    c->tree_on = true;
    c->tree_theta = theta;
    c->tree_ncrit = ncrit;
    c->tree_nleaf = nleaf;
    drop_graph(c);
    return PG_OK;
}

int pg_set_tree_quadrupole(pg_ctx *c, int on)
{
    if (!c) return PG_EINVAL;
    c->tree_quad = on != 0;
    return PG_OK;
}

int pg_set_tree_walk(pg_ctx *c, int mode)
{
    if (!c) return PG_EINVAL;
    if (mode != PG_TREE_WALK_AUTO && mode != PG_TREE_WALK_LEVEL)
        return fail(c, PG_EINVAL, "tree walk mode must be PG_TREE_WALK_AUTO or PG_TREE_WALK_LEVEL");
    c->tree_walk_mode = mode;
    return PG_OK;
}

int pg_get_tree_stats(pg_ctx *c, long long *out, int nout)
{
    if (!c || (!out && nout > 0)) return PG_EINVAL;
    for (int k = 0; k < nout && k < 4; ++k) out[k] = c->tree_stats[k];
    return PG_OK;
}

int pg_set_pm(pg_ctx *c, int ngrid, int split, double scale)
{
    if (!c) return PG_EINVAL;
    if (ngrid <= 0) {
        if (c->pm_n) drop_graph(c);
        c->pm_n = 0;
        return PG_OK;
    }
    if (ngrid < 8 || ngrid > 1024 || (ngrid & 1))
        return fail(c, PG_EINVAL, "the PM mesh needs an even size from 8 to 1024");
    if (split != PG_SPLIT_GAUSS && split != PG_SPLIT_S2)
        return fail(c, PG_EINVAL, "split must be PG_SPLIT_GAUSS or PG_SPLIT_S2");
    if (!(scale > 0.0) || !std::isfinite(scale)) return fail(c, PG_EINVAL, "scale must be finite and > 0");
    if (!c->pm) c->pm = pm_create();
    pm_set_fft(c->pm, c->pm_fft);
    c->pm_n = ngrid;
    c->pm_split = split;
    c->pm_scale = scale;
    drop_graph(c);
    return PG_OK;
}

int pg_set_pm_fft(pg_ctx *c, int mode)
{
    if (!c) return PG_EINVAL;
    if (mode != PG_FFT_AUTO && mode != PG_FFT_LIBRARY)
        return fail(c, PG_EINVAL, "the PM FFT mode must be PG_FFT_AUTO or PG_FFT_LIBRARY");
    if (mode != c->pm_fft) drop_graph(c);
    c->pm_fft = mode;
    if (c->pm) pm_set_fft(c->pm, mode);
    return PG_OK;
}

int pg_get_pm_fft(pg_ctx *c, int *kind)
{
    if (!c || !kind) return PG_EINVAL;
    *kind = c->pm ? pm_last_fft(c->pm) : 0;
    return PG_OK;
}

int pg_pm_forces_dev(pg_ctx *c, const double *x, const double *m, long long n, double *a, double *phi)
{
    if (!c) return PG_EINVAL;
    if (n < 0 || (n > 0 && (!x || !m || !a))) return fail(c, PG_EINVAL, "bad arrays or count");
    if (c->pm_n <= 0) return fail(c, PG_ESTATE, "pg_set_pm has not been called");
    if (!(c->box > 0.0)) return fail(c, PG_ESTATE, "the PM force needs pg_set_periodic");
    if (n == 0) return PG_OK;
    int rc;
    if ((rc = ensure(c, c->pm_rec, (size_t)n * 32)) || (rc = prep_sort(c, n))) return rc;
    PG_CUDA(c, launch_pack_j(x, m, (double4 *)c->pm_rec.p, n, c->stream));
    std::string err;
    int launches = 1;
    rc = pm_run(c->pm, (const double4 *)c->pm_rec.p, n, (const double4 *)c->pm_rec.p, n, c->box, c->pm_n,
                c->pm_split, c->pm_scale, a, phi, false, c->sort, c->stream, &launches, err);
    if (rc) return fail(c, rc, err);
    c->last_launches = launches;
    return PG_OK;
}

int pg_pm_deposit_dev(pg_ctx *c, const double *x, const double *m, long long n, float *rho)
{
    if (!c) return PG_EINVAL;
    if (n < 0 || (n > 0 && (!x || !m)) || !rho) return fail(c, PG_EINVAL, "bad arrays or count");
    if (c->pm_n <= 0) return fail(c, PG_ESTATE, "pg_set_pm has not been called");
    if (!(c->box > 0.0)) return fail(c, PG_ESTATE, "the PM force needs pg_set_periodic");
    int rc;
    const long long nn = std::max<long long>(n, 1);
    if ((rc = ensure(c, c->pm_rec, (size_t)nn * 32)) || (rc = prep_sort(c, nn))) return rc;
    if (n > 0) PG_CUDA(c, launch_pack_j(x, m, (double4 *)c->pm_rec.p, n, c->stream));
    std::string err;
    int launches = n > 0 ? 1 : 0;
    rc = pm_deposit(c->pm, (const double4 *)c->pm_rec.p, n, c->box, c->pm_n, c->pm_split, c->pm_scale, rho,
                    c->sort, c->stream, &launches, err);
    if (rc) return fail(c, rc, err);
    c->last_launches = launches;
    return PG_OK;
}

int pg_pm_solve_dev(pg_ctx *c, const float *rho, const double *x, long long n, double *a, double *phi)
{
    if (!c) return PG_EINVAL;
    if (n < 0 || (n > 0 && (!x || !a)) || !rho) return fail(c, PG_EINVAL, "bad arrays or count");
    if (c->pm_n <= 0) return fail(c, PG_ESTATE, "pg_set_pm has not been called");
    if (!(c->box > 0.0)) return fail(c, PG_ESTATE, "the PM force needs pg_set_periodic");
    if (n == 0) return PG_OK;
    int rc;
    if ((rc = ensure(c, c->pm_rec, (size_t)n * 32)) || (rc = prep_sort(c, n))) return rc;
    PG_CUDA(c, launch_pack_i(x, (double4 *)c->pm_rec.p, n, c->stream));
    std::string err;
    int launches = 1;
    rc = pm_solve(c->pm, rho, (const double4 *)c->pm_rec.p, n, c->box, c->pm_n, c->pm_split, c->pm_scale, a,
                  phi, false, c->sort, c->stream, &launches, err);
    if (rc) return fail(c, rc, err);
    c->last_launches = launches;
    return PG_OK;
}

int pg_pm_forces(pg_ctx *c, const double *x, const double *m, long long n, double *a, double *phi)
{
    if (!c) return PG_EINVAL;
    if (n < 0 || (n > 0 && (!x || !m || !a))) return fail(c, PG_EINVAL, "bad arrays or count");
    if (n == 0) return PG_OK;
    int rc;
    if ((rc = ensure(c, c->pm_x, (size_t)n * 24)) || (rc = ensure(c, c->pm_m, (size_t)n * 8)) ||
        (rc = ensure(c, c->pm_acc, (size_t)n * 24)) || (rc = ensure(c, c->pm_pot, (size_t)n * 8)))
        return rc;
    PG_CUDA(c, cudaMemcpyAsync(c->pm_x.p, x, (size_t)n * 24, cudaMemcpyHostToDevice, c->stream));
    PG_CUDA(c, cudaMemcpyAsync(c->pm_m.p, m, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream));
    if ((rc = pg_pm_forces_dev(c, (const double *)c->pm_x.p, (const double *)c->pm_m.p, n,
                               (double *)c->pm_acc.p, phi ? (double *)c->pm_pot.p : nullptr)))
        return rc;
    PG_CUDA(c, cudaMemcpyAsync(a, c->pm_acc.p, (size_t)n * 24, cudaMemcpyDeviceToHost, c->stream));
    if (phi) PG_CUDA(c, cudaMemcpyAsync(phi, c->pm_pot.p, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    return PG_OK;
}

int pg_get_tree_pseudo(pg_ctx *c, double *rec)
{
    if (!c || !rec) return PG_EINVAL;
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    const long long n = c->tree_sizes[0], cnt = c->tree_sizes[1] * c->tree_sizes[5];
    if (cnt <= 0) return PG_OK;
    PG_CUDA(c, cudaMemcpy(rec, (const double4 *)c->tb[pg_ctx::TB_JREC2].p + n, (size_t)cnt * 32,
                          cudaMemcpyDeviceToHost));
    return PG_OK;
}

int pg_get_tree(pg_ctx *c, long long *sizes, long long *perm, long long *g_i0, long long *g_ni,
                long long *j_off, long long *jlist)
{
    if (!c || !sizes) return PG_EINVAL;
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 6; ++k) sizes[k] = c->tree_sizes[k];
    const long long n = c->tree_sizes[0], ng = c->tree_sizes[2], nl = c->tree_sizes[3];
    if (n == 0) return PG_OK;
    auto copy32 = [&](int b, long long cnt, long long *out, bool is_signed) -> int {
        if (!out || cnt <= 0) return PG_OK;
        std::vector<unsigned> h((size_t)cnt);
        PG_CUDA(c, cudaMemcpy(h.data(), c->tb[b].p, (size_t)cnt * 4, cudaMemcpyDeviceToHost));
        for (long long k = 0; k < cnt; ++k)
            out[k] = is_signed ? (long long)(int)h[(size_t)k] : (long long)h[(size_t)k];
        return PG_OK;
    };
    int rc;
    if ((rc = copy32(pg_ctx::TB_PERM, n, perm, false)) || (rc = copy32(pg_ctx::TB_GI0, ng, g_i0, true)) ||
        (rc = copy32(pg_ctx::TB_GNI, ng, g_ni, true)) || (rc = copy32(pg_ctx::TB_JLIST, nl, jlist, true)))
        return rc;
    if (j_off)
        PG_CUDA(c, cudaMemcpy(j_off, c->tb[pg_ctx::TB_JOFF].p, (size_t)(ng + 1) * 8,
                              cudaMemcpyDeviceToHost));
    return PG_OK;
}

int pg_set_table_pot(pg_ctx *c, double (*p)(double, void *), void *user)
{
    if (!c) return PG_EINVAL;
    if (!p) {
        if (c->have_pot) drop_graph(c);
        c->have_pot = false;
        return PG_OK;
    }
    if (!c->have_table) return fail(c, PG_ESTATE, "set the force table first");
    double sc2 = (c->s_max - 2.0) / (c->r_cut * c->r_cut);
    std::vector<float> v(c->ntab);
    for (int k = 0; k < c->ntab; ++k) {
        double r = std::sqrt(((double)knot_s(k, c->F) - 2.0) / sc2);
        double pv = p(r, user);
        if (!std::isfinite(pv)) return fail(c, PG_EINVAL, "psi(r) is not finite at a knot");
        v[k] = (float)pv;
    }
    return upload_pot(c, v);
}

int pg_set_table_pot_values(pg_ctx *c, const float *v, long long n)
{
    if (!c) return PG_EINVAL;
    if (!c->have_table) return fail(c, PG_ESTATE, "set the force table first");
    if (!v) return fail(c, PG_EINVAL, "v is NULL");
    if (n != c->ntab) return fail(c, PG_EINVAL, "n must be 2^(E+F) of the force table");
    for (long long k = 0; k < n; ++k)
        if (!std::isfinite(v[k])) return fail(c, PG_EINVAL, "a knot value is not finite");
    return upload_pot(c, std::vector<float>(v, v + n));
}

static int clear_epsi(pg_ctx *c)
{
    if (c->have_epsi) {
        c->w_dirty = true;     // the i records still carry eps^2
        drop_graph(c);
    }
    c->have_epsi = false;
    c->n_epsi = 0;
    return PG_OK;
}

int pg_set_eps_i(pg_ctx *c, const double *eps, long long n)
{
    if (!c) return PG_EINVAL;
    if (n < 0) return fail(c, PG_EINVAL, "n must be >= 0");
    if (!eps || n == 0) return clear_epsi(c);
    for (long long k = 0; k < n; ++k)
        if (!(eps[k] >= 0.0) || !std::isfinite(eps[k]))
            return fail(c, PG_EINVAL, "every eps must be finite and >= 0");
    int rc;
    if ((rc = ensure(c, c->epsi, (size_t)n * 8))) return rc;
    // a previous run may still read the buffer; the host array may go away
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    PG_CUDA(c, cudaMemcpy(c->epsi.p, eps, (size_t)n * 8, cudaMemcpyHostToDevice));
    if (!c->have_epsi) drop_graph(c);
    c->have_epsi = true;
    c->epsi_applied = false;
    c->n_epsi = n;
    return PG_OK;
}

int pg_set_eps_i_dev(pg_ctx *c, const double *eps, long long n)
{
    if (!c) return PG_EINVAL;
    if (n < 0) return fail(c, PG_EINVAL, "n must be >= 0");
    if (!eps || n == 0) return clear_epsi(c);
    int rc;
    if ((rc = ensure(c, c->epsi, (size_t)n * 8))) return rc;
    PG_CUDA(c, cudaMemcpyAsync(c->epsi.p, eps, (size_t)n * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (!c->have_epsi) drop_graph(c);
    c->have_epsi = true;
    c->epsi_applied = false;
    c->n_epsi = n;
    return PG_OK;
}

int pg_set_n(pg_ctx *c, long long nj)
{
    if (!c) return PG_EINVAL;
    if (nj < 0) return fail(c, PG_EINVAL, "nj must be >= 0");
    if (nj > c->nj_hw) return fail(c, PG_ESTATE, "set_n beyond the j-particles written");
    if (nj != c->nj_n) drop_graph(c);
    c->nj_n = nj;
    return PG_OK;
}

static int grow_j(pg_ctx *c, long long end)
{
    size_t need = (size_t)end * sizeof(double4);
    if (need > c->jrec.cap) {
        // keep the records already written
        DevBuf nb;
        size_t want = std::max(need, c->jrec.cap + c->jrec.cap / 2);
        if (cudaMalloc(&nb.p, want) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(c, PG_ENOMEM, "device allocation for j records failed");
        }
        nb.cap = want;
        if (c->jrec.p && c->nj_hw > 0)
            PG_CUDA(c, cudaMemcpyAsync(nb.p, c->jrec.p, c->nj_hw * sizeof(double4),
                                       cudaMemcpyDeviceToDevice, c->stream));
        PG_CUDA(c, cudaStreamSynchronize(c->stream));
        free_dev(c->jrec);
        c->jrec = nb;
        drop_graph(c);
    }
    return PG_OK;
}

int pg_set_j(pg_ctx *c, long long adr, long long nj, const double *x, const double *m)
{
    if (!c) return PG_EINVAL;
    if (adr < 0 || nj < 0) return fail(c, PG_EINVAL, "adr and nj must be >= 0");
    if (nj > 0 && (!x || !m)) return fail(c, PG_EINVAL, "x or m is NULL");
    if (nj == 0) return PG_OK;
    int rc;
    if ((rc = grow_j(c, adr + nj))) return rc;
    size_t bx = (size_t)nj * 24, bm = (size_t)nj * 8;
    if ((rc = ensure(c, c->stage, bx + bm))) return rc;
    if (host_pinned(x) && host_pinned(m)) {
        // page-locked input: DMA straight from it
        if ((rc = copy_pinned_in(c, c->stage.p, x, bx, c->pin_j)) ||
            (rc = copy_pinned_in(c, (char *)c->stage.p + bx, m, bm, c->pin_j)))
            return rc;
    } else {
        if ((rc = ensure_pin(c, c->pin_j, bx + bm))) return rc;
        std::memcpy(c->pin_j.p, x, bx);
        std::memcpy((char *)c->pin_j.p + bx, m, bm);
        PG_CUDA(c, cudaMemcpyAsync(c->stage.p, c->pin_j.p, bx + bm, cudaMemcpyHostToDevice, c->stream));
        PG_CUDA(c, cudaEventRecord(c->pin_j.done, c->stream));
    }
    const double *dx = (const double *)c->stage.p;
    PG_CUDA(c, launch_pack_j(dx, dx + 3 * nj, (double4 *)c->jrec.p + adr, nj, c->stream));
    c->nj_hw = std::max(c->nj_hw, adr + nj);
    c->jhl_n = -1;
    return PG_OK;
}

int pg_set_j_rec_dev(pg_ctx *c, long long adr, long long nj, const double *rec)
{
    if (!c) return PG_EINVAL;
    if (adr < 0 || nj < 0) return fail(c, PG_EINVAL, "adr and nj must be >= 0");
    if (nj > 0 && !rec) return fail(c, PG_EINVAL, "rec is NULL");
    if (nj == 0) return PG_OK;
    int rc;
    if ((rc = grow_j(c, adr + nj))) return rc;
    PG_CUDA(c, cudaMemcpyAsync((double4 *)c->jrec.p + adr, rec, (size_t)nj * sizeof(double4),
                               cudaMemcpyDeviceToDevice, c->stream));
    c->nj_hw = std::max(c->nj_hw, adr + nj);
    c->jhl_n = -1;
    return PG_OK;
}

int pg_set_j_dev(pg_ctx *c, long long adr, long long nj, const double *x, const double *m)
{
    if (!c) return PG_EINVAL;
    if (adr < 0 || nj < 0) return fail(c, PG_EINVAL, "adr and nj must be >= 0");
    if (nj > 0 && (!x || !m)) return fail(c, PG_EINVAL, "x or m is NULL");
    if (nj == 0) return PG_OK;
    int rc;
    if ((rc = grow_j(c, adr + nj))) return rc;
    PG_CUDA(c, launch_pack_j(x, m, (double4 *)c->jrec.p + adr, nj, c->stream));
    c->nj_hw = std::max(c->nj_hw, adr + nj);
    c->jhl_n = -1;
    return PG_OK;
}

// the i records and their double-float pairs (written together by set_i)
static int grow_i(pg_ctx *c, long long ni)
{
    if ((size_t)ni * sizeof(double4) > c->xi.cap || (size_t)ni * 32 > c->g_ihl.cap) drop_graph(c);
    int rc = ensure(c, c->xi, (size_t)std::max<long long>(ni, 1) * sizeof(double4));
    if (!rc) rc = ensure(c, c->g_ihl, (size_t)std::max<long long>(ni, 1) * 32);
    return rc;
}

int pg_set_i(pg_ctx *c, long long ni, const double *x)
{
    if (!c) return PG_EINVAL;
    if (ni < 0) return fail(c, PG_EINVAL, "ni must be >= 0");
    if (ni > 0 && !x) return fail(c, PG_EINVAL, "x is NULL");
    int rc;
    if ((rc = grow_i(c, ni))) return rc;
    if (ni != c->ni) drop_graph(c);
    c->ni = ni;
    c->i_dirty = true;
    c->epsi_applied = false;   // new i records: eps^2 not yet in them
    if (ni == 0) return PG_OK;
    size_t bx = (size_t)ni * 24;
    // the device staging area is only touched in stream order, so j and i
    // copies can share it
    if ((rc = ensure(c, c->stage, bx))) return rc;
    if (host_pinned(x)) {
        if ((rc = copy_pinned_in(c, c->stage.p, x, bx, c->pin_i))) return rc;
    } else {
        if ((rc = ensure_pin(c, c->pin_i, bx))) return rc;
        std::memcpy(c->pin_i.p, x, bx);
        PG_CUDA(c, cudaMemcpyAsync(c->stage.p, c->pin_i.p, bx, cudaMemcpyHostToDevice, c->stream));
        PG_CUDA(c, cudaEventRecord(c->pin_i.done, c->stream));
    }
    PG_CUDA(c, launch_pack_i((const double *)c->stage.p, (double4 *)c->xi.p, ni, c->stream,
                             (float4 *)c->g_ihl.p));
    c->ihl_n = ni;
    return PG_OK;
}

int pg_set_i_dev(pg_ctx *c, long long ni, const double *x)
{
    if (!c) return PG_EINVAL;
    if (ni < 0) return fail(c, PG_EINVAL, "ni must be >= 0");
    if (ni > 0 && !x) return fail(c, PG_EINVAL, "x is NULL");
    int rc;
    if ((rc = grow_i(c, ni))) return rc;
    if (ni != c->ni) drop_graph(c);
    c->ni = ni;
    c->i_dirty = true;
    c->epsi_applied = false;   // new i records: eps^2 not yet in them
    if (ni > 0) PG_CUDA(c, launch_pack_i(x, (double4 *)c->xi.p, ni, c->stream, (float4 *)c->g_ihl.p));
    c->ihl_n = ni;
    return PG_OK;
}

int pg_set_self(pg_ctx *c, int on)
{
    if (!c) return PG_EINVAL;
    if ((on != 0) != (c->self != 0) || c->self_off != 0) drop_graph(c);
    c->self = on != 0;
    c->self_off = 0;
    return PG_OK;
}

int pg_set_self_offset(pg_ctx *c, long long lo)
{
    if (!c) return PG_EINVAL;
    if (lo < 0) return fail(c, PG_EINVAL, "the self offset must be >= 0");
    if (!c->self || lo != c->self_off) drop_graph(c);
    c->self = 1;
    c->self_off = lo;
    return PG_OK;
}

int pg_set_graph(pg_ctx *c, int on)
{
    if (!c) return PG_EINVAL;
    c->use_graph = on != 0;
    if (!c->use_graph) drop_graph(c);
    return PG_OK;
}

int pg_set_allpairs_path(pg_ctx *c, int path)
{
    if (!c) return PG_EINVAL;
    if (path != PG_PATH_AUTO && path != PG_PATH_TILED && path != PG_PATH_NARROW)
        return fail(c, PG_EINVAL, "path must be PG_PATH_AUTO, PG_PATH_TILED or PG_PATH_NARROW");
    if (path != c->path) drop_graph(c);
    c->path = path;
    return PG_OK;
}

int pg_set_shape(pg_ctx *c, int np, int ctas_per_sm, int packed)
{
    if (!c) return PG_EINVAL;
    if (np != 0 && np != 1 && np != 2 && np != 4) return fail(c, PG_EINVAL, "np must be 0, 1, 2 or 4");
    if (ctas_per_sm < 0) return fail(c, PG_EINVAL, "ctas_per_sm must be >= 0");
    if (packed < -1 || packed > 1) return fail(c, PG_EINVAL, "packed must be -1, 0 or 1");
    c->np = np;   // 0: chosen by problem size
    c->ctas_per_sm = ctas_per_sm;
    if (packed >= 0) c->packed = packed;
    c->i_dirty = true;
    drop_graph(c);
    return PG_OK;
}

int pg_set_groups_tile(pg_ctx *c, int tj, int nt)
{
    if (!c) return PG_EINVAL;
    if (tj == 0 && nt == 0) {
        if (c->g_tj || c->g_nt) drop_graph(c);
        c->g_tj = c->g_nt = 0;
        return PG_OK;
    }
    if (!groups_tile_ok(tj, nt, true))
        return fail(c, PG_EINVAL, "no batched kernel of that j-tile depth and block size is compiled");
    if (tj != c->g_tj || nt != c->g_nt) drop_graph(c);
    c->g_tj = tj;
    c->g_nt = nt;
    return PG_OK;
}

int pg_set_differencing(pg_ctx *c, int mode)
{
    if (!c) return PG_EINVAL;
    if (mode != PG_DIFF_AUTO && mode != PG_DIFF_SINGLE && mode != PG_DIFF_DOUBLE)
        return fail(c, PG_EINVAL, "differencing mode must be PG_DIFF_AUTO, PG_DIFF_SINGLE or PG_DIFF_DOUBLE");
    if (mode != c->diff_mode) drop_graph(c);
    c->diff_mode = mode;
    return PG_OK;
}

int pg_set_split(pg_ctx *c, int items_per_warp)
{
    if (!c) return PG_EINVAL;
    if (items_per_warp < 0 || items_per_warp > 8)
        return fail(c, PG_EINVAL, "items per warp must be 0 to 8");
    c->split = items_per_warp;
    drop_graph(c);
    return PG_OK;
}

int pg_info(pg_ctx *c, long long *out, int n)
{
    if (!c || !out || n < 0) return PG_EINVAL;
    if (c->pairs_on_device && c->c_pairs.p) {
        unsigned long long v = 0;
        PG_CUDA(c, cudaMemcpyAsync(&v, c->c_pairs.p, 8, cudaMemcpyDeviceToHost, c->stream));
        PG_CUDA(c, cudaStreamSynchronize(c->stream));
        c->last_pairs = (long long)v;
        c->pairs_on_device = false;
    }
    long long v[10] = {c->last_pairs, c->last_launches, 2LL * c->last_np, c->last_grid,
                       c->last_slots, c->last_df ? 1LL : (long long)c->packed, c->last_split,
                       (long long)c->last_df, c->last_tj, c->last_nt};
    int k = std::min(n, 10);
    for (int i = 0; i < k; ++i) out[i] = v[i];
    return k;
}

int pg_set_timing(pg_ctx *c, int on)
{
    if (!c) return PG_EINVAL;
    if (on && !c->tk0) {
        PG_CUDA(c, cudaEventCreate(&c->tk0));
        PG_CUDA(c, cudaEventCreate(&c->tk1));
    }
    if ((on != 0) != c->timing) drop_graph(c);
    c->timing = on != 0;
    c->timed = false;
    return PG_OK;
}

int pg_kernel_time(pg_ctx *c, double *ms)
{
    if (!c || !ms) return PG_EINVAL;
    if (!c->timed) return fail(c, PG_ESTATE, "no timed run (pg_set_timing(ctx, 1) first)");
    PG_CUDA(c, cudaEventSynchronize(c->tk1));
    float f = 0;
    PG_CUDA(c, cudaEventElapsedTime(&f, c->tk0, c->tk1));
    *ms = f;
    return PG_OK;
}

int pg_sync(pg_ctx *c)
{
    if (!c) return PG_EINVAL;
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    return read_status(c);
}

int pg_selftest_wait(pg_ctx *c, double limit_ms)
{
    if (!c) return PG_EINVAL;
    if (!(limit_ms > 0.0 && limit_ms <= 2000.0)) return fail(c, PG_EINVAL, "limit_ms must be in (0, 2000]");
    PG_CUDA(c, launch_wait_selftest((int *)c->status.p, (unsigned long long)(limit_ms * 1e6), c->stream));
    return read_status(c);
}

}  // extern "C"

// ====================================================================== runs

namespace {

struct Plan {
    long long ni, nj;
    int np, Bi, ntiles, njsub, grid, slots;
    long long W;
    bool df;               // double-float differencing (tiles not compact)
};

// i-particles per thread / 2 when not fixed by pg_set_shape: more per thread
// (more independent work per warp) for large sets, fewer (more tiles to fill
// the SMs) for small ones
int auto_np(long long ni) { return ni >= 65536 ? 4 : ni >= 8192 ? 2 : 1; }

// the kernels' EXT variant: Newton with per-i softening or eps = 0 (a zero
// guard), table mode with the potential table
bool use_ext(const pg_ctx *c)
{
    if (c->mode == PG_TABLE) return c->have_pot;
    return c->have_epsi || (float)(c->eps * c->eps) == 0.0f;
}

// the table's size as staged in shared memory, in float2 units
int tab_units(const pg_ctx *c) { return c->have_pot ? 2 * c->ntab : c->ntab; }

// the tiled path puts its i-particles in Morton order (compact tiles) from
// 16384 on, where the sort pays for itself
bool tiles_sorted(const pg_ctx *c, long long ni)
{
    return c->sort_mode == 1 || (c->sort_mode < 0 && ni >= 16384);
}

// Double-float differencing on the tiled path. One FP32 offset per particle
// from the tile's FP64 centre carries an error of about 2^-24 of the tile's
// extent, which for a close pair in a wide tile is not small against |d|.
// Tiles are compact only when the i-particles are Morton-ordered and dense in
// the j-set (at most eight j per i: a tile of B i spans about (8 B)^(1/3) j
// spacings, twice the extent of an i-set that is the j-set); every
// other tiled run differences in double-float (3 more lane operations per
// component and pair). pg_set_differencing overrides the choice.
bool tiled_df(const pg_ctx *c, long long ni, long long nj)
{
    if (c->diff_mode == PG_DIFF_SINGLE) return false;
    if (c->diff_mode == PG_DIFF_DOUBLE) return true;
    // the tabulated shape falls steeply toward r_cut, which multiplies a
    // difference's relative error into the interpolant: double-float there
    return c->mode == PG_TABLE || !tiles_sorted(c, ni) || nj > 8 * ni;
}

// the narrow path's i chunks are the caller's i-particles in the caller's
// order, as spread as they come: double-float unless single is asked for
bool narrow_df(const pg_ctx *c) { return c->diff_mode != PG_DIFF_SINGLE; }

// the combine's fields for the self term and the potential
void combine_ext(const pg_ctx *c, CombineArgs &cb)
{
    const bool table = c->mode == PG_TABLE;
    cb.newton = !table;
    cb.tabpot = table && c->have_pot;
    cb.agp = c->have_pot ? (const float4 *)c->AGP.p : nullptr;
    cb.epsi = !table && c->have_epsi;
    cb.xi = (const double4 *)c->xi.p;
}

int plan_allpairs(pg_ctx *c, Plan &p)
{
    p.ni = c->ni;
    p.nj = nj_of(c);
    p.np = c->np ? c->np : auto_np(p.ni);
    p.Bi = allpairs_bi(p.np);
    p.ntiles = (int)((p.ni + p.Bi - 1) / p.Bi);
    p.njsub = (int)((p.nj + kTJ - 1) / kTJ);
    p.W = (long long)p.ntiles * p.njsub;
    p.df = tiled_df(c, p.ni, p.nj);
    int occ = allpairs_max_blocks_per_sm(p.np, c->mode == PG_TABLE, tab_units(c), c->packed != 0,
                                         use_ext(c), p.df);
    int per = c->ctas_per_sm > 0 ? std::min(c->ctas_per_sm, occ) : occ;
    long long g = (long long)c->sms * per;
    p.grid = (int)std::max<long long>(0, std::min<long long>(g, p.W));
    p.slots = 1;
    for (long long t = 0; t < p.ntiles && p.grid > 0; ++t) {
        long long bf = stream_k_first(t * p.njsub, p.grid, p.W);
        long long bl = stream_k_first((t + 1) * p.njsub - 1, p.grid, p.W);
        p.slots = std::max<int>(p.slots, (int)(bl - bf + 1));
    }
    return PG_OK;
}

// the i ordering and tile centres (sort only when it pays)
int enqueue_tiles(pg_ctx *c, const Plan &p)
{
    int rc;
    long long n = p.ni;
    if ((rc = ensure(c, c->xt, (size_t)std::max<long long>(n, 1) * sizeof(double4))) ||
        (rc = ensure(c, c->ctr, (size_t)std::max(p.ntiles, 1) * sizeof(double4))))
        return rc;
    bool do_sort = tiles_sorted(c, n);
    c->perm = nullptr;
    if (do_sort && n > 1) {
        size_t hn = sort_hist_entries(n);
        size_t nb = (hn + 4095) / 4096 + 1;
        if ((rc = ensure(c, c->skeys0, n * 4)) || (rc = ensure(c, c->skeys1, n * 4)) ||
            (rc = ensure(c, c->svals0, n * 4)) || (rc = ensure(c, c->svals1, n * 4)) ||
            (rc = ensure(c, c->shist, hn * 4)) || (rc = ensure(c, c->ssums, nb * 4)) ||
            (rc = ensure(c, c->sbbox, 6 * 8)))
            return rc;
        c->sort.keys[0] = (unsigned *)c->skeys0.p;
        c->sort.keys[1] = (unsigned *)c->skeys1.p;
        c->sort.vals[0] = (unsigned *)c->svals0.p;
        c->sort.vals[1] = (unsigned *)c->svals1.p;
        c->sort.hist = (unsigned *)c->shist.p;
        c->sort.sums = (unsigned *)c->ssums.p;
        c->sort.bbox = (unsigned long long *)c->sbbox.p;
        PG_CUDA(c, launch_morton_sort((const double4 *)c->xi.p, n, c->sort, &c->perm, c->stream));
        c->last_launches += 3 + 5 * 4;
    }
    PG_CUDA(c, launch_tile_prep((const double4 *)c->xi.p, c->perm, n, p.Bi, (double4 *)c->xt.p,
                                (double4 *)c->ctr.p, c->stream));
    c->last_launches += 1;
    c->tiled_np = p.np;
    return PG_OK;
}

// The small path: a Newton run on an i-set below the Morton threshold (tiles
// in the caller's order, double-float differences) whose j records fit
// chunks of at most kSmallMaxChunk, with the launch shape left to the
// library. One launch does the pair loop and the combine (pg_small.cu).
// Sets its chunk count (a multiple of the cluster size, as many clusters as
// fit on the device at once: one wave) and chunk size.
bool use_small(pg_ctx *c, const Plan &p, int &nchunk, int &jchunk)
{
    if (c->mode != PG_NEWTON || c->np != 0 || p.ni <= 0 || p.nj <= 0 || tiles_sorted(c, p.ni) || !p.df)
        return false;
    const bool ext = use_ext(c);
    int &clusters = c->small_clusters[ext ? 1 : 0];
    if (clusters < 0) clusters = small_max_clusters(ext);
    if (clusters <= 0) return false;
    const long long ntiles = (p.ni + small_bi() - 1) / small_bi();
    const long long cs = small_cluster();
    long long nc = cs * std::max<long long>(1, clusters / ntiles);
    long long jc = (p.nj + nc - 1) / nc;
    if (jc > kSmallMaxChunk) {
        jc = kSmallMaxChunk;
        nc = ((p.nj + jc - 1) / jc + cs - 1) / cs * cs;
    }
    if (ntiles * nc > (long long)clusters * cs * 4) return false;   // more than a few waves
    nchunk = (int)nc;
    jchunk = (int)jc;
    return true;
}

int enqueue_small(pg_ctx *c, const Plan &p, int nchunk, int jchunk, double *acc, double *pot)
{
    int rc;
    const long long ntiles = (p.ni + small_bi() - 1) / small_bi();
    if ((rc = ensure(c, c->part, (size_t)ntiles * (nchunk / small_cluster()) * 8 * small_bi() * sizeof(float))) ||
        (rc = ensure(c, c->tickets, (size_t)ntiles * sizeof(unsigned))) ||
        (rc = ensure(c, c->g_jhl, (size_t)p.nj * 32)) || (rc = ensure(c, c->g_ihl, (size_t)p.ni * 32)))
        return rc;
    if (c->tickets_zeroed < c->tickets.cap) {
        PG_CUDA(c, cudaMemsetAsync(c->tickets.p, 0, c->tickets.cap, c->stream));
        c->tickets_zeroed = c->tickets.cap;
    }
    // double-float records: j repacked only after new j records; i written by
    // set_i (repacked here only if another path reused the buffer since)
    if ((rc = pack_j_hilo(c, p.nj))) return rc;
    if (c->ihl_n != p.ni) {
        PG_CUDA(c, launch_pack_hilo((const double4 *)c->xi.p, p.ni, (float4 *)c->g_ihl.p, c->stream));
        c->ihl_n = p.ni;
        c->last_launches += 1;
    }
    SmallArgs a{};
    a.ihl = (const float4 *)c->g_ihl.p;
    a.xi = (const double4 *)c->xi.p;
    a.jhl = (const float4 *)c->g_jhl.p;
    a.ni = p.ni;
    a.nj = p.nj;
    a.nchunk = nchunk;
    a.jchunk = jchunk;
    a.eps2 = (float)(c->eps * c->eps);
    a.epsi = c->have_epsi;
    a.self = c->self;
    a.self_off = c->self_off;
    a.part = (float *)c->part.p;
    a.ticket = (unsigned *)c->tickets.p;
    a.acc = acc;
    a.pot = pot;
    if (c->timing) PG_CUDA(c, record_timing(c, c->tk0));
    PG_CUDA(c, launch_small(a, use_ext(c), c->stream));
    if (c->timing) PG_CUDA(c, record_timing(c, c->tk1));
    c->timed = c->timing;
    c->last_launches += 1;
    c->last_np = 1;
    c->last_df = true;
    c->last_pairs = p.ni * p.nj;
    c->last_grid = (int)(ntiles * nchunk);
    c->last_slots = nchunk;
    return PG_OK;
}

int enqueue_allpairs(pg_ctx *c, const Plan &p, double *acc, double *pot)
{
    int rc;
    bool table = c->mode == PG_TABLE;
    int nchunk = 0, jchunk = 0;
    if (use_small(c, p, nchunk, jchunk)) return enqueue_small(c, p, nchunk, jchunk, acc, pot);
    if (p.ni > 0 && (c->i_dirty || c->use_graph || c->tiled_np != p.np)) {
        if ((rc = enqueue_tiles(c, p))) return rc;
        c->i_dirty = false;
    }
    if (p.ni == 0) return PG_OK;
    if ((rc = ensure(c, c->part, (size_t)p.ntiles * p.slots * p.Bi * sizeof(double4)))) return rc;
    AllPairsArgs a{};
    a.xi = (const double4 *)c->xt.p;
    a.ctr = (const double4 *)c->ctr.p;
    a.jrec = (const double4 *)c->jrec.p;
    if (!table && !p.df) {   // the single-form Newton kernel stages double-float j records
        if ((rc = ensure(c, c->g_jhl, (size_t)std::max<long long>(p.nj, 1) * 32)) ||
            (rc = pack_j_hilo(c, p.nj)))
            return rc;
        a.jhl = (const float4 *)c->g_jhl.p;
    }
    a.ni = p.ni;
    a.nj = p.nj;
    a.ntiles = p.ntiles;
    a.njsub = p.njsub;
    a.W = p.W;
    a.smax_slots = p.slots;
    a.eps2 = (float)(c->eps * c->eps);
    if (table) a.tab = table_dev(c);
    a.part = (double4 *)c->part.p;
    a.status = (int *)c->status.p;
    const bool ext = use_ext(c);
    size_t smem = allpairs_smem(p.np, table, tab_units(c), ext, p.df);
    c->last_np = p.np;
    c->last_df = p.df;
    if (p.grid > 0) {
        if (c->timing) PG_CUDA(c, record_timing(c, c->tk0));
        PG_CUDA(c, launch_allpairs(a, p.grid, p.np, table, ext, c->packed != 0, p.df, smem, c->stream));
        if (c->timing) PG_CUDA(c, record_timing(c, c->tk1));
        c->timed = c->timing;
        c->last_launches += 1;
    }
    CombineArgs cb{};
    cb.part = a.part;
    cb.perm = c->perm;
    cb.jrec = a.jrec;
    cb.ni = p.ni;
    cb.Bi = p.Bi;
    cb.njsub = p.njsub;
    cb.smax_slots = p.slots;
    cb.grid = std::max(p.grid, 1);
    cb.W = std::max<long long>(p.W, 1);
    cb.self = c->self;
    cb.self_off = c->self_off;
    combine_ext(c, cb);
    cb.eps2 = a.eps2;
    cb.accscale = table ? 1.0 / c->scale : 1.0;
    cb.acc = acc;
    cb.pot = pot;
    PG_CUDA(c, launch_combine(cb, c->stream));
    c->last_launches += 1;
    c->last_pairs = p.ni * p.nj;
    c->last_grid = p.grid;
    c->last_slots = p.slots;
    return PG_OK;
}

int check_run_state(pg_ctx *c)
{
    if (c->ni < 0) return fail(c, PG_ESTATE, "pg_set_i has not been called");
    if (c->mode == PG_TABLE && !c->have_table) return fail(c, PG_ESTATE, "table mode without a table");
    if (c->have_epsi) {
        if (c->mode != PG_NEWTON) return fail(c, PG_ESTATE, "per-i softening is for PG_NEWTON");
        if (c->n_epsi != c->ni)
            return fail(c, PG_ESTATE, "per-i softening needs one eps per i-particle of pg_set_i");
    }
    if (c->self_off != 0 && (c->tree_on || c->have_groups || c->box > 0.0))
        return fail(c, PG_ESTATE, "a self offset is for the all-pairs paths");
    if (c->tree_on) {
        if (c->mode != PG_NEWTON) return fail(c, PG_ESTATE, "the tree is for PG_NEWTON");
        if (!c->self || c->ni != nj_of(c) || c->have_groups || c->box > 0.0 || c->have_epsi)
            return fail(c, PG_ESTATE, "the tree needs the self mode with ni == nj, no groups, no "
                                      "periodic box and the global eps");
        if (c->ni + 16 * c->ni >= (1LL << 31))
            return fail(c, PG_EINVAL, "too many particles for the tree");
        return PG_OK;
    }
    if (c->have_groups) {
        if (c->h_ioff.back() > c->ni)
            return fail(c, PG_ESTATE, "groups cover more i-particles than pg_set_i gave");
        if (c->g_maxj >= nj_of(c)) return fail(c, PG_ESTATE, "a j-list index is beyond the j-particles");
        return PG_OK;
    }
    if (c->box > 0.0) {
        if (c->mode != PG_TABLE) return fail(c, PG_ESTATE, "the periodic cell path needs PG_TABLE");
        if (!c->self || c->ni != nj_of(c))
            return fail(c, PG_ESTATE, "the periodic cell path needs the self mode with ni == nj");
        if (c->r_cut * 3.0 > c->box) return fail(c, PG_ESTATE, "periodic path needs r_cut <= box / 3");
        return PG_OK;
    }
    if (c->self && c->self_off + c->ni > nj_of(c))
        return fail(c, PG_ESTATE, "self mode needs offset + ni <= nj (i-particle k is j-particle offset + k)");
    return PG_OK;
}

// host items for the groups: chunks of at most Bi i-particles, longest first
// largest i-pairs per thread of the groups kernel (items may use half of it):
// 4 for the caller's groups (hundreds of i against thousands of j); 2 for
// the tree's lists (groups of at most ncrit against about 2000 entries:
// measured 1.29 against 1.42 ms on 2^20 Plummer, monopoles) and the cells
int groups_np(const pg_ctx *c) { return c->np ? c->np : (c->have_groups ? 4 : 2); }

// the caller's plain Newton lists (no per-i softening, eps > 0) can run any
// compiled tile shape of the batched kernel; everything else the default
bool groups_plain(const pg_ctx *c) { return c->mode == PG_NEWTON && !use_ext(c); }
int groups_tj(const pg_ctx *c) { return c->g_tj && groups_plain(c) ? c->g_tj : kGroupsTJ; }
int groups_nt(const pg_ctx *c) { return c->g_nt && groups_plain(c) ? c->g_nt : kGroupsNT; }

int upload_group_items(pg_ctx *c)
{
    int Bi = groups_bi(groups_np(c), groups_nt(c));
    std::vector<GroupItem> items;
    std::vector<long long> cost;
    for (long long g = 0; g < c->ngroups; ++g) {
        long long i0 = c->h_ioff[g], ni = c->h_ioff[g + 1] - i0;
        long long nj = c->h_joff[g + 1] - c->h_joff[g];
        for (long long k = 0; k < ni; k += Bi) {
            GroupItem it;
            it.group = (int)g;
            it.i0 = (int)(i0 + k);
            it.ni = (int)std::min<long long>(Bi, ni - k);
            it.pad = 0;
            items.push_back(it);
            cost.push_back((long long)it.ni * nj);
        }
    }
    // CTA-sized items first, longest first, then the warp-sized ones (at
    // most 32 i-particles and 32768 pairs), longest first
    auto warp_sized = [&](size_t k) { return items[k].ni <= 32 && cost[k] <= 32768; };
    std::vector<size_t> order(items.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        bool sa = warp_sized(a), sb = warp_sized(b);
        if (sa != sb) return !sa;
        return cost[a] > cost[b];
    });
    c->g_warp_from = 0;
    for (size_t k = 0; k < items.size(); ++k) c->g_warp_from += warp_sized(k) ? 0 : 1;
    std::vector<GroupItem> sorted(items.size());
    for (size_t k = 0; k < order.size(); ++k) sorted[k] = items[order[k]];
    int rc;
    if ((rc = ensure(c, c->g_items, std::max<size_t>(sorted.size(), 1) * sizeof(GroupItem)))) return rc;
    if (!sorted.empty())
        PG_CUDA(c, cudaMemcpy(c->g_items.p, sorted.data(), sorted.size() * sizeof(GroupItem),
                              cudaMemcpyHostToDevice));
    c->g_nitems = (int)sorted.size();
    c->g_items_np = groups_np(c);
    c->g_items_nt = groups_nt(c);
    return PG_OK;
}

GroupArgs group_args(pg_ctx *c)
{
    GroupArgs g{};
    g.eps2 = (float)(c->eps * c->eps);
    if (c->mode == PG_TABLE) g.tab = table_dev(c);
    g.accscale = c->mode == PG_TABLE ? 1.0 / c->scale : 1.0;
    g.status = (int *)c->status.p;
    g.queue = (int *)c->g_queue.p;
    return g;
}

// df: double-float differencing (the narrow path's items); tj, nt: the
// kernel's j-tile depth and threads per CTA (the caller's plain lists only)
int launch_group_kernel(pg_ctx *c, const GroupArgs &g, bool cell, bool df = false, int tj = kGroupsTJ,
                        int nt = kGroupsNT)
{
    bool table = c->mode == PG_TABLE;
    int np = groups_np(c);
    c->last_np = np;
    c->last_df = df;
    c->last_tj = tj;
    c->last_nt = nt;
    const bool ext = use_ext(c);
    int occ = groups_max_blocks_per_sm(np, table, tab_units(c), cell, ext, df, tj, nt);
    int per = c->ctas_per_sm > 0 ? std::min(c->ctas_per_sm, occ) : occ;
    // cell lists: the warp-mode items (the small cells) in a second launch
    // whose lighter blocks fit more warps on an SM
    const int wper = cell && table ? groups_warp_blocks_per_sm(true, true, ext, tab_units(c), false) : 0;
    // That launch starts by programmatic dependent launch, each block as soon
    // as an SM has room for it. By default the CTA-mode kernel takes one CTA
    // fewer per SM than fit, which leaves room for one warp-mode block beside
    // it from the start: the shared-memory-bound clump cells and the
    // latency-bound small cells then overlap (2^21 clustered box: 2.29 ->
    // 2.18 ms for both kernels, bit-identical forces).
    if (wper > 0 && c->ctas_per_sm <= 0 && occ > 1) per = occ - 1;
    int grid = c->sms * per;
    GroupArgs gg = g;
    if (wper > 0) gg.queue_w = (int *)c->g_queue.p + 1;
    PG_CUDA(c, cudaMemsetAsync(c->g_queue.p, 0, 2 * sizeof(int), c->stream));
    if (c->timing) PG_CUDA(c, record_timing(c, c->tk0));
    PG_CUDA(c, launch_groups(gg, grid, np, table, cell, ext, df, tj, nt,
                             groups_smem(np, table, tab_units(c), df, tj, nt), c->stream));
    if (wper > 0)
        PG_CUDA(c, launch_groups_warp(gg, c->sms * wper, true, true, ext, tab_units(c), true, false,
                                      c->stream));
    if (c->timing) PG_CUDA(c, record_timing(c, c->tk1));
    c->timed = c->timing;
    c->last_grid = grid;
    c->last_launches += wper > 0 ? 2 : 1;
    return PG_OK;
}

// items that are all warp-sized (narrow all-pairs): the warp-mode kernel
// alone, wper blocks per SM, claiming items 0, 1, ... from the second counter
// (zeroed by the narrow path's preparation kernel)
int launch_group_warp_kernel(pg_ctx *c, const GroupArgs &g, int wper, bool df)
{
    const bool table = c->mode == PG_TABLE;
    const int per = c->ctas_per_sm > 0 ? std::min(c->ctas_per_sm, wper) : wper;
    const int grid = c->sms * per;
    GroupArgs gg = g;
    gg.queue_w = (int *)c->g_queue.p + 1;
    gg.warp_from = 0;
    c->last_np = 1;                     // one i-pair per lane
    c->last_df = df;
    if (c->timing) PG_CUDA(c, record_timing(c, c->tk0));
    PG_CUDA(c, launch_groups_warp(gg, grid, table, false, use_ext(c), tab_units(c), false, df, c->stream));
    if (c->timing) PG_CUDA(c, record_timing(c, c->tk1));
    c->timed = c->timing;
    c->last_grid = grid;
    c->last_launches += 1;
    return PG_OK;
}

// the j records as double-float pairs for the groups kernel; repacked only
// after the records changed. A captured graph does not hold the packing: the
// uncaptured run just before the capture packed the records, and a replay
// packs them first when they changed since (run_into)
int pack_j_hilo(pg_ctx *c, long long nj)
{
    if (c->capturing) {
        c->graph_jhl = true;
        return PG_OK;
    }
    if (c->jhl_n == nj) return PG_OK;
    PG_CUDA(c, launch_pack_hilo((const double4 *)c->jrec.p, nj, (float4 *)c->g_jhl.p, c->stream));
    c->last_launches += 1;
    c->jhl_n = nj;
    return PG_OK;
}

// Narrow all-pairs: a few i-particles against many j (the individual time
// step regime of Section 5, where one call evaluates only the particles due
// for an update). Tiles of the tiled path would stay mostly empty, so the
// i-set is cut into chunks of at most Bi particles and the j records into
// chunks of jchunk, about one (i chunk, j chunk) item per warp of the
// launch; the items run in the groups kernel with the identity j-list
// (small ones one per warp), each writing FP64 partial sums, and a second
// kernel adds each i's partials in chunk order.
bool use_narrow(const pg_ctx *c)
{
    if (c->path == PG_PATH_NARROW) return true;
    if (c->path == PG_PATH_TILED) return false;
    // measured on 2^20 j: narrow 2.7x faster per call at 16 i, even near 256,
    // 10 % faster at 2048 to 4096; tiles win once the i-set fills the GPU
    return c->ni > 0 && c->ni <= 4096 && nj_of(c) >= 64 * c->ni;
}

int enqueue_narrow(pg_ctx *c, double *acc, double *pot)
{
    int rc;
    const long long ni = c->ni, nj = nj_of(c);
    c->last_pairs = ni * nj;
    if (ni == 0) return PG_OK;
    if (nj == 0) {
        PG_CUDA(c, cudaMemsetAsync(acc, 0, (size_t)ni * 24, c->stream));
        if (pot) PG_CUDA(c, cudaMemsetAsync(pot, 0, (size_t)ni * 8, c->stream));
        return PG_OK;
    }
    const bool table = c->mode == PG_TABLE;
    const int np = groups_np(c);
    const int Bi = groups_bi(np);
    const int nic = (int)((ni + Bi - 1) / Bi);
    const bool df = narrow_df(c);
    const int occ = groups_max_blocks_per_sm(np, table, tab_units(c), false, use_ext(c), df);
    // j chunk: about `split` items per warp of the launch, whole warp tiles
    const long long spl = c->split > 0 ? c->split : 1;
    c->last_split = spl;
    auto chunk = [&](long long warps) {
        const long long per = std::max<long long>(1, warps * spl / nic);
        const long long jc = (nj + per - 1) / per;
        return std::max<long long>(128, (jc + 127) / 128 * 128);
    };
    // items are all alike: warp mode for all of them when an i chunk is
    // small (one warp pass, at most 64 i) and short, else CTA mode.
    // Warp-mode items run in the warp-mode kernel alone, which fits more
    // warps on an SM; chunks are sized for it
    const long long ich = std::min<long long>(Bi, ni);
    const int wper = ich <= 64 ? groups_warp_blocks_per_sm(table, false, use_ext(c), tab_units(c), df) : 0;
    long long jc = chunk((long long)c->sms * occ * 4);
    bool warp = false;
    if (wper > 0) {
        const long long jw = chunk((long long)c->sms * wper * groups_warp_warps_per_block());
        if (ich * jw <= 32768) {
            jc = jw;
            warp = true;
        }
    }
    const long long nch = (nj + jc - 1) / jc;
    if ((long long)nic * nch >= (1LL << 31) || jc >= (1LL << 31))
        return fail(c, PG_EINVAL, "too many narrow items");
    const long long nitems = (long long)nic * nch;
    if ((rc = ensure(c, c->g_ctr, (size_t)nic * sizeof(double4))) || (rc = ensure(c, c->g_queue, 16)) ||
        (rc = ensure(c, c->n_part, (size_t)nch * ni * sizeof(double4))) ||
        (rc = ensure(c, c->g_jhl, (size_t)nj * 32)) || (rc = ensure(c, c->g_ihl, (size_t)ni * 32)))
        return rc;
    // chunk centres, double-float i records and zeroed work counters in one launch
    PG_CUDA(c, launch_narrow_prep((const double4 *)c->xi.p, ni, Bi, nic, (double4 *)c->g_ctr.p,
                                  (float4 *)c->g_ihl.p, (int *)c->g_queue.p, c->stream));
    c->ihl_n = ni;
    if ((rc = pack_j_hilo(c, nj))) return rc;
    c->last_launches += 1;
    GroupArgs g = group_args(c);
    g.xi = (const double4 *)c->xi.p;
    g.jrec = (const double4 *)c->jrec.p;
    g.j_off = nullptr;
    g.jlist = nullptr;
    g.items = nullptr;
    g.gctr = (const double4 *)c->g_ctr.p;
    g.jhl = (const float4 *)c->g_jhl.p;
    g.ihl = (const float4 *)c->g_ihl.p;
    g.nitems = (int)nitems;
    g.warp_from = (int)nitems;
    g.nj = nj;
    g.perm = nullptr;
    g.jchunk = (int)jc;
    g.nchunks = (int)nch;
    g.ichunk = Bi;
    g.ni = ni;
    g.part = (double4 *)c->n_part.p;
    g.part_stride = ni;
    g.acc = acc;
    g.pot = pot;
    if ((rc = warp ? launch_group_warp_kernel(c, g, wper, df) : launch_group_kernel(c, g, false, df))) return rc;
    CombineArgs cb{};
    cb.part = (const double4 *)c->n_part.p;
    cb.jrec = (const double4 *)c->jrec.p;
    cb.ni = ni;
    cb.self = c->self;
    cb.self_off = c->self_off;
    combine_ext(c, cb);
    cb.eps2 = g.eps2;
    cb.accscale = g.accscale;
    cb.acc = acc;
    cb.pot = pot;
    PG_CUDA(c, launch_group_partials_combine(cb, (int)nch, c->stream));
    c->last_launches += 1;
    c->last_slots = nch;
    return PG_OK;
}

// device address of tree buffer b, grown to `bytes`
template <typename T>
int tbuf(pg_ctx *c, int b, size_t bytes, T *&out)
{
    int rc = ensure(c, c->tb[b], std::max<size_t>(bytes, 16));
    out = (T *)c->tb[b].p;
    return rc;
}

// grows buffer b of the tree scratch to hold bytes, keeping its first keep
// bytes (a larger buffer is allocated, the kept part copied, the old freed)
int tgrow(pg_ctx *c, int b, size_t bytes, size_t keep)
{
    DevBuf &d = c->tb[b];
    if (bytes <= d.cap) return PG_OK;
    const size_t want = std::max(bytes, d.cap + d.cap / 2);
    void *p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(c, PG_ENOMEM, "device allocation of " + std::to_string(want) + " bytes failed");
    }
    if (d.p) {
        cudaError_t e = keep ? cudaMemcpyAsync(p, d.p, keep, cudaMemcpyDeviceToDevice, c->stream)
                             : cudaSuccess;
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(d.p);
        if (e != cudaSuccess) {
            cudaFree(p);
            d.p = nullptr;
            d.cap = 0;
            return cuda_fail(c, e, "tree scratch growth");
        }
    }
    d.p = p;
    d.cap = want;
    return PG_OK;
}

// room for the walk's visits (with nf_keep + 1 scanned children of the
// current level kept), and the pointers into it
int walk_room(pg_ctx *c, TreeScratch &t, long long visits, long long v_keep, long long c_keep)
{
    const size_t v = (size_t)visits + 1;
    int rc;
    if ((rc = tgrow(c, pg_ctx::TB_VG, v * 4, (size_t)v_keep * 4)) ||
        (rc = tgrow(c, pg_ctx::TB_VK, v * 4, (size_t)v_keep * 4)) ||
        (rc = tgrow(c, pg_ctx::TB_VE, v * 4, (size_t)v_keep * 4)) ||
        (rc = tgrow(c, pg_ctx::TB_VC, v * 4, (size_t)c_keep * 4)) ||
        (rc = tgrow(c, pg_ctx::TB_VSUMS, (v / 4096 + 2) * 4, 0)))
        return rc;
    t.vg = (int *)c->tb[pg_ctx::TB_VG].p;
    t.vk = (int *)c->tb[pg_ctx::TB_VK].p;
    t.ve = (unsigned *)c->tb[pg_ctx::TB_VE].p;
    t.vc = (unsigned *)c->tb[pg_ctx::TB_VC].p;
    t.vsums = (unsigned *)c->tb[pg_ctx::TB_VSUMS].p;
    return PG_OK;
}

int read_dev(pg_ctx *c, void *dst, const void *src, size_t bytes)
{
    PG_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    return PG_OK;
}

// the radix sort's scratch for n keys, in c->sort
int prep_sort(pg_ctx *c, long long n)
{
    const size_t hn = sort_hist_entries(n);
    const size_t nb = (std::max<size_t>(hn, (size_t)n + 1) + 4095) / 4096 + 1;
    int rc;
    if ((rc = ensure(c, c->skeys0, n * 4)) || (rc = ensure(c, c->skeys1, n * 4)) ||
        (rc = ensure(c, c->svals0, n * 4)) || (rc = ensure(c, c->svals1, n * 4)) ||
        (rc = ensure(c, c->shist, hn * 4)) || (rc = ensure(c, c->ssums, nb * 4)))
        return rc;
    c->sort.keys[0] = (unsigned *)c->skeys0.p;
    c->sort.keys[1] = (unsigned *)c->skeys1.p;
    c->sort.vals[0] = (unsigned *)c->svals0.p;
    c->sort.vals[1] = (unsigned *)c->svals1.p;
    c->sort.hist = (unsigned *)c->shist.p;
    c->sort.sums = (unsigned *)c->ssums.p;
    return PG_OK;
}

// room for a count that was x: an eighth and 256 more, at most bound
long long tree_room(long long x, long long bound) { return std::min(bound, x + x / 8 + 256); }

// buffers whose size follows the room for nodes, groups and list entries
int tree_node_bufs(pg_ctx *c, TreeScratch &t, long long n)
{
    const long long k = std::max(t.cap_nodes, 1LL), P = t.npseudo;
    int rc;
    if ((rc = tbuf(c, pg_ctx::TB_FIRST, k * 4, t.first)) || (rc = tbuf(c, pg_ctx::TB_COUNT, k * 4, t.count)) ||
        (rc = tbuf(c, pg_ctx::TB_CHILD0, k * 4, t.child0)) || (rc = tbuf(c, pg_ctx::TB_CHILDN, k * 4, t.childn)) ||
        (rc = tbuf(c, pg_ctx::TB_LEV, k, t.lev)) || (rc = tbuf(c, pg_ctx::TB_M, k * 8, t.M)) ||
        (rc = tbuf(c, pg_ctx::TB_S, k * 24, t.S)) ||
        (rc = tbuf(c, pg_ctx::TB_JREC2, (n + P * k) * 32, t.jrec2)) ||
        (rc = tbuf(c, pg_ctx::TB_COM, k * 32, t.com)) ||
        (rc = tbuf(c, pg_ctx::TB_T, (P == 3 ? k : 1) * 48, t.T)) ||
        (rc = tbuf(c, pg_ctx::TB_BIG, (P == 3 ? k : 1) * 4, t.big_list)) ||
        (rc = tbuf(c, pg_ctx::TB_NBIG, 4, t.nbig)) ||
        (rc = tbuf(c, pg_ctx::TB_NODEW, k * sizeof(TreeNodeW), t.nodew)) ||
        (rc = ensure(c, c->g_jhl, (size_t)(n + P * k) * 32)))
        return rc;
    return PG_OK;
}

int tree_group_bufs(pg_ctx *c, TreeScratch &t, long long n, int Bi)
{
    const long long g = std::max(t.cap_groups, 1LL);
    int rc;
    if ((rc = tbuf(c, pg_ctx::TB_GBOX, g * 48, t.gbox)) || (rc = tbuf(c, pg_ctx::TB_GBOXF, g * 32, t.gboxf)) ||
        (rc = tbuf(c, pg_ctx::TB_JCOUNT, (g + 1) * 4, t.jcount)) ||
        (rc = tbuf(c, pg_ctx::TB_JOFF, (g + 1) * 8, t.j_off)) ||
        (rc = tbuf(c, pg_ctx::TB_ITEMOFF, (g + 1) * 4, t.item_off)) ||
        (rc = tbuf(c, pg_ctx::TB_ITEMS, (g + n / Bi + 1) * sizeof(GroupItem), t.items)) ||
        (rc = ensure(c, c->g_ctr, (size_t)g * 32)))
        return rc;
    t.gctr = (double4 *)c->g_ctr.p;
    return PG_OK;
}

// the level walk, with a read-back per level to size the next frontier
int tree_level_walk(pg_ctx *c, TreeScratch &t, long long n, long long ng, int &reads)
{
    int rc;
    if ((rc = tbuf(c, pg_ctx::TB_SEG, 2 * 11 * ng * 4, t.seg)) ||
        (rc = tbuf(c, pg_ctx::TB_BASE, 11 * ng * 8, t.base)) ||
        (rc = walk_room(c, t, std::max(8 * n, 2 * ng), 0, 0)))
        return rc;
    long long lev_v[12] = {0, ng};
    int nlev = 1;
    PG_CUDA(c, tree_walk_init(ng, t, c->stream));
    for (int L = 0; L < 11; ++L) {
        const long long o = lev_v[L], nf = lev_v[L + 1] - o;
        if (nf > (1LL << 28))
            return fail(c, PG_EINVAL, "tree walk frontier too large: raise theta or ncrit");
        PG_CUDA(c, tree_walk_level(n, ng, L, o, nf, c->tree_theta, c->tree_nleaf, t, c->stream));
        if (L == 10) break;       // the finest level opens nothing
        unsigned nnext = 0;
        ++reads;
        if ((rc = read_dev(c, &nnext, t.vc + nf, sizeof(unsigned)))) return rc;
        if (nnext == 0) break;
        if ((rc = walk_room(c, t, lev_v[L + 1] + nnext, lev_v[L + 1], nf + 1))) return rc;
        PG_CUDA(c, tree_walk_expand(o, nf, t, c->stream));
        lev_v[L + 2] = lev_v[L + 1] + nnext;
        nlev = L + 2;
    }
    PG_CUDA(c, tree_walk_lists(ng, lev_v, nlev, t, c->sort, c->stream));
    TreeMeta h;
    ++reads;
    if ((rc = read_dev(c, &h, t.meta, sizeof h))) return rc;
    if (h.ent >= (1ull << 32) || (unsigned long long)h.nlist != h.ent)
        return fail(c, PG_EINVAL, "tree interaction lists too long: raise theta or lower ncrit");
    t.cap_list = tree_room(h.nlist, 1LL << 32);
    if ((rc = tbuf(c, pg_ctx::TB_JLIST, std::max(t.cap_list, 1LL) * 4, t.jlist))) return rc;
    PG_CUDA(c, tree_walk_fill(n, ng, lev_v, nlev, t, (int *)c->status.p, c->stream));
    return PG_OK;
}

// The tree front end (Section 5.1's tree usage): build the tree over the
// particles, walk it per group, and evaluate the lists in the batched-group
// kernel. Every stage reads the counts it needs (level offsets, groups,
// list length, items) from the device record t.meta. With exact = false
// the buffers have the room the last exact call left, nothing is read back
// before the end, and one read there says whether every count fitted
// (*redo = true when one did not: the results are void and the caller runs
// the call again exact). With exact = true each count is read back before
// the stage that sizes a buffer by it, and the level walk takes over when a
// group's queue overflows (or when asked for).
int tree_call(pg_ctx *c, double *acc, double *pot, bool exact, bool *redo, int &reads)
{
    int rc;
    const long long n = c->ni;
    *redo = false;
    TreeScratch t{};
    t.npseudo = c->tree_quad ? 3 : 1;
    const long long P = t.npseudo;
    const long long kNoRoomCheck = 1LL << 60;
    if (exact) {
        t.cap_nodes = kNoRoomCheck;
        t.cap_groups = n;            // groups never outnumber particles
        t.cap_list = kNoRoomCheck;
    } else {
        t.cap_nodes = c->tree_cap[0];
        t.cap_groups = c->tree_cap[1];
        t.cap_list = c->tree_cap[2];
    }
    for (int L = 0; L < 11; ++L) t.hint_runs[L] = c->tree_hint[L];
    const int Bi = groups_bi(groups_np(c));
    float4 *hl = nullptr;
    if ((rc = prep_sort(c, n)) ||
        (rc = tbuf(c, pg_ctx::TB_BBOX, 48, t.bbox)) || (rc = tbuf(c, pg_ctx::TB_GEO, 48, t.geo)) ||
        (rc = tbuf(c, pg_ctx::TB_KEY, n * 4, t.key)) || (rc = tbuf(c, pg_ctx::TB_PERM, n * 4, t.perm)) ||
        (rc = tbuf(c, pg_ctx::TB_XS, n * 32, t.xs)) || (rc = tbuf(c, pg_ctx::TB_XI0, n * 32, t.xi0)) ||
        (rc = tbuf(c, pg_ctx::TB_SCAN, (11 * (n + 1) + 1) * 4, t.scan)) ||
        (rc = tbuf(c, pg_ctx::TB_TSUMS, ((11 * (n + 1) + 1) / 4096 + 2) * 4, t.tsums)) ||
        (rc = tbuf(c, pg_ctx::TB_META, sizeof(TreeMeta), t.meta)) ||
        (rc = tbuf(c, pg_ctx::TB_GAT, n * 4, t.gat)) || (rc = tbuf(c, pg_ctx::TB_GSCAN, (n + 1) * 4, t.gscan)) ||
        (rc = tbuf(c, pg_ctx::TB_GI0, n * 4, t.g_i0)) || (rc = tbuf(c, pg_ctx::TB_GNI, n * 4, t.g_ni)) ||
        (rc = tbuf(c, pg_ctx::TB_IOFF, (n + 1) * 8, t.i_off)) ||
        (rc = tbuf(c, pg_ctx::TB_FILT, sizeof(WalkFilter), t.filt)) ||
        (rc = tbuf(c, pg_ctx::TB_HL, n * 32, hl)) ||
        (rc = ensure(c, c->g_ihl, (size_t)n * 32)) || (rc = ensure(c, c->g_queue, 16)))
        return rc;
    if (!exact && ((rc = tree_node_bufs(c, t, n)) || (rc = tree_group_bufs(c, t, n, Bi)) ||
                   (rc = tbuf(c, pg_ctx::TB_JLIST, std::max(t.cap_list, 1LL) * 4, t.jlist))))
        return rc;
    if (!exact) {
        // the count pass records each group's decisions for the fill pass:
        // its emitters never outnumber its list entries
        t.emit_cap = std::max(t.cap_list, 1LL);
        if ((rc = tbuf(c, pg_ctx::TB_EMIT, t.emit_cap * 4, t.emit)) ||
            (rc = tbuf(c, pg_ctx::TB_WSCR, group_walk_warps(c->sms) * kGroupWalkScratch * 4, t.wscratch)) ||
            (rc = tbuf(c, pg_ctx::TB_GEMIT, std::max(t.cap_groups, 1LL) * 8, t.gemit)))
            return rc;
    }
    if (!c->side_stream) {
        PG_CUDA(c, cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
        for (cudaEvent_t &e : c->tree_ev) PG_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        PG_CUDA(c, cudaEventRecord(c->tree_ev[2], c->side_stream));
    }
    // nothing of an earlier call (one that returned between its fork and
    // join) still runs on the side stream
    PG_CUDA(c, cudaStreamWaitEvent(c->stream, c->tree_ev[2], 0));
    PG_CUDA(c, cudaMemsetAsync(t.meta, 0, sizeof(TreeMeta), c->stream));
    TreeMeta h{};

    // keys, sort, level offsets
    PG_CUDA(c, tree_stage_keys((const double4 *)c->jrec.p, n, t, c->sort, c->stream));
    if (exact) {
        ++reads;
        if ((rc = read_dev(c, &h, t.meta, sizeof h))) return rc;
        if (h.flags & kTreeTooLarge)
            return fail(c, PG_EINVAL, "tree too large: particles + pseudo-particles must stay below 2^27");
        t.cap_nodes = tree_room(h.nnodes, 11 * n + 1);
        for (int L = 0; L < 11; ++L) t.hint_runs[L] = h.lev_off[L + 1] - h.lev_off[L];
        if ((rc = tree_node_bufs(c, t, n))) return rc;
    }
    // node links; then the moments, the pseudo-particles and the records'
    // double-float packing on the side stream, beside the groups and the walk
    // (which waits for the moments only; the force kernel for the packing)
    PG_CUDA(c, tree_stage_links(n, t, c->stream));
    PG_CUDA(c, cudaEventRecord(c->tree_ev[0], c->stream));
    PG_CUDA(c, cudaStreamWaitEvent(c->side_stream, c->tree_ev[0], 0));
    PG_CUDA(c, tree_stage_moments(n, t, c->side_stream));
    PG_CUDA(c, cudaEventRecord(c->tree_ev[1], c->side_stream));
    PG_CUDA(c, tree_stage_jrec(n, c->sms, t, c->side_stream));
    const long long nj_room = n + P * (exact ? h.nnodes : t.cap_nodes);
    PG_CUDA(c, launch_pack_hilo(t.jrec2, nj_room, (float4 *)c->g_jhl.p, c->side_stream));
    PG_CUDA(c, cudaEventRecord(c->tree_ev[2], c->side_stream));
    c->jhl_n = -1;      // the buffer now holds the tree's records
    PG_CUDA(c, tree_stage_groups(n, c->tree_ncrit, t, c->sort, c->stream));
    if (exact) {
        ++reads;
        if ((rc = read_dev(c, &h, t.meta, sizeof h))) return rc;
        t.cap_groups = tree_room(h.ngroups, n);
        if ((rc = tree_group_bufs(c, t, n, Bi))) return rc;
    }
    PG_CUDA(c, tree_walk_prep(c->tree_theta, t, c->stream));
    PG_CUDA(c, cudaStreamWaitEvent(c->stream, c->tree_ev[1], 0));
    // the walk
    int walk = 1;
    if (!exact || c->tree_walk_mode == PG_TREE_WALK_AUTO)
        PG_CUDA(c, tree_group_walk(false, n, c->tree_theta, c->tree_nleaf, c->sms, t, c->sort, nullptr,
                                   c->stream));
    if (exact) {
        if (c->tree_walk_mode == PG_TREE_WALK_AUTO) {
            ++reads;
            if ((rc = read_dev(c, &h, t.meta, sizeof h))) return rc;
            if (h.flags & kTreeWalkQueue) walk = 2;
            else if (h.flags & kTreeListLong)
                return fail(c, PG_EINVAL, "tree interaction lists too long: raise theta or lower ncrit");
        } else {
            walk = 2;
        }
        c->tree_stats[2] = h.qmax;
        if (walk == 2) {
            if ((rc = tree_level_walk(c, t, n, h.ngroups, reads))) return rc;
        } else {
            t.cap_list = tree_room(h.nlist, 1LL << 32);
            if ((rc = tbuf(c, pg_ctx::TB_JLIST, std::max(t.cap_list, 1LL) * 4, t.jlist))) return rc;
        }
    }
    if (walk == 1)
        PG_CUDA(c, tree_group_walk(true, n, c->tree_theta, c->tree_nleaf, c->sms, t, c->sort,
                                   (int *)c->status.p, c->stream));
    // work items, then (with the packed records) the forces
    PG_CUDA(c, tree_stage_records(Bi, t, c->sort, c->stream));
    PG_CUDA(c, cudaStreamWaitEvent(c->stream, c->tree_ev[2], 0));
    // the i records' double-float pairs: the j records' own (the first n are
    // the particles in key order), unless the kernel reads each i's eps^2
    // from the i pair's w (eps = 0), which the j pair holds its mass in
    const float4 *ihl = (const float4 *)c->g_jhl.p;
    if (use_ext(c)) {
        PG_CUDA(c, launch_pack_hilo(t.xi0, n, (float4 *)c->g_ihl.p, c->stream));
        ihl = (const float4 *)c->g_ihl.p;
        t.launches += 1;
    }
    c->ihl_n = -1;      // the i buffer no longer holds the last set_i's records
    GroupArgs g = group_args(c);
    g.xi = t.xi0;
    g.jrec = t.jrec2;
    g.j_off = t.j_off;
    g.jlist = t.jlist;
    g.items = t.items;
    g.gctr = (const double4 *)c->g_ctr.p;
    g.jhl = (const float4 *)c->g_jhl.p;
    g.ihl = ihl;
    g.nitems = -1;                   // the item count is read on the device
    g.nitems_dev = &t.meta->nitems;
    g.warp_from = -1;                // lists are long: every item in CTA mode
    g.warp_from_dev = &t.meta->nitems;
    g.nj = nj_room;
    g.perm = t.perm;
    g.list_self = 1;
    g.acc = acc;
    g.pot = pot;
    g.ni = n;
    // the kernel writes FP32 (hi, lo) sums; the finish kernel converts them
    // on full warps (the FP64 output from each set's first lane was a fifth
    // of the kernel's pipe time on tree lists)
    g.hl = hl;
    if ((rc = launch_group_kernel(c, g, false))) return rc;
    PG_CUDA(c, launch_groups_finish(g, c->stream));
    c->last_launches += t.launches + 2;     // the stages; finish, the j pack
    // the one read-back of a run from room: did every count fit?
    ++reads;
    if ((rc = read_dev(c, &h, t.meta, sizeof h))) return rc;
    if (h.flags) {
        if (!exact) {
            *redo = true;
            return PG_OK;
        }
        if (h.flags & kTreeTooLarge)
            return fail(c, PG_EINVAL, "tree too large: particles + pseudo-particles must stay below 2^27");
        return fail(c, PG_EINVAL, "tree interaction lists too long: raise theta or lower ncrit");
    }
    c->last_pairs = (long long)h.pairs;
    c->last_slots = h.ngroups;
    c->tree_sizes[0] = n;
    c->tree_sizes[1] = h.nnodes;
    c->tree_sizes[2] = h.ngroups;
    c->tree_sizes[3] = h.nlist;
    c->tree_sizes[4] = h.nitems;
    c->tree_sizes[5] = P;
    if (exact) {
        // the room this call left serves the next ones, with the group walk
        c->tree_cap[0] = t.cap_nodes;
        c->tree_cap[1] = t.cap_groups;
        c->tree_cap[2] = t.cap_list;
        c->tree_cap_n = n;
        c->tree_cap_p = (int)P;
        c->tree_fast = walk == 1;
    } else {
        c->tree_stats[2] = h.qmax;
    }
    for (int L = 0; L < 11; ++L) c->tree_hint[L] = h.lev_off[L + 1] - h.lev_off[L];
    c->tree_stats[0] = walk;
    c->tree_stats[1] = exact ? 1 : 0;
    return PG_OK;
}

int enqueue_tree(pg_ctx *c, double *acc, double *pot)
{
    c->last_pairs = 0;
    const long long n = c->ni;
    if (n == 0) return PG_OK;
    int reads = 0, rc;
    bool redo = false;
    const long long P = c->tree_quad ? 3 : 1;
    if (c->tree_fast && c->tree_walk_mode == PG_TREE_WALK_AUTO && c->tree_cap_n == n && c->tree_cap_p == P) {
        if ((rc = tree_call(c, acc, pot, false, &redo, reads))) return rc;
        if (!redo) {
            c->tree_stats[3] = reads;
            return PG_OK;
        }
    }
    rc = tree_call(c, acc, pot, true, &redo, reads);
    c->tree_stats[3] = reads;
    return rc;
}

int enqueue_groups(pg_ctx *c, double *acc, double *pot)
{
    int rc;
    if ((c->g_items_np != groups_np(c) || c->g_items_nt != groups_nt(c)) && (rc = upload_group_items(c)))
        return rc;
    if ((rc = ensure(c, c->g_ctr, (size_t)std::max<long long>(c->ngroups, 1) * sizeof(double4))) ||
        (rc = ensure(c, c->g_queue, 16)))
        return rc;
    if (c->h_ioff.back() < c->ni) {   // i-particles outside every group get zeros
        PG_CUDA(c, cudaMemsetAsync(acc, 0, (size_t)c->ni * 24, c->stream));
        if (pot) PG_CUDA(c, cudaMemsetAsync(pot, 0, (size_t)c->ni * 8, c->stream));
    }
    PG_CUDA(c, launch_group_ctr((const double4 *)c->xi.p, (const long long *)c->g_ioff.p,
                                c->ngroups, 0, 0, (double4 *)c->g_ctr.p, c->stream));
    // double-float copies of the j records and i positions for the FP32 differencing
    long long nj = nj_of(c);
    if ((rc = ensure(c, c->g_jhl, (size_t)std::max<long long>(nj, 1) * 32)) ||
        (rc = ensure(c, c->g_ihl, (size_t)std::max<long long>(c->ni, 1) * 32)))
        return rc;
    if ((rc = pack_j_hilo(c, nj))) return rc;
    PG_CUDA(c, launch_pack_hilo((const double4 *)c->xi.p, c->ni, (float4 *)c->g_ihl.p, c->stream));
    c->ihl_n = c->ni;
    c->last_launches += 2;
    GroupArgs g = group_args(c);
    g.xi = (const double4 *)c->xi.p;
    g.jrec = (const double4 *)c->jrec.p;
    g.j_off = (const long long *)c->g_joff.p;
    g.jlist = (const int *)c->g_jlist.p;
    g.items = (const GroupItem *)c->g_items.p;
    g.gctr = (const double4 *)c->g_ctr.p;
    g.jhl = (const float4 *)c->g_jhl.p;
    g.ihl = (const float4 *)c->g_ihl.p;
    g.nitems = c->g_nitems;
    g.warp_from = c->g_warp_from;
    g.nj = nj_of(c);
    g.perm = nullptr;
    g.acc = acc;
    g.pot = pot;
    if ((rc = launch_group_kernel(c, g, false, false, groups_tj(c), groups_nt(c)))) return rc;
    c->last_pairs = c->g_pairs;
    return PG_OK;
}

int enqueue_cells(pg_ctx *c, double *acc, double *pot)
{
    int rc;
    long long n = c->ni;
    int nc = (int)std::floor(c->box / c->r_cut);
    if (nc > 1024) nc = 1024;
    long long ncell = (long long)nc * nc * nc;
    int Bi = groups_bi(groups_np(c));
    long long item_cap = ncell + n / Bi + 1;
    long long sn = std::max(n, item_cap);
    CellScratch &s = c->cells;
    size_t hn = sort_hist_entries(sn);
    size_t nb = (std::max<size_t>(hn, ncell + 1) + 4095) / 4096 + 1;
    if ((rc = ensure(c, c->c_wrapped, n * 32)) || (rc = ensure(c, c->c_xs, n * 32)) ||
        (rc = ensure(c, c->c_xo, n * 16)) ||
        (rc = ensure(c, c->c_perm, n * 4)) || (rc = ensure(c, c->c_start, (ncell + 1) * 4)) ||
        (rc = ensure(c, c->c_jcount, ncell * 4)) || (rc = ensure(c, c->c_icount, ncell * 4)) ||
        (rc = ensure(c, c->c_ioff, (ncell + 1) * 4)) ||
        (rc = ensure(c, c->c_items_raw, item_cap * sizeof(GroupItem))) ||
        (rc = ensure(c, c->c_items, item_cap * sizeof(GroupItem))) ||
        (rc = ensure(c, c->c_pairs, 16)) ||
        (rc = ensure(c, c->skeys0, sn * 4)) || (rc = ensure(c, c->skeys1, sn * 4)) ||
        (rc = ensure(c, c->svals0, sn * 4)) || (rc = ensure(c, c->svals1, sn * 4)) ||
        (rc = ensure(c, c->shist, hn * 4)) || (rc = ensure(c, c->ssums, nb * 4)) ||
        (rc = ensure(c, c->g_queue, 16)))
        return rc;
    if (n >= (1LL << 31)) return fail(c, PG_EINVAL, "too many particles for the cell path");
    s.wrapped = (double4 *)c->c_wrapped.p;
    s.xs = (double4 *)c->c_xs.p;
    s.xo = (float4 *)c->c_xo.p;
    s.perm = (unsigned *)c->c_perm.p;
    s.start = (unsigned *)c->c_start.p;
    s.jcount = (unsigned *)c->c_jcount.p;
    s.icount = (unsigned *)c->c_icount.p;
    s.ioff = (unsigned *)c->c_ioff.p;
    s.items_raw = (GroupItem *)c->c_items_raw.p;
    s.items = (GroupItem *)c->c_items.p;
    s.item_cap = item_cap;
    s.pairs = (unsigned long long *)c->c_pairs.p;
    s.ncta = (unsigned *)((char *)c->c_pairs.p + 8);
    c->sort.keys[0] = (unsigned *)c->skeys0.p;
    c->sort.keys[1] = (unsigned *)c->skeys1.p;
    c->sort.vals[0] = (unsigned *)c->svals0.p;
    c->sort.vals[1] = (unsigned *)c->svals1.p;
    c->sort.hist = (unsigned *)c->shist.p;
    c->sort.sums = (unsigned *)c->ssums.p;
    PG_CUDA(c, launch_cell_build((const double4 *)c->jrec.p, n, c->box, nc, Bi, c->scale, s,
                                 c->sort, c->stream));
    // kernels of the build: key, count, gather, sizes, pairs, iota, items,
    // permute (8), two scans (6), the 8-bit item sort (5) and the cell sort
    // (5 per 8 key bits)
    int cell_bits = 0;
    while ((1LL << cell_bits) < ncell) ++cell_bits;
    c->last_launches += 19 + 5 * ((cell_bits + 7) / 8);
    GroupArgs g = group_args(c);
    g.xi = s.xs;
    g.jrec = s.xs;
    g.j_off = nullptr;
    g.jlist = nullptr;
    g.cstart = s.start;
    g.nc = nc;
    g.items = s.items;
    g.gctr = nullptr;
    g.nitems = -1;
    g.nitems_dev = s.ioff + ncell;
    g.warp_from = -1;
    g.warp_from_dev = s.ncta;
    g.nj = n;
    g.xo = s.xo;
    g.cell_h = (float)(c->box / nc * c->scale);
    g.perm = s.perm;
    g.acc = acc;
    g.pot = pot;
    if ((rc = launch_group_kernel(c, g, true))) return rc;
    c->pairs_on_device = true;
    return PG_OK;
}

int enqueue_run(pg_ctx *c, double *acc, double *pot)
{
    c->last_launches = 0;
    c->last_split = 0;
    c->last_tj = c->last_nt = 0;
    // per-i softening lives in the i records' w (read by every path); a
    // captured graph writes it on every replay, as the records may be new
    if (c->have_epsi && (c->capturing || !c->epsi_applied)) {
        PG_CUDA(c, launch_set_w((double4 *)c->xi.p, (const double *)c->epsi.p, c->ni, c->stream));
        c->epsi_applied = true;
        c->i_dirty = true;
        c->last_launches += 1;
    } else if (!c->have_epsi && c->w_dirty) {
        PG_CUDA(c, launch_set_w((double4 *)c->xi.p, nullptr, c->ni, c->stream));
        c->w_dirty = false;
        c->i_dirty = true;
        c->last_launches += 1;
    }
    if (c->tree_on) return enqueue_tree(c, acc, pot);
    if (c->have_groups) return enqueue_groups(c, acc, pot);
    if (c->box > 0.0) {
        int rc = enqueue_cells(c, acc, pot);
        if (rc || c->pm_n <= 0 || c->ni <= 0) return rc;
        // PPPM / TreePM: the mesh's long-range part added to the PP forces
        if ((rc = prep_sort(c, std::max<long long>(nj_of(c), c->ni)))) return rc;
        std::string err;
        int launches = 0;
        // the targets are the cell list's particles: its cell order keeps
        // neighbours together for the interpolation, so no second sort
        rc = pm_run(c->pm, (const double4 *)c->jrec.p, nj_of(c), (const double4 *)c->xi.p, c->ni, c->box,
                    c->pm_n, c->pm_split, c->pm_scale, acc, pot, true, c->sort, c->stream, &launches, err,
                    c->cells.perm);
        if (rc) return fail(c, rc, err);
        c->last_launches += launches;
        return PG_OK;
    }
    if (use_narrow(c)) return enqueue_narrow(c, acc, pot);
    Plan p;
    plan_allpairs(c, p);
    return enqueue_allpairs(c, p, acc, pot);
}

int run_into(pg_ctx *c, double *acc, double *pot)
{
    int rc = check_run_state(c);
    if (rc) return rc;
    if (!c->use_graph || c->tree_on) return enqueue_run(c, acc, pot);   // a tree run reads counts back

    char key[320];
    snprintf(key, sizeof key, "%d|%d|%g|%lld|%lld|%d|%d|%d|%g|%d|%p|%p|%p|%p|%d|%d|%d|%lld|%d",
             (int)c->have_groups, c->mode, c->box, c->ni, nj_of(c), c->np, c->packed,
             c->ctas_per_sm, c->eps, c->self,
             (void *)acc, (void *)pot, c->jrec.p, c->xi.p, c->sort_mode, (int)c->timing,
             c->g_nitems, c->ngroups,
             (c->path * 4 + (c->have_epsi ? 2 : 0) + (c->have_pot ? 1 : 0)) * 16 + c->split);
    {
        char sk[64];
        snprintf(sk, sizeof sk, "|so%lld|df%d", c->self_off, c->diff_mode);
        strncat(key, sk, sizeof key - strlen(key) - 1);
    }
    if (c->pm_n > 0) {
        char pk[96];
        snprintf(pk, sizeof pk, "|pm%d|%d|%.17g", c->pm_n, c->pm_split, c->pm_scale);
        strncat(key, pk, sizeof key - strlen(key) - 1);
    }
    if (!c->gexec || c->gkey != key) {
        drop_graph(c);
        // this call runs uncaptured, which also makes every allocation the
        // sequence needs; the capture below records the replay for later calls
        c->i_dirty = true;
        if ((rc = enqueue_run(c, acc, pot))) return rc;
        // a default stream cannot be captured: record on the context's own
        // stream (capture runs nothing) and launch on the caller's stream
        cudaStream_t run_stream = c->stream;
        bool deflt = run_stream == nullptr || run_stream == cudaStreamLegacy ||
                     run_stream == cudaStreamPerThread;
        if (deflt) c->stream = c->own_stream;
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            c->stream = run_stream;
            return cuda_fail(c, e, "cudaStreamBeginCapture");
        }
        c->capturing = true;
        rc = enqueue_run(c, acc, pot);
        c->capturing = false;
        e = cudaStreamEndCapture(c->stream, &graph);
        c->stream = run_stream;
        if (rc) {
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
        c->gkey = key;
        return PG_OK;
    }
    if (c->graph_jhl && c->jhl_n != nj_of(c)) {      // new j records since the capture
        PG_CUDA(c, launch_pack_hilo((const double4 *)c->jrec.p, nj_of(c), (float4 *)c->g_jhl.p,
                                    c->stream));
        c->jhl_n = nj_of(c);
    }
    PG_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
    return PG_OK;
}

}  // namespace

extern "C" {

int pg_run(pg_ctx *c)
{
    if (!c) return PG_EINVAL;
    if (c->ni < 0) return fail(c, PG_ESTATE, "pg_set_i has not been called");
    int rc;
    size_t n = (size_t)std::max<long long>(c->ni, 1);
    if ((rc = ensure(c, c->acc, n * 24)) || (rc = ensure(c, c->pot, n * 8))) return rc;
    return run_into(c, (double *)c->acc.p, (double *)c->pot.p);
}

int pg_run_dev(pg_ctx *c, double *a, double *phi)
{
    if (!c) return PG_EINVAL;
    if (!a && c->ni > 0) return fail(c, PG_EINVAL, "a is NULL");
    return run_into(c, a, phi);
}

int pg_get_force(pg_ctx *c, double *a, double *phi, long long ni)
{
    if (!c) return PG_EINVAL;
    if (ni != c->ni) return fail(c, PG_EINVAL, "ni differs from the count given to pg_set_i");
    if (ni > 0 && !a) return fail(c, PG_EINVAL, "a is NULL");
    if (!c->acc.p) return fail(c, PG_ESTATE, "pg_run has not been called");
    if (ni == 0) return pg_sync(c);
    int rc;
    size_t ba = (size_t)ni * 24, bp = phi ? (size_t)ni * 8 : 0;
    if (host_pinned(a) && (!phi || host_pinned(phi))) {
        // page-locked output: DMA straight into it
        PG_CUDA(c, cudaMemcpyAsync(a, c->acc.p, ba, cudaMemcpyDeviceToHost, c->stream));
        if (phi) PG_CUDA(c, cudaMemcpyAsync(phi, c->pot.p, bp, cudaMemcpyDeviceToHost, c->stream));
        return pg_sync(c);
    }
    if ((rc = ensure_pin(c, c->pin_o, ba + bp))) return rc;
    PG_CUDA(c, cudaMemcpyAsync(c->pin_o.p, c->acc.p, ba, cudaMemcpyDeviceToHost, c->stream));
    if (phi)
        PG_CUDA(c, cudaMemcpyAsync((char *)c->pin_o.p + ba, c->pot.p, bp, cudaMemcpyDeviceToHost,
                                   c->stream));
    PG_CUDA(c, cudaEventRecord(c->pin_o.done, c->stream));
    if ((rc = pg_sync(c))) return rc;
    std::memcpy(a, c->pin_o.p, ba);
    if (phi) std::memcpy(phi, (char *)c->pin_o.p + ba, bp);
    return PG_OK;
}

int pg_set_groups(pg_ctx *c, long long ngroups, const long long *i_off, const long long *j_off,
                  const int *jlist)
{
    if (!c) return PG_EINVAL;
    if (ngroups < 0 || (ngroups > 0 && (!i_off || !j_off)))
        return fail(c, PG_EINVAL, "ngroups < 0 or NULL offsets");
    if (ngroups == 0) return pg_clear_groups(c);
    if (i_off[0] != 0 || j_off[0] != 0) return fail(c, PG_EINVAL, "offsets must start at 0");
    long long pairs = 0;
    for (long long g = 0; g < ngroups; ++g) {
        if (i_off[g + 1] < i_off[g] || j_off[g + 1] < j_off[g])
            return fail(c, PG_EINVAL, "offsets must be non-decreasing");
        pairs += (i_off[g + 1] - i_off[g]) * (j_off[g + 1] - j_off[g]);
    }
    long long nlist = j_off[ngroups];
    if (nlist > 0 && !jlist) return fail(c, PG_EINVAL, "jlist is NULL");
    if (i_off[ngroups] >= (1LL << 31)) return fail(c, PG_EINVAL, "too many i-particles in groups");
    long long maxj = -1;
    for (long long k = 0; k < nlist; ++k) {
        if (jlist[k] < 0 || jlist[k] >= (1 << 27))
            return fail(c, PG_EINVAL, "jlist entries must be in [0, 2^27)");
        maxj = std::max<long long>(maxj, jlist[k]);
    }
    int rc;
    if ((rc = ensure(c, c->g_ioff, (ngroups + 1) * 8)) || (rc = ensure(c, c->g_joff, (ngroups + 1) * 8)) ||
        (rc = ensure(c, c->g_jlist, std::max<long long>(nlist, 1) * 4)))
        return rc;
    PG_CUDA(c, cudaStreamSynchronize(c->stream));
    PG_CUDA(c, cudaMemcpy(c->g_ioff.p, i_off, (ngroups + 1) * 8, cudaMemcpyHostToDevice));
    PG_CUDA(c, cudaMemcpy(c->g_joff.p, j_off, (ngroups + 1) * 8, cudaMemcpyHostToDevice));
    if (nlist > 0) PG_CUDA(c, cudaMemcpy(c->g_jlist.p, jlist, nlist * 4, cudaMemcpyHostToDevice));
    c->h_ioff.assign(i_off, i_off + ngroups + 1);
    c->h_joff.assign(j_off, j_off + ngroups + 1);
    c->ngroups = ngroups;
    c->g_pairs = pairs;
    c->g_maxj = maxj;
    c->have_groups = true;
    drop_graph(c);
    return upload_group_items(c);
}

int pg_clear_groups(pg_ctx *c)
{
    if (!c) return PG_EINVAL;
    c->have_groups = false;
    c->ngroups = 0;
    c->h_ioff.clear();
    c->h_joff.clear();
    drop_graph(c);
    return PG_OK;
}

int pg_set_periodic(pg_ctx *c, double box)
{
    if (!c) return PG_EINVAL;
    if (!(box >= 0.0) || !std::isfinite(box)) return fail(c, PG_EINVAL, "box must be >= 0 and finite");
    if (box != c->box) drop_graph(c);
    c->box = box;
    return PG_OK;
}

int pg_backward_dev(pg_ctx *c, const double *w, double *dx, double *dm, float *dv)
{
    if (!c) return PG_EINVAL;
    if (!w || !dx || !dm) return fail(c, PG_EINVAL, "w, dx and dm must be device pointers");
    if (c->mode == PG_TABLE && !c->have_table) return fail(c, PG_ESTATE, "table mode without a table");
    if (!c->self || c->self_off != 0 || c->have_groups || c->box > 0.0 || c->ni < 0 || c->ni != nj_of(c))
        return fail(c, PG_ESTATE, "the backward pass needs the all-pairs self mode with ni == nj");
    if (c->have_epsi && c->mode == PG_NEWTON)
        return fail(c, PG_ESTATE, "the backward pass has no per-i softening");
    bool table = c->mode == PG_TABLE;
    long long n = c->ni;
    if (n == 0) return PG_OK;
    int rc;
    const int Bi = backward_bi();
    int ntiles = (int)((n + Bi - 1) / Bi);
    int njsub = (int)((n + kTJ - 1) / kTJ);
    long long W = (long long)ntiles * njsub;
    int occ = backward_max_blocks_per_sm(table, c->ntab);
    int per = c->ctas_per_sm > 0 ? std::min(c->ctas_per_sm, occ) : occ;
    int grid = (int)std::min<long long>((long long)c->sms * per, W);
    int slots = 1;
    for (long long t = 0; t < ntiles; ++t) {
        long long bf = stream_k_first(t * njsub, grid, W);
        long long bl = stream_k_first((t + 1) * njsub - 1, grid, W);
        slots = std::max<int>(slots, (int)(bl - bf + 1));
    }
    if ((rc = ensure(c, c->xt, n * sizeof(double4))) || (rc = ensure(c, c->ctr, ntiles * sizeof(double4))) ||
        (rc = ensure(c, c->bw_wj, n * sizeof(double4))) || (rc = ensure(c, c->bw_wt, n * sizeof(double4))) ||
        (rc = ensure(c, c->part, (size_t)ntiles * slots * Bi * sizeof(double4))) ||
        (rc = ensure(c, c->bw_dv, std::max(c->ntab, 1) * sizeof(double))))
        return rc;
    c->last_launches = 0;
    // tile order: the Morton order of the particles when it pays
    c->perm = nullptr;
    if (n >= 16384) {
        size_t hn = sort_hist_entries(n);
        size_t nb = (hn + 4095) / 4096 + 1;
        if ((rc = ensure(c, c->skeys0, n * 4)) || (rc = ensure(c, c->skeys1, n * 4)) ||
            (rc = ensure(c, c->svals0, n * 4)) || (rc = ensure(c, c->svals1, n * 4)) ||
            (rc = ensure(c, c->shist, hn * 4)) || (rc = ensure(c, c->ssums, nb * 4)) ||
            (rc = ensure(c, c->sbbox, 6 * 8)))
            return rc;
        c->sort.keys[0] = (unsigned *)c->skeys0.p;
        c->sort.keys[1] = (unsigned *)c->skeys1.p;
        c->sort.vals[0] = (unsigned *)c->svals0.p;
        c->sort.vals[1] = (unsigned *)c->svals1.p;
        c->sort.hist = (unsigned *)c->shist.p;
        c->sort.sums = (unsigned *)c->ssums.p;
        c->sort.bbox = (unsigned long long *)c->sbbox.p;
        PG_CUDA(c, launch_morton_sort((const double4 *)c->jrec.p, n, c->sort, &c->perm, c->stream));
        c->last_launches += 3 + 5 * 4;
    }
    c->i_dirty = true;      // the tile buffers now hold the backward's order
    PG_CUDA(c, launch_tile_prep((const double4 *)c->jrec.p, c->perm, n, Bi, (double4 *)c->xt.p,
                                (double4 *)c->ctr.p, c->stream));
    PG_CUDA(c, launch_pack_w(w, c->perm, n, (double4 *)c->bw_wj.p, (double4 *)c->bw_wt.p, c->stream));
    if (table && dv) PG_CUDA(c, cudaMemsetAsync(c->bw_dv.p, 0, c->ntab * sizeof(double), c->stream));
    BackwardArgs a{};
    a.xi = (const double4 *)c->xt.p;
    a.wv = (const double4 *)c->bw_wt.p;
    a.ctr = (const double4 *)c->ctr.p;
    // Newton: the j records in the i-particles' tile order, so that the own
    // pair falls in the sub-tiles beside the diagonal (the kernel tests for
    // it only there); the table kernel keeps the records' order
    a.jx = (const double4 *)(table ? c->jrec.p : c->xt.p);
    a.jwv = (const double4 *)(table ? c->bw_wj.p : c->bw_wt.p);
    a.n = n;
    a.ntiles = ntiles;
    a.njsub = njsub;
    a.W = W;
    a.smax_slots = slots;
    a.eps2 = (float)(c->eps * c->eps);
    if (table) a.tab = table_dev(c);
    a.part = (double4 *)c->part.p;
    a.dv = (table && dv) ? (double *)c->bw_dv.p : nullptr;
    a.perm = c->perm;
    a.status = (int *)c->status.p;
    if (c->timing) PG_CUDA(c, record_timing(c, c->tk0));
    PG_CUDA(c, launch_backward(a, grid, table, backward_smem(table, c->ntab), c->stream));
    if (c->timing) PG_CUDA(c, record_timing(c, c->tk1));
    c->timed = c->timing;
    double inv = table ? 1.0 / c->scale : 1.0;
    PG_CUDA(c, launch_backward_combine(a.part, c->perm, n, njsub, slots, grid, W, inv, dx, dm,
                                       c->stream));
    if (table && dv) PG_CUDA(c, launch_dv_out((const double *)c->bw_dv.p, c->ntab, inv, dv, c->stream));
    c->last_launches += 5;
    c->last_pairs = n * n;
    c->last_grid = grid;
    c->last_slots = slots;
    return PG_OK;
}

// The autotuner: runs the current workload once per candidate launch shape
// (one warm-up run, then three timed ones on the context's stream) and keeps
// the fastest. Candidates, per path:
//   - all-pairs tiles: i per thread 2 np (np 1, 2, 4) x packed FP32x2 or
//     scalar x CTAs per SM (the occupancy limit and one below);
//   - the batched kernel (groups, tree lists, cell list): np x CTAs per SM;
//   - narrow all-pairs: np x items per warp of the launch (1, 2, 4), the
//     split of the j records into chunks.
// Threads per CTA and j-tile depths are compile-time constants of the
// kernels (register and shared-memory budgets follow from them).
int pg_tune(pg_ctx *c)
{
    if (!c) return PG_EINVAL;
    int rc = check_run_state(c);
    if (rc) return rc;
    if (c->ni <= 0) return PG_OK;
    size_t n = (size_t)c->ni;
    if ((rc = ensure(c, c->acc, n * 24)) || (rc = ensure(c, c->pot, n * 8))) return rc;
    bool graph = c->use_graph;
    c->use_graph = false;
    cudaEvent_t e0, e1;
    PG_CUDA(c, cudaEventCreate(&e0));
    PG_CUDA(c, cudaEventCreate(&e1));
    int best_np = c->np, best_cta = c->ctas_per_sm, best_pk = c->packed, best_split = c->split;
    int best_tj = c->g_tj, best_nt = c->g_nt;
    float best = 1e30f;
    const bool groups_path = c->have_groups || c->box > 0.0 || c->tree_on;
    const bool narrow = !groups_path && use_narrow(c);
    const bool table = c->mode == PG_TABLE;
    // the caller's plain Newton lists also try every compiled tile shape
    const bool tiles = c->have_groups && !c->tree_on && groups_plain(c);
    auto chk = [&](cudaError_t e, const char *where) { return e == cudaSuccess ? PG_OK : cuda_fail(c, e, where); };
    auto trial = [&](int np, int pk, int cta, int split, int tj, int nt) {
        c->np = np;
        c->packed = pk;
        c->ctas_per_sm = cta;
        c->split = split;
        c->g_tj = tj;
        c->g_nt = nt;
        c->i_dirty = true;
        if ((rc = run_into(c, (double *)c->acc.p, (double *)c->pot.p))) return;
        if ((rc = chk(cudaEventRecord(e0, c->stream), "cudaEventRecord"))) return;
        for (int r = 0; r < 3 && !rc; ++r) rc = run_into(c, (double *)c->acc.p, (double *)c->pot.p);
        if (rc) return;
        if ((rc = chk(cudaEventRecord(e1, c->stream), "cudaEventRecord"))) return;
        if ((rc = chk(cudaEventSynchronize(e1), "cudaEventSynchronize"))) return;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_np = np;
            best_cta = cta;
            best_pk = pk;
            best_split = split;
            best_tj = tj;
            best_nt = nt;
        }
    };
    const int nps[3] = {1, 2, 4};
    const int shapes[4][2] = {{kGroupsTJ, kGroupsNT}, {256, 128}, {1024, 256}, {512, 256}};
    for (int np : nps) {
        if (rc) break;
        if (narrow) {
            for (int split = 1; split <= 4 && !rc; split *= 2) trial(np, c->packed, 0, split, c->g_tj, c->g_nt);
            continue;
        }
        // the double-float tiled variant is packed only
        const bool df = !groups_path && tiled_df(c, c->ni, nj_of(c));
        for (int sh = 0; sh < (tiles ? 4 : 1) && !rc; ++sh) {
            const int tj = tiles ? shapes[sh][0] : c->g_tj, nt = tiles ? shapes[sh][1] : c->g_nt;
            for (int pk = groups_path || df ? 1 : 0; pk <= 1 && !rc; ++pk) {
                const int occ = groups_path
                                    ? groups_max_blocks_per_sm(np, table, tab_units(c), c->box > 0.0 && !c->have_groups,
                                                               use_ext(c), false, tj ? tj : kGroupsTJ,
                                                               nt ? nt : kGroupsNT)
                                    : allpairs_max_blocks_per_sm(np, table, tab_units(c), pk != 0, use_ext(c), df);
                for (int cta = std::max(1, occ - 1); cta <= occ && !rc; ++cta) trial(np, pk, cta, c->split, tj, nt);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->np = best_np;
    c->ctas_per_sm = best_cta;
    c->packed = best_pk;
    c->split = best_split;
    c->g_tj = best_tj;
    c->g_nt = best_nt;
    c->i_dirty = true;
    c->use_graph = graph;
    drop_graph(c);
    if (rc) return rc;
    return read_status(c);
}

}  // extern "C"
