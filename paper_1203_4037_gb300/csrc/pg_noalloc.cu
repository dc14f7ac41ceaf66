// pg_noalloc.cu -- an all-pairs Newton entry point that allocates nothing.
//
// Some callers cannot allocate device memory when they want forces: a host
// application whose own memory pool has reserved the whole GPU up front (so
// cudaMalloc fails), or a time-critical step of a simulation loop that must
// not stall on the device-wide synchronisation cudaMalloc and cudaFree can
// cause. They pass their own inputs and outputs;
// the scratch the force loop needs (a status word, packed j records,
// i-particles in tile order, tile centres, per-CTA partial sums) lives in
// the fixed array `g_noalloc_scratch` below, which every GPU that loads this
// library holds until the process exits (about 3.6 MiB).
//
// The array's name in host code is only a host-side stand-in, so the first
// call on each device, with that device current, looks up its device address
// with cudaGetSymbolAddress and keeps it. Make that first call before any
// stream capture. Every call shares the one array and leaves its contents
// behind: each call clears the status word (cudaMemsetAsync, which allocates
// nothing) and writes every other scratch word it reads before reading it,
// but calls that overlap on the GPU (different streams, or different host
// threads without ordering) race on it.
//
// The i-particles are not Morton-ordered here (that would need sort
// scratch), so the force kernel differences in double-float: a pair's
// difference keeps FP32 precision relative to |d| however spread a tile is.
// If a device-side wait of the force kernel gives up (a bounded wait of at
// most two seconds), every output of the call is NaN.
#include <algorithm>
#include <mutex>

#include "pg.h"
#include "pg_internal.h"

namespace pg {

namespace {

constexpr long long kNoAllocMaxN = PG_NOALLOC_MAX_N;
constexpr int kNoAllocNP = 2;                                   // i per thread / 2
constexpr int kNoAllocBi = kNT * 2 * kNoAllocNP;                // 512 i per tile
constexpr long long kMaxTiles = (kNoAllocMaxN + kNoAllocBi - 1) / kNoAllocBi;
constexpr int kMaxSlots = 5;                                    // grid <= 4 CTAs per tile
constexpr size_t kStatusBytes = 256;                            // two ints, padded
constexpr size_t kJrecBytes = (size_t)kNoAllocMaxN * sizeof(double4);
constexpr size_t kXtBytes = (size_t)kNoAllocMaxN * sizeof(double4);
constexpr size_t kCtrBytes = (size_t)kMaxTiles * sizeof(double4);
constexpr size_t kPartBytes = (size_t)kMaxTiles * kMaxSlots * kNoAllocBi * sizeof(double4);
constexpr size_t kScratchBytes = kStatusBytes + kJrecBytes + kXtBytes + kCtrBytes + kPartBytes;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_setup_mu;
void *g_scratch_ptr[256] = {};   // device address of the array, per device

// device address of the scratch array on the current device (looked up once)
cudaError_t scratch_on_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = (unsigned char *)g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" int pg_newton_allpairs_noalloc(const double *x, const double *m, long long n,
                                          double eps, double *a, double *phi, void *cuda_stream)
{
    if (n < 0 || n > kNoAllocMaxN) return PG_EINVAL;
    if (!(eps >= 0.0)) return PG_EINVAL;
    if (n > 0 && (!x || !m || !a)) return PG_EINVAL;
    if (n == 0) return PG_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char *base = nullptr;
    if (scratch_on_current_device(&base) != cudaSuccess) {
        (void)cudaGetLastError();
        return PG_ECUDA;
    }
    int *status = (int *)base;
    double4 *jrec = (double4 *)(base + kStatusBytes);
    double4 *xt = (double4 *)(base + kStatusBytes + kJrecBytes);
    double4 *ctr = (double4 *)(base + kStatusBytes + kJrecBytes + kXtBytes);
    double4 *part = (double4 *)(base + kStatusBytes + kJrecBytes + kXtBytes + kCtrBytes);

    // launch shape: NP = 2, at most 4 CTAs per i-tile so that each tile's
    // partial sums come from at most kMaxSlots CTAs
    const float eps2 = (float)(eps * eps);
    const bool ext = eps2 == 0.0f;     // the zero guard for coincident pairs at eps = 0
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (int)((n + kNoAllocBi - 1) / kNoAllocBi);
    const int njsub = (int)((n + kTJ - 1) / kTJ);
    const long long W = (long long)ntiles * njsub;
    int occ = allpairs_max_blocks_per_sm(kNoAllocNP, false, 0, true, ext, true);
    long long G = std::min<long long>(std::min<long long>(W, 4LL * ntiles), (long long)sms * occ);
    int slots = 1;
    for (long long t = 0; t < ntiles; ++t) {
        long long bf = stream_k_first(t * njsub, (int)G, W);
        long long bl = stream_k_first((t + 1) * njsub - 1, (int)G, W);
        slots = std::max<int>(slots, (int)(bl - bf + 1));
    }
    if (slots > kMaxSlots) return PG_EINVAL;   // cannot happen for n within the limit

    cudaError_t e = cudaMemsetAsync(status, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = launch_pack_j(x, m, jrec, n, st);
    if (e == cudaSuccess) e = launch_tile_prep(jrec, nullptr, n, kNoAllocBi, xt, ctr, st);
    // the i records' fourth value is each i's eps^2 for the kernel's EXT form;
    // the copies of the j records hold the masses there, so clear it
    if (e == cudaSuccess && ext) e = launch_set_w(xt, nullptr, n, st);
    AllPairsArgs ap{};
    ap.xi = xt;
    ap.ctr = ctr;
    ap.jrec = jrec;
    ap.ni = n;
    ap.nj = n;
    ap.ntiles = ntiles;
    ap.njsub = njsub;
    ap.W = W;
    ap.smax_slots = slots;
    ap.eps2 = eps2;
    ap.part = part;
    ap.status = status;
    if (e == cudaSuccess)
        e = launch_allpairs(ap, (int)G, kNoAllocNP, false, ext, true, true,
                            allpairs_smem(kNoAllocNP, false, 0, ext, true), st);
    CombineArgs cb{};
    cb.part = part;
    cb.perm = nullptr;
    cb.jrec = jrec;
    cb.ni = n;
    cb.Bi = kNoAllocBi;
    cb.njsub = njsub;
    cb.smax_slots = slots;
    cb.grid = (int)G;
    cb.W = W;
    cb.self = 1;
    cb.newton = 1;
    cb.eps2 = eps2;
    cb.accscale = 1.0;
    cb.acc = a;
    cb.pot = phi;
    cb.fail_nan = status;
    if (e == cudaSuccess) e = launch_combine(cb, st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return PG_ECUDA;
    }
    return PG_OK;
}
