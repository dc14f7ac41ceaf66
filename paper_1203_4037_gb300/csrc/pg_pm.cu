// pg_pm.cu -- the particle-mesh (PM) long-range force of the PPPM and TreePM
// methods whose short-range part the arbitrary-shape force loop evaluates
// (Section 4.2: PP with R(r, eps) - R(r, r_cut) plus PM with R(r, r_cut)
// make the full softened force; the Gaussian split pairs the same way).
//
// In a periodic cube of side L on an N^3 mesh (points at j h, h = L / N):
//  0. sources and targets put in mesh order (a radix sort on the nearest
//     mesh point), so that the threads of a warp share stencil points;
//  1. TSC assignment: around the nearest mesh point j0 = floor(u + 1/2) of
//     u = x / h, offset d = u - j0, weights 1/2 (1/2 - d)^2, 3/4 - d^2,
//     1/2 (1/2 + d)^2 per axis; density m w / h^3, FP32 atomics;
//  2. real-to-complex FFT: the hand-written FFTs of pg_fft.cu for a
//     power-of-two mesh from 8 to 512 (steps 2-4 fused there), cuFFT for
//     the other sizes or on request (pm_set_fft);
//  3. per mode k = 2 pi n / L: phi_k = rho_k G(n^2) / (W(n_x) W(n_y) W(n_z)),
//     G = -4 pi D(k) / (k^2 N^3) with the split factor D (Gaussian
//     exp(-k^2 r_s^2), or the S2 clouds' S(k a)^2), W = sinc^6(pi n / N)
//     (the TSC window, once for the assignment and once for the
//     interpolation); the k = 0 mode and the Nyquist planes are dropped;
//     written as the four spectra -i k_x phi, -i k_y phi, -i k_z phi, phi;
//  4. one batched complex-to-real FFT of the four;
//  5. TSC interpolation of the four fields at every particle (the same
//     stencil as the assignment).
// G and 1/W come from small FP64-built tables (G depends on k only through
// n^2), so the per-mode work is FP32 loads and multiplies.
#include <cufft.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "pg.h"
#include "pg_device.cuh"

namespace pg {

struct PmState {
    int N = 0, split = -1;
    double L = 0.0, scale = 0.0;
    cufftHandle r2c = 0, c2r = 0;
    bool have_r2c = false, have_c2r = false;
    int fft_mode = 0;            // 0: hand-written where the mesh allows, 1: cuFFT
    int last_fft = 0;            // the last solve: 1 hand-written, 2 cuFFT
    float2 *twid = nullptr;      // N: e^{-2 pi i m / N} (hand-written FFTs)
    float *rho = nullptr;        // N^3
    float2 *rk = nullptr;        // N^2 (N/2 + 1)
    float2 *spec = nullptr;      // 4 N^2 (N/2 + 1)
    float *field = nullptr;      // 4 N^3
    float *gtab = nullptr;       // 3 (N/2)^2 + 1: G by n^2
    float *wtab = nullptr;       // N: 1 / sinc^6(pi n / N) by index
    // mesh records (nearest point, FP32 offsets and mass), in input order and
    // in mesh order
    int4 *mj_raw = nullptr, *mj_tgt = nullptr;
    float4 *md_raw = nullptr, *md_tgt = nullptr;
    unsigned *perm_tgt = nullptr;                     // mesh order -> target index
    long long cap = 0;
};

namespace {

__device__ __forceinline__ int wrap_index(int j, int N) { return j < 0 ? j + N : j >= N ? j - N : j; }

// one coordinate in mesh units: the nearest mesh point j0 in [0, N) and the
// offset d = u - j0 in [-1/2, 1/2] of u = x / h. u is formed in 32.32 fixed
// point, t = u 2^32 rounded to an integer (one FP64 multiply by 2^32 / h and
// one conversion: GB300 issues FP64 at about two operations per SM-clock),
// wrapped into [0, N 2^32) with integer arithmetic; j0 = floor(u + 1/2)
// and d come from t's integer and fraction bits. d is within 2^-33 of the
// FP64 offset, far below its own FP32 rounding. Coordinates up to 2^29
// boxes from the origin are wrapped exactly; farther ones are reduced in
// FP64 first.
__device__ __forceinline__ int mesh_axis(double x, double scale32, int N, float &d)
{
    const long long P = (long long)N << 32;             // the box in fixed point
    double u = x * scale32;
    if (!(fabs(u) < 0x1p61)) u -= (double)P * floor(u / (double)P);
    long long t = __double2ll_rn(u);
    if (t < 0 || t >= P) {
        t %= P;
        if (t < 0) t += P;
    }
    const long long j = (t + (1LL << 31)) >> 32;
    d = (float)(int)(t - (j << 32)) * 0x1p-32f;
    return (int)(j >= N ? j - N : j);
}

__device__ __forceinline__ void tsc_weights(float d, float w[3])
{
    w[0] = 0.5f * (0.5f - d) * (0.5f - d);
    w[1] = 0.75f - d * d;
    w[2] = 0.5f * (0.5f + d) * (0.5f + d);
}

// the three cells z0 - 1 .. z0 + 1 of one stencil row with weights w0, w1,
// w2: vector atomics on the aligned groups of four cells that hold them
// (one or two; the other lanes add +0, which leaves a cell unchanged), or
// three scalar atomics when the row wraps around the box or vec is off (the
// host sets it when N is a multiple of four and the mesh 16-byte aligned,
// so that every row is)
__device__ __forceinline__ void deposit_row(float *__restrict__ row, int zc, int N, bool vec, float w0, float w1,
                                            float w2)
{
    if (!vec || zc < 0 || zc + 2 >= N) {
        atomicAdd(row + wrap_index(zc, N), w0);
        atomicAdd(row + wrap_index(zc + 1, N), w1);
        atomicAdd(row + wrap_index(zc + 2, N), w2);
        return;
    }
    const int a4 = zc & ~3, o = zc - a4;
    float4 *g = reinterpret_cast<float4 *>(row + a4);
    if (o == 0) {
        atomicAdd(g, make_float4(w0, w1, w2, 0.0f));
    } else if (o == 1) {
        atomicAdd(g, make_float4(0.0f, w0, w1, w2));
    } else if (o == 2) {
        atomicAdd(g, make_float4(0.0f, 0.0f, w0, w1));
        atomicAdd(g + 1, make_float4(w2, 0.0f, 0.0f, 0.0f));
    } else {
        atomicAdd(g, make_float4(0.0f, 0.0f, 0.0f, w0));
        atomicAdd(g + 1, make_float4(w1, w2, 0.0f, 0.0f));
    }
}

__global__ void k_pm_assign(const int4 *__restrict__ mj, const float4 *__restrict__ md, long long n, int N,
                            float vinv, float *__restrict__ rho, int vec)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 j = mj[i];
    const float4 d = md[i];
    float wx[3], wy[3], wz[3];
    tsc_weights(d.x, wx);
    tsc_weights(d.y, wy);
    tsc_weights(d.z, wz);
    const float mv = d.w * vinv;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long ix = wrap_index(j.x + a - 1, N);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const long long row = (ix * N + wrap_index(j.y + b - 1, N)) * N;
            const float wab = mv * wx[a] * wy[b];
            deposit_row(rho + row, j.z - 1, N, vec != 0, wab * wz[0], wab * wz[1], wab * wz[2]);
        }
    }
}

// The same deposit from records in an order that keeps particles of one
// mesh point together (mesh or cell-list order). The lanes of a warp that
// hold the same nearest mesh point (a run of consecutive lanes) would add to
// the same 27 cells in the same instructions, and those atomics serialise:
// the run's weights are summed in the warp first (a segmented scan over the
// lanes), and the run's last lane adds the 27 sums. A warp whose lanes all
// hold different points takes the plain path.
__global__ void __launch_bounds__(256) k_pm_assign_runs(const int4 *__restrict__ mj, const float4 *__restrict__ md,
                                                        long long n, int N, float vinv, float *__restrict__ rho,
                                                        int vec)
{
    constexpr unsigned kFull = 0xffffffffu;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < n;
    const int4 j = valid ? mj[i] : make_int4(0, 0, 0, 0);
    const float4 d = valid ? md[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    // a lane past the end gets a key no record has
    const long long key = valid ? ((long long)j.x * N + j.y) * N + j.z : -1 - (long long)lane;
    const long long prev = __shfl_up_sync(kFull, key, 1);
    const unsigned heads = __ballot_sync(kFull, lane == 0 || prev != key);
    if (!valid && heads == kFull) return;          // past the end, and no lane waits for a shuffle
    float wx[3], wy[3], wz[3];
    tsc_weights(d.x, wx);
    tsc_weights(d.y, wy);
    tsc_weights(d.z, wz);
    const float mv = valid ? d.w * vinv : 0.0f;
    if (heads == kFull) {                          // no two lanes share a point
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const long long ix = wrap_index(j.x + a - 1, N);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const long long row = (ix * N + wrap_index(j.y + b - 1, N)) * N;
                const float wab = mv * wx[a] * wy[b];
                deposit_row(rho + row, j.z - 1, N, vec != 0, wab * wz[0], wab * wz[1], wab * wz[2]);
            }
        }
        return;
    }
    // first lane of this lane's run, and whether this lane ends it
    const unsigned upto = lane == 31 ? heads : heads & ((2u << lane) - 1u);   // heads at lanes <= this one
    const int start = 31 - __clz(upto);
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    float w[27];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) w[9 * a + 3 * b + c] = mv * wx[a] * wy[b] * wz[c];
#pragma unroll
    for (int sft = 1; sft < 32; sft <<= 1) {
        const bool take = lane - sft >= start;
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            const float t = __shfl_up_sync(kFull, w[q], sft);
            if (take) w[q] += t;
        }
    }
    if (!valid || !tail) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long ix = wrap_index(j.x + a - 1, N);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const long long row = (ix * N + wrap_index(j.y + b - 1, N)) * N;
            deposit_row(rho + row, j.z - 1, N, vec != 0, w[9 * a + 3 * b], w[9 * a + 3 * b + 1],
                        w[9 * a + 3 * b + 2]);
        }
    }
}

// mesh order: a record's key is the row-major index of its nearest mesh
// point, so that neighbouring threads share stencil points; the mesh record
// (point; offsets and mass) is written here once, in input order
__global__ void k_pm_keys(const double4 *__restrict__ rec, long long n, double scale32, int N,
                          unsigned *__restrict__ keys, unsigned *__restrict__ vals, int4 *__restrict__ mj,
                          float4 *__restrict__ md)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 v = rec[i];
    float dx, dy, dz;
    const int jx = mesh_axis(v.x, scale32, N, dx), jy = mesh_axis(v.y, scale32, N, dy),
              jz = mesh_axis(v.z, scale32, N, dz);
    keys[i] = ((unsigned)jx * (unsigned)N + (unsigned)jy) * (unsigned)N + (unsigned)jz;
    vals[i] = (unsigned)i;
    mj[i] = make_int4(jx, jy, jz, 0);
    md[i] = make_float4(dx, dy, dz, (float)v.w);
}

__global__ void k_pm_gather(const int4 *__restrict__ mj, const float4 *__restrict__ md,
                            const unsigned *__restrict__ perm, long long n, int4 *__restrict__ mj_out,
                            float4 *__restrict__ md_out)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned p = perm[i];
    mj_out[i] = mj[p];
    md_out[i] = md[p];
}

// the four spectra of every mode (index t over N x N x (N/2 + 1), z fastest)
__global__ void k_pm_green(const float2 *__restrict__ rk, int N, float kf, const float *__restrict__ gtab,
                           const float *__restrict__ wtab, float2 *__restrict__ spec)
{
    const int nz2 = N / 2 + 1;
    const long long M = (long long)N * N * nz2;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= M) return;
    const int iz = (int)(t % nz2);
    const long long r = t / nz2;
    const int iy = (int)(r % N), ix = (int)(r / N);
    const int half = N / 2;
    const int nx = ix < half ? ix : ix - N, ny = iy < half ? iy : iy - N, nz = iz;
    float g = 0.0f;
    if (ix != half && iy != half && iz != half)     // the Nyquist planes are dropped
        g = gtab[nx * nx + ny * ny + nz * nz] * wtab[ix] * wtab[iy] * wtab[iz];
    const float2 v = rk[t];
    const float pr = v.x * g, pi = v.y * g;          // phi_k
    const float kx = kf * nx, ky = kf * ny, kz = kf * nz;
    spec[t] = make_float2(kx * pi, -kx * pr);        // -i k phi
    spec[M + t] = make_float2(ky * pi, -ky * pr);
    spec[2 * M + t] = make_float2(kz * pi, -kz * pr);
    spec[3 * M + t] = make_float2(pr, pi);
}

__global__ void k_pm_interp(const int4 *__restrict__ mj, const float4 *__restrict__ md,
                            const unsigned *__restrict__ perm, long long n, int N,
                            const float *__restrict__ field, double *__restrict__ acc,
                            double *__restrict__ pot, int add)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 j = mj[i];
    const float4 d = md[i];
    float wx[3], wy[3], wz[3];
    tsc_weights(d.x, wx);
    tsc_weights(d.y, wy);
    tsc_weights(d.z, wz);
    const int jx = j.x, jy = j.y, jz = j.z;
    const long long N3 = (long long)N * N * N;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long ix = wrap_index(jx + a - 1, N);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const long long row = (ix * N + wrap_index(jy + b - 1, N)) * N;
            const float wab = wx[a] * wy[b];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long p = row + wrap_index(jz + c - 1, N);
                const float w = wab * wz[c];
#pragma unroll
                for (int q = 0; q < 4; ++q) s[q] = fmaf(w, __ldg(field + q * N3 + p), s[q]);
            }
        }
    }
    const long long o = perm[i];             // the target's own index
    for (int q = 0; q < 3; ++q) acc[3 * o + q] = add ? acc[3 * o + q] + (double)s[q] : (double)s[q];
    if (pot) pot[o] = add ? pot[o] + (double)s[3] : (double)s[3];
}

unsigned blocks256(long long n) { return (unsigned)((std::max(n, 1LL) + 255) / 256); }

void release(PmState &s)
{
    if (s.have_r2c) cufftDestroy(s.r2c);
    if (s.have_c2r) cufftDestroy(s.c2r);
    s.have_r2c = s.have_c2r = false;
    for (void *p : {(void *)s.rho, (void *)s.rk, (void *)s.spec, (void *)s.field, (void *)s.gtab,
                    (void *)s.wtab, (void *)s.mj_raw, (void *)s.mj_tgt, (void *)s.md_raw, (void *)s.md_tgt,
                    (void *)s.perm_tgt, (void *)s.twid})
        if (p) cudaFree(p);
    s.twid = nullptr;
    s.rho = nullptr;
    s.rk = s.spec = nullptr;
    s.field = s.gtab = s.wtab = nullptr;
    s.mj_raw = s.mj_tgt = nullptr;
    s.md_raw = s.md_tgt = nullptr;
    s.perm_tgt = nullptr;
    s.cap = 0;
    s.N = 0;
    s.split = -1;
}

// S2 cloud form factor S(q), q = k a / 2 (FP64; the series below 0.1 where
// the closed form cancels)
double s2_form(double q)
{
    if (q < 0.1) return 1.0 - q * q / 15.0 + q * q * q * q / 560.0 - std::pow(q, 6) / 37800.0;
    return 12.0 * (2.0 - 2.0 * std::cos(q) - q * std::sin(q)) / (q * q * q * q);
}

}  // namespace

PmState *pm_create() { return new PmState(); }

void pm_destroy(PmState *s)
{
    if (!s) return;
    release(*s);
    delete s;
}

void pm_set_fft(PmState *s, int mode) { s->fft_mode = mode; }
int pm_last_fft(const PmState *s) { return s->last_fft; }

namespace {

// mesh, plans and tables for (N, split, scale, L); room for n records
int ensure(PmState *s, double L, int N, int split, double scale, long long n, std::string &err)
{
    const int nz2 = N / 2 + 1;
    const long long N3 = (long long)N * N * N, M = (long long)N * N * nz2;
    if (s->N != N) {
        release(*s);
        if (cudaMalloc(&s->rho, N3 * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&s->rk, M * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&s->spec, 4 * M * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&s->field, 4 * N3 * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&s->gtab, ((size_t)3 * (N / 2) * (N / 2) + 1) * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&s->wtab, (size_t)N * sizeof(float)) != cudaSuccess) {
            (void)cudaGetLastError();
            release(*s);
            err = "PM mesh allocation failed";
            return PG_ENOMEM;
        }
        if (fft_mesh_ok(N)) {
            std::vector<float2> tw((size_t)N);
            fft_twiddles(N, tw.data());
            if (cudaMalloc(&s->twid, (size_t)N * sizeof(float2)) != cudaSuccess ||
                cudaMemcpy(s->twid, tw.data(), (size_t)N * sizeof(float2), cudaMemcpyHostToDevice) !=
                    cudaSuccess) {
                (void)cudaGetLastError();
                release(*s);
                err = "PM twiddle table allocation failed";
                return PG_ENOMEM;
            }
        }
        s->N = N;
        s->split = -1;
    }
    if (s->split != split || s->scale != scale || s->L != L) {
        // G(n^2) = -4 pi D(k) / (k^2 N^3) and 1 / sinc^6(pi n / N), in FP64
        const int half = N / 2;
        std::vector<float> g((size_t)3 * half * half + 1), w((size_t)N);
        const double kf = 2.0 * M_PI / L;
        g[0] = 0.0f;
        for (size_t q = 1; q < g.size(); ++q) {
            const double k2 = kf * kf * (double)q, k = std::sqrt(k2);
            double D;
            if (split == 0) {
                D = std::exp(-k2 * scale * scale);
            } else {
                const double f = s2_form(0.5 * k * scale);
                D = f * f;
            }
            g[q] = (float)(-4.0 * M_PI * D / (k2 * (double)N3));
        }
        for (int i = 0; i < N; ++i) {
            const int nn = i < half ? i : i - N;
            const double x = M_PI * nn / N;
            const double sn = nn == 0 ? 1.0 : std::sin(x) / x;
            w[(size_t)i] = (float)(1.0 / std::pow(sn, 6));
        }
        if (cudaMemcpy(s->gtab, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(s->wtab, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            err = "PM table upload failed";
            return PG_ECUDA;
        }
        s->split = split;
        s->scale = scale;
        s->L = L;
    }
    if (n > s->cap) {
        for (void *p : {(void *)s->mj_raw, (void *)s->mj_tgt, (void *)s->md_raw, (void *)s->md_tgt,
                        (void *)s->perm_tgt})
            if (p) cudaFree(p);
        s->mj_raw = s->mj_tgt = nullptr;
        s->md_raw = s->md_tgt = nullptr;
        s->perm_tgt = nullptr;
        s->cap = 0;
        bool ok = true;
        for (int4 **p : {&s->mj_raw, &s->mj_tgt})
            ok = ok && cudaMalloc(p, n * sizeof(int4)) == cudaSuccess;
        for (float4 **p : {&s->md_raw, &s->md_tgt})
            ok = ok && cudaMalloc(p, n * sizeof(float4)) == cudaSuccess;
        ok = ok && cudaMalloc(&s->perm_tgt, n * sizeof(unsigned)) == cudaSuccess;
        if (!ok) {
            (void)cudaGetLastError();
            err = "PM record allocation failed";
            return PG_ENOMEM;
        }
        s->cap = n;
    }
    return PG_OK;
}

int key_bits_of(int N)
{
    const unsigned long long N3 = (unsigned long long)N * N * N;
    int b = 1;
    while (b < 32 && (1ull << b) < N3) ++b;
    return b;
}

// the mesh records of n records (input order, in mj_raw / md_raw); with
// sorted, also in mesh order (mj_out / md_out) and perm_keep = mesh order ->
// input index
// mesh records of n particles; sorted: also gathered into an interpolation
// order kept in perm_keep, mesh order by a radix sort of the keys, or the
// caller's order (a permutation of 0 .. n-1 that already keeps neighbours
// together, such as the cell list's) without a sort
cudaError_t records(PmState *s, const double4 *rec, long long n, bool sorted, int4 *mj_out, float4 *md_out,
                    unsigned *perm_keep, SortScratch &sort, cudaStream_t st, int *launches,
                    const unsigned *order = nullptr)
{
    const int N = s->N;
    k_pm_keys<<<blocks256(n), 256, 0, st>>>(rec, n, std::ldexp(N / s->L, 32), N, sort.keys[0], sort.vals[0],
                                            s->mj_raw, s->md_raw);
    if (launches) *launches += 1;
    if (!sorted) return cudaGetLastError();
    const unsigned *perm = order;
    if (!perm) {
        const int kb = key_bits_of(N);
        unsigned *ko = nullptr, *sp = nullptr;
        cudaError_t e = launch_radix_sort(sort.keys[0], sort.vals[0], n, kb, sort, &ko, &sp, st);
        if (e != cudaSuccess) return e;
        perm = sp;
        if (launches) *launches += (kb + 7) / 8 * 5;
    }
    k_pm_gather<<<blocks256(n), 256, 0, st>>>(s->mj_raw, s->md_raw, perm, n, mj_out, md_out);
    cudaMemcpyAsync(perm_keep, perm, n * sizeof(unsigned), cudaMemcpyDeviceToDevice, st);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// the TSC deposit of n records into rho (cleared first): records in input
// order (runs = false), or in an order that keeps the particles of a mesh
// point together, whose runs of one point the warp sums first (runs = true;
// in input order neighbouring threads rarely share a point)
void deposit(PmState *s, const int4 *mj, const float4 *md, long long n, float *rho, bool runs, cudaStream_t st,
             int *launches)
{
    const int N = s->N;
    const long long N3 = (long long)N * N * N;
    const float vinv = (float)((double)N3 / (s->L * s->L * s->L));     // 1 / h^3
    cudaMemsetAsync(rho, 0, N3 * sizeof(float), st);
    const int vec = (N % 4 == 0 && ((uintptr_t)rho & 15) == 0) ? 1 : 0;
    if (runs)
        k_pm_assign_runs<<<blocks256(n), 256, 0, st>>>(mj, md, n, N, vinv, rho, vec);
    else
        k_pm_assign<<<blocks256(n), 256, 0, st>>>(mj, md, n, N, vinv, rho, vec);
    if (launches) *launches += 1;
}

// the cuFFT plans of the mesh (made on first use)
int lib_plans(PmState *s, std::string &err)
{
    if (s->have_r2c && s->have_c2r) return PG_OK;
    const int N = s->N;
    const long long N3 = (long long)N * N * N, M = (long long)N * N * (N / 2 + 1);
    if (!s->have_r2c) {
        if (cufftPlan3d(&s->r2c, N, N, N, CUFFT_R2C) != CUFFT_SUCCESS) {
            err = "cufftPlan3d failed";
            return PG_ECUDA;
        }
        s->have_r2c = true;
    }
    int dims[3] = {N, N, N};
    if (cufftPlanMany(&s->c2r, 3, dims, nullptr, 1, (int)M, nullptr, 1, (int)N3, CUFFT_C2R, 4) != CUFFT_SUCCESS) {
        err = "cufftPlanMany failed";
        return PG_ECUDA;
    }
    s->have_c2r = true;
    return PG_OK;
}

// rho -> the four fields (FFT, Green's function, batched inverse FFT)
int solve_fields(PmState *s, float *rho, cudaStream_t st, int *launches, std::string &err)
{
    const int N = s->N;
    const long long M = (long long)N * N * (N / 2 + 1);
    if (s->fft_mode == 0 && fft_mesh_ok(N)) {
        const cudaError_t e = fft_solve(rho, s->field, s->rk, s->spec, s->twid, s->gtab, s->wtab,
                                        (float)(2.0 * M_PI / s->L), N, st);
        if (e != cudaSuccess) {
            err = cudaGetErrorString(e);
            return PG_ECUDA;
        }
        if (launches) *launches += 5;
        s->last_fft = 1;
        return PG_OK;
    }
    int rc = lib_plans(s, err);
    if (rc) return rc;
    s->last_fft = 2;
    if (cufftSetStream(s->r2c, st) != CUFFT_SUCCESS || cufftSetStream(s->c2r, st) != CUFFT_SUCCESS) {
        err = "cufftSetStream failed";
        return PG_ECUDA;
    }
    if (cufftExecR2C(s->r2c, rho, (cufftComplex *)s->rk) != CUFFT_SUCCESS) {
        err = "cufftExecR2C failed";
        return PG_ECUDA;
    }
    k_pm_green<<<blocks256(M), 256, 0, st>>>(s->rk, N, (float)(2.0 * M_PI / s->L), s->gtab, s->wtab, s->spec);
    if (cufftExecC2R(s->c2r, (cufftComplex *)s->spec, s->field) != CUFFT_SUCCESS) {
        err = "cufftExecC2R failed";
        return PG_ECUDA;
    }
    if (launches) *launches += 1;      // cuFFT's own kernels are not counted
    return PG_OK;
}

int finish(std::string &err)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return PG_ECUDA;
    }
    return PG_OK;
}

}  // namespace

int pm_run(PmState *s, const double4 *src, long long ns, const double4 *tgt, long long nt, double L, int N,
           int split, double scale, double *acc, double *pot, bool add, SortScratch &sort, cudaStream_t st,
           int *launches, std::string &err, const unsigned *tgt_order)
{
    int rc = ensure(s, L, N, split, scale, std::max(ns, nt), err);
    if (rc) return rc;
    // the targets interpolated in mesh order; the sources deposited in that
    // order when they are the same particles (one set of records), else in
    // input order
    const bool same = src == tgt && ns == nt;
    cudaError_t e = records(s, src, ns, same, s->mj_tgt, s->md_tgt, s->perm_tgt, sort, st, launches,
                            same ? tgt_order : nullptr);
    if (e == cudaSuccess) {
        if (same)
            deposit(s, s->mj_tgt, s->md_tgt, ns, s->rho, true, st, launches);
        else
            deposit(s, s->mj_raw, s->md_raw, ns, s->rho, false, st, launches);
        if (!same)
            e = records(s, tgt, nt, true, s->mj_tgt, s->md_tgt, s->perm_tgt, sort, st, launches, tgt_order);
    }
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return PG_ECUDA;
    }
    if ((rc = solve_fields(s, s->rho, st, launches, err))) return rc;
    k_pm_interp<<<blocks256(nt), 256, 0, st>>>(s->mj_tgt, s->md_tgt, s->perm_tgt, nt, N, s->field, acc, pot,
                                               add ? 1 : 0);
    if (launches) *launches += 1;
    return finish(err);
}

int pm_deposit(PmState *s, const double4 *src, long long ns, double L, int N, int split, double scale,
               float *rho, SortScratch &sort, cudaStream_t st, int *launches, std::string &err)
{
    int rc = ensure(s, L, N, split, scale, ns, err);
    if (rc) return rc;
    cudaError_t e = records(s, src, ns, false, nullptr, nullptr, nullptr, sort, st, launches);
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return PG_ECUDA;
    }
    deposit(s, s->mj_raw, s->md_raw, ns, rho, false, st, launches);
    return finish(err);
}

int pm_solve(PmState *s, const float *rho, const double4 *tgt, long long nt, double L, int N, int split,
             double scale, double *acc, double *pot, bool add, SortScratch &sort, cudaStream_t st,
             int *launches, std::string &err)
{
    int rc = ensure(s, L, N, split, scale, nt, err);
    if (rc) return rc;
    // the caller's mesh is copied: the forward FFT may not leave its input
    cudaMemcpyAsync(s->rho, rho, (size_t)N * N * N * sizeof(float), cudaMemcpyDeviceToDevice, st);
    cudaError_t e = records(s, tgt, nt, true, s->mj_tgt, s->md_tgt, s->perm_tgt, sort, st, launches);
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return PG_ECUDA;
    }
    if ((rc = solve_fields(s, s->rho, st, launches, err))) return rc;
    k_pm_interp<<<blocks256(nt), 256, 0, st>>>(s->mj_tgt, s->md_tgt, s->perm_tgt, nt, N, s->field, acc, pot,
                                               add ? 1 : 0);
    if (launches) *launches += 1;
    return finish(err);
}

}  // namespace pg
