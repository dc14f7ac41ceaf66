// pg_pm.cu -- the particle-mesh (PM) long-range force of the PPPM and TreePM
// methods whose short-range part the arbitrary-shape force loop evaluates
// (Section 4.2: PP with R(r, eps) - R(r, r_cut) plus PM with R(r, r_cut)
// make the full softened force; the Gaussian split pairs the same way).
//
// In a periodic cube of side L on an N^3 mesh (points at j h, h = L / N):
//  1. TSC assignment: around the nearest mesh point j0 = floor(u + 1/2) of
//     u = x / h, offset d = u - j0, weights 1/2 (1/2 - d)^2, 3/4 - d^2,
//     1/2 (1/2 + d)^2 per axis; density m w / h^3, FP32 atomics;
//  2. real-to-complex FFT (cuFFT, a plain library FFT);
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
    float *rho = nullptr;        // N^3
    float2 *rk = nullptr;        // N^2 (N/2 + 1)
    float2 *spec = nullptr;      // 4 N^2 (N/2 + 1)
    float *field = nullptr;      // 4 N^3
    float *gtab = nullptr;       // 3 (N/2)^2 + 1: G by n^2
    float *wtab = nullptr;       // N: 1 / sinc^6(pi n / N) by index
};

namespace {

__device__ __forceinline__ int wrap_index(int j, int N) { return j < 0 ? j + N : j >= N ? j - N : j; }

// TSC stencil of one coordinate: the nearest point and the three weights
__device__ __forceinline__ int tsc_axis(double x, double inv_h, int N, float w[3])
{
    double u = x * inv_h;
    u -= N * floor(u / N);                 // into [0, N)
    const double j0 = floor(u + 0.5);
    const float d = (float)(u - j0);
    w[0] = 0.5f * (0.5f - d) * (0.5f - d);
    w[1] = 0.75f - d * d;
    w[2] = 0.5f * (0.5f + d) * (0.5f + d);
    return (int)j0;                        // 0 .. N
}

__global__ void k_pm_assign(const double4 *__restrict__ rec, long long n, double inv_h, int N, float vinv,
                            float *__restrict__ rho)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 v = rec[i];
    float wx[3], wy[3], wz[3];
    const int jx = tsc_axis(v.x, inv_h, N, wx), jy = tsc_axis(v.y, inv_h, N, wy),
              jz = tsc_axis(v.z, inv_h, N, wz);
    const float mv = (float)v.w * vinv;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long ix = wrap_index(jx + a - 1, N);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const long long row = (ix * N + wrap_index(jy + b - 1, N)) * N;
            const float wab = mv * wx[a] * wy[b];
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(rho + row + wrap_index(jz + c - 1, N), wab * wz[c]);
        }
    }
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

__global__ void k_pm_interp(const double4 *__restrict__ rec, long long n, double inv_h, int N,
                            const float *__restrict__ field, double *__restrict__ acc,
                            double *__restrict__ pot, int add)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 v = rec[i];
    float wx[3], wy[3], wz[3];
    const int jx = tsc_axis(v.x, inv_h, N, wx), jy = tsc_axis(v.y, inv_h, N, wy),
              jz = tsc_axis(v.z, inv_h, N, wz);
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
    for (int q = 0; q < 3; ++q) acc[3 * i + q] = add ? acc[3 * i + q] + (double)s[q] : (double)s[q];
    if (pot) pot[i] = add ? pot[i] + (double)s[3] : (double)s[3];
}

unsigned blocks256(long long n) { return (unsigned)((std::max(n, 1LL) + 255) / 256); }

void release(PmState &s)
{
    if (s.have_r2c) cufftDestroy(s.r2c);
    if (s.have_c2r) cufftDestroy(s.c2r);
    s.have_r2c = s.have_c2r = false;
    for (void *p : {(void *)s.rho, (void *)s.rk, (void *)s.spec, (void *)s.field, (void *)s.gtab,
                    (void *)s.wtab})
        if (p) cudaFree(p);
    s.rho = nullptr;
    s.rk = s.spec = nullptr;
    s.field = s.gtab = s.wtab = nullptr;
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

int pm_run(PmState *s, const double4 *src, long long ns, const double4 *tgt, long long nt, double L, int N,
           int split, double scale, double *acc, double *pot, bool add, cudaStream_t st, int *launches,
           std::string &err)
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
        if (cufftPlan3d(&s->r2c, N, N, N, CUFFT_R2C) != CUFFT_SUCCESS) {
            release(*s);
            err = "cufftPlan3d failed";
            return PG_ECUDA;
        }
        s->have_r2c = true;
        int dims[3] = {N, N, N};
        if (cufftPlanMany(&s->c2r, 3, dims, nullptr, 1, (int)M, nullptr, 1, (int)N3, CUFFT_C2R, 4) !=
            CUFFT_SUCCESS) {
            release(*s);
            err = "cufftPlanMany failed";
            return PG_ECUDA;
        }
        s->have_c2r = true;
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
    const double inv_h = N / L;
    const float vinv = (float)((double)N3 / (L * L * L));     // 1 / h^3
    if (cufftSetStream(s->r2c, st) != CUFFT_SUCCESS || cufftSetStream(s->c2r, st) != CUFFT_SUCCESS) {
        err = "cufftSetStream failed";
        return PG_ECUDA;
    }
    cudaMemsetAsync(s->rho, 0, N3 * sizeof(float), st);
    k_pm_assign<<<blocks256(ns), 256, 0, st>>>(src, ns, inv_h, N, vinv, s->rho);
    if (cufftExecR2C(s->r2c, s->rho, (cufftComplex *)s->rk) != CUFFT_SUCCESS) {
        err = "cufftExecR2C failed";
        return PG_ECUDA;
    }
    k_pm_green<<<blocks256(M), 256, 0, st>>>(s->rk, N, (float)(2.0 * M_PI / L), s->gtab, s->wtab, s->spec);
    if (cufftExecC2R(s->c2r, (cufftComplex *)s->spec, s->field) != CUFFT_SUCCESS) {
        err = "cufftExecC2R failed";
        return PG_ECUDA;
    }
    k_pm_interp<<<blocks256(nt), 256, 0, st>>>(tgt, nt, inv_h, N, s->field, acc, pot, add ? 1 : 0);
    if (launches) *launches += 3;      // the library's FFT kernels are not counted
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return PG_ECUDA;
    }
    return PG_OK;
}

}  // namespace pg
