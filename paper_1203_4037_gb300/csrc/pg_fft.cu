// pg_fft.cu -- the particle-mesh solve with hand-written FFTs: density in,
// the four fields (-d phi / dx, dy, dz, phi) out, for power-of-two meshes.
//
// Layouts (N = 2^p, H = N / 2): the density and the fields are real N^3
// arrays, z fastest (index (x N + y) N + z). The spectra keep kz = 0 .. H-1
// only, index (x N + y) H + kz: the kz = H (Nyquist) plane is one of the
// planes the Green's function sets to zero, so it is never formed.
//
// Five passes, each over tiles of C lines (C consecutive z-lines, or C
// consecutive kz columns of an x- or y-line family):
//  1. z, forward, real to complex: two real samples per complex value, an
//     H-point complex FFT, then X[k] = E[k] + e^{-2 pi i k / N} O[k] with the
//     even / odd spectra E = (Z[k] + conj Z[H-k]) / 2,
//     O = (Z[k] - conj Z[H-k]) / 2i;
//  2. y, forward, in place;
//  3. x: forward; phi = rho G(n) / (W(nx) W(ny) W(nz)) as in the cuFFT
//     solve (G by n^2, the TSC window by index, Nyquist planes dropped);
//     then the inverse x-FFT of phi (A) and of -i kx phi (B). ky and kz are
//     constant along an x-line, so -i ky phi and -i kz phi need no x-FFT of
//     their own;
//  4. y, inverse: Y = F^-1 A (in place) and Yy = F^-1 (-i ky A) from one
//     read of A, then Yx = F^-1 B (in place);
//  5. z, inverse, complex to real, one field per block: for a half
//     spectrum X (X[H] = 0) the H-point inverse of Z[k] = (X[k] + conj
//     X[H-k]) + i (X[k] - conj X[H-k]) e^{2 pi i k / N} holds
//     x[2m] + i x[2m+1]; phi from Y, -dphi/dz from -i kz Y, -dphi/dy from
//     Yy, -dphi/dx from Yx.
// Every transform is unnormalised (the Green's table carries 1 / N^3).
//
// A line of len = R1 R2 points is transformed in two Stockham stages (the
// self-sorting form: natural order in and out). Stage A: butterfly j < R2
// takes rows j + r R2 (r < R1), an R1-point DFT in registers, and puts its
// outputs at rows j R1 + r. Stage B: butterfly j < R1 takes rows j + r R1
// (r < R2), multiplies row r by W_len^{r j}, an R2-point DFT, outputs back
// at rows j + r R1. One exchange through shared memory sits between the
// stages; stage A of the y- and x-passes reads global memory directly, and
// their stage B writes it. In the x-pass the inverse transforms take the
// forward's stage-B butterflies in the other order (radix R2 first, over the
// same rows j + r R1), so the Green's function and the first inverse stage
// run on the registers the forward transform left. The DFTs in registers
// are radix-2 decimation in time, fully unrolled, with the 32nd roots of
// unity as constants; the stage twiddles come from one table of
// e^{-2 pi i m / N}, m < N, built in FP64 on the host.
#include <algorithm>
#include <cmath>

#include "pg_device.cuh"
#include "pg_internal.h"

namespace pg {

namespace {

constexpr int kFftThreads = 256;
constexpr int kFftC = 16;          // lines per tile (fewer when H < 16)

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// -i k a
__device__ __forceinline__ float2 mul_mik(float k, float2 a) { return make_float2(k * a.y, -k * a.x); }

// cos(m pi / 16), m = 0 .. 8
__host__ __device__ constexpr float cos16(int m)
{
    return m == 0 ? 1.0f : m == 1 ? 0.98078528040323045f : m == 2 ? 0.92387953251128676f
         : m == 3 ? 0.83146961230254524f : m == 4 ? 0.70710678118654752f : m == 5 ? 0.55557023301960222f
         : m == 6 ? 0.38268343236508977f : m == 7 ? 0.19509032201612827f : 0.0f;
}
// cos and sin of 2 pi m / 32
__host__ __device__ constexpr float cos32(int m)
{
    return ((m & 31) >> 3) == 0 ? cos16(m & 7) : ((m & 31) >> 3) == 1 ? -cos16(8 - (m & 7))
         : ((m & 31) >> 3) == 2 ? -cos16(m & 7) : cos16(8 - (m & 7));
}
__host__ __device__ constexpr float sin32(int m)
{
    return ((m & 31) >> 3) == 0 ? cos16(8 - (m & 7)) : ((m & 31) >> 3) == 1 ? cos16(m & 7)
         : ((m & 31) >> 3) == 2 ? -cos16(8 - (m & 7)) : -cos16(m & 7);
}

// v times e^{-+2 pi i m / 32} (forward: minus), m a compile-time constant
// after unrolling; the quarter turns are exact
template <bool INV>
__device__ __forceinline__ float2 rot32(float2 v, int m)
{
    m &= 31;
    if (m == 0) return v;
    if (m == 16) return make_float2(-v.x, -v.y);
    if (m == 8) return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    if (m == 24) return INV ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
    const float c = cos32(m), s = INV ? sin32(m) : -sin32(m);
    return make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
}

__host__ __device__ constexpr int brev(int i, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// the R-point DFT of v[0 .. R-1] in registers, natural order in and out
template <int R, bool INV>
__device__ __forceinline__ void dft(float2 *v)
{
    constexpr int bits = ilog2(R);
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = brev(i, bits);
        if (j > i) {
            const float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int half = 1; half < R; half <<= 1) {
#pragma unroll
        for (int k = 0; k < half; ++k) {
#pragma unroll
            for (int b = 0; b < R; b += 2 * half) {
                const float2 t = rot32<INV>(v[b + k + half], k * (16 / half));
                const float2 u = v[b + k];
                v[b + k] = cadd(u, t);
                v[b + k + half] = csub(u, t);
            }
        }
    }
}

// stage-B twiddles: v[r] times W_len^{-+r j} (forward: e^{-2 pi i r j / len})
template <int R, bool INV>
__device__ __forceinline__ void twiddle(float2 *v, int j, const float2 *tw, int scale)
{
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const float2 w = tw[r * j * scale];
        v[r] = cmul(v[r], INV ? cconj(w) : w);
    }
}

__device__ __forceinline__ void load_twiddles(float2 *tw, const float2 *__restrict__ g, int N)
{
    for (int m = threadIdx.x; m < N; m += blockDim.x) tw[m] = g[m];
}

// ---------------------------------------------------------------- pass 1
// z-lines l0 .. l0 + C - 1 of rho (N reals, H complex each) -> spec rows.
// Shared tiles are line-major with a padded line stride LS = H + 1.
template <int R1, int R2>
__global__ void __launch_bounds__(kFftThreads) k_fft_z_r2c(const float *__restrict__ rho, float2 *__restrict__ spec,
                                                           const float2 *__restrict__ twg, int N, int C, int lgC)
{
    constexpr int len = R1 * R2;           // H
    constexpr int LS = len + 1;
    extern __shared__ float2 sm[];
    float2 *ba = sm, *bb = ba + C * LS, *tw = bb + C * LS;
    const long long l0 = (long long)blockIdx.x * C;
    const int tid = threadIdx.x, T = blockDim.x;
    load_twiddles(tw, twg, N);
    const float2 *in = reinterpret_cast<const float2 *>(rho);
    for (int t = tid; t < C * len; t += T) {
        const int c = t / len, n = t - c * len;
        ba[c * LS + n] = in[(l0 + c) * len + n];
    }
    __syncthreads();
    // stage A (c fastest: conflict-free across the padded lines)
    for (int t = tid; t < R2 * C; t += T) {
        const int c = t & (C - 1), j = t >> lgC;
        float2 v[R1];
#pragma unroll
        for (int r = 0; r < R1; ++r) v[r] = ba[c * LS + j + r * R2];
        dft<R1, false>(v);
#pragma unroll
        for (int r = 0; r < R1; ++r) bb[c * LS + j * R1 + r] = v[r];
    }
    __syncthreads();
    const float2 *Z = bb;
    if constexpr (R2 > 1) {
        // stage B (j fastest)
        for (int t = tid; t < R1 * C; t += T) {
            const int j = t & (R1 - 1), c = t / R1;
            float2 v[R2];
#pragma unroll
            for (int r = 0; r < R2; ++r) v[r] = bb[c * LS + j + r * R1];
            twiddle<R2, false>(v, j, tw, N / len);
            dft<R2, false>(v);
#pragma unroll
            for (int r = 0; r < R2; ++r) ba[c * LS + j + r * R1] = v[r];
        }
        __syncthreads();
        Z = ba;
    }
    for (int t = tid; t < C * len; t += T) {
        const int c = t / len, k = t - c * len;
        const float2 zk = Z[c * LS + k], zm = Z[c * LS + ((len - k) & (len - 1))];
        const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        spec[(l0 + c) * len + k] = cadd(e, cmul(tw[k], o));
    }
}

// ---------------------------------------------------------------- pass 2
// the y-FFT of plane x, columns kz0 .. kz0 + C - 1, in place. Shared tiles
// are row-major with row stride S = C + 1.
template <int R1, int R2>
__global__ void __launch_bounds__(kFftThreads) k_fft_y(float2 *__restrict__ spec, const float2 *__restrict__ twg,
                                                       int N, int C, int lgC)
{
    constexpr int len = R1 * R2;           // N
    extern __shared__ float2 sm[];
    const int H = N / 2, S = C + 1, tid = threadIdx.x, T = blockDim.x;
    float2 *b0 = sm, *tw = b0 + len * S;
    const int tiles = H / C;
    const long long x = blockIdx.x / tiles;
    const int kz0 = (int)(blockIdx.x - x * tiles) * C;
    float2 *base = spec + x * N * H + kz0;
    load_twiddles(tw, twg, N);
    if constexpr (R2 == 1) {
        __syncthreads();
        for (int t = tid; t < C; t += T) {
            float2 v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = base[(long long)r * H + t];
            dft<R1, false>(v);
#pragma unroll
            for (int r = 0; r < R1; ++r) base[(long long)r * H + t] = v[r];
        }
    } else {
        for (int t = tid; t < R2 * C; t += T) {
            const int c = t & (C - 1), j = t >> lgC;
            float2 v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = base[(long long)(j + r * R2) * H + c];
            dft<R1, false>(v);
#pragma unroll
            for (int r = 0; r < R1; ++r) b0[(j * R1 + r) * S + c] = v[r];
        }
        __syncthreads();
        for (int t = tid; t < R1 * C; t += T) {
            const int c = t & (C - 1), j = t >> lgC;
            float2 v[R2];
#pragma unroll
            for (int r = 0; r < R2; ++r) v[r] = b0[(j + r * R1) * S + c];
            twiddle<R2, false>(v, j, tw, N / len);
            dft<R2, false>(v);
#pragma unroll
            for (int r = 0; r < R2; ++r) base[(long long)(j + r * R1) * H + c] = v[r];
        }
    }
}

// ---------------------------------------------------------------- pass 3
// at row y, columns kz0 .. kz0 + C - 1: the forward x-FFT, the Green's
// function, and the inverse x-FFTs of phi (to A) and -i kx phi (to B).
// Thread t < R1 C owns the forward's stage-B butterfly (j, c) = (t / C,
// t mod C) (R1 C <= 256 for every mesh), which is the inverse's first one.
template <int R1, int R2>
__global__ void __launch_bounds__(kFftThreads) k_fft_x_green(const float2 *__restrict__ spec, float2 *__restrict__ A,
                                                             float2 *__restrict__ B, const float2 *__restrict__ twg,
                                                             const float *__restrict__ gtab,
                                                             const float *__restrict__ wtab, float kf, int N, int C,
                                                             int lgC)
{
    constexpr int len = R1 * R2;           // N
    constexpr int RB = R2 > 1 ? R2 : R1;   // points of the stage held in registers
    extern __shared__ float2 sm[];
    const int H = N / 2, S = C + 1, tid = threadIdx.x, T = blockDim.x;
    float2 *b0 = sm, *tw = b0 + len * S;
    const int tiles = H / C;
    const int iy = blockIdx.x / tiles;
    const int kz0 = (blockIdx.x - iy * tiles) * C;
    const long long rowx = (long long)N * H;            // stride of x in the spectra
    const long long off = (long long)iy * H + kz0;
    load_twiddles(tw, twg, N);
    if constexpr (R2 > 1) {
        // forward stage A, from global
        for (int t = tid; t < R2 * C; t += T) {
            const int c = t & (C - 1), j = t >> lgC;
            float2 v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = spec[(j + r * R2) * rowx + off + c];
            dft<R1, false>(v);
#pragma unroll
            for (int r = 0; r < R1; ++r) b0[(j * R1 + r) * S + c] = v[r];
        }
    }
    __syncthreads();
    const bool own = tid < (R2 > 1 ? R1 : 1) * C;
    const int c = tid & (C - 1), j = tid >> lgC;
    float2 phi[RB];
    const int ny = iy < H ? iy : iy - N;
    const float wy = iy == H ? 0.0f : wtab[iy];
    if (own) {
        if constexpr (R2 > 1) {
#pragma unroll
            for (int r = 0; r < R2; ++r) phi[r] = b0[(j + r * R1) * S + c];
            twiddle<R2, false>(phi, j, tw, N / len);
            dft<R2, false>(phi);
        } else {
#pragma unroll
            for (int r = 0; r < R1; ++r) phi[r] = spec[r * rowx + off + c];
            dft<R1, false>(phi);
        }
        const int nz = kz0 + c;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const int ix = R2 > 1 ? j + r * R1 : r;
            const int nx = ix < H ? ix : ix - N;
            float g = 0.0f;
            if (ix != H && iy != H)         // the Nyquist planes are dropped (kz < H always)
                g = gtab[nx * nx + ny * ny + nz * nz] * wtab[ix] * wy * wtab[nz];
            phi[r] = make_float2(phi[r].x * g, phi[r].y * g);
        }
    }
    __syncthreads();                        // b0 free again
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        float2 *out = pass == 0 ? A : B;
        if (own) {
            float2 w[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const int ix = R2 > 1 ? j + r * R1 : r;
                const int nx = ix < H ? ix : ix - N;
                w[r] = pass == 0 ? phi[r] : mul_mik(kf * nx, phi[r]);
            }
            if constexpr (R2 > 1) {
                // inverse stage A: radix R2 over rows j + r R1, outputs at rows j R2 + r
                dft<R2, true>(w);
#pragma unroll
                for (int r = 0; r < R2; ++r) b0[(j * R2 + r) * S + c] = w[r];
            } else {
                dft<R1, true>(w);
#pragma unroll
                for (int r = 0; r < R1; ++r) out[r * rowx + off + c] = w[r];
            }
        }
        if constexpr (R2 > 1) {
            __syncthreads();
            // inverse stage B: radix R1 over rows jj + r R2, to global
            for (int t = tid; t < R2 * C; t += T) {
                const int cc = t & (C - 1), jj = t >> lgC;
                float2 u[R1];
#pragma unroll
                for (int r = 0; r < R1; ++r) u[r] = b0[(jj + r * R2) * S + cc];
                twiddle<R1, true>(u, jj, tw, N / len);
                dft<R1, true>(u);
#pragma unroll
                for (int r = 0; r < R1; ++r) out[(jj + r * R2) * rowx + off + cc] = u[r];
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- pass 4
// at plane x, columns kz0 .. kz0 + C - 1: Y = F^-1 A (in place of A) and
// Yy = F^-1 (-i ky A) from one read of A, then Yx = F^-1 B (in place of B)
template <int R1, int R2>
__global__ void __launch_bounds__(kFftThreads) k_fft_y_inv(float2 *__restrict__ A, float2 *__restrict__ B,
                                                           float2 *__restrict__ Yy, const float2 *__restrict__ twg,
                                                           float kf, int N, int C, int lgC)
{
    constexpr int len = R1 * R2;           // N
    extern __shared__ float2 sm[];
    const int H = N / 2, S = C + 1, tid = threadIdx.x, T = blockDim.x;
    float2 *b0 = sm, *b1 = b0 + len * S, *tw = b1 + len * S;
    const int tiles = H / C;
    const long long x = blockIdx.x / tiles;
    const int kz0 = (int)(blockIdx.x - x * tiles) * C;
    const long long off = x * N * H + kz0;
    float2 *pa = A + off, *pb = B + off, *py = Yy + off;
    load_twiddles(tw, twg, N);
    if constexpr (R2 == 1) {
        __syncthreads();
        for (int t = tid; t < C; t += T) {
            float2 v[R1], vy[R1], vb[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                const int ny = r < H ? r : r - N;
                v[r] = pa[(long long)r * H + t];
                vy[r] = mul_mik(kf * ny, v[r]);
                vb[r] = pb[(long long)r * H + t];
            }
            dft<R1, true>(v);
            dft<R1, true>(vy);
            dft<R1, true>(vb);
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                pa[(long long)r * H + t] = v[r];
                py[(long long)r * H + t] = vy[r];
                pb[(long long)r * H + t] = vb[r];
            }
        }
    } else {
        // A: stage A of Y and Yy together
        for (int t = tid; t < R2 * C; t += T) {
            const int c = t & (C - 1), j = t >> lgC;
            float2 v[R1], vy[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                const int y = j + r * R2;
                const int ny = y < H ? y : y - N;
                v[r] = pa[(long long)y * H + c];
                vy[r] = mul_mik(kf * ny, v[r]);
            }
            dft<R1, true>(v);
            dft<R1, true>(vy);
#pragma unroll
            for (int r = 0; r < R1; ++r) {
                b0[(j * R1 + r) * S + c] = v[r];
                b1[(j * R1 + r) * S + c] = vy[r];
            }
        }
        __syncthreads();
        for (int t = tid; t < R1 * C; t += T) {
            const int c = t & (C - 1), j = t >> lgC;
            float2 v[R2], vy[R2];
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                v[r] = b0[(j + r * R1) * S + c];
                vy[r] = b1[(j + r * R1) * S + c];
            }
            twiddle<R2, true>(v, j, tw, N / len);
            twiddle<R2, true>(vy, j, tw, N / len);
            dft<R2, true>(v);
            dft<R2, true>(vy);
#pragma unroll
            for (int r = 0; r < R2; ++r) {
                pa[(long long)(j + r * R1) * H + c] = v[r];
                py[(long long)(j + r * R1) * H + c] = vy[r];
            }
        }
        __syncthreads();
        // B -> Yx
        for (int t = tid; t < R2 * C; t += T) {
            const int c = t & (C - 1), j = t >> lgC;
            float2 v[R1];
#pragma unroll
            for (int r = 0; r < R1; ++r) v[r] = pb[(long long)(j + r * R2) * H + c];
            dft<R1, true>(v);
#pragma unroll
            for (int r = 0; r < R1; ++r) b0[(j * R1 + r) * S + c] = v[r];
        }
        __syncthreads();
        for (int t = tid; t < R1 * C; t += T) {
            const int c = t & (C - 1), j = t >> lgC;
            float2 v[R2];
#pragma unroll
            for (int r = 0; r < R2; ++r) v[r] = b0[(j + r * R1) * S + c];
            twiddle<R2, true>(v, j, tw, N / len);
            dft<R2, true>(v);
#pragma unroll
            for (int r = 0; r < R2; ++r) pb[(long long)(j + r * R1) * H + c] = v[r];
        }
    }
}

// ---------------------------------------------------------------- pass 5
// the complex-to-real pre-processing of row k of a half spectrum line
// (X[H] = 0), times -i kz first when dz
__device__ __forceinline__ float2 c2r_pre(float2 a, float2 b, int k, int H, bool dz, float kf, const float2 *tw)
{
    if (dz) {
        a = mul_mik(kf * k, a);
        b = mul_mik(kf * (H - k), b);
    }
    const float2 s = cadd(a, cconj(b)), d = csub(a, cconj(b));
    const float2 dw = cmul(d, cconj(tw[k]));           // e^{+2 pi i k / N}
    return make_float2(s.x - dw.y, s.y + dw.x);          // s + i d w
}

// z-lines l0 .. l0 + C - 1 of field q = blockIdx.y (0 .. 3: -dphi/dx from
// Yx, -dphi/dy from Yy, -dphi/dz from -i kz Y, phi from Y), N reals each;
// line-major tiles (stride H + 1). One field per block keeps a block's
// registers to one line set (Y is read by two blocks)
template <int R1, int R2>
__global__ void __launch_bounds__(kFftThreads) k_fft_z_c2r(const float2 *__restrict__ Y, const float2 *__restrict__ Yy,
                                                           const float2 *__restrict__ Yx, float *__restrict__ field,
                                                           const float2 *__restrict__ twg, float kf, int N, int C,
                                                           int lgC)
{
    constexpr int len = R1 * R2;           // H
    constexpr int LS = len + 1;
    extern __shared__ float2 sm[];
    float2 *bx = sm, *b0 = bx + C * LS, *tw = b0 + C * LS;
    const long long l0 = (long long)blockIdx.x * C;
    const long long N3 = (long long)N * N * N;
    const int tid = threadIdx.x, T = blockDim.x, q = blockIdx.y;
    const float2 *src = q == 0 ? Yx : q == 1 ? Yy : Y;
    float2 *out = reinterpret_cast<float2 *>(field + q * N3);
    const bool dz = q == 2;
    load_twiddles(tw, twg, N);
    for (int t = tid; t < C * len; t += T) {
        const int c = t / len, n = t - c * len;
        bx[c * LS + n] = src[(l0 + c) * len + n];
    }
    __syncthreads();
    for (int t = tid; t < R2 * C; t += T) {
        const int c = t & (C - 1), j = t >> lgC;
        float2 v[R1];
#pragma unroll
        for (int r = 0; r < R1; ++r) {
            const int k = j + r * R2;
            const float2 a = bx[c * LS + k];
            const float2 b = k ? bx[c * LS + len - k] : make_float2(0.0f, 0.0f);
            v[r] = c2r_pre(a, b, k, len, dz, kf, tw);
        }
        dft<R1, true>(v);
        if constexpr (R2 == 1) {
#pragma unroll
            for (int r = 0; r < R1; ++r) out[(l0 + c) * len + r] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < R1; ++r) b0[c * LS + j * R1 + r] = v[r];
        }
    }
    if constexpr (R2 > 1) {
        __syncthreads();
        // stage B, j fastest: each line's outputs go out as runs of R1 values
        for (int t = tid; t < R1 * C; t += T) {
            const int j = t & (R1 - 1), c = t / R1;
            float2 v[R2];
#pragma unroll
            for (int r = 0; r < R2; ++r) v[r] = b0[c * LS + j + r * R1];
            twiddle<R2, true>(v, j, tw, N / len);
            dft<R2, true>(v);
#pragma unroll
            for (int r = 0; r < R2; ++r) out[(l0 + c) * len + j + r * R1] = v[r];
        }
    }
}

size_t smem_rows(int len, int C, int bufs, int N) { return ((size_t)bufs * len * (C + 1) + N) * sizeof(float2); }
size_t smem_lines(int len, int C, int bufs, int N) { return ((size_t)bufs * C * (len + 1) + N) * sizeof(float2); }

template <int R1, int R2>
cudaError_t set_smem_xy(int N)
{
    const int big = (int)smem_rows(R1 * R2, kFftC, 2, N);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fft_y<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_fft_x_green<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_fft_y_inv<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) !=
            cudaSuccess)
        return e;
    return cudaSuccess;
}

template <int R1, int R2>
cudaError_t set_smem_z(int N)
{
    const int big = (int)smem_lines(R1 * R2, kFftC, 3, N);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_fft_z_r2c<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_fft_z_c2r<R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)) !=
            cudaSuccess)
        return e;
    return cudaSuccess;
}

cudaError_t fft_configure()
{
    static bool done[kMaxDevices];
    return once_per_device(done, []() {
        cudaError_t e;
        if ((e = set_smem_xy<8, 1>(8)) != cudaSuccess || (e = set_smem_xy<16, 1>(16)) != cudaSuccess ||
            (e = set_smem_xy<16, 2>(32)) != cudaSuccess || (e = set_smem_xy<16, 4>(64)) != cudaSuccess ||
            (e = set_smem_xy<16, 8>(128)) != cudaSuccess || (e = set_smem_xy<16, 16>(256)) != cudaSuccess ||
            (e = set_smem_xy<16, 32>(512)) != cudaSuccess || (e = set_smem_z<4, 1>(8)) != cudaSuccess ||
            (e = set_smem_z<8, 1>(16)) != cudaSuccess || (e = set_smem_z<16, 1>(32)) != cudaSuccess ||
            (e = set_smem_z<16, 2>(64)) != cudaSuccess || (e = set_smem_z<16, 4>(128)) != cudaSuccess ||
            (e = set_smem_z<16, 8>(256)) != cudaSuccess || (e = set_smem_z<16, 16>(512)) != cudaSuccess)
            return e;
        return cudaSuccess;
    });
}

// the five passes for one (R1 R2 = N) x (Z1 Z2 = N / 2) factorisation
template <int R1, int R2, int Z1, int Z2>
void launch_passes(const float *rho, float *field, float2 *S, float2 *A, float2 *B, float2 *Yy, const float2 *tw,
                   const float *gtab, const float *wtab, float kf, int N, int C, cudaStream_t st)
{
    const int H = N / 2, lgC = ilog2(C);
    const unsigned zlines = (unsigned)((long long)N * N / C), cols = (unsigned)((long long)N * (H / C));
    k_fft_z_r2c<Z1, Z2><<<zlines, kFftThreads, smem_lines(H, C, 2, N), st>>>(rho, S, tw, N, C, lgC);
    k_fft_y<R1, R2><<<cols, kFftThreads, smem_rows(N, C, 1, N), st>>>(S, tw, N, C, lgC);
    k_fft_x_green<R1, R2><<<cols, kFftThreads, smem_rows(N, C, 1, N), st>>>(S, A, B, tw, gtab, wtab, kf, N, C,
                                                                            lgC);
    k_fft_y_inv<R1, R2><<<cols, kFftThreads, smem_rows(N, C, 2, N), st>>>(A, B, Yy, tw, kf, N, C, lgC);
    k_fft_z_c2r<Z1, Z2><<<dim3(zlines, 4), kFftThreads, smem_lines(H, C, 2, N), st>>>(A, Yy, B, field, tw, kf, N,
                                                                                     C, lgC);
}

}  // namespace

bool fft_mesh_ok(int N) { return N >= 8 && N <= 512 && (N & (N - 1)) == 0; }

// the twiddle table of an N-point mesh: e^{-2 pi i m / N}, m < N (FP64 on
// the host, rounded to FP32)
void fft_twiddles(int N, float2 *host)
{
    for (int m = 0; m < N; ++m) {
        const double a = 2.0 * M_PI * (double)m / (double)N;
        host[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
}

// rho (N^3) -> field (4 N^3). Scratch: S (N^2 H complex) and W (3 N^2 H
// complex). Five launches.
cudaError_t fft_solve(const float *rho, float *field, float2 *S, float2 *W, const float2 *tw, const float *gtab,
                      const float *wtab, float kf, int N, cudaStream_t st)
{
    cudaError_t e = fft_configure();
    if (e != cudaSuccess) return e;
    const int H = N / 2;
    const int C = std::min(kFftC, H);
    const long long M = (long long)N * N * H;
    float2 *A = W, *B = W + M, *Yy = W + 2 * M;
    switch (N) {
    case 8: launch_passes<8, 1, 4, 1>(rho, field, S, A, B, Yy, tw, gtab, wtab, kf, N, C, st); break;
    case 16: launch_passes<16, 1, 8, 1>(rho, field, S, A, B, Yy, tw, gtab, wtab, kf, N, C, st); break;
    case 32: launch_passes<16, 2, 16, 1>(rho, field, S, A, B, Yy, tw, gtab, wtab, kf, N, C, st); break;
    case 64: launch_passes<16, 4, 16, 2>(rho, field, S, A, B, Yy, tw, gtab, wtab, kf, N, C, st); break;
    case 128: launch_passes<16, 8, 16, 4>(rho, field, S, A, B, Yy, tw, gtab, wtab, kf, N, C, st); break;
    case 256: launch_passes<16, 16, 16, 8>(rho, field, S, A, B, Yy, tw, gtab, wtab, kf, N, C, st); break;
    case 512: launch_passes<16, 32, 16, 16>(rho, field, S, A, B, Yy, tw, gtab, wtab, kf, N, C, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pg
