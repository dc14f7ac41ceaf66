// pg_table.cu -- device side of the bit-pattern force table (Section 3.4.1).
//
// The stored table is the paper's pair per knot, G0_k = f(r_k)/r_k and
// G1_k = (G0_{k+1} - G0_k) / (s_{k+1} - s_k), with the knot s_k being the
// FP32 pattern of 2.0f plus k * 2^(23-F). The force kernels keep a derived
// pair in shared memory instead: A_k = G0_k - s_k G1_k with G1_k, so that the
// interpolation G0_k + (s - s_k) G1_k of Section 3.4.2 becomes one fused
// multiply-add, g = A_k + s G1_k, and the knot s_k need not be rebuilt from
// the index bits in the pair loop.
#include "pg_device.cuh"

namespace pg {

__device__ __forceinline__ float knot_s(int k, int shift)
{
    return __uint_as_float(0x40000000u + ((unsigned)k << shift));
}

__global__ void k_table_prep(const float *__restrict__ G0, const float *__restrict__ G1,
                             float2 *__restrict__ AG1, int n, int shift)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float g1 = G1[k];
    AG1[k] = make_float2(fmaf(-knot_s(k, shift), g1, G0[k]), g1);
}

cudaError_t launch_table_prep(const float *G0, const float *G1, float2 *AG1, int E, int F,
                              cudaStream_t st)
{
    int n = 1 << (E + F);
    k_table_prep<<<(n + 255) / 256, 256, 0, st>>>(G0, G1, AG1, n, 23 - F);
    return cudaGetLastError();
}

// G0/G1 from knot values v (v[n-1] is the value at r_cut from below); the
// last entry is zero so that the force vanishes at and beyond r_cut. The
// knot spacing is a power of two, so the FP64 quotient is exact and the
// only rounding is the final one to FP32.
__global__ void k_table_from_values(const float *__restrict__ v, float *__restrict__ G0,
                                    float *__restrict__ G1, int n, int shift)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (k < n - 1) {
        double ds = (double)knot_s(k + 1, shift) - (double)knot_s(k, shift);
        G0[k] = v[k];
        G1[k] = (float)(((double)v[k + 1] - (double)v[k]) / ds);
    } else {
        G0[k] = 0.0f;
        G1[k] = 0.0f;
    }
}

cudaError_t launch_table_from_values(const float *v, float *G0, float *G1, int E, int F,
                                     cudaStream_t st)
{
    int n = 1 << (E + F);
    k_table_from_values<<<(n + 255) / 256, 256, 0, st>>>(v, G0, G1, n, 23 - F);
    return cudaGetLastError();
}

// The force table and a potential table on the same knots, interleaved as
// {A_k, G1_k, A_p,k, P1_k} (A_p,k = P0_k - s_k P1_k), so that one 16-byte
// shared load gives both interpolants: g = A + s G1, psi = A_p + s P1.
__global__ void k_table_merge(const float2 *__restrict__ AG1, const float *__restrict__ P0,
                              const float *__restrict__ P1, float4 *__restrict__ AGP, int n,
                              int shift)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float2 f = AG1[k];
    const float p1 = P1[k];
    AGP[k] = make_float4(f.x, f.y, fmaf(-knot_s(k, shift), p1, P0[k]), p1);
}

cudaError_t launch_table_merge(const float2 *AG1, const float *P0, const float *P1, float4 *AGP,
                               int E, int F, cudaStream_t st)
{
    int n = 1 << (E + F);
    k_table_merge<<<(n + 255) / 256, 256, 0, st>>>(AG1, P0, P1, AGP, n, 23 - F);
    return cudaGetLastError();
}

}  // namespace pg
