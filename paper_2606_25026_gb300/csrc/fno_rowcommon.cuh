// Device helpers shared by the forward and backward row kernels of the FNO.
//
// Each translation unit that includes this header gets its own copy of the
// x-stage tables in constant memory (the row kernels read them as warp-uniform
// broadcasts) and uploads it through its own entry point.
#pragma once
#include "fno_internal.cuh"

namespace spe {
namespace fno {

// Gx [n][16] and Fx [16][n] for n = 64 and n = 32 (rows beyond M unused).
static __constant__ float2 cG64[64 * kTableM];
static __constant__ float2 cF64[kTableM * 64];
static __constant__ float2 cG32[32 * kTableM];
static __constant__ float2 cF32[kTableM * 32];

template <int N>
__device__ __forceinline__ float2 Gx(int x, int kx)
{
    return N == 64 ? cG64[x * kTableM + kx] : cG32[x * kTableM + kx];
}

template <int N>
__device__ __forceinline__ float2 Fx(int kx, int x)
{
    return N == 64 ? cF64[kx * 64 + x] : cF32[kx * 32 + x];
}

static inline cudaError_t upload_tables_here(const float2 *G64, const float2 *F64, const float2 *G32,
                                             const float2 *F32)
{
    cudaError_t e = cudaMemcpyToSymbol(cG64, G64, sizeof(float2) * 64 * kTableM);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cF64, F64, sizeof(float2) * 64 * kTableM);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cG32, G32, sizeof(float2) * 32 * kTableM);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cF32, F32, sizeof(float2) * 32 * kTableM);
    return e;
}

__device__ __forceinline__ float act_load(const float *p) { return *p; }
__device__ __forceinline__ float act_load(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void act_store(float *p, float v) { *p = v; }
__device__ __forceinline__ void act_store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
// the value an activation holds once stored
__device__ __forceinline__ float act_round(float v, const float *) { return v; }
__device__ __forceinline__ float act_round(float v, const __nv_bfloat16 *)
{
    return __bfloat162float(__float2bfloat16_rn(v));
}

__device__ __forceinline__ float wload(const __nv_bfloat16 *w, size_t i) { return __bfloat162float(w[i]); }

constexpr float kInvSqrt2 = 0.70710678118654752440f;
constexpr float kInvSqrt2Pi = 0.39894228040143267794f;

// exact GELU u Phi(u) and its derivative Phi(u) + u phi(u)
__device__ __forceinline__ float gelu(float u) { return 0.5f * u * (1.f + erff(u * kInvSqrt2)); }
__device__ __forceinline__ float gelu_grad(float u)
{
    return 0.5f * (1.f + erff(u * kInvSqrt2)) + u * kInvSqrt2Pi * expf(-0.5f * u * u);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void zero_shared(float *sh, int count)
{
    for (int e = threadIdx.x; e < count; e += blockDim.x) sh[e] = 0.f;
}

__device__ __forceinline__ void write_partials(const float *sh, float *partials, int seg)
{
    for (int e = threadIdx.x; e < seg; e += blockDim.x) partials[(size_t)blockIdx.x * seg + e] = sh[e];
}

}  // namespace fno
}  // namespace spe
