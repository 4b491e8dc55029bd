// Deterministic grid-wide reductions in FP64.
//
// Every block reduces its values with warp shuffles, writes one partial per
// slot, and takes a ticket; the block that takes the last ticket sums all
// partials in a fixed order (thread i takes partials i, i + NT, ...; then a
// fixed shuffle tree), writes the result and returns the ticket counter to
// zero.  The result therefore does not depend on block scheduling.
#pragma once
#include <cuda_runtime.h>

namespace spe {

__device__ __forceinline__ double warp_op(double v, bool is_max)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmax(v, w) : v + w;
    }
    return v;
}

// Block-wide reduction of K values; the result is valid in thread 0.
// maxmask bit k selects max instead of sum for slot k.
template <int K, int NT>
__device__ __forceinline__ void block_reduce(double (&v)[K], int maxmask, double *sh)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_op(v[k], (maxmask >> k) & 1);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) sh[k * NW + warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double x = lane < NW ? sh[k * NW + lane] : 0.0;
            v[k] = warp_op(x, (maxmask >> k) & 1);
        }
    }
}

// The reduction over nblocks work units (tiles) numbered bid = 0 .. nblocks - 1: every unit calls
// this exactly once, from whichever block runs it.  partials holds nblocks * K doubles; counter
// starts (and ends) at 0.  With out_scaled, the results times scale are written there as well.
template <int K, int NT>
__device__ __forceinline__ void tile_reduce(double (&v)[K], int maxmask, double *partials, unsigned int *counter,
                                            double *out, double *out_scaled, double scale, unsigned int bid,
                                            unsigned int nblocks)
{
    __shared__ double sh[K * (NT / 32)];
    __shared__ int last;
    block_reduce<K, NT>(v, maxmask, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) partials[(size_t)bid * K + k] = v[k];
        __threadfence();
        unsigned int ticket = atomicAdd(counter, 1u);
        last = (ticket == nblocks - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    // the loads are independent of the running sums: unrolled, they are in flight together (the
    // order of the additions, and so the result, is unchanged)
#pragma unroll 8
    for (unsigned int b = threadIdx.x; b < nblocks; b += NT) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double x = __ldcg(&partials[(size_t)b * K + k]);
            acc[k] = ((maxmask >> k) & 1) ? fmax(acc[k], x) : acc[k] + x;
        }
    }
    block_reduce<K, NT>(acc, maxmask, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = acc[k];
        if (out_scaled) {
#pragma unroll
            for (int k = 0; k < K; ++k) out_scaled[k] = acc[k] * scale;
        }
        *counter = 0u;
    }
}

// All blocks of the launch must call this exactly once (one unit per block).
template <int K, int NT>
__device__ __forceinline__ void grid_reduce(double (&v)[K], int maxmask, double *partials,
                                            unsigned int *counter, double *out, double *out_scaled = nullptr,
                                            double scale = 1.0)
{
    const unsigned int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    tile_reduce<K, NT>(v, maxmask, partials, counter, out, out_scaled, scale, bid, nblocks);
}

}  // namespace spe
