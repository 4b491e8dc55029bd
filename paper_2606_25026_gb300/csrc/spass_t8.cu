// Strided-pass kernels with 8-column tiles (see spass_impl.cuh); separate translation units
// per width so they compile in parallel.
#include "spass_impl.cuh"

namespace spe {

cudaError_t launch_spass_t8(int n, const SParams &p, cudaStream_t st, int *blocks_out)
{
    switch (n) {
#define X(n)                                                                               \
    case n:                                                                                \
        if constexpr (tile_fits<n>(8)) return launch_s_nt<n, 8>(p, st, blocks_out);   \
        return cudaErrorInvalidValue;
        SPE_FOR_EACH_N(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t setup_spass_attributes_t8()
{
    cudaError_t e = cudaSuccess;
#define X(n)                                                                                            \
    if constexpr (tile_fits<n>(8))                                                                   \
        if (e == cudaSuccess)                                                                            \
            e = cudaFuncSetAttribute(spass_kernel<n, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)SCfg<n, 8>::smem);
    SPE_FOR_EACH_N(X)
#undef X
    return e;
}

}  // namespace spe
