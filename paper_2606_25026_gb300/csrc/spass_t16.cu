// Strided-pass kernels with 16-column tiles (see spass_impl.cuh); separate translation units
// per width so they compile in parallel.
#include "spass_impl.cuh"

namespace spe {

cudaError_t launch_spass_t16(int n, const SParams &p, cudaStream_t st, int *blocks_out)
{
    switch (n) {
#define X(n) \
    case n: return spass_launch_w<n, 16>(p, st, blocks_out);
        SPE_FOR_EACH_N(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t setup_spass_attributes_t16()
{
    cudaError_t e = cudaSuccess;
#define X(n) \
    if (e == cudaSuccess) e = spass_attr_w<n, 16>();
    SPE_FOR_EACH_N(X)
#undef X
    return e;
}

}  // namespace spe
