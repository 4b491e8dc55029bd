// Tensor-core (split FP16) instances of the x and strided passes for N = 256
// and 512: the same kernels with every radix-16 stage on tcgen05 (tc16.cuh).
#include "spass_impl.cuh"
#include "xpass_impl.cuh"

namespace spe {

template <int N>
static cudaError_t launch_x_tc(const XParams &p, cudaStream_t st, int *blocks_out)
{
    const int blocks = (p.rows + XCfg<N, true>::T - 1) / XCfg<N, true>::T;
    if (blocks_out) *blocks_out = blocks;
    xpass_kernel<N, true><<<blocks, XCfg<N, true>::NT, XCfg<N, true>::smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_xpass_tc(int nx, const XParams &p, cudaStream_t st, int *blocks_out)
{
    if (nx == 256) return launch_x_tc<256>(p, st, blocks_out);
    if (nx == 512) return launch_x_tc<512>(p, st, blocks_out);
    return cudaErrorInvalidValue;
}

cudaError_t launch_spass_tc(int n, const SParams &p, cudaStream_t st, int *blocks_out)
{
    if (n == 256) return launch_s_nt<256, 16, true>(p, st, blocks_out);
    if (n == 512) return launch_s_nt<512, 16, true>(p, st, blocks_out);
    return cudaErrorInvalidValue;
}

cudaError_t setup_tc_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(xpass_kernel<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)XCfg<256, true>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(xpass_kernel<512, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)XCfg<512, true>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(spass_kernel<256, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SCfg<256, 16, true>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(spass_kernel<512, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SCfg<512, 16, true>::smem);
    return e;
}

}  // namespace spe
