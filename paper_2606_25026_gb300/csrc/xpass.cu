// x passes (FP32 instances); the kernel is in xpass_impl.cuh.
#include "xpass_impl.cuh"

namespace spe {

template <int N>
static cudaError_t launch_x_n(const XParams &p, cudaStream_t st, int *blocks_out)
{
    const int blocks = (p.rows + XCfg<N>::T - 1) / XCfg<N>::T;
    if (blocks_out) *blocks_out = blocks;
    xpass_kernel<N, false><<<blocks, XCfg<N>::NT, XCfg<N>::smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_xpass_tc(int nx, const XParams &p, cudaStream_t st, int *blocks_out);

cudaError_t launch_xpass(int nx, const XParams &p, cudaStream_t st, int *blocks_out)
{
    if (p.tc && (nx == 256 || nx == 512)) return launch_xpass_tc(nx, p, st, blocks_out);
    switch (nx) {
#define X(n) \
    case n: return launch_x_n<n>(p, st, blocks_out);
        SPE_FOR_EACH_N(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

size_t xpass_rows_per_block(int) { return 16; }

cudaError_t setup_xpass_attributes()
{
    cudaError_t e = cudaSuccess;
#define X(n)                                                                                                    \
    if (e == cudaSuccess)                                                                                        \
        e = cudaFuncSetAttribute(xpass_kernel<n, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XCfg<n>::smem);
    SPE_FOR_EACH_N(X)
#undef X
    return e;
}

}  // namespace spe
