// x passes (FP32 instances); the kernel is in xpass_impl.cuh.
#include "xfused_impl.cuh"

namespace spe {

// The step's two x passes of a gravitating grid go to the fused kernels (xfused_impl.cuh);
// every other flag set (no gravity, static potential, absorbing layer, the final kick, the
// diagnostics) to the generic one.
constexpr int kKickFused = X_HAS_PHI | X_KICK | X_FFT;
constexpr int kDensFused = X_IFFT | X_MASS | X_R2C;

template <int N>
static cudaError_t launch_x_n(const XParams &p, cudaStream_t st, int *blocks_out)
{
    const int blocks = (p.rows + XCfg<N>::T - 1) / XCfg<N>::T;
    if (blocks_out) *blocks_out = blocks;
    constexpr int NT = XCfg<N>::NT;
    constexpr size_t SM = XCfg<N>::smem;
    if constexpr (xfused_ok<N>()) {
        const int f = p.flags;
        if (f == kKickFused) {
            xkick_fused_kernel<N, false><<<blocks, NT, SM, st>>>(p);
            return cudaGetLastError();
        }
        if (f == (kKickFused | X_WRITE_PHI)) {
            xkick_fused_kernel<N, true><<<blocks, NT, SM, st>>>(p);
            return cudaGetLastError();
        }
        if (f == kDensFused) {
            xdens_fused_kernel<N, false><<<blocks, xdens_nt<N>(), SM, st>>>(p);
            return cudaGetLastError();
        }
        if (f == (kDensFused | X_DEP)) {
            xdens_fused_kernel<N, true><<<blocks, xdens_nt<N>(), SM, st>>>(p);
            return cudaGetLastError();
        }
    }
    xpass_kernel<N, false><<<blocks, NT, SM, st>>>(p);
    return cudaGetLastError();
}

template <int N>
static cudaError_t attr_x_n()
{
    const int sm = (int)XCfg<N>::smem;
    cudaError_t e = cudaFuncSetAttribute(xpass_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if constexpr (xfused_ok<N>()) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(xkick_fused_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(xkick_fused_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(xdens_fused_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(xdens_fused_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    }
    return e;
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
#define X(n) \
    if (e == cudaSuccess) e = attr_x_n<n>();
    SPE_FOR_EACH_N(X)
#undef X
    return e;
}

}  // namespace spe
