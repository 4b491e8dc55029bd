// spe_field_energy_noalloc: the field-energy reduction for callers that
// cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or any allocating routine) at the
// point where they need a diagnostic: code running inside another
// framework's memory pool, a real-time loop with a fixed memory budget, or a
// process that must not grow its device footprint after start-up.  This
// entry point computes the same mass and self-interaction energy as
// spe_energy for a complex64 field the caller already holds on the device,
// with its reduction scratch (block partial sums, the block ticket counter
// and the result slots) in one fixed file-scope device array instead of a
// grid workspace.
//
// The array is SPE_NOALLOC_SCRATCH_DOUBLES doubles (16.5 KB); every GPU that
// loads libspe keeps it until the process exits.  All calls share it, and it
// keeps the last call's contents, so calls that overlap on the GPU (on
// different streams or host threads at the same time) race; serialise them.
// The ticket counter is cleared at the start of every call.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress while that device is current (the name is only a
// host-side stand-in, not a device address) and caches it per device.  Make
// that first call before any stream capture.  cudaDeviceReset unloads the
// module, so the cached address is stale afterwards: a process that resets a
// device must not call this entry point on that device again.
#include <mutex>
#include <stdint.h>

#include "reduce.cuh"
#include "spe.h"
#include "spe_internal.cuh"

namespace {

constexpr int kNaBlocks = 1024;    // at most this many blocks, one partial pair each
constexpr int kNaThreads = 256;
constexpr int kNaCounterSlot = 2 * kNaBlocks;       // ticket counter (first 4 bytes of the slot)
constexpr int kNaResultSlot = 2 * kNaBlocks + 8;    // two raw sums for host delivery
constexpr int kNaMaxDevices = 64;
static_assert(kNaResultSlot + 2 <= SPE_NOALLOC_SCRATCH_DOUBLES, "scratch too small");

static __device__ __align__(256) double g_noalloc_scratch[SPE_NOALLOC_SCRATCH_DOUBLES];

std::mutex g_na_mu;
double *g_na_addr[kNaMaxDevices];

// Sum |psi|^2 and |psi|^4 over n values; the last block writes
// out[0] = dv * sum|psi|^2 and out[1] = kappa / 2 * dv * sum|psi|^4.
__global__ void __launch_bounds__(kNaThreads)
field_energy_noalloc_kernel(const float2 *__restrict__ psi, size_t n, double dv, double kappa, double *scratch,
                            double *out)
{
    __shared__ double sh[2 * (kNaThreads / 32)];
    __shared__ int last;
    double acc[2] = {0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)kNaThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kNaThreads) {
        const float2 v = psi[i];
        const double a2 = (double)v.x * v.x + (double)v.y * v.y;
        acc[0] += a2;
        acc[1] += a2 * a2;
    }
    unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + kNaCounterSlot);
    spe::block_reduce<2, kNaThreads>(acc, 0, sh);
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = acc[0];
        scratch[2 * blockIdx.x + 1] = acc[1];
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double tot[2] = {0.0, 0.0};
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += kNaThreads) {
        tot[0] += __ldcg(&scratch[2 * b]);
        tot[1] += __ldcg(&scratch[2 * b + 1]);
    }
    spe::block_reduce<2, kNaThreads>(tot, 0, sh);
    if (threadIdx.x == 0) {
        out[0] = tot[0] * dv;
        out[1] = 0.5 * kappa * tot[1] * dv;
        *counter = 0u;
    }
}

}  // namespace

extern "C" int spe_field_energy_noalloc(const void *psi_c64, size_t n, double cell_volume, double kappa,
                                        double *out2, int where, void *cuda_stream)
{
    if (!psi_c64 || !out2 || n == 0 || (where != SPE_HOST && where != SPE_DEVICE)) return SPE_EINVAL;
    if (n > SPE_NOALLOC_MAX_CELLS) return SPE_EINVAL;
    if (!(cell_volume > 0) || !isfinite(cell_volume) || !isfinite(kappa)) return SPE_EINVAL;
    // the kernel reads psi as float2 and writes out2 as doubles: both need 8-byte alignment
    if (((uintptr_t)psi_c64 & 7u) != 0 || (where == SPE_DEVICE && ((uintptr_t)out2 & 7u) != 0)) return SPE_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return SPE_ECUDA;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mu);
        if (!g_na_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
                cudaGetLastError();
                return SPE_ECUDA;
            }
            g_na_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_na_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaMemsetAsync(scratch + kNaCounterSlot, 0, sizeof(unsigned int), st) != cudaSuccess) return SPE_ECUDA;
    size_t blocks = (n + kNaThreads - 1) / kNaThreads;
    if (blocks > (size_t)kNaBlocks) blocks = kNaBlocks;
    double *dst = (where == SPE_DEVICE) ? out2 : scratch + kNaResultSlot;
    field_energy_noalloc_kernel<<<(unsigned)blocks, kNaThreads, 0, st>>>(static_cast<const float2 *>(psi_c64), n,
                                                                         cell_volume, kappa, scratch, dst);
    if (cudaGetLastError() != cudaSuccess) return SPE_ECUDA;
    if (where == SPE_HOST) {
        if (cudaMemcpyAsync(out2, scratch + kNaResultSlot, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
            return SPE_ECUDA;
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? SPE_OK : SPE_ECUDA;
}
