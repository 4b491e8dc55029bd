// One persistent launch per step for a batch of independent grids.
//
// A batch step is eight phases, the passes of the kick-drift-kick step in
// order (Sec. 3.1 Eq. (SPE_solver_KDK), Algorithm 1; stars by Sec. 3.2.2):
//   0  x pass: Phi from its half spectrum, kick, forward x transform
//   1  forward y transform of psi, and the stars' kick-drift-deposit
//      (both need only phase 0)
//   2  z pass: forward z transform, drift, inverse z transform
//   3  inverse y transform of psi
//   4  x pass: inverse x transform, density (+ the stars' deposit), mass,
//      real x transform of rho
//   5  forward y transform of the half spectrum
//   6  z pass: forward z transform, Poisson multiply, inverse z transform
//   7  inverse y transform of the half spectrum
// Each phase is one work list: every member's tiles of that pass (x-row
// tiles, strided column tiles, star blocks), numbered consecutively member
// after member.  The launch is cooperative (all CTAs resident); each CTA takes
// items it, it + gridDim.x, ... of the list and runs the pass's body with 256
// threads, then all CTAs meet at a grid-wide barrier before the next phase.
// Members of different sizes therefore share every SM in every phase, and one
// kernel launch replaces the members' 8-9 launches each.
//
// The barrier is a counter that every CTA increments once per phase; thread 0
// of each CTA then polls it, at most wait_limit times.  A poll count that runs
// out sets a status bit and the CTA leaves the kernel (the batch call then
// returns SPE_ETIMEOUT and the members' state must be set again): a CTA that
// is not resident, or that faulted, cannot hang the others.
//
// Strided tiles are 16 columns wide with each length's default radix plan and
// per-thread asynchronous tile copies; the x passes, the strided passes and
// the stars run the same bodies as the stand-alone kernels, so a member's
// result is bitwise that of the same grid stepped alone.
#include "particles_impl.cuh"
#include "spass_impl.cuh"
#include "xfused_impl.cuh"

namespace spe {

namespace {

constexpr int kBT = kBatchThreads;
static_assert(kBT == kPartThreads, "the star body runs one star per thread of a 256-thread block");

constexpr size_t cmax3(size_t a, size_t b) { return a > b ? a : b; }
template <int N> constexpr size_t member_smem()
{
    return cmax3(XCfg<N>::smem, SCfg<N, kBatchTile>::smem);
}
constexpr size_t kBatchSmem =
    cmax3(cmax3(cmax3(member_smem<64>(), member_smem<96>()), cmax3(member_smem<128>(), member_smem<192>())),
          (size_t)kBoxBytes);
constexpr size_t kPrmBytes = cmax3(cmax3(sizeof(XParams), sizeof(SParams)), sizeof(PParams));

// the pass parameters of the item, copied into shared memory once per item
template <class P>
__device__ __forceinline__ const P &stage_params(const P &src, unsigned char *prm)
{
    static_assert(sizeof(P) % 4 == 0, "parameter block copied in 4-byte words");
    const unsigned *s = reinterpret_cast<const unsigned *>(&src);
    unsigned *d = reinterpret_cast<unsigned *>(prm);
    for (int k = threadIdx.x; k < (int)(sizeof(P) / 4); k += kBT) d[k] = s[k];
    __syncthreads();
    return *reinterpret_cast<const P *>(prm);
}

// Each body behind a call of its own, so that every pass gets its own register allocation instead
// of one allocation for all of them inlined together.
template <int N, bool WPHI>
__device__ __noinline__ void item_kick(const XParams &p, int tile, unsigned char *smem)
{
    xkick_fused_body<N, kBT, WPHI>(p, tile, smem);
}
template <int N, bool DEP>
__device__ __noinline__ void item_dens(const XParams &p, int tile, int ntiles, unsigned char *smem)
{
    xdens_fused_body<N, kBT, DEP>(p, tile, ntiles, smem);
}
template <int N>
__device__ __noinline__ void item_strided(const SParams &p, int cx, int b, unsigned char *smem)
{
    spass_body<N, kBatchTile, kBT>(p, nullptr, cx, b, smem);
}
__device__ __noinline__ void item_stars(const PParams &p, int block, unsigned char *smem)
{
    particles_body(p, block, smem);
}

template <int N>
__device__ __forceinline__ void run_item_n(int phase, const BatchMember &mb, int local, unsigned char *smem,
                                           unsigned char *prm)
{
    switch (phase) {
    case 0: {
        const XParams &p = stage_params(mb.xk, prm);
        if (p.flags & X_WRITE_PHI) item_kick<N, true>(p, local, smem);
        else item_kick<N, false>(p, local, smem);
        break;
    }
    case 4: {
        const XParams &p = stage_params(mb.xd, prm);
        if (p.flags & X_DEP) item_dens<N, true>(p, local, mb.xtiles, smem);
        else item_dens<N, false>(p, local, mb.xtiles, smem);
        break;
    }
    case 1: {
        const int ny_items = mb.cols_psi * N;
        if (local >= ny_items) {
            item_stars(stage_params(mb.pp, prm), local - ny_items, smem);
            break;
        }
        item_strided<N>(stage_params(mb.yf, prm), local % mb.cols_psi, local / mb.cols_psi, smem);
        break;
    }
    default: {
        const SParams *src = phase == 2 ? &mb.zd : phase == 3 ? &mb.yi : phase == 5 ? &mb.rf : phase == 6 ? &mb.rp
                                                                                                       : &mb.ri;
        const int cols = phase <= 3 ? mb.cols_psi : mb.cols_rho;
        item_strided<N>(stage_params(*src, prm), local % cols, local / cols, smem);
        break;
    }
    }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// every CTA arrives once; false when this CTA's wait ran out (the status bit is set)
__device__ __forceinline__ bool grid_barrier(const BatchLaunch &L, int phase)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(L.bar, 1u);
        const unsigned target = (unsigned)(phase + 1) * gridDim.x;
        int good = 1;
        for (long long it = 0; ld_acquire(L.bar) < target; ++it) {
            if (it >= L.wait_limit) {
                good = 0;
                atomicOr(L.status, kTcStatusTimeout);
                break;
            }
            __nanosleep(128);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

__global__ void __launch_bounds__(kBT, 3) batch_persist_kernel(BatchLaunch L)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) unsigned char prm[kPrmBytes];
    for (int phase = 0; phase < kBatchPhases; ++phase) {
        const int *off = L.offs + phase * (L.count + 1);
        const int total = off[L.count];
        for (int it = blockIdx.x; it < total; it += gridDim.x) {
            // the member holding item it: the last m with off[m] <= it
            int lo = 0, hi = L.count - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (off[mid] <= it) lo = mid;
                else hi = mid - 1;
            }
            const BatchMember &mb = L.m[lo];
            const int local = it - off[lo];
            switch (mb.n) {
            case 64: run_item_n<64>(phase, mb, local, smem, prm); break;
            case 96: run_item_n<96>(phase, mb, local, smem, prm); break;
            case 128: run_item_n<128>(phase, mb, local, smem, prm); break;
            case 192: run_item_n<192>(phase, mb, local, smem, prm); break;
            default: break;
            }
            __syncthreads();   // the next item reuses the shared memory
        }
        if (phase + 1 < kBatchPhases && !grid_barrier(L, phase)) return;
    }
}

}  // namespace

bool batch_persist_n_ok(int n) { return n == 64 || n == 96 || n == 128 || n == 192; }

size_t batch_persist_smem() { return kBatchSmem; }

cudaError_t batch_persist_setup(int *blocks_out)
{
    cudaError_t e = cudaFuncSetAttribute(batch_persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kBatchSmem);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persist_kernel, kBT, kBatchSmem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) *blocks_out = per_sm * sms;
    return e;
}

cudaError_t launch_batch_persist(const BatchLaunch &L, int blocks, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = kBatchSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_persist_kernel, L);
}

}  // namespace spe
