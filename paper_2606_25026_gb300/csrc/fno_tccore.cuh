// tcgen05 helpers of the FNO surrogate's tensor-core kernels (fno_tc.cu forward, fno_tc_bwd.cu
// backward): BF16 kind::f16 MMAs with K-major no-swizzle operands in shared memory, FP32
// accumulators in TMEM, one mbarrier per CTA with a bounded wait.
#pragma once
#include "fno_rowcommon.cuh"
#include "tc16.cuh"

namespace spe {
namespace fno {
namespace {

constexpr int kTile = 4;                       // rows per tile
constexpr int kFnoTcStatus = 1 << 2;           // status bit of a timed-out wait

// kind::f16 instruction descriptor, BF16 A and B (K-major), FP32 D, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
}

// byte offset of (row, k) in a no-swizzle K-major operand with K columns
__device__ __forceinline__ int kmaj(int row, int k, int K)
{
    return (row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t desc_k(const void *p, int K)
{
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;
    d |= (uint64_t)(128 >> 4) << 16;                // next core matrix along K
    d |= (uint64_t)((K * 16) >> 4) << 32;           // next 8-row group
    d |= 1ull << 46;
    return d;
}

// 128-byte-swizzled K-major operand: atoms of 8 rows x 64 BF16 (1024 bytes, 1024-byte aligned),
// the 16-byte chunk c of row r stored at chunk c ^ (r & 7); rows are 128 bytes apart and the K range
// splits into atoms of 64, atom a of a [rows][K] operand at byte a * rows * 128.  A column of such an
// operand (one k, consecutive rows) spreads over all banks, unlike the no-swizzle core-matrix layout.
__device__ __forceinline__ int sw128(int row, int k, int rows)
{
    return (k >> 6) * rows * 128 + row * 128 + ((((k & 63) >> 3) ^ (row & 7)) << 4) + ((k & 7) << 1);
}

// descriptor of K step s (16 elements) of a 128-byte-swizzled K-major operand with `rows` rows
__device__ __forceinline__ uint64_t desc_sw128(const void *base, int s, int rows)
{
    const uint64_t addr = smem_u32(base) + (uint32_t)((s >> 2) * rows * 128 + (s & 3) * 32);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;
    d |= (uint64_t)1 << 16;                          // leading offset: unused within a swizzle atom
    d |= (uint64_t)(1024 >> 4) << 32;                // next 8-row group
    d |= 1ull << 46;
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// warp-wide: 16 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int W>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[W])
{
    if constexpr (W == 32) {
        tmem_ld32(taddr, v);
    } else {
        static_assert(W == 16, "16 or 32 columns");
        tmem_ld16(taddr, v);
    }
}

__device__ __forceinline__ unsigned short bf16_bits(float v)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    return (uint32_t)bf16_bits(lo) | ((uint32_t)bf16_bits(hi) << 16);
}

template <int COLS>
__device__ __forceinline__ void tmem_alloc_n(uint32_t *dst)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

template <int COLS>
__device__ __forceinline__ void tmem_free_n(uint32_t base)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(COLS) : "memory");
}

struct TcCtl {
    unsigned long long mbar;
    uint32_t tmem_base;
    uint32_t phase;
};

template <int COLS>
__device__ __forceinline__ void ctl_setup(TcCtl *ctl)
{
    if (threadIdx.x == 0) {
        mbar_init(&ctl->mbar, 1);
        ctl->phase = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) tmem_alloc_n<COLS>(&ctl->tmem_base);
}

// make the generic-proxy shared-memory writes visible to the tensor cores and
// order them before the MMA issue
__device__ __forceinline__ void to_tensor_cores()
{
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void wait_mma(TcCtl *ctl, int *status)
{
    if (!mbar_wait(&ctl->mbar, ctl->phase) && (threadIdx.x & 31) == 0 && status) atomicOr(status, kFnoTcStatus);
    tc_fence_after();
}

// all threads past their TMEM reads before the phase flips and the next MMA
__device__ __forceinline__ void end_phase(TcCtl *ctl)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) ctl->phase ^= 1u;
    __syncthreads();
}

}  // namespace
}  // namespace fno
}  // namespace spe
