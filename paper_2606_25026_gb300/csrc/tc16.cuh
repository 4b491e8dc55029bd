// Radix-16 DFT stages on the 5th-generation tensor cores (tcgen05), split FP16.
//
// One Stockham radix-16 stage over a tile (see fft_tile.cuh) is a real GEMM:
// every butterfly group g (16 complex points, twiddled) is a row of 32 reals
// [Re x_0..x_15, Im x_0..x_15]; the 16-point DFT is the 32 x 32 real matrix
//   W = [[C, -S], [S, C]],  C_qr = cos(DIR 2 pi q r / 16), S_qr = sin(...),
// and the stage computes D = A W^T for A = (groups x 32).  Groups go in
// blocks of M = 128 rows, N = 32, K = 32 (two K = 16 instructions).
//
// Split FP16 with FP32 accumulation: each row is scaled by a power of two
// 2^e (so its largest entry is near 2^14), split into a = hi + lo with
// hi = fp16(a), lo = fp16(a - hi); W likewise.  The accumulator collects
// A_hi W_hi + A_lo W_hi + A_hi W_lo (the lo x lo term, ~2^-22 relative, is
// dropped) in TMEM; rows are read back with tcgen05.ld and unscaled.
//
// Shared-memory operands use the no-swizzle K-major canonical layout: core
// matrices of 8 rows x 16 bytes stored contiguously (128 B); the next core
// matrix along K is 128 B on (leading byte offset), the next 8-row group is
// 4 x 128 B on (stride byte offset).  One elected thread issues the MMAs;
// completion arrives on an mbarrier whose wait is bounded: on timeout the
// kernel records an error bit in the status word and carries on (the result
// is then wrong and the host reports SPE_ETIMEOUT), so a fault in the
// tensor path can never hang the GPU.  TMEM is allocated once per CTA and
// freed before the kernel exits.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace spe {

constexpr int kTcRows = 128;                    // M per MMA block
constexpr int kTcMaxGroups = 512;               // groups per stage and CTA
constexpr int kTcCols = 128;                    // TMEM columns: 4 blocks x N = 32
constexpr unsigned kTcWaitLimit = 1u << 24;     // mbarrier polls before giving up
constexpr int kTcStatusTimeout = 1 << 1;

// Shared-memory context of the tensor stages of one CTA.
struct TcSmem {
    __half a_hi[kTcMaxGroups * 32];   // A operand, core-matrix layout
    __half a_lo[kTcMaxGroups * 32];
    __half w_hi[2][32 * 32];          // B operands (W rows, K-major), [0] forward, [1] inverse
    __half w_lo[2][32 * 32];
    float scale[kTcMaxGroups];        // 2^-e per row
    unsigned long long mbar;
    uint32_t tmem_base;
    uint32_t phase;
};

// byte offset of element (row, k) in a no-swizzle K-major operand of K = 32
__device__ __forceinline__ int tc_off(int row, int k)
{
    return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(const void *smem_start)
{
    const uint64_t addr = smem_u32(smem_start);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;            // start address
    d |= (uint64_t)(128 >> 4) << 16;         // leading byte offset: next core matrix along K
    d |= (uint64_t)(512 >> 4) << 32;         // stride byte offset: next 8-row group
    d |= 1ull << 46;                         // descriptor version for tcgen05
    return d;                                // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: F32 accumulate, F16 A and B, both K-major, N = 32, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kTcIdesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(unsigned long long *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// bounded wait for the given phase parity; returns false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned long long *mbar, uint32_t parity)
{
    const uint32_t a = smem_u32(mbar);
    for (unsigned it = 0; it < kTcWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// warp-wide: allocate / free kTcCols TMEM columns (address written to *dst)
__device__ __forceinline__ void tmem_alloc(uint32_t *dst)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t base)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(kTcCols) : "memory");
}

// warp-wide: 32 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace spe

#include "fft_tile.cuh"

namespace spe {

// Radix plans of the tensor-core mode: every radix-16 stage runs on tcgen05.
template <int N> struct PlanTc;
template <> struct PlanTc<256> { using type = RList<16, 16>; };
template <> struct PlanTc<512> { using type = RList<16, 16, 2>; };

// Per-CTA set-up: mbarrier, W operands into shared memory, TMEM allocation.
// w: [dir][hi / lo][32 x 32 in core-matrix layout], dir 0 = forward.
__device__ __forceinline__ void tc_setup(TcSmem &c, const __half *__restrict__ w, int nt)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(w);
    uint4 *dst_hi0 = reinterpret_cast<uint4 *>(c.w_hi[0]);
    uint4 *dst_lo0 = reinterpret_cast<uint4 *>(c.w_lo[0]);
    uint4 *dst_hi1 = reinterpret_cast<uint4 *>(c.w_hi[1]);
    uint4 *dst_lo1 = reinterpret_cast<uint4 *>(c.w_lo[1]);
    for (int i = threadIdx.x; i < 128; i += nt) {  // 1024 halves = 128 uint4 per matrix
        dst_hi0[i] = src[i];
        dst_lo0[i] = src[128 + i];
        dst_hi1[i] = src[256 + i];
        dst_lo1[i] = src[384 + i];
    }
    if (threadIdx.x == 0) {
        mbar_init(&c.mbar, 1);
        c.phase = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) tmem_alloc(&c.tmem_base);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void tc_teardown(TcSmem &c)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_free(c.tmem_base);
}

// One radix-16 Stockham stage (Ns as in fft_stage) on the tensor cores.
template <int N, int T, int TP, int NT, int DIR, int Ns>
__device__ __forceinline__ void fft_stage_tc16(float2 *s, const float4 *__restrict__ tw, TcSmem &c, int *status)
{
    constexpr int R = 16, B = N / R, G = B * T, NBLK = G / kTcRows;
    static_assert(G % kTcRows == 0 && G <= kTcMaxGroups, "tensor stage needs 128-row blocks");
    static_assert(NT % 128 == 0, "tensor stage needs whole warp quarters");
    char *ah = reinterpret_cast<char *>(c.a_hi);
    char *al = reinterpret_cast<char *>(c.a_lo);
    for (int g = threadIdx.x; g < G; g += NT) {
        const int t = g % T, j = g / T, k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[(j + r * B) * TP + t];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float4 w = __ldg(&tw[k * r * (N / (Ns * R))]);
                v[r] = cmul_comp(v[r], make_float2(w.x, DIR > 0 ? -w.y : w.y), make_float2(w.z, DIR > 0 ? -w.w : w.w));
            }
        }
        float m = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) m = fmaxf(m, fmaxf(fabsf(v[r].x), fabsf(v[r].y)));
        int e = 0;
        if (m > 0.f) frexpf(m, &e);
        const float sc = ldexpf(1.f, 14 - e);
        c.scale[g] = ldexpf(1.f, e - 14);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float re = v[r].x * sc, im = v[r].y * sc;
            const __half hr = __float2half_rn(re), hi = __float2half_rn(im);
            *reinterpret_cast<__half *>(ah + tc_off(g, r)) = hr;
            *reinterpret_cast<__half *>(ah + tc_off(g, 16 + r)) = hi;
            *reinterpret_cast<__half *>(al + tc_off(g, r)) = __float2half_rn(re - __half2float(hr));
            *reinterpret_cast<__half *>(al + tc_off(g, 16 + r)) = __float2half_rn(im - __half2float(hi));
        }
    }
    fence_async_smem();
    __syncthreads();
    const int d = DIR < 0 ? 0 : 1;
    if (threadIdx.x == 0) {
        tc_fence_after();
#pragma unroll
        for (int blk = 0; blk < NBLK; ++blk) {
            const uint32_t dt = c.tmem_base + blk * 32;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const uint64_t a_hi = tc_desc(ah + blk * 8192 + kk * 256);
                const uint64_t a_lo = tc_desc(al + blk * 8192 + kk * 256);
                const uint64_t b_hi = tc_desc(reinterpret_cast<char *>(c.w_hi[d]) + kk * 256);
                const uint64_t b_lo = tc_desc(reinterpret_cast<char *>(c.w_lo[d]) + kk * 256);
                tc_mma(dt, a_hi, b_hi, kk);
                tc_mma(dt, a_lo, b_hi, 1);
                tc_mma(dt, a_hi, b_lo, 1);
            }
        }
        tc_commit(&c.mbar);
    }
    if (!mbar_wait(&c.mbar, c.phase) && (threadIdx.x & 31) == 0) atomicOr(status, kTcStatusTimeout);
    tc_fence_after();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quarter = warp & 3;
    for (int blk = warp >> 2; blk < NBLK; blk += NT / 128) {
        float y[32];
        tmem_ld32(c.tmem_base + ((uint32_t)(quarter * 32) << 16) + blk * 32, y);
        const int g = blk * kTcRows + quarter * 32 + lane;
        const int t = g % T, j = g / T, k = j % Ns;
        const float us = c.scale[g];
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) s[(base + q * Ns) * TP + t] = make_float2(y[q] * us, y[16 + q] * us);
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) c.phase ^= 1u;
}

template <int N, int T, int TP, int NT, int DIR, int Ns>
__device__ __forceinline__ void fft_stages_tc(float2 *, const float4 *, TcSmem &, int *, RList<>) {}

template <int N, int T, int TP, int NT, int DIR, int Ns, int R, int... Rest>
__device__ __forceinline__ void fft_stages_tc(float2 *s, const float4 *tw, TcSmem &c, int *status, RList<R, Rest...>)
{
    if constexpr (R == 16) fft_stage_tc16<N, T, TP, NT, DIR, Ns>(s, tw, c, status);
    else fft_stage<N, T, TP, NT, DIR, Ns, R>(s, tw);
    fft_stages_tc<N, T, TP, NT, DIR, Ns * R>(s, tw, c, status, RList<Rest...>{});
}

template <int N, int T, int TP, int NT, int DIR>
__device__ __forceinline__ void tile_fft_tc(float2 *s, const float4 *tw, TcSmem &c, int *status)
{
    fft_stages_tc<N, T, TP, NT, DIR, 1>(s, tw, c, status, typename PlanTc<N>::type{});
}

// tile_fft_fwd_op_inv with the tensor-core plan (the fused middle stage stays in registers)
template <int N, int T, int TP, int NT, class Op>
__device__ __forceinline__ void tile_fft_fwd_op_inv_tc(float2 *s, const float4 *tw, const Op &op, TcSmem &c,
                                                        int *status)
{
    using Full = typename PlanTc<N>::type;
    constexpr int R = SplitLast<Full>::last;
    using Init = typename SplitLast<Full>::init;
    constexpr int B = N / R;
    fft_stages_tc<N, T, TP, NT, -1, 1>(s, tw, c, status, Init{});
    constexpr int TOTAL = B * T;
    constexpr int PER = (TOTAL + NT - 1) / NT;
    float2 v[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int t = idx % T, j = idx / T;
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = s[(j + r * B) * TP + t];
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int t = idx % T, j = idx / T;
            if (B > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float4 w = __ldg(&tw[j * r]);
                    v[p][r] = cmul_comp(v[p][r], make_float2(w.x, w.y), make_float2(w.z, w.w));
                }
            }
            Dft<R, -1>::run(v[p]);
#pragma unroll
            for (int q = 0; q < R; ++q) v[p][q] = op(v[p][q], j + q * B, t);
            Dft<R, +1>::run(v[p]);
#pragma unroll
            for (int q = 0; q < R; ++q) s[(j * R + q) * TP + t] = v[p][q];
        }
    }
    __syncthreads();
    fft_stages_tc<N, T, TP, NT, +1, R>(s, tw, c, status, typename Reverse<Init>::type{});
}

}  // namespace spe
