// Strided passes: transforms along y or z, where consecutive points of a
// line are S complex values apart and neighbouring lines (columns) are
// adjacent in memory.
//
// One CTA owns a tile of T adjacent columns x N points (T = 32 for N < 256,
// 16 from 256 up; 8, 16 or 32 as the autotuner picks), so every row of the
// tile is one coalesced segment.  In spass_kernel the loads are asynchronous
// 16-byte copies straight into shared memory (every load of the tile in flight
// at once) and the stores are float4; spass_line_kernel (one transform alone,
// lengths 64-256) loads its first stage straight into registers and stores its
// last stage straight from them.  The tile lives in shared memory
// element-major (tile[n * T + t]) with lanes over t: the FFT stages are then
// bank-conflict free without padding.  Radix schedules: the default plan per
// length, and up to two alternatives (PL = 1, 2) the autotuner may pick.
//
// Flags select forward transform, a pointwise multiply in k space, and the
// inverse transform, all on the same tile; with a multiply, the last forward
// stage, the multiply and the first inverse stage run in registers:
//   drift   (S_FWD | S_DRIFT | S_INV on the z axis of psi):
//       psi_hat *= exp(-i eta k^2 dt / 2) / (nx ny nz) = D_xy(kx, ky) E_z(kz),
//       both factors built in FP64 on the host and applied as (hi + lo) float
//       pairs with compensated products, so that the per-mode factor carries
//       no fixed FP32 rounding that would repeat every step
//       [Sec. 3.1 step (b), Algorithm 1 "kinetic drift in Fourier space"];
//   Poisson (S_FWD | S_POISSON | S_INV on the z axis of the half spectrum):
//       rho_hat *= -4 pi G / (k^2 nx ny nz), zero at k = 0
//       [Sec. 3.1 step (c), Sec. 3.2.1: zero mode removed].
#pragma once
#include "fft_tile.cuh"
#include "reduce.cuh"
#include "spe_internal.cuh"
#include "tc16.cuh"
#include "tma.cuh"

namespace spe {

template <class L> struct MaxRadix;
template <int R> struct MaxRadix<RList<R>> { static constexpr int value = R; };
template <int R0, int R1, int... Rs> struct MaxRadix<RList<R0, R1, Rs...>> {
    static constexpr int rest = MaxRadix<RList<R1, Rs...>>::value;
    static constexpr int value = R0 > rest ? R0 : rest;
};

// Tile width (columns per CTA): 32 below N = 256 and 16 from there by default;
// the other width is the autotuner's alternative (SParams::tile).
template <int N> constexpr int default_tile() { return N >= 256 ? 16 : 32; }

template <int N, int TW, bool TC = false, int PL = 0> struct SCfg {
    static constexpr int T = TW;
    static constexpr int TP = T;
    static constexpr int W = N * T / MaxRadix<typename PlanSel<N, PL>::type>::value;  // butterflies per stage
    static constexpr int NT = W >= 512 ? 512 : (W >= 256 ? 256 : (W >= 128 ? 128 : 64));
    // + 128: the tile starts at the first 128-byte boundary of the dynamic area (TMA destination)
    static constexpr size_t base = sizeof(float2) * N * TP;
    static constexpr size_t tc_off = (base + 127) & ~(size_t)127;
    static constexpr size_t smem = (TC ? tc_off + sizeof(TcSmem) : base) + 128;
};

struct DriftOp {
    const float4 *colfac, *ez;
    __device__ __forceinline__ float2 operator()(float2 v, int n, int t) const
    {
        const float4 d = colfac[t];
        const float4 e = __ldg(&ez[n]);
        v = cmul_comp(v, make_float2(d.x, d.y), make_float2(d.z, d.w));
        return cmul_comp(v, make_float2(e.x, e.y), make_float2(e.z, e.w));
    }
};

struct PoissonOp {
    const float *colk2, *linek2;
    float scale;  // -4 pi G / (nx ny nz)
    __device__ __forceinline__ float2 operator()(float2 v, int n, int t) const
    {
        const float k2 = colk2[t] + __ldg(&linek2[n]);
        // k^2 lies between (2 pi / L)^2 and 3 (pi N / L)^2, far inside the range where the fast
        // division is within 2 ulp: a 2e-7 relative error on Phi_hat, well below its FP32 transforms'
        return cscale(v, (k2 > 0.f) ? __fdividef(scale, k2) : 0.f);
    }
};

// The body works on column tile cx of batch b with NT threads and SCfg<N, TW, TC, PL>::smem bytes of
// shared memory at smem_dyn (tm: the pass's tensor map when p.tma is set); the kernel below runs one
// tile per block, a persistent kernel any tile from any block.
template <int N, int TW, int NT, bool TC = false, int PL = 0, bool SINGLE = false>
__device__ __forceinline__ void spass_body(const SParams &p, const CUtensorMap *tm, int cx, int b,
                                           unsigned char *smem_dyn)
{
    constexpr int T = SCfg<N, TW, TC, PL>::T, TP = SCfg<N, TW, TC, PL>::TP, HT = T / 2;
    constexpr int BR = tma_box_rows(N), NB = N / BR;
    unsigned char *smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    TcSmem *tcs = nullptr;
    if constexpr (TC) {
        tcs = reinterpret_cast<TcSmem *>(smem_raw + SCfg<N, TW, TC>::tc_off);
        tc_setup(*tcs, static_cast<const __half *>(p.tcw), NT);
    }
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);
    __shared__ float4 colfac[T];
    __shared__ float colk2[T];
    __shared__ __align__(8) unsigned long long tma_bar;
    const int c0 = cx * T;
    const int tid = threadIdx.x;
    const int flags = p.flags;
    float2 *base = p.data + (size_t)b * p.bstride + c0;
    // the launcher clears p.tma when the tensor map could not be encoded for this shape
    const bool tma = !TC && p.tma;

    if (tma && tid == 0) {
        mbar_init(&tma_bar, 1);
        fence_mbar_init();
    }
    if (tid < T) {
        const int c = c0 + tid;
        if (flags & S_DRIFT)
            colfac[tid] = (c < p.W) ? __ldg(&p.dxy[(size_t)b * p.dxy_pitch + c]) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (flags & S_POISSON) colk2[tid] = (c < p.W) ? __ldg(&p.colk2[c]) + __ldg(&p.batchk2[b]) : 0.f;
    }

    if (tma) {
        __syncthreads();   // the mbarrier is initialised
        if (tid == 0) {
            mbar_expect_tx(&tma_bar, (uint32_t)(N * T * sizeof(float2)));
#pragma unroll
            for (int k = 0; k < NB; ++k) tma_load_3d(tile + k * BR * TP, tm, 2 * c0, k * BR, b, &tma_bar);
        }
        if (!mbar_wait(&tma_bar, 0) && (tid & 31) == 0) atomicOr(p.status, kTcStatusTimeout);
    } else {
        for (int idx = tid; idx < N * HT; idx += NT) {
            const int n = idx / HT, q = idx % HT;
            if (c0 + 2 * q < p.W) cp_async16(&tile[n * TP + 2 * q], base + (size_t)n * p.S + 2 * q);
            else *reinterpret_cast<float4 *>(&tile[n * TP + 2 * q]) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cp_async_wait_all();
    }
    __syncthreads();
    if (!SINGLE && (flags & (S_FWD | S_INV)) == (S_FWD | S_INV) && (flags & (S_DRIFT | S_POISSON))) {
        if constexpr (TC) {
            if (flags & S_DRIFT)
                tile_fft_fwd_op_inv_tc<N, T, TP, NT>(tile, p.tw, DriftOp{colfac, p.ez}, *tcs, p.status);
            else
                tile_fft_fwd_op_inv_tc<N, T, TP, NT>(tile, p.tw, PoissonOp{colk2, p.linek2, p.poisson * p.norm},
                                                     *tcs, p.status);
        } else if constexpr (!SINGLE) {
            if (flags & S_DRIFT) tile_fft_fwd_op_inv<N, T, TP, NT, DriftOp, PL>(tile, p.tw, DriftOp{colfac, p.ez});
            else
                // the potential's transforms take plain FP32 twiddle products (fft_tile.cuh)
                tile_fft_fwd_op_inv<N, T, TP, NT, PoissonOp, PL>(tile, PlainTw{p.tw},
                                                                 PoissonOp{colk2, p.linek2, p.poisson * p.norm});
        }
    } else if constexpr (TC) {
        if (flags & S_FWD) tile_fft_tc<N, T, TP, NT, -1>(tile, p.tw, *tcs, p.status);
        if (flags & S_INV) tile_fft_tc<N, T, TP, NT, +1>(tile, p.tw, *tcs, p.status);
    } else {
        if (flags & S_FWD) tile_fft<N, T, TP, NT, -1, PL>(tile, p.tw);
        if (flags & S_INV) tile_fft<N, T, TP, NT, +1, PL>(tile, p.tw);
    }

    if (flags & S_KIN) {
        double acc = 0.0;
        for (int idx = tid; idx < N * T; idx += NT) {
            const int n = idx / T, t = idx % T;
            if (c0 + t < p.W) {
                const float2 v = tile[n * TP + t];
                acc += (double)(__ldg(&p.linek2[n]) * (v.x * v.x + v.y * v.y));
            }
        }
        double r[1] = {acc};
        grid_reduce<1, NT>(r, 0, p.partials, p.counter, p.result);
        if constexpr (TC) tc_teardown(*tcs);
        return;
    }

    if (tma) {
        // every thread's tile writes are visible to the async proxy before one thread stores the boxes
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < NB; ++k) tma_store_3d(tm, 2 * c0, k * BR, b, tile + k * BR * TP);
            tma_store_commit_wait_read();
        }
    } else {
        for (int idx = tid; idx < N * HT; idx += NT) {
            const int n = idx / HT, q = idx % HT;
            if (c0 + 2 * q < p.W)
                *reinterpret_cast<float4 *>(base + (size_t)n * p.S + 2 * q) =
                    *reinterpret_cast<const float4 *>(&tile[n * TP + 2 * q]);
        }
    }
    if constexpr (TC) tc_teardown(*tcs);
}

template <int N, int TW, bool TC = false, int PL = 0>
__global__ void __launch_bounds__(SCfg<N, TW, TC, PL>::NT) spass_kernel(SParams p, const __grid_constant__ CUtensorMap tm)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    spass_body<N, TW, SCfg<N, TW, TC, PL>::NT, TC, PL>(p, &tm, blockIdx.x, blockIdx.y, smem_dyn);
}

// The fused passes (drift, Poisson) at 512 points with the [16, 32] plan and 8-column tiles, held to
// five CTAs of 128 threads per SM (96 registers, no spills) instead of four at 106.  A kernel of its
// own: a minimum-blocks bound of 1 on spass_kernel would lift the register cap of every other instance
// (the 16-column one then takes 216 registers).
template <int N, int TW, int PL> struct FusedMinBlocks {
    static constexpr int value = (N == 512 && PL == 2 && TW == 8) ? 5 : 1;
};

template <int N, int TW, int PL>
__global__ void __launch_bounds__(SCfg<N, TW, false, PL>::NT, FusedMinBlocks<N, TW, PL>::value)
    spass_fused_mb_kernel(SParams p, const __grid_constant__ CUtensorMap tm)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    spass_body<N, TW, SCfg<N, TW, false, PL>::NT, false, PL>(p, &tm, blockIdx.x, blockIdx.y, smem_dyn);
}

// One forward or inverse transform alone, where spass_line_kernel does not apply: the same body
// without the fused multiply, so that its register budget is its own.  At 512 points with the
// [16, 32] plan it holds three CTAs of 256 threads (16-column tiles) or six of 128 (8-column tiles)
// per SM at about 80 registers, instead of two or three at 106-133.
template <int N, int TW, int PL> struct SingleMinBlocks {
    static constexpr int value = (N == 512 && PL == 2) ? (TW == 16 ? 3 : (TW == 8 ? 6 : 1)) : 1;
};

template <int N, int TW, int PL>
__global__ void __launch_bounds__(SCfg<N, TW, false, PL>::NT, SingleMinBlocks<N, TW, PL>::value)
    spass_single_kernel(SParams p, const __grid_constant__ CUtensorMap tm)
{
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    spass_body<N, TW, SCfg<N, TW, false, PL>::NT, false, PL, true>(p, &tm, blockIdx.x, blockIdx.y, smem_dyn);
}

// One forward or inverse transform (S_FWD or S_INV alone) with FP32 stages, its first stage
// loading straight from global memory and its last storing straight back (tile_fft_direct): a
// kernel of its own, so that its register allocation is not the fused passes'.  Lengths whose
// plan has a single stage use spass_kernel.
template <int N, int TW, int PL> struct LineCfg {
    static constexpr int NT = SCfg<N, TW, false, PL>::NT;
    static constexpr int RMAX = MaxRadix<typename PlanSel<N, PL>::type>::value;
    // used where it fits 64 registers (four CTAs of 256 threads per SM): the power-of-two lengths
    // from 64 to 256, whose stages are radix 16 and smaller.  Elsewhere (radix-3 stages, 512 and
    // up) it needs 88-148 registers and ran slower than the staged kernel (512-point y passes
    // 415 -> 600 us), so those keep spass_kernel.
    static constexpr int MINB = 1024 / NT;
    static constexpr bool usable = RMAX <= 16 && N >= 64 && N <= 256 && (N & (N - 1)) == 0 &&
                                   Length<typename PlanSel<N, PL>::type>::value >= 2;
};

template <int N, int TW, int PL>
__global__ void __launch_bounds__(LineCfg<N, TW, PL>::NT, LineCfg<N, TW, PL>::MINB) spass_line_kernel(SParams p)
{
    constexpr int T = TW, NT = LineCfg<N, TW, PL>::NT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);
    float2 *base = p.data + (size_t)blockIdx.y * p.bstride + blockIdx.x * T;
    const int live = p.W - (int)blockIdx.x * T;
    const long long S = p.S;
    const auto ld = [base, live, S](int n, int t) {
        return t < live ? __ldcg(base + n * S + t) : make_float2(0.f, 0.f);
    };
    const auto st = [base, live, S](int n, int t, float2 v) {
        if (t < live) base[n * S + t] = v;
    };
    if (p.flags & S_FWD) tile_fft_direct<N, T, T, NT, -1, PL>(tile, p.tw, ld, st);
    else tile_fft_direct<N, T, T, NT, +1, PL>(tile, p.tw, ld, st);
}

// widths that fit in shared memory for length N
template <int N> constexpr bool tile_fits(int tw) { return (size_t)N * tw * sizeof(float2) <= 227 * 1024; }

template <int N, int TW, bool TC = false, int PL = 0>
static cudaError_t launch_s_nt(const SParams &p, cudaStream_t st, int *blocks_out)
{
    dim3 grid((p.W + TW - 1) / TW, p.batches);
    if (blocks_out) *blocks_out = grid.x * grid.y;
    if constexpr (!TC && LineCfg<N, TW, PL>::usable) {
        if (p.flags == S_FWD || p.flags == S_INV) {
            spass_line_kernel<N, TW, PL><<<grid, LineCfg<N, TW, PL>::NT, SCfg<N, TW, false, PL>::smem, st>>>(p);
            return cudaGetLastError();
        }
    }
    CUtensorMap tm;
    SParams q = p;
    if constexpr (TC) {
        q.tma = 0;
    } else {
        if (!encode_spass_tmap(p, N, TW, &tm)) q.tma = 0;
    }
    if (!q.tma) memset(&tm, 0, sizeof(tm));
    if constexpr (!TC && SingleMinBlocks<N, TW, PL>::value > 1) {
        if (p.flags == S_FWD || p.flags == S_INV) {
            spass_single_kernel<N, TW, PL><<<grid, SCfg<N, TW, false, PL>::NT, SCfg<N, TW, false, PL>::smem, st>>>(q, tm);
            return cudaGetLastError();
        }
    }
    if constexpr (!TC && FusedMinBlocks<N, TW, PL>::value > 1) {
        spass_fused_mb_kernel<N, TW, PL><<<grid, SCfg<N, TW, false, PL>::NT, SCfg<N, TW, false, PL>::smem, st>>>(q, tm);
        return cudaGetLastError();
    }
    spass_kernel<N, TW, TC, PL><<<grid, SCfg<N, TW, TC, PL>::NT, SCfg<N, TW, TC, PL>::smem, st>>>(q, tm);
    return cudaGetLastError();
}

template <int N, int TW, int PL>
static cudaError_t attr_s(int smem)
{
    cudaError_t e = cudaFuncSetAttribute(spass_kernel<N, TW, false, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if constexpr (LineCfg<N, TW, PL>::usable) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(spass_line_kernel<N, TW, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem);
    }
    if constexpr (SingleMinBlocks<N, TW, PL>::value > 1) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(spass_single_kernel<N, TW, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem);
    }
    if constexpr (FusedMinBlocks<N, TW, PL>::value > 1) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(spass_fused_mb_kernel<N, TW, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem);
    }
    return e;
}

}  // namespace spe

namespace spe {

// Launch / attribute set-up of width W at length n, for the per-width translation units; inside
// templates the discarded branches instantiate nothing.
template <int n, int W>
cudaError_t spass_launch_w(const SParams &p, cudaStream_t st, int *blocks_out)
{
    if constexpr (tile_fits<n>(W)) {
        if constexpr (has_plan2<n>()) {
            if (p.plan == 2) return launch_s_nt<n, W, false, 2>(p, st, blocks_out);
        }
        if constexpr (has_alt_plan<n>()) {
            if (p.plan == 1) return launch_s_nt<n, W, false, 1>(p, st, blocks_out);
        }
        return launch_s_nt<n, W>(p, st, blocks_out);
    } else {
        return cudaErrorInvalidValue;
    }
}

template <int n, int W>
cudaError_t spass_attr_w()
{
    cudaError_t e = cudaSuccess;
    if constexpr (tile_fits<n>(W)) {
        e = attr_s<n, W, 0>((int)SCfg<n, W>::smem);
        if constexpr (has_alt_plan<n>()) {
            if (e == cudaSuccess) e = attr_s<n, W, 1>((int)SCfg<n, W, false, 1>::smem);
        }
        if constexpr (has_plan2<n>()) {
            if (e == cudaSuccess) e = attr_s<n, W, 2>((int)SCfg<n, W, false, 2>::smem);
        }
    }
    return e;
}

}  // namespace spe
