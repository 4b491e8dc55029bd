// Tensor-core (tcgen05, BF16 operands, FP32 accumulation in TMEM) forward
// kernels of the FNO surrogate, used when activations are stored in BF16.
//
// Layer row kernel: a tile of 4 rows, TMEM lane m = (r, c) = r * 32 + c
// (row r of the tile, channel c), columns over x.  Per tile, three GEMMs
// (M = 128, all operands K-major, no-swizzle core-matrix layout):
//   G1  D[(r,c)][x]  = sum_(r',j) blockdiag(W)[(r,c)][(r',j)] V[r'][x][j]
//                      (K = 128; the off-diagonal blocks are zeros)
//   G2  D[(r,c)][x] += sum_kk  B'[r][kk][c] G'[x][kk]      (K = 2M)
//       with B' = (Re, Im) of the inverse-y output and G' = (Re Gx, -Im Gx),
//       so G2 is the real x inverse of the spectral path;
//   epilogue: u = D + b, v' = GELU(u) (stored), v' also into the A operand of
//   G3  E[(r,c)][kk] = sum_x V'[r][x][c] F'[kk][x]           (K = n)
//       with F' = (Re Fx, Im Fx): the next layer's x DFT (complex pairs).
// The last layer stops after G1 + G2 and stores v_L = u; the projection runs
// in its own kernel with TMEM lane = cell: H[cell][j] = sum_c V_L[cell][c]
// Q1[j][c] (M = 128 cells, N = 64, K = 32), then GELU and Q2 per thread.
//
// One thread issues the MMAs; completion arrives on an mbarrier with a
// bounded wait (on timeout a status bit is set and the kernel carries on, so
// the result is wrong but the GPU never hangs).  TMEM is allocated once per
// CTA and freed before exit.
#include "fno_tccore.cuh"

namespace spe {
namespace fno {
namespace {

// Shared-memory layout of the layer kernel (bytes), n = N, KM = 2M.
template <int N, int M>
struct LayerSmem {
    static constexpr int KM = 2 * M;
    static constexpr int A1 = 0;                              // [128][128]
    static constexpr int B1 = A1 + 128 * 128 * 2;             // [N][128]
    static constexpr int A2 = B1 + N * 128 * 2;               // [128][KM]
    static constexpr int B2 = A2 + 128 * KM * 2;              // [N][KM]
    // A3 shares B1's bytes: B1 is last read by G1, A3 first written after G1 completes, and the
    // next tile stages B1 only after G3 (which reads A3) has completed
    static constexpr int A3 = B1;                             // [128][N] <= [N][128]
    static constexpr int B3 = B2 + N * KM * 2;                // [KM][N]
    static constexpr int CTL = B3 + KM * N * 2;               // mbarrier, tmem base, phase
    static constexpr int BYTES = CTL + 64;
};


enum { kModeLayer = 0, kModeLast = 1, kModeLift = 2 };

template <int N, int M, int MODE>
__global__ void __launch_bounds__(kRowThreads) layer_fwd_tc_kernel(RowArgs a)
{
    constexpr bool LAST = MODE == kModeLast, LIFT = MODE == kModeLift;
    using S = LayerSmem<N, M>;
    constexpr int KM = S::KM;
    extern __shared__ __align__(1024) unsigned char sm[];
    TcCtl *ctl = reinterpret_cast<TcCtl *>(sm + S::CTL);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- per-CTA constants: blockdiag(W) (zero off the diagonal), G', F' (prebuilt images)
    if (!LIFT) {
        for (int e = tid; e < 128 * 128 * 2 / 16; e += kRowThreads)
            reinterpret_cast<uint4 *>(sm + S::A1)[e] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        for (int e = tid; e < kTile * kC * 4; e += kRowThreads) {
            const int r = e / (kC * 4), c = (e / 4) % kC, q = e % 4;
            *reinterpret_cast<uint4 *>(sm + S::A1 + kmaj(r * 32 + c, r * 32 + q * 8, 128)) =
                *reinterpret_cast<const uint4 *>(a.w + a.oW + c * kC + q * 8);
        }
    }
    for (int e = tid; e < N * KM * 2 / 16; e += kRowThreads) {
        reinterpret_cast<uint4 *>(sm + S::B2)[e] = a.tcG[e];
        if (!LAST) reinterpret_cast<uint4 *>(sm + S::B3)[e] = a.tcF[e];
    }
    ctl_setup<128>(ctl);
    const float bc = LIFT ? wload(a.w, a.op + lane) : wload(a.w, a.ob + lane);
    float Pr[kFin];
#pragma unroll
    for (int f = 0; f < kFin; ++f) Pr[f] = LIFT ? wload(a.w, a.oP + lane * kFin + f) : 0.f;
    float *fs = reinterpret_cast<float *>(sm + S::A1);   // lift: features [kTile][N][4] (A1 unused)
    to_tensor_cores();
    const uint32_t tbase = ctl->tmem_base;

    const __nv_bfloat16 *vin = (const __nv_bfloat16 *)a.vin;
    __nv_bfloat16 *vout = (__nv_bfloat16 *)a.vout;
    __nv_bfloat16 *uout = (__nv_bfloat16 *)a.uout;
    const int tiles = a.rows / kTile;
    const int r_ep = warp & 3, half = warp >> 2;      // epilogue: tile row, column half

    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int row0 = t * kTile;
        if (LIFT) {
            for (int e = tid; e < kTile * N; e += kRowThreads) {
                const size_t c = (size_t)row0 * N + e;
                const float2 u = a.psi[c], q = a.psib[c];
                fs[e * 4 + 0] = u.x * a.inv_A;
                fs[e * 4 + 1] = u.y * a.inv_A;
                fs[e * 4 + 2] = q.x * a.inv_A;
                fs[e * 4 + 3] = q.y * a.inv_A;
            }
            __syncthreads();
        }
        // ---- stage V (B1) and B' (A2): every load of the tile in flight before the stores
        if (!LIFT) {
            constexpr int NV = kTile * N * 4 / kRowThreads, NB = kTile * M * kC / kRowThreads;
            static_assert(NV * kRowThreads == kTile * N * 4 && NB * kRowThreads == kTile * M * kC,
                          "staging loops divide evenly");
            uint4 vv[NV];
            float2 bb[NB];
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const int e = tid + i * kRowThreads, r = e / (N * 4), x = (e / 4) % N, q = e % 4;
                vv[i] = *reinterpret_cast<const uint4 *>(vin + ((size_t)(row0 + r) * N + x) * kC + q * 8);
            }
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const int e = tid + i * kRowThreads, r = e / (M * kC), kx = (e / kC) % M, c = e % kC;
                bb[i] = a.xrow[((size_t)(row0 + r) * M + kx) * kC + c];
            }
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const int e = tid + i * kRowThreads, r = e / (N * 4), x = (e / 4) % N, q = e % 4;
                *reinterpret_cast<uint4 *>(sm + S::B1 + kmaj(x, r * 32 + q * 8, 128)) = vv[i];
            }
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const int e = tid + i * kRowThreads, r = e / (M * kC), kx = (e / kC) % M, c = e % kC;
                *reinterpret_cast<uint32_t *>(sm + S::A2 + kmaj(r * 32 + c, 2 * kx, KM)) = pack_bf16(bb[i].x, bb[i].y);
            }
        }
        if (!LIFT) {
            to_tensor_cores();
            if (tid == 0) {
                constexpr uint32_t id1 = idesc_bf16(N);
#pragma unroll
                for (int s = 0; s < 128 / 16; ++s)
                    mma_bf16(tbase, desc_k(sm + S::A1 + s * 256, 128), desc_k(sm + S::B1 + s * 256, 128), id1,
                             s > 0);
#pragma unroll
                for (int s = 0; s < KM / 16; ++s)
                    mma_bf16(tbase, desc_k(sm + S::A2 + s * 256, KM), desc_k(sm + S::B2 + s * 256, KM), id1, 1);
                tc_commit(&ctl->mbar);
            }
            wait_mma(ctl, a.status);
        }
        {
            constexpr int HW = N / 2;                 // columns per warp
            float d[HW];
            const int row = row0 + r_ep;
            if (LIFT) {
#pragma unroll
                for (int i = 0; i < HW; ++i) {
                    const float *f = fs + (r_ep * N + half * HW + i) * 4;
                    d[i] = Pr[0] * f[0] + Pr[1] * f[1] + Pr[2] * f[2] + Pr[3] * f[3];
                }
            } else {
                tmem_ld<HW>(tbase + ((uint32_t)(r_ep * 32) << 16) + half * HW, d);
            }
#pragma unroll
            for (int i = 0; i < HW; i += 8) {
                uint32_t pk[4];
#pragma unroll
                for (int k = 0; k < 8; k += 2) {
                    float v0, v1;
                    const int x0 = half * HW + i + k;
                    const float u0 = d[i + k] + bc, u1 = d[i + k + 1] + bc;
                    const size_t e0 = ((size_t)row * N + x0) * kC + lane;
                    if (LAST || LIFT) {
                        v0 = u0;
                        v1 = u1;
                    } else {
                        if (a.store_u) {
                            uout[e0] = __float2bfloat16_rn(u0);
                            uout[e0 + kC] = __float2bfloat16_rn(u1);
                        }
                        v0 = gelu(u0);
                        v1 = gelu(u1);
                    }
                    vout[e0] = __float2bfloat16_rn(v0);
                    vout[e0 + kC] = __float2bfloat16_rn(v1);
                    pk[k / 2] = pack_bf16(v0, v1);
                }
                if (!LAST)
                    *reinterpret_cast<uint4 *>(sm + S::A3 + kmaj(r_ep * 32 + lane, half * HW + i, N)) =
                        make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        if (!LIFT) end_phase(ctl);
        if (!LAST) {
            to_tensor_cores();
            if (tid == 0) {
                constexpr uint32_t id3 = idesc_bf16(KM);
#pragma unroll
                for (int s = 0; s < N / 16; ++s)
                    mma_bf16(tbase + N, desc_k(sm + S::A3 + s * 256, N), desc_k(sm + S::B3 + s * 256, N), id3,
                             s > 0);
                tc_commit(&ctl->mbar);
            }
            wait_mma(ctl, a.status);
            {
                constexpr int HW = KM / 2;           // 8 or 16 columns per warp
                // KM = 16: both halves read the same 16 columns and half 1 stores nothing
                float d[16];
                tmem_ld16(tbase + ((uint32_t)(r_ep * 32) << 16) + N + (HW == 16 ? half * 16 : 0), d);
                if (HW == 16 || half == 0) {
                    const int row = row0 + r_ep;
                    const int kx0 = (HW == 16) ? half * 8 : 0;
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        a.xrow[((size_t)row * M + kx0 + k) * kC + lane] = make_float2(d[2 * k], d[2 * k + 1]);
                }
            }
            end_phase(ctl);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free_n<128>(tbase);
}

// Projection: H[cell][j] = sum_c V_L[cell][c] Q1[j][c] on the tensor cores
// (TMEM lane = cell), then psi_pred = psi_b + sigma (Q2 GELU(H + q1) + q2).
struct ProjSmem {
    static constexpr int A = 0;                   // [128 cells][32]
    static constexpr int B = A + 128 * 32 * 2;    // [64][32]
    static constexpr int PART = B + 64 * 32 * 2;  // [128][2] partial outputs of columns 32..63
    static constexpr int PAR = PART + 128 * 2 * 4;// q1 [64], Q2 [2][64], q2 [2]
    static constexpr int CTL = PAR + (64 + 128 + 2) * 4 + 8;
    static constexpr int BYTES = CTL + 64;   // at most 8 CTAs of 256 threads per SM: 8 x 64 TMEM columns
};

__global__ void __launch_bounds__(kRowThreads) proj_tc_kernel(RowArgs a, int cells)
{
    using S = ProjSmem;
    extern __shared__ __align__(1024) unsigned char sm[];
    TcCtl *ctl = reinterpret_cast<TcCtl *>(sm + S::CTL);
    float *part = reinterpret_cast<float *>(sm + S::PART);
    float *q1 = reinterpret_cast<float *>(sm + S::PAR);
    float *q2w = q1 + 64;
    float *q2b = q2w + 128;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < kH * 4; e += kRowThreads) {
        const int j = e / 4, q = e % 4;
        *reinterpret_cast<uint4 *>(sm + S::B + kmaj(j, q * 8, 32)) =
            *reinterpret_cast<const uint4 *>(a.w + a.oQ1 + j * kC + q * 8);
    }
    for (int e = tid; e < kH; e += kRowThreads) q1[e] = wload(a.w, a.oq1 + e);
    for (int e = tid; e < 2 * kH; e += kRowThreads) q2w[e] = wload(a.w, a.oQ2 + e);
    if (tid < 2) q2b[tid] = wload(a.w, a.oq2 + tid);
    ctl_setup<64>(ctl);
    to_tensor_cores();
    const uint32_t tbase = ctl->tmem_base;
    const __nv_bfloat16 *vin = (const __nv_bfloat16 *)a.vin;
    const int tiles = cells / 128;
    const int quarter = warp & 3, half = warp >> 2;

    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const size_t cell0 = (size_t)t * 128;
        for (int e = tid; e < 128 * 4; e += kRowThreads) {
            const int m = e / 4, q = e % 4;
            *reinterpret_cast<uint4 *>(sm + S::A + kmaj(m, q * 8, 32)) =
                *reinterpret_cast<const uint4 *>(vin + (cell0 + m) * kC + q * 8);
        }
        to_tensor_cores();
        if (tid == 0) {
            constexpr uint32_t id = idesc_bf16(64);
#pragma unroll
            for (int s = 0; s < 2; ++s)
                mma_bf16(tbase, desc_k(sm + S::A + s * 256, 32), desc_k(sm + S::B + s * 256, 32), id, s > 0);
            tc_commit(&ctl->mbar);
        }
        wait_mma(ctl, a.status);
        float h[32];
        tmem_ld32(tbase + ((uint32_t)(quarter * 32) << 16) + half * 32, h);
        float o0 = 0.f, o1 = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int j = half * 32 + i;
            const float g = gelu(h[i] + q1[j]);
            o0 = fmaf(q2w[j], g, o0);
            o1 = fmaf(q2w[kH + j], g, o1);
        }
        const int m = quarter * 32 + lane;
        if (half == 1) {
            part[2 * m] = o0;
            part[2 * m + 1] = o1;
        }
        end_phase(ctl);
        if (half == 0) {
            o0 += part[2 * m] + q2b[0];
            o1 += part[2 * m + 1] + q2b[1];
            const size_t cell = cell0 + m;
            const float2 pb = a.psib[cell];
            a.out[cell] = make_float2(pb.x + a.sigma * o0, pb.y + a.sigma * o1);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free_n<64>(tbase);
}

template <int N, int M, int MODE>
cudaError_t layer_tc_run(const RowArgs &a, int grid, cudaStream_t st)
{
    constexpr int bytes = LayerSmem<N, M>::BYTES;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(layer_fwd_tc_kernel<N, M, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    layer_fwd_tc_kernel<N, M, MODE><<<grid, kRowThreads, bytes, st>>>(a);
    return cudaGetLastError();
}

template <int N, int M>
cudaError_t layer_tc_mode(int mode, const RowArgs &a, int grid, cudaStream_t st)
{
    if (mode == kModeLift) return layer_tc_run<N, M, kModeLift>(a, grid, st);
    if (mode == kModeLast) return layer_tc_run<N, M, kModeLast>(a, grid, st);
    return layer_tc_run<N, M, kModeLayer>(a, grid, st);
}

}  // namespace

cudaError_t launch_layer_fwd_tc(int n, int M, int mode, const RowArgs &a, int grid, cudaStream_t st)
{
    if (a.rows % kTile) return cudaErrorInvalidValue;
#define SPE_FNO_TC_CASE(NN, MM) \
    if (n == NN && M == MM) return layer_tc_mode<NN, MM>(mode, a, grid, st);
    SPE_FNO_TC_CASE(64, 16)
    SPE_FNO_TC_CASE(64, 8)
    SPE_FNO_TC_CASE(32, 16)
    SPE_FNO_TC_CASE(32, 8)
#undef SPE_FNO_TC_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_proj_tc(const RowArgs &a, int cells, int grid, cudaStream_t st)
{
    if (cells % 128) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(proj_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             ProjSmem::BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    proj_tc_kernel<<<grid, kRowThreads, ProjSmem::BYTES, st>>>(a, cells);
    return cudaGetLastError();
}


}  // namespace fno
}  // namespace spe
