// Tensor-core (tcgen05, BF16 operands, FP32 accumulation in TMEM) backward row kernels of the FNO
// surrogate, used when activations are stored in BF16 (the FP32-activation network keeps the
// CUDA-core kernels of fno_bwd.cu, whose gradients match the FP64 reference to 1e-4).
//
// Cotangents as in fno_bwd.cu: for a Fourier layer u_l = W_l v_{l-1} + b_l + Re(Fx-inverse of the
// spectral path), v bar = W^T u bar + Re(Fx^H a bar) and the spectral path's x-stage cotangent is
// Bbar = Gx^H u bar.  A tile is 4 rows; TMEM lane m = (r, c) = r * 32 + c (row r of the tile,
// channel c), as in the forward kernels.  Per tile (all operands K-major, no swizzle):
//   G1  D[(r,c)][x]   = sum_(r',j) blockdiag(W^T)[(r,c)][(r',j)] Ubar[r'][x][j]       (K = 128)
//   G2  D[(r,c)][x]  += sum_kk Abar'[r][kk][c] F''[x][kk]                             (K = 2M)
//       with Abar' = (Re, Im) of the row's x-stage cotangent and F''[x] = (Re Fx, Im Fx)[kk],
//       so D = v bar of the row;
//   epilogue: u bar_{l-1} = D GELU'(u_{l-1}) (stored in FP32, and in BF16 into the A operand of)
//   G3  E[(r,c)][kk]  = sum_x Ubar'[r][x][c] G''[kk][x]                               (K = n)
//       with G'' = (Re Gx, -Im Gx): the previous layer's x-stage cotangent Gx^H u bar;
//   G4  S[(r,c)][(r',j)] += sum_x Ubar'[r][x][c] V[r'][x][j]                          (K = n)
//       accumulated in TMEM over all tiles of the CTA; the blocks r = r' summed over r are the
//       CTA's partial dL/dW (the off-diagonal blocks are computed and ignored).
// Modes: layer (G1-G4), start (u bar of the last layer given: G3, G4), lift (G1, G2, then dL/dP
// and dL/dp from the four input features on the CUDA cores).  Every CTA writes one partial segment
// (W [C][C] | b [C], or P [C][4] | p [C]) in a fixed order, so the fixed-order reduction of the
// partials is deterministic.
//
// One thread issues the MMAs; completion arrives on an mbarrier with a bounded wait (on timeout a
// status bit is set and the kernel carries on).  TMEM (256 columns) is allocated once per CTA and
// freed before exit.
#include "fno_tccore.cuh"

namespace spe {
namespace fno {
namespace {

constexpr int kBwdLayer = kTcBwdLayer, kBwdStart = kTcBwdStart, kBwdLift = kTcBwdLift;

constexpr int kColE = 64;    // TMEM column of E (D takes columns 0 .. n - 1)
constexpr int kColS = 128;   // TMEM column of S (128 columns)

template <int N, int M>
struct BwdSmem {
    static constexpr int KM = 2 * M;
    static constexpr int A1 = 0;                       // blockdiag(W^T) [128][128]
    static constexpr int B1 = A1 + 128 * 128 * 2;      // Ubar [N][128]
    static constexpr int A2 = B1 + N * 128 * 2;        // Abar' [128][KM]
    static constexpr int B2 = A2 + 128 * KM * 2;       // F'' [N][KM]
    static constexpr int A3 = B2 + N * KM * 2;         // Ubar' [128][N]
    static constexpr int B3 = A3 + 128 * N * 2;        // G'' [KM][N]
    static constexpr int B4 = B3 + KM * N * 2;         // V as [(r',j)][x]: [128][N]
    static constexpr int FS = B4;                      // lift: features [kTile][N][4] floats
    static constexpr int CTL = B4 + 128 * N * 2;
    static constexpr int BYTES = CTL + 64;
    // after the tile loop A1 .. B1 hold the reduction scratch
    static_assert(4 * 32 * 32 * 4 + kRowWarps * 32 * 5 * 4 <= B2, "reduction scratch");
    static_assert(kTile * N * 4 * 4 <= 128 * N * 2, "lift features");
};

// 8 floats as 8 BF16 in one 16-byte word
__device__ __forceinline__ uint4 pack8(const float4 &a, const float4 &b)
{
    return make_uint4(pack_bf16(a.x, a.y), pack_bf16(a.z, a.w), pack_bf16(b.x, b.y), pack_bf16(b.z, b.w));
}

template <int N, int M, int MODE>
__global__ void __launch_bounds__(kRowThreads, 2) layer_bwd_tc_kernel(RowArgs a)
{
    constexpr bool START = MODE == kBwdStart, LIFT = MODE == kBwdLift;
    using S = BwdSmem<N, M>;
    constexpr int KM = S::KM;
    constexpr int HW = N / 2;                          // epilogue columns per warp
    extern __shared__ __align__(1024) unsigned char sm[];
    TcCtl *ctl = reinterpret_cast<TcCtl *>(sm + S::CTL);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r_ep = warp & 3, half = warp >> 2;       // epilogue: tile row (TMEM quadrant), column half

    // ---- per-CTA constants: blockdiag(W^T) (zero off the diagonal), F'', G''
    if (!START) {
        for (int e = tid; e < 128 * 128 * 2 / 16; e += kRowThreads)
            reinterpret_cast<uint4 *>(sm + S::A1)[e] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        for (int e = tid; e < kTile * kC * 4; e += kRowThreads) {
            const int r = e / (kC * 4), c = (e / 4) % kC, q = e % 4;
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const unsigned short lo = __bfloat16_as_ushort(a.w[a.oW + (size_t)(q * 8 + 2 * i) * kC + c]);
                const unsigned short hi = __bfloat16_as_ushort(a.w[a.oW + (size_t)(q * 8 + 2 * i + 1) * kC + c]);
                w[i] = (uint32_t)lo | ((uint32_t)hi << 16);
            }
            *reinterpret_cast<uint4 *>(sm + S::A1 + kmaj(r * 32 + c, r * 32 + q * 8, 128)) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
        for (int e = tid; e < N * KM * 2 / 16; e += kRowThreads)
            reinterpret_cast<uint4 *>(sm + S::B2)[e] = a.tcFt[e];
    }
    if (!LIFT)
        for (int e = tid; e < N * KM * 2 / 16; e += kRowThreads) reinterpret_cast<uint4 *>(sm + S::B3)[e] = a.tcGt[e];
    ctl_setup<256>(ctl);
    float Pr[kFin];                                    // lift: this lane's dL/dP row partial
    float gacc = 0.f;                                  // dL/db or dL/dp partial of channel `lane`
#pragma unroll
    for (int f = 0; f < kFin; ++f) Pr[f] = 0.f;
    float *fs = reinterpret_cast<float *>(sm + S::FS);
    to_tensor_cores();
    const uint32_t tbase = ctl->tmem_base;

    const __nv_bfloat16 *vin = (const __nv_bfloat16 *)a.vin;
    const __nv_bfloat16 *upre = (const __nv_bfloat16 *)a.upre;
    const int tiles = a.rows / kTile;
    int done = 0;

    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++done) {
        const int row0 = t * kTile;
        const int row = row0 + r_ep;
        // the tile's global loads first, all in flight together, then their conversions and stores
        constexpr int NB1 = kTile * N * 4 / kRowThreads, NA2 = kTile * M * kC / kRowThreads;
        constexpr int NB4 = kTile * (N / 16) / kRowWarps;
        static_assert(NB1 * kRowThreads == kTile * N * 4 && NA2 * kRowThreads == kTile * M * kC &&
                          NB4 * kRowWarps == kTile * (N / 16),
                      "staging loops divide evenly");
        float4 ub[START ? 1 : NB1][2];
        float2 ab[START ? 1 : NA2];
        uint4 vv[LIFT ? 1 : NB4][2];
        if (!START) {
#pragma unroll
            for (int i = 0; i < NB1; ++i) {
                const int e = tid + i * kRowThreads, r = e / (N * 4), x = (e / 4) % N, q = e % 4;
                const float4 *u = reinterpret_cast<const float4 *>(a.ubar + ((size_t)(row0 + r) * N + x) * kC + q * 8);
                ub[i][0] = u[0];
                ub[i][1] = u[1];
            }
#pragma unroll
            for (int i = 0; i < NA2; ++i) {
                const int e = tid + i * kRowThreads, r = e / (M * kC), kx = (e / kC) % M, c = e % kC;
                ab[i] = a.xrow[((size_t)(row0 + r) * M + kx) * kC + c];
            }
        }
        // V as [(r',j)][x]: each lane takes two neighbouring x of 8 channels and stores the eight
        // (x, x + 1) pairs of BF16 as 32-bit words
        const int vp = lane & 3, vq = lane >> 2;
        if (!LIFT) {
#pragma unroll
            for (int i = 0; i < NB4; ++i) {
                const int it = warp + i * kRowWarps, rr = it / (N / 16), xb = (it % (N / 16)) * 16;
                const int x = xb + (vq & 1) * 8 + 2 * vp, j0 = (vq >> 1) * 8;
                const __nv_bfloat16 *src = vin + ((size_t)(row0 + rr) * N + x) * kC + j0;
                vv[i][0] = *reinterpret_cast<const uint4 *>(src);
                vv[i][1] = *reinterpret_cast<const uint4 *>(src + kC);
            }
        }
        // layer: the pre-activations the epilogue needs (this lane's channel, this warp's columns)
        unsigned short up[LIFT || START ? 1 : HW];
        if (!LIFT && !START) {
            const unsigned short *ur = reinterpret_cast<const unsigned short *>(upre) + ((size_t)row * N + half * HW) * kC + lane;
#pragma unroll
            for (int i = 0; i < HW; ++i) up[i] = ur[(size_t)i * kC];
        }
        if (!START) {
#pragma unroll
            for (int i = 0; i < NB1; ++i) {
                const int e = tid + i * kRowThreads, r = e / (N * 4), x = (e / 4) % N, q = e % 4;
                *reinterpret_cast<uint4 *>(sm + S::B1 + kmaj(x, r * 32 + q * 8, 128)) = pack8(ub[i][0], ub[i][1]);
            }
#pragma unroll
            for (int i = 0; i < NA2; ++i) {
                const int e = tid + i * kRowThreads, r = e / (M * kC), kx = (e / kC) % M, c = e % kC;
                *reinterpret_cast<uint32_t *>(sm + S::A2 + kmaj(r * 32 + c, 2 * kx, KM)) = pack_bf16(ab[i].x, ab[i].y);
            }
        }
        if (!LIFT) {
#pragma unroll
            for (int i = 0; i < NB4; ++i) {
                const int it = warp + i * kRowWarps, rr = it / (N / 16), xb = (it % (N / 16)) * 16;
                const int x = xb + (vq & 1) * 8 + 2 * vp, j0 = (vq >> 1) * 8;
                const uint32_t w0[4] = {vv[i][0].x, vv[i][0].y, vv[i][0].z, vv[i][0].w};
                const uint32_t w1[4] = {vv[i][1].x, vv[i][1].y, vv[i][1].z, vv[i][1].w};
#pragma unroll
                for (int jj = 0; jj < 8; ++jj)
                    *reinterpret_cast<uint32_t *>(sm + S::B4 + kmaj(rr * 32 + j0 + jj, x, N)) =
                        __byte_perm(w0[jj >> 1], w1[jj >> 1], (jj & 1) ? 0x7632 : 0x5410);
            }
        }
        if (LIFT) {
            for (int e = tid; e < kTile * N; e += kRowThreads) {
                const size_t c = (size_t)row0 * N + e;
                const float2 u = a.psi[c], q = a.psib[c];
                fs[e * 4 + 0] = u.x * a.inv_A;
                fs[e * 4 + 1] = u.y * a.inv_A;
                fs[e * 4 + 2] = q.x * a.inv_A;
                fs[e * 4 + 3] = q.y * a.inv_A;
            }
        }
        if (START) {
            // the given u bar straight into the A operand of G3 / G4
#pragma unroll
            for (int i = 0; i < HW; i += 8) {
                uint32_t pk[4];
#pragma unroll
                for (int k = 0; k < 8; k += 2) {
                    const size_t e0 = ((size_t)row * N + half * HW + i + k) * kC + lane;
                    const float u0 = a.ubar[e0], u1 = a.ubar[e0 + kC];
                    gacc += u0;
                    gacc += u1;
                    pk[k / 2] = pack_bf16(u0, u1);
                }
                *reinterpret_cast<uint4 *>(sm + S::A3 + kmaj(r_ep * 32 + lane, half * HW + i, N)) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        to_tensor_cores();
        if (!START) {
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
            float d[HW];
            tmem_ld<HW>(tbase + ((uint32_t)(r_ep * 32) << 16) + half * HW, d);
            if (LIFT) {
                // v bar of the lift: dL/dp += v bar, dL/dP[c][f] += v bar * feature f
#pragma unroll
                for (int i = 0; i < HW; ++i) {
                    const float *f = fs + (r_ep * N + half * HW + i) * 4;
                    gacc += d[i];
#pragma unroll
                    for (int q = 0; q < kFin; ++q) Pr[q] = fmaf(d[i], f[q], Pr[q]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < HW; i += 8) {
                    uint32_t pk[4];
#pragma unroll
                    for (int k = 0; k < 8; k += 2) {
                        const size_t e0 = ((size_t)row * N + half * HW + i + k) * kC + lane;
                        const float u0 = d[i + k] * gelu_grad(__bfloat162float(__ushort_as_bfloat16(up[i + k])));
                        const float u1 = d[i + k + 1] * gelu_grad(__bfloat162float(__ushort_as_bfloat16(up[i + k + 1])));
                        a.ubar[e0] = u0;
                        a.ubar[e0 + kC] = u1;
                        gacc += u0;
                        gacc += u1;
                        pk[k / 2] = pack_bf16(u0, u1);
                    }
                    *reinterpret_cast<uint4 *>(sm + S::A3 + kmaj(r_ep * 32 + lane, half * HW + i, N)) =
                        make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
            }
            end_phase(ctl);
        }
        if (!LIFT) {
            to_tensor_cores();
            if (tid == 0) {
                constexpr uint32_t id3 = idesc_bf16(KM), id4 = idesc_bf16(128);
#pragma unroll
                for (int s = 0; s < N / 16; ++s)
                    mma_bf16(tbase + kColE, desc_k(sm + S::A3 + s * 256, N), desc_k(sm + S::B3 + s * 256, N), id3,
                             s > 0);
#pragma unroll
                for (int s = 0; s < N / 16; ++s)
                    mma_bf16(tbase + kColS, desc_k(sm + S::A3 + s * 256, N), desc_k(sm + S::B4 + s * 256, N), id4,
                             (s > 0 || done > 0) ? 1u : 0u);
                tc_commit(&ctl->mbar);
            }
            wait_mma(ctl, a.status);
            {
                constexpr int EW = KM / 2;          // 8 or 16 columns per warp
                // KM = 16: both halves read the same 16 columns and half 1 stores nothing
                float d[16];
                tmem_ld16(tbase + ((uint32_t)(r_ep * 32) << 16) + kColE + (EW == 16 ? half * 16 : 0), d);
                if (EW == 16 || half == 0) {
                    const int kx0 = (EW == 16) ? half * 8 : 0;
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        a.xrow[((size_t)row * M + kx0 + k) * kC + lane] = make_float2(d[2 * k], d[2 * k + 1]);
                }
            }
            end_phase(ctl);
        }
        __syncthreads();   // the next tile restages the operands
    }

    // ---- the CTA's partial segment, in a fixed order
    float *red = reinterpret_cast<float *>(sm + S::A1);          // [4][32][32] diagonal blocks of S
    float *gred = red + 4 * 32 * 32;                              // [8 warps][32][5]
    const int seg = LIFT ? kLiftSeg : kLayerSeg;
    float *out = a.partials + (size_t)blockIdx.x * seg;
    if (!LIFT && done > 0) {
        float sv[16];
        tmem_ld16(tbase + ((uint32_t)(r_ep * 32) << 16) + kColS + r_ep * 32 + half * 16, sv);
#pragma unroll
        for (int i = 0; i < 16; ++i) red[(r_ep * 32 + lane) * 32 + half * 16 + i] = sv[i];
    }
    gred[(warp * 32 + lane) * 5 + 0] = gacc;
#pragma unroll
    for (int f = 0; f < kFin; ++f) gred[(warp * 32 + lane) * 5 + 1 + f] = Pr[f];
    __syncthreads();
    if (LIFT) {
        for (int e = tid; e < kC * kFin; e += kRowThreads) {
            const int c = e / kFin, f = e % kFin;
            float s = 0.f;
            for (int w = 0; w < kRowWarps; ++w) s += gred[(w * 32 + c) * 5 + 1 + f];
            out[c * kFin + f] = s;
        }
        for (int c = tid; c < kC; c += kRowThreads) {
            float s = 0.f;
            for (int w = 0; w < kRowWarps; ++w) s += gred[(w * 32 + c) * 5];
            out[kC * kFin + c] = s;
        }
    } else {
        for (int e = tid; e < kC * kC; e += kRowThreads) {
            float s = 0.f;
            if (done > 0)
                for (int r = 0; r < 4; ++r) s += red[(r * 32 + e / kC) * 32 + e % kC];
            out[e] = s;
        }
        for (int c = tid; c < kC; c += kRowThreads) {
            float s = 0.f;
            for (int w = 0; w < kRowWarps; ++w) s += gred[(w * 32 + c) * 5];
            out[kC * kC + c] = s;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free_n<256>(tbase);
}

template <int N, int M, int MODE>
cudaError_t bwd_tc_run(const RowArgs &a, int grid, cudaStream_t st)
{
    constexpr int bytes = BwdSmem<N, M>::BYTES;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(layer_bwd_tc_kernel<N, M, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    layer_bwd_tc_kernel<N, M, MODE><<<grid, kRowThreads, bytes, st>>>(a);
    return cudaGetLastError();
}

template <int N, int M>
cudaError_t bwd_tc_mode(int mode, const RowArgs &a, int grid, cudaStream_t st)
{
    if (mode == kBwdLift) return bwd_tc_run<N, M, kBwdLift>(a, grid, st);
    if (mode == kBwdStart) return bwd_tc_run<N, M, kBwdStart>(a, grid, st);
    return bwd_tc_run<N, M, kBwdLayer>(a, grid, st);
}

// Projection backward on the tensor cores: a tile of 128 cells, TMEM lane = cell.
//   GA  H[cell][j]   = sum_c V[cell][c] Q1[j][c]                 (K = 32), h = H + q1
//   epilogue: g = GELU(h), o = Q2 g + q2, the loss term, ob = dL/do, hb = (Q2^T ob) GELU'(h)
//   GB  VB[cell][c]  = sum_j Hb[cell][j] Q1[j][c]                (K = 64): u bar of the last layer
//   GW  W[m][k]     += sum_cell Aw[m][cell] Bw[k][cell]           (K = 128 cells, accumulated in
//       TMEM over the CTA's tiles) with rows m < 64 = Hb^T and m >= 64 = G^T, columns k < 32 = V^T,
//       k = 32, 33 the two ob and k = 34 ones: dL/dQ1[j][c] = W[j][c], dL/dq1[j] = W[j][34],
//       dL/dQ2[o][j] = W[64 + j][32 + o].  dL/dq2 and the loss are summed on the CUDA cores.
struct ProjBwdSmem {
    static constexpr int AV = 0;                  // V [128][32]
    static constexpr int BQ = AV + 128 * 32 * 2;  // Q1 [64][32]
    static constexpr int AH = BQ + 64 * 32 * 2;   // Hb [128][64]
    static constexpr int BQT = AH + 128 * 64 * 2; // Q1^T [32][64]
    static constexpr int AW = BQT + 32 * 64 * 2;  // [Hb^T; G^T] [128][128], 128-byte swizzle (column writes)
    static constexpr int BW = AW + 128 * 128 * 2; // [V^T; ob; 1; 0] [48][128], 128-byte swizzle
    static_assert(AW % 1024 == 0 && BW % 1024 == 0 && (48 * 128) % 1024 == 0, "swizzle atoms 1024-byte aligned");
    static constexpr int PART = BW + 48 * 128 * 2;// [2 halves][128][2] partial o
    static constexpr int PAR = PART + 2 * 128 * 2 * 4;   // q1 [64], Q2 [2][64], q2 [2]
    static constexpr int RED = PAR + (64 + 128 + 2) * 4; // [128][3] loss and dL/dq2 partials
    static constexpr int CTL = (RED + 128 * 3 * 4 + 63) & ~63;
    static constexpr int BYTES = CTL + 64;
};

__device__ __forceinline__ void put_bf16(unsigned char *base, int off, float v)
{
    *reinterpret_cast<unsigned short *>(base + off) = bf16_bits(v);
}

__global__ void __launch_bounds__(kRowThreads, 2) proj_bwd_tc_kernel(RowArgs a, int cells)
{
    using S = ProjBwdSmem;
    constexpr int kColH = 0, kColVB = 64, kColW = 128;
    extern __shared__ __align__(1024) unsigned char sm[];
    TcCtl *ctl = reinterpret_cast<TcCtl *>(sm + S::CTL);
    float *part = reinterpret_cast<float *>(sm + S::PART);
    float *q1 = reinterpret_cast<float *>(sm + S::PAR);
    float *q2w = q1 + 64;
    float *q2b = q2w + 128;
    float *red = reinterpret_cast<float *>(sm + S::RED);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int qd = warp & 3, half = warp >> 2;
    const int m = qd * 32 + lane;                 // this thread's cell (TMEM lane) in the tile

    // ---- per-CTA constants: Q1, Q1^T, the ones row and zero rows of Bw, q1, Q2, q2
    for (int e = tid; e < kH * 4; e += kRowThreads) {
        const int j = e / 4, q = e % 4;
        *reinterpret_cast<uint4 *>(sm + S::BQ + kmaj(j, q * 8, 32)) =
            *reinterpret_cast<const uint4 *>(a.w + a.oQ1 + j * kC + q * 8);
    }
    for (int e = tid; e < kC * kH; e += kRowThreads) {
        const int c = e / kH, j = e % kH;
        *reinterpret_cast<unsigned short *>(sm + S::BQT + kmaj(c, j, 64)) =
            __bfloat16_as_ushort(a.w[a.oQ1 + (size_t)j * kC + c]);
    }
    for (int e = tid; e < 16 * 128; e += kRowThreads) {
        const int k = 32 + e / 128, cell = e % 128;
        put_bf16(sm + S::BW, sw128(k, cell, 48), k == 34 ? 1.f : 0.f);
    }
    for (int e = tid; e < kH; e += kRowThreads) q1[e] = wload(a.w, a.oq1 + e);
    for (int e = tid; e < 2 * kH; e += kRowThreads) q2w[e] = wload(a.w, a.oQ2 + e);
    if (tid < 2) q2b[tid] = wload(a.w, a.oq2 + tid);
    ctl_setup<256>(ctl);
    to_tensor_cores();
    const uint32_t tbase = ctl->tmem_base;
    const uint32_t lrow = (uint32_t)(qd * 32) << 16;
    const __nv_bfloat16 *vin = (const __nv_bfloat16 *)a.vin;
    const int tiles = cells / 128;
    float loss = 0.f, gq2a = 0.f, gq2b = 0.f;
    int done = 0;

    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++done) {
        const size_t cell0 = (size_t)t * 128;
        const size_t cell = cell0 + m;
        // V [cell][c] (A of GA) and V^T [c][cell] (rows 0..31 of Bw, pairs of cells per word)
        for (int e = tid; e < 128 * 4; e += kRowThreads) {
            const int mm = e / 4, q = e % 4;
            *reinterpret_cast<uint4 *>(sm + S::AV + kmaj(mm, q * 8, 32)) =
                *reinterpret_cast<const uint4 *>(vin + (cell0 + mm) * kC + q * 8);
        }
        {
            const int p = lane & 3, q = lane >> 2;
            // each warp takes 16 cells: lanes (p, q) hold cells mm, mm + 1 of channels j0 .. j0 + 7
            const int mm = warp * 16 + (q & 1) * 8 + 2 * p, j0 = (q >> 1) * 8;
            const __nv_bfloat16 *src = vin + (cell0 + mm) * kC + j0;
            const uint4 v0 = *reinterpret_cast<const uint4 *>(src);
            const uint4 v1 = *reinterpret_cast<const uint4 *>(src + kC);
            const uint32_t w0[4] = {v0.x, v0.y, v0.z, v0.w}, w1[4] = {v1.x, v1.y, v1.z, v1.w};
#pragma unroll
            for (int jj = 0; jj < 8; ++jj)
                *reinterpret_cast<uint32_t *>(sm + S::BW + sw128(j0 + jj, mm, 48)) =
                    __byte_perm(w0[jj >> 1], w1[jj >> 1], (jj & 1) ? 0x7632 : 0x5410);
        }
        to_tensor_cores();
        if (tid == 0) {
            constexpr uint32_t id = idesc_bf16(64);
#pragma unroll
            for (int s = 0; s < 2; ++s)
                mma_bf16(tbase + kColH, desc_k(sm + S::AV + s * 256, 32), desc_k(sm + S::BQ + s * 256, 32), id, s > 0);
            tc_commit(&ctl->mbar);
        }
        wait_mma(ctl, a.status);
        float h[32];
        tmem_ld32(tbase + lrow + kColH + half * 32, h);
        float o0 = 0.f, o1 = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            // GELU(u) = u Phi(u) and GELU'(u) = Phi(u) + u phi(u) share the normal CDF Phi; h[i]
            // keeps GELU'(u) for the cotangent below
            const int j = half * 32 + i;
            const float u = h[i] + q1[j];
            const float cdf = 0.5f * (1.f + erff(u * kInvSqrt2));
            const float g = u * cdf;
            h[i] = fmaf(u * kInvSqrt2Pi, expf(-0.5f * u * u), cdf);
            o0 = fmaf(q2w[j], g, o0);
            o1 = fmaf(q2w[kH + j], g, o1);
            put_bf16(sm + S::AW, sw128(64 + j, m, 128), g);
        }
        part[(half * 128 + m) * 2] = o0;
        part[(half * 128 + m) * 2 + 1] = o1;
        end_phase(ctl);      // also orders the partial sums of o before they are read
        const float O0 = part[m * 2] + part[(128 + m) * 2] + q2b[0];
        const float O1 = part[m * 2 + 1] + part[(128 + m) * 2 + 1] + q2b[1];
        const float2 pb = a.psib[cell], tg = a.target[cell];
        const float dx = pb.x + a.sigma * O0 - tg.x, dy = pb.y + a.sigma * O1 - tg.y;
        const float ob0 = a.loss_scale * dx, ob1 = a.loss_scale * dy;
        if (half == 0) {
            loss = fmaf(dx, dx, loss);
            loss = fmaf(dy, dy, loss);
            gq2a += ob0;
            gq2b += ob1;
            put_bf16(sm + S::BW, sw128(32, m, 48), ob0);
            put_bf16(sm + S::BW, sw128(33, m, 48), ob1);
        }
#pragma unroll
        for (int i = 0; i < 32; i += 8) {
            uint32_t pk[4];
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                const int j = half * 32 + i + k;
                const float hb0 = (q2w[j] * ob0 + q2w[kH + j] * ob1) * h[i + k];
                const float hb1 = (q2w[j + 1] * ob0 + q2w[kH + j + 1] * ob1) * h[i + k + 1];
                put_bf16(sm + S::AW, sw128(j, m, 128), hb0);
                put_bf16(sm + S::AW, sw128(j + 1, m, 128), hb1);
                pk[k / 2] = pack_bf16(hb0, hb1);
            }
            *reinterpret_cast<uint4 *>(sm + S::AH + kmaj(m, half * 32 + i, 64)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        to_tensor_cores();
        if (tid == 0) {
            constexpr uint32_t idb = idesc_bf16(32), idw = idesc_bf16(48);
#pragma unroll
            for (int s = 0; s < 4; ++s)
                mma_bf16(tbase + kColVB, desc_k(sm + S::AH + s * 256, 64), desc_k(sm + S::BQT + s * 256, 64), idb,
                         s > 0);
#pragma unroll
            for (int s = 0; s < 8; ++s)
                mma_bf16(tbase + kColW, desc_sw128(sm + S::AW, s, 128), desc_sw128(sm + S::BW, s, 48), idw,
                         (s > 0 || done > 0) ? 1u : 0u);
            tc_commit(&ctl->mbar);
        }
        wait_mma(ctl, a.status);
        {
            float vb[16];
            tmem_ld16(tbase + lrow + kColVB + half * 16, vb);
            float4 *dst = reinterpret_cast<float4 *>(a.ubar + cell * kC + half * 16);
#pragma unroll
            for (int i = 0; i < 4; ++i) dst[i] = make_float4(vb[4 * i], vb[4 * i + 1], vb[4 * i + 2], vb[4 * i + 3]);
        }
        end_phase(ctl);
    }

    // ---- the CTA's partial segment: Q1 [H][C] | q1 [H] | Q2 [2][H] | q2 [2] | loss
    constexpr int q1o = kH * kC, q2o = kH * kC + kH;
    float *out = a.partials + (size_t)blockIdx.x * kTopSeg;
    if (done > 0) {
        if (half == 0) {
            float w[32];
            tmem_ld32(tbase + lrow + kColW, w);
            if (m < 64) {
#pragma unroll
                for (int c = 0; c < kC; ++c) out[m * kC + c] = w[c];
            }
        } else {
            float w[16];
            tmem_ld16(tbase + lrow + kColW + 32, w);
            if (m < 64) out[q1o + m] = w[2];
            else {
                out[q2o + (m - 64)] = w[0];
                out[q2o + kH + (m - 64)] = w[1];
            }
        }
    } else {
        for (int e = tid; e < q2o + 2 * kH; e += kRowThreads) out[e] = 0.f;
    }
    if (half == 0) {
        red[m * 3 + 0] = gq2a;
        red[m * 3 + 1] = gq2b;
        red[m * 3 + 2] = loss;
    }
    __syncthreads();
    if (tid < 3) {
        float s = 0.f;
        for (int k = 0; k < 128; ++k) s += red[k * 3 + tid];
        out[kTopSeg - 3 + tid] = s;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free_n<256>(tbase);
}

}  // namespace

cudaError_t launch_layer_bwd_tc(int n, int M, int mode, const RowArgs &a, int grid, cudaStream_t st)
{
    if (a.rows % kTile || grid < 1 || grid > a.rows / kTile) return cudaErrorInvalidValue;
#define SPE_FNO_TC_CASE(NN, MM) \
    if (n == NN && M == MM) return bwd_tc_mode<NN, MM>(mode, a, grid, st);
    SPE_FNO_TC_CASE(64, 16)
    SPE_FNO_TC_CASE(64, 8)
    SPE_FNO_TC_CASE(32, 16)
    SPE_FNO_TC_CASE(32, 8)
#undef SPE_FNO_TC_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_proj_bwd_tc(const RowArgs &a, int cells, int grid, cudaStream_t st)
{
    if (cells % 128 || grid < 1 || grid > cells / 128) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(proj_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             ProjBwdSmem::BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    proj_bwd_tc_kernel<<<grid, kRowThreads, ProjBwdSmem::BYTES, st>>>(a, cells);
    return cudaGetLastError();
}

}  // namespace fno
}  // namespace spe
