// Forward row kernels of the FNO surrogate.
//
// One block of 8 warps handles one (b, z, y) row of n cells at a time and
// loops over rows with a fixed grid; lane c owns channel c.  Per row:
//   lift   : v_0 = P f + p from the features of psi and psi_b, then the
//            truncated x DFT a[kx][c] = sum_x Fx[kx][x] v_0[x][c];
//   layer l: u = W v + b + Re sum_kx Gx[x][kx] B[kx][c]  (B: the inverse y
//            output of the layer's spectral path, i.e. its last inverse
//            stage is fused here), v' = GELU(u), then the next layer's x DFT;
//   last   : v_L = u and the projection o = Q2 GELU(Q1 v_L + q1) + q2, giving
//            psi_pred = psi_b + sigma (o_0 + i o_1).
// Weights are read from the BF16 mirror and accumulated in FP32.
#include "fno_rowcommon.cuh"

namespace spe {
namespace fno {
namespace {

template <int N, int M, typename Act>
__global__ void __launch_bounds__(kRowThreads) lift_fwd_kernel(RowArgs a)
{
    __shared__ float fs[N][kFin];
    __shared__ float vs[N][kC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float Pr[kFin];
#pragma unroll
    for (int f = 0; f < kFin; ++f) Pr[f] = wload(a.w, a.oP + lane * kFin + f);
    const float pc = wload(a.w, a.op + lane);
    Act *vout = (Act *)a.vout;

    for (int r = blockIdx.x; r < a.rows; r += gridDim.x) {
        for (int x = threadIdx.x; x < N; x += kRowThreads) {
            const float2 u = a.psi[(size_t)r * N + x], q = a.psib[(size_t)r * N + x];
            fs[x][0] = u.x * a.inv_A;
            fs[x][1] = u.y * a.inv_A;
            fs[x][2] = q.x * a.inv_A;
            fs[x][3] = q.y * a.inv_A;
        }
        __syncthreads();
        for (int x = warp; x < N; x += kRowWarps) {
            float v = pc;
#pragma unroll
            for (int f = 0; f < kFin; ++f) v = fmaf(Pr[f], fs[x][f], v);
            const size_t e = ((size_t)r * N + x) * kC + lane;
            act_store(vout + e, v);
            vs[x][lane] = act_round(v, vout);
        }
        __syncthreads();
        for (int kx = warp; kx < M; kx += kRowWarps) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
            for (int x = 0; x < N; ++x) {
                const float2 f = Fx<N>(kx, x);
                const float v = vs[x][lane];
                acc.x = fmaf(f.x, v, acc.x);
                acc.y = fmaf(f.y, v, acc.y);
            }
            a.xrow[((size_t)r * M + kx) * kC + lane] = acc;
        }
        __syncthreads();
    }
}

template <int N, int M, typename Act, bool LAST>
__global__ void __launch_bounds__(kRowThreads) layer_fwd_kernel(RowArgs a)
{
    __shared__ float vs[N][kC];
    __shared__ float2 bs[M][kC];
    __shared__ float vo[N][kC];
    __shared__ float q1s[LAST ? kH : 1][kC + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float Wr[kC];
#pragma unroll
    for (int j = 0; j < kC; ++j) Wr[j] = wload(a.w, a.oW + lane * kC + j);
    const float bc = wload(a.w, a.ob + lane);
    float q1a = 0.f, q1b = 0.f, q2w[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, q2b0 = 0.f, q2b1 = 0.f;
    if (LAST) {
        for (int e = threadIdx.x; e < kH * kC; e += kRowThreads) q1s[e / kC][e % kC] = wload(a.w, a.oQ1 + e);
        q1a = wload(a.w, a.oq1 + lane);
        q1b = wload(a.w, a.oq1 + lane + 32);
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            q2w[o][0] = wload(a.w, a.oQ2 + o * kH + lane);
            q2w[o][1] = wload(a.w, a.oQ2 + o * kH + lane + 32);
        }
        q2b0 = wload(a.w, a.oq2);
        q2b1 = wload(a.w, a.oq2 + 1);
    }
    const Act *vin = (const Act *)a.vin;
    Act *vout = (Act *)a.vout;
    Act *uout = (Act *)a.uout;

    for (int r = blockIdx.x; r < a.rows; r += gridDim.x) {
        const Act *vr = vin + (size_t)r * N * kC;
        for (int e = threadIdx.x; e < N * kC; e += kRowThreads) vs[e / kC][e % kC] = act_load(vr + e);
        const float2 *br = a.xrow + (size_t)r * M * kC;
        for (int e = threadIdx.x; e < M * kC; e += kRowThreads) bs[e / kC][e % kC] = br[e];
        __syncthreads();
        for (int x = warp; x < N; x += kRowWarps) {
            float u = bc;
#pragma unroll
            for (int j = 0; j < kC; ++j) u = fmaf(Wr[j], vs[x][j], u);
#pragma unroll
            for (int kx = 0; kx < M; ++kx) {
                const float2 g = Gx<N>(x, kx);
                const float2 q = bs[kx][lane];
                u = fmaf(g.x, q.x, u);
                u = fmaf(-g.y, q.y, u);
            }
            const size_t e = ((size_t)r * N + x) * kC + lane;
            if (!LAST) {
                if (a.store_u) act_store(uout + e, u);
                const float v = gelu(u);
                act_store(vout + e, v);
                vo[x][lane] = act_round(v, vout);
            } else {
                act_store(vout + e, u);
                vo[x][lane] = act_round(u, vout);
                __syncwarp();
                float h0 = q1a, h1 = q1b;
#pragma unroll 8
                for (int c = 0; c < kC; ++c) {
                    const float vv = vo[x][c];
                    h0 = fmaf(q1s[lane][c], vv, h0);
                    h1 = fmaf(q1s[lane + 32][c], vv, h1);
                }
                const float g0 = gelu(h0), g1 = gelu(h1);
                const float o0 = warp_sum(q2w[0][0] * g0 + q2w[0][1] * g1);
                const float o1 = warp_sum(q2w[1][0] * g0 + q2w[1][1] * g1);
                if (lane == 0) {
                    const size_t c = (size_t)r * N + x;
                    const float2 pb = a.psib[c];
                    a.out[c] = make_float2(pb.x + a.sigma * (o0 + q2b0), pb.y + a.sigma * (o1 + q2b1));
                }
            }
        }
        __syncthreads();
        if (!LAST) {
            for (int kx = warp; kx < M; kx += kRowWarps) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
                for (int x = 0; x < N; ++x) {
                    const float2 f = Fx<N>(kx, x);
                    const float v = vo[x][lane];
                    acc.x = fmaf(f.x, v, acc.x);
                    acc.y = fmaf(f.y, v, acc.y);
                }
                a.xrow[((size_t)r * M + kx) * kC + lane] = acc;
            }
            __syncthreads();
        }
    }
}

template <int N, int M, typename Act>
cudaError_t lift_nm(const RowArgs &a, int grid, cudaStream_t st)
{
    lift_fwd_kernel<N, M, Act><<<grid, kRowThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <int N, int M, typename Act>
cudaError_t layer_nm(bool last, const RowArgs &a, int grid, cudaStream_t st)
{
    if (last)
        layer_fwd_kernel<N, M, Act, true><<<grid, kRowThreads, 0, st>>>(a);
    else
        layer_fwd_kernel<N, M, Act, false><<<grid, kRowThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename F>
cudaError_t dispatch(int n, int M, bool fp32, F &&f)
{
#define SPE_FNO_CASE(NN, MM)                                                     \
    if (n == NN && M == MM)                                                      \
        return fp32 ? f.template run<NN, MM, float>() : f.template run<NN, MM, __nv_bfloat16>();
    SPE_FNO_CASE(64, 16)
    SPE_FNO_CASE(64, 8)
    SPE_FNO_CASE(32, 16)
    SPE_FNO_CASE(32, 8)
#undef SPE_FNO_CASE
    return cudaErrorInvalidValue;
}

struct LiftRun {
    const RowArgs &a;
    int grid;
    cudaStream_t st;
    template <int N, int M, typename Act>
    cudaError_t run() const { return lift_nm<N, M, Act>(a, grid, st); }
};

struct LayerRun {
    const RowArgs &a;
    int grid;
    cudaStream_t st;
    bool last;
    template <int N, int M, typename Act>
    cudaError_t run() const { return layer_nm<N, M, Act>(last, a, grid, st); }
};

}  // namespace

cudaError_t upload_fwd_tables(const float2 *G64, const float2 *F64, const float2 *G32, const float2 *F32)
{
    return upload_tables_here(G64, F64, G32, F32);
}

cudaError_t launch_lift_fwd(int n, int M, bool fp32, const RowArgs &a, int grid, cudaStream_t st)
{
    return dispatch(n, M, fp32, LiftRun{a, grid, st});
}

cudaError_t launch_layer_fwd(int n, int M, bool fp32, bool last, const RowArgs &a, int grid, cudaStream_t st)
{
    return dispatch(n, M, fp32, LayerRun{a, grid, st, last});
}

}  // namespace fno
}  // namespace spe
