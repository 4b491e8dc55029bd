// Backward row kernels of the FNO surrogate (same row blocking as the forward).
//
// Cotangents follow the convention  z_bar = dL/dRe z + i dL/dIm z  for complex
// z, so a complex linear map y = A x back-propagates as x_bar = A^H y_bar, a
// real-input map y = A x (x real) as x_bar = Re(A^H y_bar), and a real-output
// map y = Re(A x) as x_bar = A^H y_bar.
//   top       : from psi_pred - psi_target back through the projection:
//               gradients of Q1, q1, Q2, q2 and the loss, and
//               ubar_{L-1} = v_L bar (the last layer has no activation);
//   grad_start: W_{L-1}, b_{L-1} gradients and Bbar = Gx^H ubar_{L-1};
//   layer l   : v_l bar = W_l^T ubar_l + Re(Fx^H abar_l),
//               ubar_{l-1} = v_l bar * GELU'(u_{l-1}), gradients of W_{l-1},
//               b_{l-1}, and Bbar_{l-1} = Gx^H ubar_{l-1};
//   lift      : v_0 bar as above, gradients of P and p.
// Weight gradients are summed per block in a fixed warp order and written as
// one partial per block; a separate kernel adds the partials in block order.
#include "fno_rowcommon.cuh"

namespace spe {
namespace fno {
namespace {

template <int N, typename Act>
__global__ void __launch_bounds__(kRowThreads) top_bwd_kernel(RowArgs a)
{
    __shared__ float vs[N][kC];
    __shared__ float q1s[kH][kC + 1];
    __shared__ float hb[kRowWarps][kH];
    __shared__ float acc_s[kTopSeg];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < kH * kC; e += kRowThreads) q1s[e / kC][e % kC] = wload(a.w, a.oQ1 + e);
    zero_shared(acc_s, kTopSeg);
    const float q1a = wload(a.w, a.oq1 + lane), q1b = wload(a.w, a.oq1 + lane + 32);
    float q2w[2][2];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        q2w[o][0] = wload(a.w, a.oQ2 + o * kH + lane);
        q2w[o][1] = wload(a.w, a.oQ2 + o * kH + lane + 32);
    }
    const float q2b0 = wload(a.w, a.oq2), q2b1 = wload(a.w, a.oq2 + 1);
    float gQ1[2][kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) gQ1[0][c] = gQ1[1][c] = 0.f;
    float gq1[2] = {0.f, 0.f}, gQ2[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, gq2[2] = {0.f, 0.f}, loss = 0.f;
    const Act *vin = (const Act *)a.vin;

    for (int r = blockIdx.x; r < a.rows; r += gridDim.x) {
        const Act *vr = vin + (size_t)r * N * kC;
        __syncthreads();
        for (int e = threadIdx.x; e < N * kC; e += kRowThreads) vs[e / kC][e % kC] = act_load(vr + e);
        __syncthreads();
        for (int x = warp; x < N; x += kRowWarps) {
            float h0 = q1a, h1 = q1b;
#pragma unroll 8
            for (int c = 0; c < kC; ++c) {
                const float vv = vs[x][c];
                h0 = fmaf(q1s[lane][c], vv, h0);
                h1 = fmaf(q1s[lane + 32][c], vv, h1);
            }
            const float g0 = gelu(h0), g1 = gelu(h1);
            const float o0 = warp_sum(q2w[0][0] * g0 + q2w[0][1] * g1) + q2b0;
            const float o1 = warp_sum(q2w[1][0] * g0 + q2w[1][1] * g1) + q2b1;
            const size_t cell = (size_t)r * N + x;
            const float2 pb = a.psib[cell], tg = a.target[cell];
            const float dx = pb.x + a.sigma * o0 - tg.x, dy = pb.y + a.sigma * o1 - tg.y;
            if (lane == 0) {
                loss = fmaf(dx, dx, loss);
                loss = fmaf(dy, dy, loss);
            }
            const float ob0 = a.loss_scale * dx, ob1 = a.loss_scale * dy;
            gQ2[0][0] = fmaf(ob0, g0, gQ2[0][0]);
            gQ2[0][1] = fmaf(ob0, g1, gQ2[0][1]);
            gQ2[1][0] = fmaf(ob1, g0, gQ2[1][0]);
            gQ2[1][1] = fmaf(ob1, g1, gQ2[1][1]);
            if (lane == 0) {
                gq2[0] += ob0;
                gq2[1] += ob1;
            }
            const float hb0 = (q2w[0][0] * ob0 + q2w[1][0] * ob1) * gelu_grad(h0);
            const float hb1 = (q2w[0][1] * ob0 + q2w[1][1] * ob1) * gelu_grad(h1);
            gq1[0] += hb0;
            gq1[1] += hb1;
#pragma unroll
            for (int c = 0; c < kC; ++c) {
                const float vv = vs[x][c];
                gQ1[0][c] = fmaf(hb0, vv, gQ1[0][c]);
                gQ1[1][c] = fmaf(hb1, vv, gQ1[1][c]);
            }
            hb[warp][lane] = hb0;
            hb[warp][lane + 32] = hb1;
            __syncwarp();
            float vb = 0.f;
#pragma unroll 8
            for (int j = 0; j < kH; ++j) vb = fmaf(q1s[j][lane], hb[warp][j], vb);
            a.ubar[cell * kC + lane] = vb;
            __syncwarp();
        }
    }
    __syncthreads();
    // segment: Q1 [H][C] | q1 [H] | Q2 [2][H] | q2 [2] | loss, summed warp by warp
    constexpr int q1o = kH * kC, q2o = kH * kC + kH;
    for (int w = 0; w < kRowWarps; ++w) {
        if (warp == w) {
#pragma unroll
            for (int c = 0; c < kC; ++c) {
                acc_s[lane * kC + c] += gQ1[0][c];
                acc_s[(lane + 32) * kC + c] += gQ1[1][c];
            }
            acc_s[q1o + lane] += gq1[0];
            acc_s[q1o + lane + 32] += gq1[1];
            acc_s[q2o + lane] += gQ2[0][0];
            acc_s[q2o + lane + 32] += gQ2[0][1];
            acc_s[q2o + kH + lane] += gQ2[1][0];
            acc_s[q2o + kH + lane + 32] += gQ2[1][1];
            if (lane == 0) {
                acc_s[kTopSeg - 3] += gq2[0];
                acc_s[kTopSeg - 2] += gq2[1];
                acc_s[kTopSeg - 1] += loss;
            }
        }
        __syncthreads();
    }
    write_partials(acc_s, a.partials, kTopSeg);
}

// Adds a lane's W-gradient row (gW[j] = dL/dW[lane][j]) and b-gradient into
// the block's shared segment W [C][C] | b [C], warp by warp.
__device__ __forceinline__ void accumulate_layer_seg(float *acc_s, const float (&gW)[kC], float gb)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w = 0; w < kRowWarps; ++w) {
        if (warp == w) {
#pragma unroll
            for (int j = 0; j < kC; ++j) acc_s[lane * kC + j] += gW[j];
            acc_s[kC * kC + lane] += gb;
        }
        __syncthreads();
    }
}

template <int N, int M, typename Act>
__global__ void __launch_bounds__(kRowThreads) grad_start_kernel(RowArgs a)
{
    __shared__ float us[N][kC];
    __shared__ float vs[N][kC];
    __shared__ float acc_s[kLayerSeg];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    zero_shared(acc_s, kLayerSeg);
    float gW[kC], gb = 0.f;
#pragma unroll
    for (int j = 0; j < kC; ++j) gW[j] = 0.f;
    const Act *vin = (const Act *)a.vin;

    for (int r = blockIdx.x; r < a.rows; r += gridDim.x) {
        __syncthreads();
        const float *ur = a.ubar + (size_t)r * N * kC;
        const Act *vr = vin + (size_t)r * N * kC;
        for (int e = threadIdx.x; e < N * kC; e += kRowThreads) {
            us[e / kC][e % kC] = ur[e];
            vs[e / kC][e % kC] = act_load(vr + e);
        }
        __syncthreads();
        for (int x = warp; x < N; x += kRowWarps) {
            const float uu = us[x][lane];
            gb += uu;
#pragma unroll
            for (int j = 0; j < kC; ++j) gW[j] = fmaf(uu, vs[x][j], gW[j]);
        }
        for (int kx = warp; kx < M; kx += kRowWarps) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
            for (int x = 0; x < N; ++x) {
                const float2 g = Gx<N>(x, kx);
                const float u = us[x][lane];
                acc.x = fmaf(g.x, u, acc.x);
                acc.y = fmaf(-g.y, u, acc.y);
            }
            a.xrow[((size_t)r * M + kx) * kC + lane] = acc;
        }
    }
    __syncthreads();
    accumulate_layer_seg(acc_s, gW, gb);
    write_partials(acc_s, a.partials, kLayerSeg);
}

template <int N, int M, typename Act>
__global__ void __launch_bounds__(kRowThreads) layer_bwd_kernel(RowArgs a)
{
    __shared__ float us[N][kC];      // ubar_l
    __shared__ float2 as[M][kC];     // abar_l
    __shared__ float vs[N][kC];      // v_{l-1}
    __shared__ float un[N][kC];      // ubar_{l-1}
    __shared__ float acc_s[kLayerSeg];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    zero_shared(acc_s, kLayerSeg);
    float Wc[kC];                    // column lane of W_l
#pragma unroll
    for (int j = 0; j < kC; ++j) Wc[j] = wload(a.w, a.oW + j * kC + lane);
    float gW[kC], gb = 0.f;
#pragma unroll
    for (int j = 0; j < kC; ++j) gW[j] = 0.f;
    const Act *vin = (const Act *)a.vin;
    const Act *upre = (const Act *)a.upre;

    for (int r = blockIdx.x; r < a.rows; r += gridDim.x) {
        __syncthreads();
        const float *ur = a.ubar + (size_t)r * N * kC;
        const Act *vr = vin + (size_t)r * N * kC;
        for (int e = threadIdx.x; e < N * kC; e += kRowThreads) {
            us[e / kC][e % kC] = ur[e];
            vs[e / kC][e % kC] = act_load(vr + e);
        }
        const float2 *ar = a.xrow + (size_t)r * M * kC;
        for (int e = threadIdx.x; e < M * kC; e += kRowThreads) as[e / kC][e % kC] = ar[e];
        __syncthreads();
        for (int x = warp; x < N; x += kRowWarps) {
            float vb = 0.f;
#pragma unroll
            for (int j = 0; j < kC; ++j) vb = fmaf(Wc[j], us[x][j], vb);
#pragma unroll
            for (int kx = 0; kx < M; ++kx) {
                const float2 f = Fx<N>(kx, x);
                const float2 q = as[kx][lane];
                vb = fmaf(f.x, q.x, vb);
                vb = fmaf(f.y, q.y, vb);
            }
            const size_t e = ((size_t)r * N + x) * kC + lane;
            const float ub = vb * gelu_grad(act_load(upre + e));
            un[x][lane] = ub;
            a.ubar[e] = ub;
            gb += ub;
#pragma unroll
            for (int j = 0; j < kC; ++j) gW[j] = fmaf(ub, vs[x][j], gW[j]);
        }
        __syncthreads();
        for (int kx = warp; kx < M; kx += kRowWarps) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
            for (int x = 0; x < N; ++x) {
                const float2 g = Gx<N>(x, kx);
                const float u = un[x][lane];
                acc.x = fmaf(g.x, u, acc.x);
                acc.y = fmaf(-g.y, u, acc.y);
            }
            a.xrow[((size_t)r * M + kx) * kC + lane] = acc;
        }
    }
    __syncthreads();
    accumulate_layer_seg(acc_s, gW, gb);
    write_partials(acc_s, a.partials, kLayerSeg);
}

template <int N, int M, typename Act>
__global__ void __launch_bounds__(kRowThreads) lift_bwd_kernel(RowArgs a)
{
    __shared__ float us[N][kC];
    __shared__ float2 as[M][kC];
    __shared__ float fs[N][kFin];
    __shared__ float acc_s[kLiftSeg];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    zero_shared(acc_s, kLiftSeg);
    float Wc[kC];
#pragma unroll
    for (int j = 0; j < kC; ++j) Wc[j] = wload(a.w, a.oW + j * kC + lane);
    float gP[kFin] = {0.f, 0.f, 0.f, 0.f}, gp = 0.f;

    for (int r = blockIdx.x; r < a.rows; r += gridDim.x) {
        __syncthreads();
        const float *ur = a.ubar + (size_t)r * N * kC;
        for (int e = threadIdx.x; e < N * kC; e += kRowThreads) us[e / kC][e % kC] = ur[e];
        const float2 *ar = a.xrow + (size_t)r * M * kC;
        for (int e = threadIdx.x; e < M * kC; e += kRowThreads) as[e / kC][e % kC] = ar[e];
        for (int x = threadIdx.x; x < N; x += kRowThreads) {
            const float2 u = a.psi[(size_t)r * N + x], q = a.psib[(size_t)r * N + x];
            fs[x][0] = u.x * a.inv_A;
            fs[x][1] = u.y * a.inv_A;
            fs[x][2] = q.x * a.inv_A;
            fs[x][3] = q.y * a.inv_A;
        }
        __syncthreads();
        for (int x = warp; x < N; x += kRowWarps) {
            float vb = 0.f;
#pragma unroll
            for (int j = 0; j < kC; ++j) vb = fmaf(Wc[j], us[x][j], vb);
#pragma unroll
            for (int kx = 0; kx < M; ++kx) {
                const float2 f = Fx<N>(kx, x);
                const float2 q = as[kx][lane];
                vb = fmaf(f.x, q.x, vb);
                vb = fmaf(f.y, q.y, vb);
            }
            gp += vb;
#pragma unroll
            for (int f = 0; f < kFin; ++f) gP[f] = fmaf(vb, fs[x][f], gP[f]);
        }
    }
    __syncthreads();
    for (int w = 0; w < kRowWarps; ++w) {
        if (warp == w) {
#pragma unroll
            for (int f = 0; f < kFin; ++f) acc_s[lane * kFin + f] += gP[f];
            acc_s[kC * kFin + lane] += gp;
        }
        __syncthreads();
    }
    write_partials(acc_s, a.partials, kLiftSeg);
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

enum class Kind { Top, Start, Layer, Lift };

struct Run {
    const RowArgs &a;
    int grid;
    cudaStream_t st;
    Kind kind;
    template <int N, int M, typename Act>
    cudaError_t run() const
    {
        switch (kind) {
            case Kind::Top: top_bwd_kernel<N, Act><<<grid, kRowThreads, 0, st>>>(a); break;
            case Kind::Start: grad_start_kernel<N, M, Act><<<grid, kRowThreads, 0, st>>>(a); break;
            case Kind::Layer: layer_bwd_kernel<N, M, Act><<<grid, kRowThreads, 0, st>>>(a); break;
            case Kind::Lift: lift_bwd_kernel<N, M, Act><<<grid, kRowThreads, 0, st>>>(a); break;
        }
        return cudaGetLastError();
    }
};

}  // namespace

cudaError_t upload_bwd_tables(const float2 *G64, const float2 *F64, const float2 *G32, const float2 *F32)
{
    return upload_tables_here(G64, F64, G32, F32);
}

cudaError_t launch_top_bwd(int n, bool fp32, const RowArgs &a, int grid, cudaStream_t st)
{
    // the projection does not depend on M; any instantiated M serves
    return dispatch(n, 16, fp32, Run{a, grid, st, Kind::Top});
}

cudaError_t launch_grad_start(int n, int M, bool fp32, const RowArgs &a, int grid, cudaStream_t st)
{
    return dispatch(n, M, fp32, Run{a, grid, st, Kind::Start});
}

cudaError_t launch_layer_bwd(int n, int M, bool fp32, const RowArgs &a, int grid, cudaStream_t st)
{
    return dispatch(n, M, fp32, Run{a, grid, st, Kind::Layer});
}

cudaError_t launch_lift_bwd(int n, int M, bool fp32, const RowArgs &a, int grid, cudaStream_t st)
{
    return dispatch(n, M, fp32, Run{a, grid, st, Kind::Lift});
}

}  // namespace fno
}  // namespace spe
