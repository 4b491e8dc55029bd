// Mode-space and elementwise kernels of the FNO surrogate: the y and z stages
// of the truncated DFTs (a complex contraction along one axis), the per-mode
// channel mixing and its adjoint, the fixed-order sum of per-block gradient
// partials, Adam, and the difference norms the judge uses.
#include "fno_internal.cuh"
#include "reduce.cuh"

namespace spe {
namespace fno {
namespace {

constexpr int kAxisThreads = 128;

// out[o][m][i] = scale * sum_j mat[m][j] in[o][j][i] for m in this block's
// MT outputs; threads run over i (contiguous), blocks over (i, o, m chunk).
template <int NIN, int MT>
__global__ void __launch_bounds__(kAxisThreads) axis_kernel(const float2 *__restrict__ in, float2 *__restrict__ out,
                                                           const float2 *__restrict__ mat, int I, int Mout,
                                                           float scale)
{
    __shared__ float2 ms[MT][NIN];
    const int o = blockIdx.y, m0 = blockIdx.z * MT;
    for (int e = threadIdx.x; e < MT * NIN; e += kAxisThreads) ms[e / NIN][e % NIN] = mat[(size_t)m0 * NIN + e];
    __syncthreads();
    const int i = blockIdx.x * kAxisThreads + threadIdx.x;
    if (i >= I) return;
    float2 acc[MT];
#pragma unroll
    for (int t = 0; t < MT; ++t) acc[t] = make_float2(0.f, 0.f);
    const float2 *src = in + (size_t)o * NIN * I + i;
    // eight loads of the strided input in flight per thread (the contraction is short and latency-bound)
#pragma unroll 8
    for (int j = 0; j < NIN; ++j) {
        const float2 x = src[(size_t)j * I];
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            const float2 m = ms[t][j];
            acc[t].x = fmaf(m.x, x.x, fmaf(-m.y, x.y, acc[t].x));
            acc[t].y = fmaf(m.x, x.y, fmaf(m.y, x.x, acc[t].y));
        }
    }
    float2 *dst = out + ((size_t)o * Mout + m0) * I + i;
#pragma unroll
    for (int t = 0; t < MT; ++t) dst[(size_t)t * I] = make_float2(acc[t].x * scale, acc[t].y * scale);
}

template <int NIN, int MT>
cudaError_t axis_run(const float2 *in, float2 *out, const float2 *mat, int Mout, int O, int I, float scale,
                     cudaStream_t st)
{
    dim3 grid((I + kAxisThreads - 1) / kAxisThreads, O, Mout / MT);
    axis_kernel<NIN, MT><<<grid, kAxisThreads, 0, st>>>(in, out, mat, I, Mout, scale);
    return cudaGetLastError();
}

// Y[b][k][o] = sum_i R[k][i][o] X[b][k][i]: one warp per mode k, lane o holds
// column o of R[k].
__global__ void __launch_bounds__(256) mix_fwd_kernel(const float2 *__restrict__ X, float2 *__restrict__ Y,
                                                     const __nv_bfloat162 *__restrict__ R, int K, int B)
{
    __shared__ float2 xs[8][kC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * 8 + warp;
    if (k >= K) return;
    float2 rc[kC];
#pragma unroll
    for (int i = 0; i < kC; ++i) rc[i] = __bfloat1622float2(R[((size_t)k * kC + i) * kC + lane]);
    for (int b = 0; b < B; ++b) {
        const size_t base = ((size_t)b * K + k) * kC;
        xs[warp][lane] = X[base + lane];
        __syncwarp();
        float2 y = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < kC; ++i) {
            const float2 x = xs[warp][i];
            y.x = fmaf(rc[i].x, x.x, fmaf(-rc[i].y, x.y, y.x));
            y.y = fmaf(rc[i].x, x.y, fmaf(rc[i].y, x.x, y.y));
        }
        Y[base + lane] = y;
        __syncwarp();
    }
}

// Xbar[b][k][i] = sum_o conj(R[k][i][o]) Ybar[b][k][o] and
// dL/dR[k][i][o] = sum_b Ybar[b][k][o] conj(X[b][k][i]) (written, not added):
// one warp per mode, lane i holds row i of R[k] and of its gradient.
__global__ void __launch_bounds__(256) mix_bwd_kernel(const float2 *__restrict__ Yb, const float2 *__restrict__ X,
                                                     float2 *__restrict__ Xb, const __nv_bfloat162 *__restrict__ R,
                                                     float2 *__restrict__ gR, int K, int B)
{
    __shared__ float2 ys[8][kC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.x * 8 + warp;
    if (k >= K) return;
    __nv_bfloat162 rr[kC];
#pragma unroll
    for (int o = 0; o < kC; ++o) rr[o] = R[((size_t)k * kC + lane) * kC + o];
    float2 g[kC];
#pragma unroll
    for (int o = 0; o < kC; ++o) g[o] = make_float2(0.f, 0.f);
    for (int b = 0; b < B; ++b) {
        const size_t base = ((size_t)b * K + k) * kC;
        ys[warp][lane] = Yb[base + lane];
        const float2 xi = X[base + lane];
        __syncwarp();
        float2 xb = make_float2(0.f, 0.f);
#pragma unroll
        for (int o = 0; o < kC; ++o) {
            const float2 r = __bfloat1622float2(rr[o]);
            const float2 y = ys[warp][o];
            xb.x = fmaf(r.x, y.x, fmaf(r.y, y.y, xb.x));
            xb.y = fmaf(r.x, y.y, fmaf(-r.y, y.x, xb.y));
            g[o].x = fmaf(y.x, xi.x, fmaf(y.y, xi.y, g[o].x));
            g[o].y = fmaf(y.y, xi.x, fmaf(-y.x, xi.y, g[o].y));
        }
        Xb[base + lane] = xb;
        __syncwarp();
    }
    float2 *dst = gR + ((size_t)k * kC + lane) * kC;
#pragma unroll
    for (int o = 0; o < kC; ++o) dst[o] = g[o];
}

// The mode-space stage of a layer for one (ky, kx) column, fused: z DFT
// X[kz][c] = sum_z Efwd[kz][z] A[z][c], mixing Y[kz][o] = sum_i R[k][i][o]
// X[kz][i] (k = kz M^2 + ky M + kx), z inverse Z[z][c] = (1/n) sum_kz
// Einv[z][kz] Y[kz][c]; Z overwrites A in place (the block owns the column).
// X is kept for the backward pass when Xsave is given.  Lane = channel.  One block per
// (column, batch entry): blockIdx.x the column, blockIdx.y the entry.
template <int N, int M>
__global__ void __launch_bounds__(256) zmix_fwd_kernel(float2 *__restrict__ A, float2 *__restrict__ Xsave,
                                                      const __nv_bfloat162 *__restrict__ R,
                                                      const float2 *__restrict__ Efwd, const float2 *__restrict__ Einv)
{
    __shared__ float2 as[N][kC];
    __shared__ float2 xs[M][kC];
    __shared__ float2 ys[M][kC];
    __shared__ float2 ef[M][N];
    __shared__ float2 ei[N][M];
    constexpr int K = M * M * M, COLS = M * M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = blockIdx.x;
    for (int e = threadIdx.x; e < M * N; e += 256) {
        ef[e / N][e % N] = Efwd[e];
        ei[e / M][e % M] = Einv[e];
    }
    const float inv_n = 1.f / N;
    const int b = blockIdx.y;
    __syncthreads();
    for (int e = threadIdx.x; e < N * kC; e += 256) {
        const int z = e / kC, c = e % kC;
        as[z][c] = A[(((size_t)b * N + z) * COLS + col) * kC + c];
    }
    __syncthreads();
    for (int kz = warp; kz < M; kz += 8) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 8
        for (int z = 0; z < N; ++z) {
            const float2 m = ef[kz][z], x = as[z][lane];
            acc.x = fmaf(m.x, x.x, fmaf(-m.y, x.y, acc.x));
            acc.y = fmaf(m.x, x.y, fmaf(m.y, x.x, acc.y));
        }
        xs[kz][lane] = acc;
        if (Xsave) Xsave[((size_t)b * K + (size_t)kz * COLS + col) * kC + lane] = acc;
    }
    __syncthreads();
    for (int kz = warp; kz < M; kz += 8) {
        const __nv_bfloat162 *Rk = R + ((size_t)kz * COLS + col) * kC * kC;
        float2 y = make_float2(0.f, 0.f);
#pragma unroll 8
        for (int i = 0; i < kC; ++i) {
            const float2 r = __bfloat1622float2(Rk[i * kC + lane]);
            const float2 x = xs[kz][i];
            y.x = fmaf(r.x, x.x, fmaf(-r.y, x.y, y.x));
            y.y = fmaf(r.x, x.y, fmaf(r.y, x.x, y.y));
        }
        ys[kz][lane] = y;
    }
    __syncthreads();
    for (int z = warp; z < N; z += 8) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int kz = 0; kz < M; ++kz) {
            const float2 m = ei[z][kz], y = ys[kz][lane];
            acc.x = fmaf(m.x, y.x, fmaf(-m.y, y.y, acc.x));
            acc.y = fmaf(m.x, y.y, fmaf(m.y, y.x, acc.y));
        }
        A[(((size_t)b * N + z) * COLS + col) * kC + lane] = make_float2(acc.x * inv_n, acc.y * inv_n);
    }
}

// Column sums of the per-block partials in FP64, in a fixed order: a block takes 32 consecutive
// entries; its 8 warps each sum the partials b = w, w + 8, ... of those entries (lanes over the
// entries, so every load is coalesced), and the 8 warp sums are added in warp order.
__global__ void __launch_bounds__(256) reduce_partials_kernel(const float *__restrict__ part, int seg, int nblk,
                                                             float *__restrict__ dst, int ndst,
                                                             double *__restrict__ extra)
{
    __shared__ double ws[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (e < seg) {
#pragma unroll 4
        for (int b = warp; b < nblk; b += 8) s += (double)part[(size_t)b * seg + e];
    }
    ws[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && e < seg) {
        double t = ws[0][lane];
#pragma unroll
        for (int w = 1; w < 8; ++w) t += ws[w][lane];
        if (e < ndst)
            dst[e] = (float)t;
        else
            extra[e - ndst] = t;
    }
}

__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, __nv_bfloat16 *__restrict__ w, size_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = pi;
        w[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void mirror_kernel(const float *__restrict__ p, __nv_bfloat16 *__restrict__ w, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        w[i] = __float2bfloat16_rn(p[i]);
}

__global__ void __launch_bounds__(256) diff_norms_kernel(const float2 *__restrict__ a, const float2 *__restrict__ b,
                                                        size_t n, double *partials, unsigned int *counter,
                                                        double *out)
{
    double v[2] = {0.0, 0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 x = a[i], y = b[i];
        const double dx = (double)x.x - y.x, dy = (double)x.y - y.y;
        v[0] += dx * dx + dy * dy;
        v[1] += (double)y.x * y.x + (double)y.y * y.y;
    }
    grid_reduce<2, 256>(v, 0, partials, counter, out);
}

}  // namespace

template <int NIN>
cudaError_t axis_nin(int MT, const float2 *in, float2 *out, const float2 *mat, int Mout, int O, int I, float scale,
                     cudaStream_t st)
{
    switch (MT) {
        case 1: return axis_run<NIN, 1>(in, out, mat, Mout, O, I, scale, st);
        case 2: return axis_run<NIN, 2>(in, out, mat, Mout, O, I, scale, st);
        case 4: return axis_run<NIN, 4>(in, out, mat, Mout, O, I, scale, st);
        case 8: return axis_run<NIN, 8>(in, out, mat, Mout, O, I, scale, st);
        default: return axis_run<NIN, 16>(in, out, mat, Mout, O, I, scale, st);
    }
}

// Outputs per thread: as many as keep about 128 K threads in flight (the
// contractions are short; latency, not arithmetic, bounds them), at most 16.
int pick_mt(int Mout, long long OI)
{
    int mt = 16;
    while (mt > 1 && (Mout % mt != 0 || OI * (Mout / mt) < (128ll << 10))) mt >>= 1;
    return mt;
}

cudaError_t launch_axis_any(const float2 *in, float2 *out, const float2 *mat, int nin, int Mout, int O, int I,
                            float scale, cudaStream_t st)
{
    const int mt = pick_mt(Mout, (long long)O * I);
    switch (nin) {
        case 64: return axis_nin<64>(mt, in, out, mat, Mout, O, I, scale, st);
        case 32: return axis_nin<32>(mt, in, out, mat, Mout, O, I, scale, st);
        case 16: return axis_nin<16>(mt, in, out, mat, Mout, O, I, scale, st);
        case 8: return axis_nin<8>(mt, in, out, mat, Mout, O, I, scale, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_axis(const float2 *in, float2 *out, const float2 *mat, int n, int M, bool fwd, int O, int I,
                        float scale, cudaStream_t st)
{
    return launch_axis_any(in, out, mat, fwd ? n : M, fwd ? M : n, O, I, scale, st);
}

cudaError_t launch_zmix_fwd(int n, int M, float2 *A, float2 *Xsave, const __nv_bfloat16 *R, const float2 *Efwd,
                            const float2 *Einv, int B, cudaStream_t st)
{
    const __nv_bfloat162 *R2 = (const __nv_bfloat162 *)R;
    if (n == 64 && M == 16) zmix_fwd_kernel<64, 16><<<dim3(M * M, B), 256, 0, st>>>(A, Xsave, R2, Efwd, Einv);
    else if (n == 64 && M == 8) zmix_fwd_kernel<64, 8><<<dim3(M * M, B), 256, 0, st>>>(A, Xsave, R2, Efwd, Einv);
    else if (n == 32 && M == 16) zmix_fwd_kernel<32, 16><<<dim3(M * M, B), 256, 0, st>>>(A, Xsave, R2, Efwd, Einv);
    else if (n == 32 && M == 8) zmix_fwd_kernel<32, 8><<<dim3(M * M, B), 256, 0, st>>>(A, Xsave, R2, Efwd, Einv);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_mix_fwd(int M, const float2 *X, float2 *Y, const __nv_bfloat16 *R, int B, cudaStream_t st)
{
    const int K = M * M * M;
    mix_fwd_kernel<<<K / 8, 256, 0, st>>>(X, Y, (const __nv_bfloat162 *)R, K, B);
    return cudaGetLastError();
}

cudaError_t launch_mix_bwd(int M, const float2 *Ybar, const float2 *X, float2 *Xbar, const __nv_bfloat16 *R,
                           float *gradR, int B, cudaStream_t st)
{
    const int K = M * M * M;
    mix_bwd_kernel<<<K / 8, 256, 0, st>>>(Ybar, X, Xbar, (const __nv_bfloat162 *)R, (float2 *)gradR, K, B);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const float *partials, int seg, int nblk, float *dst, int ndst, double *extra,
                                   cudaStream_t st)
{
    reduce_partials_kernel<<<(seg + 31) / 32, 256, 0, st>>>(partials, seg, nblk, dst, ndst, extra);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, float *m, float *v, const float *g, __nv_bfloat16 *w, size_t n, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t st)
{
    adam_kernel<<<152 * 8, 256, 0, st>>>(p, m, v, g, w, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_mirror(const float *p, __nv_bfloat16 *w, size_t n, cudaStream_t st)
{
    mirror_kernel<<<152 * 8, 256, 0, st>>>(p, w, n);
    return cudaGetLastError();
}

cudaError_t launch_diff_norms(const float2 *a, const float2 *b, size_t n, double *partials, unsigned int *counter,
                              double *out, cudaStream_t st)
{
    diff_norms_kernel<<<kDiffBlocks, 256, 0, st>>>(a, b, n, partials, counter, out);
    return cudaGetLastError();
}

}  // namespace fno
}  // namespace spe
