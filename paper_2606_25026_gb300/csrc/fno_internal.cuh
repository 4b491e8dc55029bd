// Internal interface of the Fourier-neural-operator surrogate kernels.
//
// Layout conventions (B = batch, n = grid points per axis, C = 32 channels,
// M = kept modes per axis; a "row" is one (b, z, y) line of n cells):
//   activations  v_l, u_l        [B][z][y][x][C]  float or bf16 (channel fastest)
//   x-row buffer                 [B][z][y][kx][C] complex float (kx < M): the
//                                x-stage DFT of a row and, in place, the spectral
//                                input of the next row kernel
//   y-stage buffer               [B][z][ky][kx][C] complex float
//   modes X_l, Y                 [B][kz][ky][kx][C] complex float
//   ubar (cotangent of u)        [B][z][y][x][C]  float
// Tables (FP64-computed, stored as float2):
//   Efwd [M][n] = e^{-2 pi i f(m) j / n},   Einv [n][M] = e^{+2 pi i f(m) j / n}
//   Fx   [M][n] = e^{-2 pi i kx x / n},     Gx   [n][M] = w(kx) e^{+2 pi i kx x / n} / n,
//   w(0) = 1, w(kx > 0) = 2, f(m) = m for m < M/2 and m - M otherwise.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "spe.h"

#include <cstddef>

namespace spe {
namespace fno {

constexpr int kC = 32;               // channels (one per lane)
constexpr int kH = 64;               // projection hidden width
constexpr int kFin = 4;              // feature channels
constexpr int kFout = 2;             // output channels (re, im)
constexpr int kRowThreads = 256;     // 8 warps per row block
constexpr int kRowWarps = kRowThreads / 32;
// Row kernels run a fixed grid that loops over rows, so every block's partial
// weight-gradient sums, and their fixed-order reduction, do not depend on
// scheduling: 2 blocks per SM on 152 SMs.
constexpr int kRowBlocks = 304;
constexpr int kTableN = 64;          // largest n with x tables in constant memory
constexpr int kTableM = 16;          // largest M

constexpr int kTopSeg = kH * kC + kH + kFout * kH + kFout + 1;   // Q1, q1, Q2, q2, loss
constexpr int kLayerSeg = kC * kC + kC;                           // W, b
constexpr int kLiftSeg = kC * kFin + kC;                          // P, p

struct Offsets {
    size_t P, p, W[8], b[8], R[8], Q1, q1, Q2, q2, total;
};

struct RowArgs {
    int rows;                       // B * n * n
    int store_u;                    // forward: keep u_l
    const float2 *psi, *psib, *target;
    float2 *out;                    // proposal (last forward layer)
    const void *vin;                // v_l (forward), v_{l-1} (backward), v_L (top)
    void *vout, *uout;              // forward outputs
    const void *upre;               // backward: u_{l-1}
    float2 *xrow;                   // in/out, in place per row
    float *ubar;                    // in/out, in place per row
    const __nv_bfloat16 *w;         // BF16 parameter mirror
    size_t oW, ob, oP, op, oQ1, oq1, oQ2, oq2;
    float inv_A, sigma, loss_scale;
    float *partials;                // [gridDim.x][segment]
    int *status;                    // device status word (tensor-core wait timeouts)
    const uint4 *tcG, *tcF;         // BF16 operand images of G' [n][2M] and F' [2M][n] (K-major)
    const uint4 *tcFt, *tcGt;       // backward images: F'' [n][2M] = (Re Fx, Im Fx) and G'' [2M][n] = (Re Gx, -Im Gx)
};

// forward row kernels (fno_fwd.cu)
cudaError_t upload_fwd_tables(const float2 *G64, const float2 *F64, const float2 *G32, const float2 *F32);
cudaError_t launch_lift_fwd(int n, int M, bool fp32, const RowArgs &a, int grid, cudaStream_t st);
cudaError_t launch_layer_fwd(int n, int M, bool fp32, bool last, const RowArgs &a, int grid, cudaStream_t st);

// backward row kernels (fno_bwd.cu)
cudaError_t upload_bwd_tables(const float2 *G64, const float2 *F64, const float2 *G32, const float2 *F32);
cudaError_t launch_top_bwd(int n, bool fp32, const RowArgs &a, int grid, cudaStream_t st);
cudaError_t launch_grad_start(int n, int M, bool fp32, const RowArgs &a, int grid, cudaStream_t st);
cudaError_t launch_layer_bwd(int n, int M, bool fp32, const RowArgs &a, int grid, cudaStream_t st);
cudaError_t launch_lift_bwd(int n, int M, bool fp32, const RowArgs &a, int grid, cudaStream_t st);

// tensor-core forward kernels, BF16 activations (fno_tc.cu)
// mode: 0 = Fourier layer, 1 = last Fourier layer (no GELU, no next x DFT), 2 = lift
constexpr int kTcTile = 4;          // rows per tensor-core tile
constexpr int kTcBlocks = 456;      // 3 CTAs per SM (about 66 KB of shared memory each)
constexpr int kProjBlocks = 1216;   // up to 8 CTAs per SM
cudaError_t launch_layer_fwd_tc(int n, int M, int mode, const RowArgs &a, int grid, cudaStream_t st);
cudaError_t launch_proj_tc(const RowArgs &a, int cells, int grid, cudaStream_t st);

// tensor-core backward row kernels, BF16 activations (fno_tc_bwd.cu); grid <= rows / kTcTile CTAs,
// each writing one partial segment (kLayerSeg, or kLiftSeg for the lift)
constexpr int kTcBwdLayer = 0;      // v bar, u bar_{l-1}, Bbar_{l-1}, dL/dW_{l-1}, dL/db_{l-1}
constexpr int kTcBwdStart = 1;      // Bbar_{L-1}, dL/dW_{L-1}, dL/db_{L-1} from the given u bar_{L-1}
constexpr int kTcBwdLift = 2;       // v bar_0, dL/dP, dL/dp
cudaError_t launch_layer_bwd_tc(int n, int M, int mode, const RowArgs &a, int grid, cudaStream_t st);
// projection backward (top of the backward pass): u bar of the last layer, dL/dQ1, dL/dq1, dL/dQ2,
// dL/dq2 and the loss; cells a multiple of 128, grid <= cells / 128, one kTopSeg partial per CTA
cudaError_t launch_proj_bwd_tc(const RowArgs &a, int cells, int grid, cudaStream_t st);

// mode-space and elementwise kernels (fno_modes.cu)
// out[o][m][i] = scale * sum_j Mat[m][j] in[o][j][i] with Mat = Efwd [M][n]
// (fwd: j < n, m < M) or Einv [n][M] (j < M, m < n); I a multiple of 64
cudaError_t launch_axis(const float2 *in, float2 *out, const float2 *mat, int n, int M, bool fwd, int O, int I,
                        float scale, cudaStream_t st);
// fused z DFT + mixing + z inverse of one layer, in place over the y-stage buffer
cudaError_t launch_zmix_fwd(int n, int M, float2 *A, float2 *Xsave, const __nv_bfloat16 *R, const float2 *Efwd,
                            const float2 *Einv, int B, cudaStream_t st);
cudaError_t launch_mix_fwd(int M, const float2 *X, float2 *Y, const __nv_bfloat16 *R, int B, cudaStream_t st);
cudaError_t launch_mix_bwd(int M, const float2 *Ybar, const float2 *X, float2 *Xbar, const __nv_bfloat16 *R,
                           float *gradR, int B, cudaStream_t st);
cudaError_t launch_reduce_partials(const float *partials, int seg, int nblk, float *dst, int ndst, double *extra,
                                   cudaStream_t st);
cudaError_t launch_adam(float *p, float *m, float *v, const float *g, __nv_bfloat16 *w, size_t n, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t st);
cudaError_t launch_mirror(const float *p, __nv_bfloat16 *w, size_t n, cudaStream_t st);
// out[0] = sum |a - b|^2, out[1] = sum |b|^2 (FP64, deterministic)
cudaError_t launch_diff_norms(const float2 *a, const float2 *b, size_t n, double *partials, unsigned int *counter,
                              double *out, cudaStream_t st);
constexpr int kDiffBlocks = 304;

}  // namespace fno
}  // namespace spe

struct spe_fno;

namespace spe {
namespace fno {

// spe_fno_forward issued as direct launches on another stream, never as a graph
// replay (for use inside a stream capture)
int forward_direct(spe_fno *f, cudaStream_t st, const void *psi, const void *psi_b, void *psi_out, int batch);

// grid points per axis and stream of a network (fno.cu)
int net_n(const spe_fno *f);
cudaStream_t net_stream(const spe_fno *f);
// spe_fno_forward issued on another stream (the caller serialises use of f)
int forward_on_stream(spe_fno *f, cudaStream_t st, const void *psi, const void *psi_b, void *psi_out, int batch);

}  // namespace fno
}  // namespace spe

namespace spe {

// solver internals the judge uses (api.cu)
constexpr int kEnergyRaw = 18;   // raw energy sums copied per spe_energy
int energy_issue(spe_grid *g, double *host_raw, bool copy_to_host);
// apply the grid's deferred closing half kick, if any (spe_settle)
int settle(spe_grid *g);
int energy_from_raw(spe_grid *g, const double *raw, spe_energy_t *out);
float2 *grid_psi(spe_grid *g);
cudaStream_t grid_stream(spe_grid *g);

}  // namespace spe
