/*
 * libspe surrogate -- a Fourier neural operator (FNO) that proposes psi K steps
 * ahead, trained on trajectories of the solver in spe.h, and the judge that
 * accepts or rejects each proposal against that solver.
 *
 * None of this has a counterpart in the paper (Meng & Dong 2026); the paper's
 * split-step method (spe.h) stays the reference and the fallback.  The network:
 *
 *   features  f = (Re psi, Im psi, Re psi_b, Im psi_b) * inv_A   (4 channels)
 *             psi_b = one solver step of length K dt from psi (the coarse step)
 *   lift      v_0 = P f + p                                         (4 -> C)
 *   layer l   u_l = W_l v_l + b_l + Re IDFT[ R_l . DFT_M(v_l) ]
 *             v_{l+1} = GELU(u_l) for l < L-1, v_L = u_{L-1}
 *   project   o = Q2 GELU(Q1 v_L + q1) + q2                       (C -> H -> 2)
 *   proposal  psi_pred = psi_b + sigma (o_0 + i o_1)
 *
 * C = 32 channels, H = 64, GELU the exact erf form.  DFT_M keeps the mode box
 * kx in [0, M) (x is the half-spectrum axis), ky, kz in [-M/2, M/2); the
 * forward DFT is unnormalised, the inverse carries 1/n^3 and is the real
 * inverse of the half spectrum (the imaginary part of a kx = 0 term is
 * dropped after the z and y inverses).
 *
 * Parameters are one flat float vector, in this order:
 *   P [C][4], p [C],
 *   per layer l: W_l [C][C] (row = output channel), b_l [C],
 *                R_l [M^3][C_in][C_out][2]  (re, im; mode k = (kz*M + ky)*M + kx,
 *                signed frequency m for m < M/2 and m - M otherwise),
 *   Q1 [H][C], q1 [H], Q2 [2][H], q2 [2].
 * The library keeps an FP32 master copy (Adam updates it) and a BF16 mirror;
 * every kernel reads the BF16 weights and accumulates in FP32.  Activations
 * are stored in BF16 (default) or FP32 (SPE_FNO_ACT_FP32).  With BF16
 * activations the forward pass runs its dense row stages (W v, the real x
 * inverse, the next x DFT, the projection) on the tensor cores with BF16
 * operands (the DFT tables and the spectral inputs rounded to BF16); with FP32
 * activations every stage runs on the CUDA cores in FP32.
 *
 * Batch loss (spe_fno_backward):  sum_b sum_cells |psi_pred - psi_target|^2
 *                                 / (sigma^2 B n^3).
 *
 * Field pointers are DEVICE pointers on the network's device, complex64
 * [batch][n][n][n] (z, y, x; x fastest), borrowed for the call.  All device
 * work is ordered on cfg.cuda_stream.  Every entry point returns SPE_OK or a
 * negative status from spe.h.
 */
#ifndef SPE_FNO_H
#define SPE_FNO_H

#include "spe.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SPE_FNO_WIDTH   32
#define SPE_FNO_HIDDEN  64

/* flags of spe_fno_config */
#define SPE_FNO_TRAIN     (1 << 0)  /* keep activations for spe_fno_backward */
#define SPE_FNO_ACT_FP32  (1 << 1)  /* store activations in FP32 instead of BF16 */
#define SPE_FNO_NO_GRAPH  (1 << 2)  /* never replay the inference forward as a CUDA graph */
#define SPE_FNO_PROFILE   (1 << 3)  /* CUDA events around every kernel (no graph replay) */

typedef struct spe_fno spe_fno;

typedef struct {
    int n;             /* grid points per axis: 32 or 64 */
    int layers;        /* L, 1..8 */
    int modes;         /* M, 8 or 16, M <= n/2 */
    int max_batch;     /* largest batch of a forward / backward call, 1..256 */
    int flags;         /* SPE_FNO_* */
    double inv_A;      /* feature scale 1/A (A: the field's rms amplitude) */
    double sigma;      /* output scale of the correction */
    void *cuda_stream; /* cudaStream_t, NULL = legacy default stream */
} spe_fno_config;

/* Number of floats in the flat parameter vector of this configuration.
 * Host only.  SPE_EINVAL for an unsupported configuration. */
SPE_API int spe_fno_param_count(const spe_fno_config *cfg, size_t *count);

/* Allocate a network (parameters zero, Adam state zero) and its activation
 * buffers for cfg->max_batch samples.  SPE_ENOMEM if device memory runs out. */
SPE_API int spe_fno_create(const spe_fno_config *cfg, spe_fno **out);
SPE_API int spe_fno_destroy(spe_fno *f);

/* Copy the flat FP32 parameter vector in (refreshing the BF16 mirror) or out.
 * count must equal spe_fno_param_count; where = SPE_HOST or SPE_DEVICE. */
SPE_API int spe_fno_set_params(spe_fno *f, const float *params, size_t count, int where);
SPE_API int spe_fno_get_params(spe_fno *f, float *params, size_t count, int where);

/* Gradient of the last spe_fno_backward, same layout as the parameters. */
SPE_API int spe_fno_get_grads(spe_fno *f, float *grads, size_t count, int where);

/* psi_out[b] = the proposal for (psi[b], psi_b[b]), b < batch.  psi_out may be
 * psi_b (in place).  With SPE_FNO_TRAIN the activations are kept for
 * spe_fno_backward.  Asynchronous on the stream.  SPE_EINVAL if batch is out
 * of [1, max_batch].  Without SPE_FNO_TRAIN a call that repeats the previous
 * call's buffers, batch and stream is captured once as a CUDA graph and
 * replayed (results are bitwise the same; parameter updates need no
 * re-capture since the kernels read the weights in place). */
SPE_API int spe_fno_forward(spe_fno *f, const void *psi, const void *psi_b, void *psi_out, int batch);

/* Gradient of the batch loss of the last forward against psi_target
 * ([batch][n^3] complex64, device) into the gradient buffer (overwritten), and
 * the loss into *loss_out if loss_out is not NULL (this synchronises the
 * stream).  The psi and psi_b buffers of that forward must still hold its
 * inputs.  SPE_ESTATE without SPE_FNO_TRAIN, without a forward before it, or
 * after an in-place forward (psi_out == psi_b). */
SPE_API int spe_fno_backward(spe_fno *f, const void *psi_target, double *loss_out);

/* One Adam step (Kingma & Ba 2015) on the FP32 master with the current
 * gradient, then refresh the BF16 mirror.  Asynchronous. */
SPE_API int spe_fno_adam(spe_fno *f, double lr, double beta1, double beta2, double eps);

/* Synchronise the network's stream; SPE_ETIMEOUT if a bounded device-side wait
 * of a tensor-core kernel gave up since the last call (the affected results
 * are wrong; the flag is cleared). */
SPE_API int spe_fno_sync(spe_fno *f);

/* With SPE_FNO_PROFILE: per kernel kind, the launches and summed CUDA-event
 * milliseconds since the last call (then reset).  Fills up to cap entries of
 * names / launches / ms and returns the number of kinds (>= 0), or a negative
 * status (SPE_ESTATE without the flag).  Synchronises the stream. */
SPE_API int spe_fno_profile_read(spe_fno *f, const char **names, unsigned long long *launches, double *ms, int cap);

/* Kernels launched by this network since creation (or the last reset). */
SPE_API int spe_fno_launch_count(spe_fno *f, unsigned long long *count_out, int reset);

/* ---- the judge ------------------------------------------------------------
 * spe_surrogate_advance moves a grid K steps of dt, by the network's proposal
 * if the judge accepts it, else by the solver:
 *   1. psi_b = one solver step of length K dt from the grid's psi (on a private
 *      coarse grid with the CFL check off);
 *   2. the proposal from the network;
 *   3. mass drift |M(prop) - M(psi)| / M(psi) and energy drift
 *      |E(prop) - E(psi)| / |E(psi)| (spe_energy's total);
 *   4. if spot_check: the solver runs the K steps on the grid and the relative
 *      L2 error of the proposal against it is measured; the grid keeps the
 *      solver's result and accepted reports the verdict;
 *      else: if both drifts are within limits the grid takes the proposal,
 *      otherwise the solver runs the K steps (fallback).
 * Grids with star particles are not supported (SPE_EINVAL): the network sees
 * psi only.  The grid's n must equal the network's n on every axis. */
typedef struct {
    double max_mass_drift;
    double max_energy_drift;
    double max_rel_l2;
} spe_judge_config;

typedef struct {
    int accepted;          /* 1 if the proposal passed every check made */
    int spot_checked;      /* 1 if the solver rollout was run and compared */
    int used_proposal;     /* 1 if the grid now holds the proposal */
    double mass_drift;
    double energy_drift;
    double rel_l2;         /* -1 when not spot-checked */
} spe_judge_result;

typedef struct spe_surrogate spe_surrogate;

/* Bind a network to grids of configuration grid_cfg (its coarse grid and
 * scratch are allocated here).  The network must outlive the surrogate. */
SPE_API int spe_surrogate_create(const spe_config *grid_cfg, spe_fno *f, const spe_judge_config *jc,
                                 spe_surrogate **out);
SPE_API int spe_surrogate_destroy(spe_surrogate *s);
SPE_API int spe_surrogate_advance(spe_surrogate *s, spe_grid *g, int K, double dt, int spot_check,
                                  spe_judge_result *out);

/* Kernels the surrogate's advances ran (the network's, the coarse grid's and
 * the kernels they launched on the caller's grid; CUDA-graph nodes counted per
 * replay) since creation or the last reset. */
SPE_API int spe_surrogate_launch_count(spe_surrogate *s, unsigned long long *count_out, int reset);

#ifdef __cplusplus
}
#endif
#endif
