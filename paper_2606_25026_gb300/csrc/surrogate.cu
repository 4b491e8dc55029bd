// The judge of the FNO surrogate (include/spe_fno.h): propose psi K steps
// ahead, check the proposal's mass and energy drift (and, when asked, its
// error against the solver's own K steps), and fall back to the solver when a
// check fails.  Built from the public solver API and the network's API.
//
// The coarse step, the network and the proposal's energy run on a private
// stream (the coarse grid's), so the energy of the current state, computed on
// the grid's stream, overlaps them; the coarse grid steps without host syncs.
#include <cuda_runtime.h>

#include <cmath>
#include <new>

#include "fno_internal.cuh"
#include "spe_fno.h"

using namespace spe::fno;

struct spe_surrogate {
    spe_config gcfg;
    spe_fno *f;
    spe_judge_config jc;
    spe_grid *coarse;
    float2 *psi0, *psib, *prop;
    double *partials, *out;
    unsigned int *counter;
    size_t ncells;
    cudaStream_t st;      // the grids' stream (grid_cfg.cuda_stream)
    cudaStream_t own;     // private stream of the coarse grid and the network
    cudaEvent_t ready;
};

namespace {

void release(spe_surrogate *s)
{
    if (s->coarse) spe_destroy(s->coarse);
    cudaFree(s->psi0);
    cudaFree(s->psib);
    cudaFree(s->prop);
    cudaFree(s->partials);
    cudaFree(s->out);
    cudaFree(s->counter);
    if (s->ready) cudaEventDestroy(s->ready);
    if (s->own) cudaStreamDestroy(s->own);
}

}  // namespace

extern "C" {

SPE_API int spe_surrogate_create(const spe_config *grid_cfg, spe_fno *f, const spe_judge_config *jc,
                                 spe_surrogate **out)
{
    if (!grid_cfg || !f || !jc || !out) return SPE_EINVAL;
    *out = nullptr;
    const int nf = net_n(f);
    if (grid_cfg->nx != nf || grid_cfg->ny != nf || grid_cfg->nz != nf) return SPE_EINVAL;
    spe_surrogate *s = new (std::nothrow) spe_surrogate();
    if (!s) return SPE_ENOMEM;
    s->gcfg = *grid_cfg;
    s->f = f;
    s->jc = *jc;
    s->st = (cudaStream_t)grid_cfg->cuda_stream;
    s->ncells = (size_t)grid_cfg->nx * grid_cfg->ny * grid_cfg->nz;
    int rc = SPE_OK;
    if (cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ready, cudaEventDisableTiming) != cudaSuccess)
        rc = SPE_ECUDA;
    spe_config cc = *grid_cfg;
    cc.flags |= SPE_NO_CFL_CHECK | SPE_ASYNC;
    cc.max_particles = 0;
    cc.cuda_stream = s->own;
    if (rc == SPE_OK) rc = spe_create_grid(&cc, nullptr, 0, &s->coarse);
    cudaError_t e = cudaSuccess;
    if (rc == SPE_OK) {
        e = cudaMalloc(&s->psi0, s->ncells * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&s->psib, s->ncells * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&s->prop, s->ncells * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&s->partials, kDiffBlocks * 2 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&s->out, 2 * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&s->counter, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(s->counter, 0, sizeof(unsigned int));
        if (e != cudaSuccess) rc = (e == cudaErrorMemoryAllocation) ? SPE_ENOMEM : SPE_ECUDA;
    }
    if (rc != SPE_OK) {
        release(s);
        delete s;
        return rc;
    }
    *out = s;
    return SPE_OK;
}

SPE_API int spe_surrogate_destroy(spe_surrogate *s)
{
    if (!s) return SPE_EINVAL;
    cudaStreamSynchronize(s->st);
    release(s);
    delete s;
    return SPE_OK;
}

SPE_API int spe_surrogate_advance(spe_surrogate *s, spe_grid *g, int K, double dt, int spot_check,
                                  spe_judge_result *out)
{
    if (!s || !g || !out || K < 1 || !std::isfinite(dt)) return SPE_EINVAL;
    size_t np = 0;
    int rc = spe_particle_count(g, &np);
    if (rc) return rc;
    if (np) return SPE_EINVAL;
    spe_judge_result r{};
    r.rel_l2 = -1.0;
    // 1. the state, handed to the private stream
    if ((rc = spe_get_psi(g, s->psi0, SPE_DEVICE))) return rc;
    if (cudaEventRecord(s->ready, s->st) != cudaSuccess || cudaStreamWaitEvent(s->own, s->ready, 0) != cudaSuccess)
        return SPE_ECUDA;
    // 2. the coarse step and the proposal (private stream, no host sync)
    if ((rc = spe_set_ic(s->coarse, s->psi0, s->ncells, SPE_DEVICE))) return rc;
    if ((rc = spe_step(s->coarse, 1, K * dt))) return rc;
    if ((rc = spe_get_psi(s->coarse, s->psib, SPE_DEVICE))) return rc;
    if ((rc = forward_on_stream(s->f, s->own, s->psi0, s->psib, s->prop, 1))) return rc;
    if ((rc = spe_set_ic(s->coarse, s->prop, s->ncells, SPE_DEVICE))) return rc;
    // 3. the state's energy on the grid's stream meanwhile, then the proposal's
    spe_energy_t e0{}, e1{};
    if ((rc = spe_energy(g, &e0))) return rc;
    if ((rc = spe_energy(s->coarse, &e1))) return rc;
    if ((rc = spe_fno_sync(s->f))) return rc;
    r.mass_drift = std::fabs(e1.mass - e0.mass) / std::fabs(e0.mass);
    r.energy_drift = std::fabs(e1.total - e0.total) / std::fabs(e0.total);
    const bool drift_ok = std::isfinite(r.mass_drift) && std::isfinite(r.energy_drift) &&
                          r.mass_drift <= s->jc.max_mass_drift && r.energy_drift <= s->jc.max_energy_drift;
    // 4. spot check or accept / fall back
    if (spot_check) {
        if ((rc = spe_step(g, K, dt))) return rc;
        if ((rc = spe_get_psi(g, s->psib, SPE_DEVICE))) return rc;
        if ((rc = spe_sync(g))) return rc;
        cudaError_t e = launch_diff_norms(s->prop, s->psib, s->ncells, s->partials, s->counter, s->out, s->st);
        double h[2] = {0.0, 0.0};
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, s->out, sizeof(h), cudaMemcpyDeviceToHost, s->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
        if (e != cudaSuccess) return SPE_ECUDA;
        r.rel_l2 = std::sqrt(h[0] / h[1]);
        r.spot_checked = 1;
        r.accepted = drift_ok && std::isfinite(r.rel_l2) && r.rel_l2 <= s->jc.max_rel_l2;
        r.used_proposal = 0;
    } else if (drift_ok) {
        if ((rc = spe_set_ic(g, s->prop, s->ncells, SPE_DEVICE))) return rc;
        if ((rc = spe_sync(g))) return rc;
        r.accepted = 1;
        r.used_proposal = 1;
    } else {
        if ((rc = spe_step(g, K, dt))) return rc;
        r.accepted = 0;
    }
    *out = r;
    return SPE_OK;
}

}  // extern "C"
