// The judge of the FNO surrogate (include/spe_fno.h): propose psi K steps
// ahead, check the proposal's mass and energy drift (and, when asked, its
// error against the solver's own K steps), and fall back to the solver when a
// check fails.  Built from the public solver API and the network's API.
//
// The coarse step, the network and the proposal's energy run on a private
// stream (the coarse grid's), so the energy of the current state, computed on
// the grid's stream, overlaps them.  That private-stream work is captured as
// one CUDA graph the second time an advance repeats K dt, and replayed after
// (the coarse grid's tables are built by the first, direct advance); the
// proposal's raw energy sums come back through a pinned buffer, so an advance
// has one wait for the private stream.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <vector>

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
    double *h_raw;        // pinned: the proposal's raw energy sums
    double *h_raw0;       // pinned: the state's raw energy sums
    cudaGraphExec_t exec; // the private-stream work of an advance, for key_dt
    double key_dt;
    int seen;
    bool graph_ok;
    unsigned long long graph_kernels;  // kernel nodes of exec
    unsigned long long launches;       // kernels this surrogate ran (graph nodes included)
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
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->own) cudaStreamDestroy(s->own);
    if (s->h_raw) cudaFreeHost(s->h_raw);
    if (s->h_raw0) cudaFreeHost(s->h_raw0);
}

// coarse step of K dt from psi0, the proposal, the proposal's energy kernels and
// the copy of its raw sums to the pinned buffer: all on the private stream, no
// host synchronisation (capturable)
int issue_private(spe_surrogate *s, double kdt)
{
    int rc;
    if ((rc = spe_set_ic(s->coarse, s->psi0, s->ncells, SPE_DEVICE))) return rc;
    if ((rc = spe_step(s->coarse, 1, kdt))) return rc;
    if ((rc = spe::settle(s->coarse))) return rc;
    if (cudaMemcpyAsync(s->psib, spe::grid_psi(s->coarse), s->ncells * sizeof(float2), cudaMemcpyDeviceToDevice,
                        s->own) != cudaSuccess)
        return SPE_ECUDA;
    if ((rc = forward_direct(s->f, s->own, s->psi0, s->psib, s->prop, 1))) return rc;
    if ((rc = spe_set_ic(s->coarse, s->prop, s->ncells, SPE_DEVICE))) return rc;
    return spe::energy_issue(s->coarse, s->h_raw, true);
}

int capture_private(spe_surrogate *s, double kdt)
{
    if (s->exec) {
        cudaGraphExecDestroy(s->exec);
        s->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s->own, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SPE_ECUDA;
    int rc = issue_private(s, kdt);
    const cudaError_t ec = cudaStreamEndCapture(s->own, &graph);
    if (rc == SPE_OK && ec != cudaSuccess) rc = SPE_ECUDA;
    if (rc == SPE_OK && cudaGraphInstantiate(&s->exec, graph, 0) != cudaSuccess) {
        s->exec = nullptr;
        rc = SPE_ECUDA;
    }
    s->graph_kernels = 0;
    if (graph) {
        size_t n = 0;
        if (cudaGraphGetNodes(graph, nullptr, &n) == cudaSuccess && n) {
            std::vector<cudaGraphNode_t> nodes(n);
            if (cudaGraphGetNodes(graph, nodes.data(), &n) == cudaSuccess)
                for (size_t i = 0; i < n; ++i) {
                    cudaGraphNodeType t;
                    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                        ++s->graph_kernels;
                }
        }
        cudaGraphDestroy(graph);
    }
    cudaGetLastError();
    return rc;
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
    cc.flags &= ~SPE_PROFILE;
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
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_raw, spe::kEnergyRaw * sizeof(double));
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_raw0, spe::kEnergyRaw * sizeof(double));
        s->graph_ok = true;
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
    unsigned long long g0 = 0, c0 = 0, f0 = 0;
    spe_launch_count(g, &g0, 0);
    spe_launch_count(s->coarse, &c0, 0);
    spe_fno_launch_count(s->f, &f0, 0);
    bool replayed = false;
    // 1. the state (with any closing half kick it still owes), handed to the private stream
    if ((rc = spe::settle(g))) return rc;
    if (cudaMemcpyAsync(s->psi0, spe::grid_psi(g), s->ncells * sizeof(float2), cudaMemcpyDeviceToDevice,
                        spe::grid_stream(g)) != cudaSuccess)
        return SPE_ECUDA;
    if (cudaEventRecord(s->ready, spe::grid_stream(g)) != cudaSuccess ||
        cudaStreamWaitEvent(s->own, s->ready, 0) != cudaSuccess)
        return SPE_ECUDA;
    // 2. coarse step, proposal, the proposal's energy (private stream; a graph replay once K dt repeats)
    const double kdt = K * dt;
    if (s->graph_ok && s->seen >= 1 && s->key_dt == kdt) {
        if (!s->exec && (rc = capture_private(s, kdt))) {
            s->graph_ok = false;          // capture unavailable: stay on direct launches
            if ((rc = issue_private(s, kdt))) return rc;
        } else if (cudaGraphLaunch(s->exec, s->own) != cudaSuccess) {
            return SPE_ECUDA;
        } else {
            replayed = true;
        }
    } else {
        if (s->exec) {
            cudaGraphExecDestroy(s->exec);
            s->exec = nullptr;
        }
        if ((rc = issue_private(s, kdt))) return rc;
        s->key_dt = kdt;
        s->seen = 1;
    }
    // 3. the state's energy on the grid's stream meanwhile; then both sets of raw sums
    spe_energy_t e0{}, e1{};
    if ((rc = spe::energy_issue(g, s->h_raw0, true))) return rc;
    if (cudaStreamSynchronize(spe::grid_stream(g)) != cudaSuccess || cudaStreamSynchronize(s->own) != cudaSuccess)
        return SPE_ECUDA;
    if ((rc = spe::energy_from_raw(g, s->h_raw0, &e0))) return rc;
    if ((rc = spe::energy_from_raw(s->coarse, s->h_raw, &e1))) return rc;
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
    unsigned long long g1 = 0, c1 = 0, f1 = 0;
    spe_launch_count(g, &g1, 0);
    spe_launch_count(s->coarse, &c1, 0);
    spe_fno_launch_count(s->f, &f1, 0);
    // the counters also moved while a graph was captured (its kernels did not run then)
    if (!replayed) s->launches += (g1 - g0) + (c1 - c0) + (f1 - f0);
    else s->launches += (g1 - g0) + s->graph_kernels;
    *out = r;
    return SPE_OK;
}

SPE_API int spe_surrogate_launch_count(spe_surrogate *s, unsigned long long *count_out, int reset)
{
    if (!s || !count_out) return SPE_EINVAL;
    *count_out = s->launches;
    if (reset) s->launches = 0;
    return SPE_OK;
}

}  // extern "C"
