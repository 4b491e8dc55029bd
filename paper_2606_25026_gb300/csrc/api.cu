// libspe C ABI: grid state, workspace layout and the per-step schedule.
//
// Per kick-drift-kick step (Sec. 3.1 Eq. (SPE_solver_KDK), Algorithm 1) the
// device runs, on the grid's stream:
//   1. x pass  : Phi rows from the x half spectrum, kick psi by (Phi +
//                kappa|psi|^2) dt_k / eta, forward x transform of psi  [(a)/(d), (b)]
//   2. stars   : v += g dt_k, x += v dt, CIC deposit                  [Sec. 3.2.2]
//   3. y pass  : forward y transform of psi                           [(b)]
//   4. z pass  : forward z, drift exp(-i eta k^2 dt / 2) / N^3, inverse z  [(b)]
//   5. y pass  : inverse y transform of psi                           [(b)]
//   6. x pass  : inverse x transform, rho = |psi|^2 + rho_*, mass, forward
//                real x transform of rho                               [(b), (c)]
//   7. y pass  : forward y transform of rho_hat                       [(c)]
//   8. z pass  : forward z, * -4 pi G / (k^2 N^3) (k = 0 -> 0), inverse z   [(c)]
//   9. y pass  : inverse y transform                                  [(c)]
// leaving Phi as an x half spectrum that the next step's pass 1 turns into
// real-space Phi.  Within one spe_step call the second half kick of a step
// and the first of the next are one full kick (dt_k = dt); the call starts
// and ends with a half kick (dt_k = dt/2).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <cuda_fp16.h>

#include "spe.h"
#include "fno_internal.cuh"
#include "spe_internal.cuh"

namespace spe {
cudaError_t setup_xpass_attributes();
cudaError_t setup_spass_attributes();

bool supported_n(int n)
{
    switch (n) {
#define X(v) case v:
        SPE_FOR_EACH_N(X)
#undef X
        return true;
    default: return false;
    }
}

cudaError_t setup_kernel_attributes()
{
    cudaError_t e = setup_xpass_attributes();
    if (e == cudaSuccess) e = setup_spass_attributes();
    return e;
}
}  // namespace spe

using namespace spe;

namespace {

const double kPi = 3.14159265358979323846264338327950288;

enum Kind {
    KIND_X_KICK_FFT = 0,
    KIND_X_IFFT_DENSITY,
    KIND_Y_PSI,
    KIND_Z_DRIFT,
    KIND_Y_RHO,
    KIND_Z_POISSON,
    KIND_PARTICLES,
    KIND_X_KICK_FINAL,
    KIND_X_POTENTIAL,
    KIND_DIAG,
    KIND_COPY,
    KIND_SORT,
    KIND_COUNT
};

const char *kKindNames[KIND_COUNT] = {
    "x_kick_fwd", "x_inv_density_r2c", "y_fft_psi", "z_fft_drift", "y_fft_rho", "z_fft_poisson",
    "particles_kdk_deposit", "x_kick_final", "x_potential", "diagnostics", "layout_copy", "particles_sort",
};

struct ProfRec {
    int kind;
    cudaEvent_t e0, e1;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t psi, phik, phi, phib, dep, dflag, part, bins, tw, k2, drift, absorb, tcw, partials, counter, diag, status,
        total;
};

int compute_layout(const spe_config *c, Layout *L, int *W, int *P)
{
    if (!c) return SPE_EINVAL;
    if (!supported_n(c->nx) || !supported_n(c->ny) || !supported_n(c->nz)) return SPE_EINVAL;
    if (!(c->Lx > 0) || !(c->Ly > 0) || !(c->Lz > 0) || !(c->hbar_over_m > 0)) return SPE_EINVAL;
    if (!isfinite(c->G) || !isfinite(c->kappa)) return SPE_EINVAL;
    if (!isfinite(c->absorb_alpha) || c->absorb_alpha < 0 || (c->absorb_alpha > 0 && c->absorb_nb <= 0))
        return SPE_EINVAL;
    if (c->max_particles > (size_t)0x7fffffff) return SPE_EINVAL;
    const size_t ncells = (size_t)c->nx * c->ny * c->nz;
    const int w = c->nx / 2 + 1;
    const int p = (w + 3) & ~3;
    size_t off = 0;
    L->psi = off;      off = align256(off + ncells * sizeof(float2));
    L->phik = off;     off = align256(off + (size_t)c->ny * c->nz * p * sizeof(float2));
    L->phi = off;      off = align256(off + ncells * sizeof(float));
    L->phib = off;     off = align256(off + ((c->flags & SPE_STATIC_POTENTIAL) ? ncells * sizeof(float) : 0));
    L->dep = off;      off = align256(off + (c->max_particles ? ncells * sizeof(long long) : 0));
    // one byte per row marking the rows whose deposit may be nonzero (padded: read 16 at a time)
    L->dflag = off;    off = align256(off + (c->max_particles ? (size_t)c->ny * c->nz + 16 : 0));
    // two sets of star arrays (x, y, z, vx, vy, vz, m, id) for reordering, sort keys, block counters
    L->part = off;     off = align256(off + 17 * align256(c->max_particles * sizeof(float)));
    // block counters, then the span totals of their scan (one per 2048 counters)
    const size_t nbins = (size_t)((c->nx + 3) / 4) * ((c->ny + 3) / 4) * ((c->nz + 3) / 4);
    L->bins = off;     off = align256(off + sizeof(int) * (nbins + (nbins + 2047) / 2048));
    L->tw = off;       off = align256(off + (size_t)(c->nx + c->ny + c->nz) * sizeof(float4));
    L->k2 = off;       off = align256(off + (size_t)(c->nx + c->ny + c->nz) * sizeof(float));
    L->drift = off;    off = align256(off + ((size_t)c->nx * c->ny + c->nz) * sizeof(float4));
    L->absorb = off;   off = align256(off + (size_t)(c->nx + c->ny + c->nz) * sizeof(float));
    L->tcw = off;      off = align256(off + 4 * 1024 * sizeof(uint16_t));
    L->partials = off; off = align256(off + (size_t)kMaxPartials * 5 * sizeof(double));
    L->counter = off;  off = align256(off + 256);
    L->diag = off;     off = align256(off + 64 * sizeof(double));
    L->status = off;   off = align256(off + sizeof(int));
    L->total = off;
    *W = w;
    *P = p;
    return SPE_OK;
}

}  // namespace

struct spe_grid {
    spe_config cfg;
    int device;
    int n[3];
    double L[3], dx[3], dv;
    size_t ncells;
    int W, P;
    cudaStream_t st;
    bool gravity;
    unsigned char *ws;
    bool owns_ws;
    float2 *psi, *phik;
    float *phi;
    long long *dep;
    unsigned char *dflag;   // rows whose deposit may be nonzero (set by the star kernel, cleared by the density pass)
    float *px, *py, *pz, *vx, *vy, *vz, *pm;
    unsigned int *pid;            // insertion index of the star in each memory slot
    float *alt[7];                // second set of star arrays (reordering target)
    unsigned int *alt_id;
    int *skey, *bins;
    int nbins, nbx, nby;
    unsigned long long steps_done;
    float4 *tw[3];
    float *k2[3];
    float4 *dxy;      // exp(-i eta (kx^2 + ky^2) dt / 2) / (nx ny nz), (hi, lo)
    float4 *ez;       // exp(-i eta kz^2 dt / 2), (hi, lo)
    double *partials;
    unsigned int *counter;
    double *diag;
    float4 *h_stage;  // pinned staging for the drift and absorbing-layer tables
    float *phib;      // static external potential (SPE_STATIC_POTENTIAL)
    bool static_set;
    float *absorb;    // absorbing-layer factors per axis: nx, ny, nz floats (dt dependent)
    bool absorbing;
    int stile[3];     // strided-pass tile width per axis (0 = default; set by the autotuner)
    int splan[3];     // strided-pass radix schedule per axis (0 default, 1 alternative)
    int htile[3];     // the half spectrum's strided passes (rho, Phi): 0 = as psi's, else set by the autotuner
    int hplan[3];
    int tc;           // SPE_PREC_SPLIT16
    __half *tcw;      // 32 x 32 DFT operands for the tensor stages: [dir][hi, lo][core layout]
    int *status;      // device status word
    // CUDA graph of one full step (dt_k = dt), replayed on the caller's stream
    cudaStream_t cap_st;
    // the stars' kick-drift-deposit runs on side_st while the y and z transforms of psi run on st
    // (fork after the kick pass, join before the density pass); profile mode keeps them serial
    cudaStream_t side_st;
    cudaEvent_t fork_ev, join_ev;
    cudaGraphExec_t step_exec;
    double graph_dt;
    size_t graph_np;
    bool graph_static;
    int graph_tiles;
    unsigned long long graph_nodes;
    bool capturing;
    size_t np;
    double mstar;
    double quantum;
    bool phi_valid;
    // the closing half kick of the last spe_step, not yet applied: the next spe_step with the same
    // dt merges it into its leading kick, anything that reads or changes the state applies it first
    bool sort_due;          // reorder the stars by cell block at the next step (stars were added)
    bool kick_pending;
    double pending_h;
    double pending_dt;
    // the raw mass sum a blocking spe_step read back (valid until anything writes diag[0] again)
    double host_mass;
    bool host_mass_valid;
    bool tables_valid;
    double table_dt;
    unsigned long long launches;
    bool profile;
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> evfree;
};

namespace {

int cuerr(cudaError_t e) { return e == cudaSuccess ? SPE_OK : SPE_ECUDA; }

cudaEvent_t take_event(spe_grid *g)
{
    if (!g->evfree.empty()) {
        cudaEvent_t e = g->evfree.back();
        g->evfree.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Issue one kernel launch, counting it and (with SPE_PROFILE) timing it.
template <class F>
int launch(spe_grid *g, int kind, F &&f)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (g->profile) {
        e0 = take_event(g);
        cudaEventRecord(e0, g->st);
    }
    cudaError_t e = f();
    g->launches++;
    if (g->profile) {
        e1 = take_event(g);
        cudaEventRecord(e1, g->st);
        g->prof.push_back(ProfRec{kind, e0, e1});
    }
    return cuerr(e);
}

double wavenumber(int j, int n, double L)
{
    const int s = (2 * j < n) ? j : j - n;
    return 2.0 * kPi * (double)s / L;
}

XParams base_x(spe_grid *g)
{
    XParams p;
    memset(&p, 0, sizeof(p));
    p.psi = g->psi;
    p.phik = g->phik;
    p.phi_out = g->phi;
    p.dep = g->dep;
    p.dflag = g->dflag;
    p.tw = g->tw[0];
    p.k2 = g->k2[0];
    p.rows = g->n[1] * g->n[2];
    p.P = g->P;
    p.kappa = (float)g->cfg.kappa;
    p.dep_scale = (float)(g->quantum / g->dv);
    p.partials = g->partials;
    p.counter = g->counter;
    p.result = g->diag;
    p.mass_scale = g->dv;
    p.absorb_x = g->absorb;
    p.absorb_y = g->absorb + g->n[0];
    p.absorb_z = g->absorb + g->n[0] + g->n[1];
    p.phib = g->phib;
    p.ny = g->n[1];
    p.tc = g->tc;
    p.tcw = g->tcw;
    p.status = g->status;
    return p;
}

// Transform along y of a field with W live columns at row pitch P.
SParams base_y(spe_grid *g, float2 *data, int W, int P)
{
    SParams p;
    memset(&p, 0, sizeof(p));
    p.data = data;
    const bool half = W != g->n[0] && g->htile[1];   // the half spectrum, with a schedule of its own
    p.tile = half ? g->htile[1] : g->stile[1];
    p.plan = half ? g->hplan[1] : g->splan[1];
    p.tc = g->tc;
    p.tma = !g->tc && !(g->cfg.flags & SPE_NO_TMA);
    p.tcw = g->tcw;
    p.status = g->status;
    p.S = P;
    p.bstride = (long long)P * g->n[1];
    p.W = W;
    p.batches = g->n[2];
    p.tw = g->tw[1];
    p.linek2 = g->k2[1];
    p.partials = g->partials;
    p.counter = g->counter;
    p.result = g->diag;
    return p;
}

// Transform along z.
SParams base_z(spe_grid *g, float2 *data, int W, int P)
{
    SParams p;
    memset(&p, 0, sizeof(p));
    p.data = data;
    const bool half = W != g->n[0] && g->htile[2];
    p.tile = half ? g->htile[2] : g->stile[2];
    p.plan = half ? g->hplan[2] : g->splan[2];
    p.tc = g->tc;
    p.tma = !g->tc && !(g->cfg.flags & SPE_NO_TMA);
    p.tcw = g->tcw;
    p.status = g->status;
    p.S = (long long)P * g->n[1];
    p.bstride = P;
    p.W = W;
    p.batches = g->n[1];
    p.tw = g->tw[2];
    p.dxy = g->dxy;
    p.ez = g->ez;
    p.dxy_pitch = g->n[0];
    p.colk2 = g->k2[0];
    p.batchk2 = g->k2[1];
    p.linek2 = g->k2[2];
    p.norm = (float)(1.0 / (double)g->ncells);
    p.poisson = (float)(-4.0 * kPi * g->cfg.G);
    p.partials = g->partials;
    p.counter = g->counter;
    p.result = g->diag;
    return p;
}

PParams base_p(spe_grid *g)
{
    PParams p;
    memset(&p, 0, sizeof(p));
    p.x = g->px; p.y = g->py; p.z = g->pz;
    p.vx = g->vx; p.vy = g->vy; p.vz = g->vz;
    p.m = g->pm;
    p.phi = g->phi;
    p.dep = g->dep;
    p.dflag = g->dflag;
    p.n = (int)g->np;
    p.nx = g->n[0]; p.ny = g->n[1]; p.nz = g->n[2];
    p.Lx = (float)g->L[0]; p.Ly = (float)g->L[1]; p.Lz = (float)g->L[2];
    p.inv_dx = (float)(1.0 / g->dx[0]);
    p.inv_dy = (float)(1.0 / g->dx[1]);
    p.inv_dz = (float)(1.0 / g->dx[2]);
    p.gx_scale = (float)(0.5 / g->dx[0]);
    p.gy_scale = (float)(0.5 / g->dx[1]);
    p.gz_scale = (float)(0.5 / g->dx[2]);
    p.inv_quantum = (float)(1.0 / g->quantum);
    return p;
}

int run_x(spe_grid *g, int kind, XParams p)
{
    return launch(g, kind, [&] { return launch_xpass(g->n[0], p, g->st, nullptr); });
}

int run_s(spe_grid *g, int kind, int n, SParams p)
{
    return launch(g, kind, [&] { return launch_spass(n, p, g->st, nullptr); });
}

float4 split_c(double re, double im)
{
    const float hr = (float)re, hi = (float)im;
    return make_float4(hr, hi, (float)(re - (double)hr), (float)(im - (double)hi));
}

// Drift factors for step size dt, built in FP64: D_xy = exp(-i eta (kx^2 +
// ky^2) dt / 2) / (nx ny nz) per (kx, ky) and E_z = exp(-i eta kz^2 dt / 2),
// phases reduced modulo 2 pi in FP64, each stored as a (hi, lo) float pair.
int ensure_drift_tables(spe_grid *g, double dt)
{
    if (g->tables_valid && g->table_dt == dt) return SPE_OK;
    cudaError_t e = cudaStreamSynchronize(g->st);  // the staging buffer may still be in flight
    if (e != cudaSuccess) return SPE_ECUDA;
    const double eta = g->cfg.hbar_over_m, twopi = 2.0 * kPi;
    const double norm = 1.0 / (double)g->ncells;
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    std::vector<double> px(nx), py(ny);
    for (int i = 0; i < nx; ++i) {
        const double k = wavenumber(i, nx, g->L[0]);
        px[i] = fmod(eta * k * k * dt * 0.5, twopi);
    }
    for (int j = 0; j < ny; ++j) {
        const double k = wavenumber(j, ny, g->L[1]);
        py[j] = fmod(eta * k * k * dt * 0.5, twopi);
    }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const double ph = px[i] + py[j];
            g->h_stage[(size_t)j * nx + i] = split_c(norm * cos(ph), -norm * sin(ph));
        }
    float4 *ezh = g->h_stage + (size_t)nx * ny;
    for (int k = 0; k < nz; ++k) {
        const double kk = wavenumber(k, nz, g->L[2]);
        const double ph = fmod(eta * kk * kk * dt * 0.5, twopi);
        ezh[k] = split_c(cos(ph), -sin(ph));
    }
    e = cudaMemcpyAsync(g->dxy, g->h_stage, ((size_t)nx * ny + nz) * sizeof(float4), cudaMemcpyHostToDevice,
                        g->st);
    if (e != cudaSuccess) return SPE_ECUDA;
    if (g->absorbing) {
        // Sec. 3.1 layer per axis: exp(-alpha dt (2 - [tanh((x + L/2)/(L/N_b)) - tanh((x - L/2)/(L/N_b))]));
        // the product over the three axes is the printed 3D factor
        float *ab = reinterpret_cast<float *>(g->h_stage + (size_t)nx * ny + nz);
        int off = 0;
        for (int a = 0; a < 3; ++a) {
            const double La = g->L[a], w = La / g->cfg.absorb_nb;
            for (int i = 0; i < g->n[a]; ++i) {
                const double x = -0.5 * La + i * g->dx[a];
                const double sa = tanh((x + 0.5 * La) / w) - tanh((x - 0.5 * La) / w);
                ab[off + i] = (float)exp(-g->cfg.absorb_alpha * dt * (2.0 - sa));
            }
            off += g->n[a];
        }
        e = cudaMemcpyAsync(g->absorb, ab, (size_t)off * sizeof(float), cudaMemcpyHostToDevice, g->st);
        if (e != cudaSuccess) return SPE_ECUDA;
    }
    g->tables_valid = true;
    g->table_dt = dt;
    return SPE_OK;
}

bool has_kick(spe_grid *g) { return g->gravity || g->cfg.kappa != 0.0 || g->static_set; }
// stars feel a potential (self gravity and / or the static one)
bool stars_kicked(spe_grid *g) { return g->gravity || g->static_set; }
int static_flag(spe_grid *g) { return g->static_set ? X_STATIC : 0; }

// Phi from the current psi and particles (the state at n = 0 of Algorithm 1,
// or after set_ic / add_particles).
int compute_phi(spe_grid *g)
{
    int rc = SPE_OK;
    g->host_mass_valid = false;   // the density pass below rewrites diag[0]
    if (!g->gravity) {
        g->phi_valid = true;
        return SPE_OK;
    }
    const bool parts = g->np > 0;
    if (parts) {
        PParams pp = base_p(g);
        pp.flags = PK_DEPOSIT;
        rc = launch(g, KIND_PARTICLES, [&] { return launch_particles(pp, g->st); });
        if (rc) return rc;
    }
    XParams xp = base_x(g);
    xp.flags = X_MASS | X_R2C | (parts ? X_DEP : 0);
    if ((rc = run_x(g, KIND_X_IFFT_DENSITY, xp))) return rc;
    SParams y = base_y(g, g->phik, g->W, g->P);
    y.flags = S_FWD;
    if ((rc = run_s(g, KIND_Y_RHO, g->n[1], y))) return rc;
    SParams z = base_z(g, g->phik, g->W, g->P);
    z.flags = S_FWD | S_POISSON | S_INV;
    if ((rc = run_s(g, KIND_Z_POISSON, g->n[2], z))) return rc;
    y.flags = S_INV;
    if ((rc = run_s(g, KIND_Y_RHO, g->n[1], y))) return rc;
    g->phi_valid = true;
    return SPE_OK;
}

// Reorder the star arrays by 4x4x4 cell block every kSortEvery steps so a
// warp's Phi gathers and deposit atomics hit few L2 lines (stars cross a cell
// in hundreds of CFL-limited steps, so the order stays useful that long).
constexpr unsigned long long kSortEvery = 64;

int sort_particles(spe_grid *g)
{
    SortParams sp;
    memset(&sp, 0, sizeof(sp));
    float *cur[7] = {g->px, g->py, g->pz, g->vx, g->vy, g->vz, g->pm};
    for (int a = 0; a < 7; ++a) {
        sp.src[a] = cur[a];
        sp.dst[a] = g->alt[a];
    }
    sp.src_id = g->pid;
    sp.dst_id = g->alt_id;
    sp.key = g->skey;
    sp.count = g->bins;
    sp.totals = g->bins + g->nbins;
    sp.n = (int)g->np;
    sp.nbins = g->nbins;
    sp.nx = g->n[0]; sp.ny = g->n[1]; sp.nz = g->n[2];
    sp.nbx = g->nbx; sp.nby = g->nby;
    sp.Lx = (float)g->L[0]; sp.Ly = (float)g->L[1]; sp.Lz = (float)g->L[2];
    sp.inv_dx = (float)(1.0 / g->dx[0]);
    sp.inv_dy = (float)(1.0 / g->dx[1]);
    sp.inv_dz = (float)(1.0 / g->dx[2]);
    int extra = 0;
    int rc = launch(g, KIND_SORT, [&] { return launch_particle_sort(sp, g->st, &extra); });
    g->launches += extra > 0 ? extra - 1 : 0;
    if (rc) return rc;
    g->sort_due = false;
    // copy the reordered arrays back so that the star arrays never move (captured graphs hold
    // their addresses)
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < 7 && e == cudaSuccess; ++a)
        e = cudaMemcpyAsync(cur[a], g->alt[a], g->np * sizeof(float), cudaMemcpyDeviceToDevice, g->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->pid, g->alt_id, g->np * sizeof(unsigned int), cudaMemcpyDeviceToDevice, g->st);
    return cuerr(e);
}

int ensure_side_stream(spe_grid *g)
{
    if (!g->side_st && cudaStreamCreateWithFlags(&g->side_st, cudaStreamNonBlocking) != cudaSuccess) return SPE_ECUDA;
    if (!g->fork_ev && cudaEventCreateWithFlags(&g->fork_ev, cudaEventDisableTiming) != cudaSuccess) return SPE_ECUDA;
    if (!g->join_ev && cudaEventCreateWithFlags(&g->join_ev, cudaEventDisableTiming) != cudaSuccess) return SPE_ECUDA;
    return SPE_OK;
}

// One KDK step whose leading kick has size dtk (dt/2 for the first step of
// a call, dt afterwards).
// absorb_prev: apply the absorbing layer of the previous step (all steps of a
// call but the first; the call's last step gets it in the final kick pass).
int step_body(spe_grid *g, double dtk, double dt, bool absorb_prev)
{
    int rc;
    g->host_mass_valid = false;
    const bool grav = g->gravity;
    const bool parts = g->np > 0;
    const bool skick = parts && stars_kicked(g);
    XParams xp = base_x(g);
    xp.flags = X_FFT | (has_kick(g) ? X_KICK : 0) | (grav ? X_HAS_PHI : 0) | (skick ? X_WRITE_PHI : 0) |
               static_flag(g) | ((absorb_prev && g->absorbing) ? X_ABSORB : 0);
    xp.kick_scale = (float)(dtk / g->cfg.hbar_over_m);
    if ((rc = run_x(g, KIND_X_KICK_FFT, xp))) return rc;
    // The stars need only the kick pass (the real Phi it writes) and the density pass needs their
    // deposit, so they run beside the y and z transforms of psi, which touch neither.
    const bool side = parts && !g->profile;
    if (parts) {
        if (!g->capturing && (g->sort_due || g->steps_done % kSortEvery == 0) && (rc = sort_particles(g))) return rc;
        PParams pp = base_p(g);
        pp.flags = PK_DRIFT | (skick ? PK_KICK : 0) | (grav ? PK_DEPOSIT : 0);
        pp.kick = (float)dtk;
        pp.drift = (float)dt;
        if (side) {
            if ((rc = ensure_side_stream(g))) return rc;
            if (cudaEventRecord(g->fork_ev, g->st) != cudaSuccess ||
                cudaStreamWaitEvent(g->side_st, g->fork_ev, 0) != cudaSuccess)
                return SPE_ECUDA;
            rc = launch(g, KIND_PARTICLES, [&] { return launch_particles(pp, g->side_st); });
            if (cudaEventRecord(g->join_ev, g->side_st) != cudaSuccess && !rc) rc = SPE_ECUDA;
            if (rc) {
                cudaStreamWaitEvent(g->st, g->join_ev, 0);   // rejoin the side stream before failing
                return rc;
            }
        } else if ((rc = launch(g, KIND_PARTICLES, [&] { return launch_particles(pp, g->st); }))) {
            return rc;
        }
    }
    SParams y = base_y(g, g->psi, g->n[0], g->n[0]);
    y.flags = S_FWD;
    if ((rc = run_s(g, KIND_Y_PSI, g->n[1], y))) return rc;
    SParams z = base_z(g, g->psi, g->n[0], g->n[0]);
    z.flags = S_FWD | S_DRIFT | S_INV;
    if ((rc = run_s(g, KIND_Z_DRIFT, g->n[2], z))) return rc;
    y.flags = S_INV;
    if ((rc = run_s(g, KIND_Y_PSI, g->n[1], y))) return rc;
    if (side && cudaStreamWaitEvent(g->st, g->join_ev, 0) != cudaSuccess) return SPE_ECUDA;
    xp.flags = X_IFFT | X_MASS | (grav ? X_R2C : 0) | ((parts && grav) ? X_DEP : 0);
    if ((rc = run_x(g, KIND_X_IFFT_DENSITY, xp))) return rc;
    if (grav) {
        SParams yr = base_y(g, g->phik, g->W, g->P);
        yr.flags = S_FWD;
        if ((rc = run_s(g, KIND_Y_RHO, g->n[1], yr))) return rc;
        SParams zr = base_z(g, g->phik, g->W, g->P);
        zr.flags = S_FWD | S_POISSON | S_INV;
        if ((rc = run_s(g, KIND_Z_POISSON, g->n[2], zr))) return rc;
        yr.flags = S_INV;
        if ((rc = run_s(g, KIND_Y_RHO, g->n[1], yr))) return rc;
    }
    return SPE_OK;
}

// everything about the strided passes' launch shapes that a captured graph bakes in
int schedule_key(const spe_grid *g)
{
    auto t = [](int w) { return w == 8 ? 1 : (w == 16 ? 2 : (w == 32 ? 3 : 0)); };
    int k = 0;
    for (int a = 1; a <= 2; ++a)
        k = (((k * 4 + t(g->stile[a])) * 4 + g->splan[a]) * 4 + t(g->htile[a])) * 4 + g->hplan[a];
    return k;
}

bool graphs_enabled(spe_grid *g) { return !(g->cfg.flags & (SPE_NO_GRAPH | SPE_PROFILE)); }

// One full step (dt_k = dt, the previous step's absorbing layer applied) as an
// executable CUDA graph, captured on the grid's private stream and launched on
// the caller's.  Re-captured when anything baked into the launches changes.
int ensure_step_graph(spe_grid *g, double dt)
{
    const int tiles = schedule_key(g);
    if (g->step_exec && g->graph_dt == dt && g->graph_np == g->np && g->graph_static == g->static_set &&
        g->graph_tiles == tiles)
        return SPE_OK;
    if (g->step_exec) {
        cudaGraphExecDestroy(g->step_exec);
        g->step_exec = nullptr;
    }
    if (!g->cap_st && cudaStreamCreateWithFlags(&g->cap_st, cudaStreamNonBlocking) != cudaSuccess) return SPE_ECUDA;
    cudaStream_t user = g->st;
    const unsigned long long before = g->launches;
    g->st = g->cap_st;
    g->capturing = true;
    cudaError_t e = cudaStreamBeginCapture(g->cap_st, cudaStreamCaptureModeThreadLocal);
    int rc = (e == cudaSuccess) ? step_body(g, dt, dt, true) : SPE_ECUDA;
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = (e == cudaSuccess) ? cudaStreamEndCapture(g->cap_st, &graph) : e;
    g->st = user;
    g->capturing = false;
    g->graph_nodes = g->launches - before;
    g->launches = before;
    if (rc || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc ? rc : SPE_ECUDA;
    }
    e = cudaGraphInstantiate(&g->step_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g->step_exec = nullptr;
        cudaGetLastError();
        return SPE_ECUDA;
    }
    g->graph_dt = dt;
    g->graph_np = g->np;
    g->graph_static = g->static_set;
    g->graph_tiles = tiles;
    return SPE_OK;
}

// Full steps (dt_k = dt, the previous step's absorbing layer applied), by graph replay when
// allowed: from two steps up, or from one when single is set (a run of single-step calls, whose
// every step is a full one).
int run_full_steps(spe_grid *g, int count, double dt, bool single = false)
{
    int rc;
    if (count <= 0) return SPE_OK;
    if (!graphs_enabled(g) || (count < 2 && !single)) {
        for (int s = 0; s < count; ++s) {
            if ((rc = step_body(g, dt, dt, true))) return rc;
            g->steps_done++;
        }
        return SPE_OK;
    }
    if ((rc = ensure_step_graph(g, dt))) return rc;
    for (int s = 0; s < count; ++s) {
        if (g->np && (g->sort_due || g->steps_done % kSortEvery == 0) && (rc = sort_particles(g))) return rc;
        if (cudaGraphLaunch(g->step_exec, g->st) != cudaSuccess) return SPE_ECUDA;
        g->launches += g->graph_nodes;
        g->steps_done++;
    }
    return SPE_OK;
}

int final_half_kick(spe_grid *g, double h)
{
    int rc;
    const bool grav = g->gravity;
    const bool parts = g->np > 0;
    const bool skick = parts && stars_kicked(g);
    if (has_kick(g) || g->absorbing) {
        XParams xp = base_x(g);
        xp.flags = (has_kick(g) ? X_KICK : 0) | (grav ? X_HAS_PHI : 0) | (skick ? X_WRITE_PHI : 0) | static_flag(g) |
                   (g->absorbing ? X_ABSORB : 0);
        xp.kick_scale = (float)(h / g->cfg.hbar_over_m);
        if ((rc = run_x(g, KIND_X_KICK_FINAL, xp))) return rc;
    }
    if (skick) {
        PParams pp = base_p(g);
        pp.flags = PK_KICK;
        pp.kick = (float)h;
        if ((rc = launch(g, KIND_PARTICLES, [&] { return launch_particles(pp, g->st); }))) return rc;
    }
    return SPE_OK;
}

}  // namespace

namespace spe {

// Apply the deferred closing half kick, if any (asynchronously, on the grid's stream).
int settle(spe_grid *g)
{
    if (!g->kick_pending) return SPE_OK;
    g->kick_pending = false;
    return final_half_kick(g, g->pending_h);
}

}  // namespace spe

namespace {

using spe::settle;

// Real-space Phi into g->phi.
int potential_to_phi(spe_grid *g)
{
    int rc;
    if (!g->phi_valid && (rc = compute_phi(g))) return rc;
    if (!g->gravity) {
        if (g->static_set)
            return cuerr(cudaMemcpyAsync(g->phi, g->phib, g->ncells * sizeof(float), cudaMemcpyDeviceToDevice, g->st));
        return cuerr(cudaMemsetAsync(g->phi, 0, g->ncells * sizeof(float), g->st));
    }
    XParams xp = base_x(g);
    xp.flags = X_HAS_PHI | X_WRITE_PHI | static_flag(g);
    return run_x(g, KIND_X_POTENTIAL, xp);
}

int deposit_only(spe_grid *g)
{
    if (!g->np) return SPE_OK;
    PParams pp = base_p(g);
    pp.flags = PK_DEPOSIT;
    return launch(g, KIND_PARTICLES, [&] { return launch_particles(pp, g->st); });
}

int copy_out(spe_grid *g, void *dst, const void *src, size_t bytes, int where)
{
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, where == SPE_HOST ? cudaMemcpyDeviceToHost
                                                                       : cudaMemcpyDeviceToDevice, g->st);
    if (e != cudaSuccess) return SPE_ECUDA;
    return cuerr(cudaStreamSynchronize(g->st));
}

void update_quantum(spe_grid *g)
{
    g->quantum = (g->mstar > 0.0) ? g->mstar * ldexp(1.0, -50) : 1.0;
}

}  // namespace

namespace spe {

// Launch every kernel of spe_energy on the grid's stream; the raw sums land in
// diag[8 .. 8 + kEnergyRaw).  With host_raw they are also copied there
// asynchronously (a pinned buffer; nothing waits).
int energy_issue(spe_grid *g, double *host_raw, bool copy_to_host)
{
    int rc;
    if ((rc = settle(g))) return rc;
    if ((rc = potential_to_phi(g))) return rc;
    if ((rc = deposit_only(g))) return rc;
    if ((rc = launch(g, KIND_DIAG, [&] {
             return launch_grid_diag(g->psi, g->phi, g->np ? g->dep : nullptr, (float)(g->quantum / g->dv),
                                     (float)g->cfg.kappa, g->dv, g->ncells, g->partials, g->counter, g->diag + 8,
                                     g->st);
         })))
        return rc;
    if (g->static_set) {
        // the static potential counts once, not halved: 1/2 sum (|psi|^2 + rho_*) Phi_b dV lands in diag[25]
        if ((rc = deposit_only(g))) return rc;
        if ((rc = launch(g, KIND_DIAG, [&] {
                 return launch_grid_diag(g->psi, g->phib, g->np ? g->dep : nullptr, (float)(g->quantum / g->dv),
                                         0.f, g->dv, g->ncells, g->partials, g->counter, g->diag + 24, g->st);
             })))
            return rc;
    }
    // kinetic: sum over axes of (1/N_a) sum_lines sum_k k_a^2 |F_a line|^2
    XParams xp = base_x(g);
    xp.flags = X_KIN;
    xp.result = g->diag + 16;
    if ((rc = run_x(g, KIND_DIAG, xp))) return rc;
    SParams y = base_y(g, g->psi, g->n[0], g->n[0]);
    y.flags = S_FWD | S_KIN;
    y.result = g->diag + 17;
    if ((rc = run_s(g, KIND_DIAG, g->n[1], y))) return rc;
    SParams z = base_z(g, g->psi, g->n[0], g->n[0]);
    z.flags = S_FWD | S_KIN;
    z.result = g->diag + 18;
    if ((rc = run_s(g, KIND_DIAG, g->n[2], z))) return rc;
    if (g->np) {
        if ((rc = launch(g, KIND_DIAG, [&] {
                 return launch_particle_ke(g->vx, g->vy, g->vz, g->pm, (int)g->np, g->partials, g->counter,
                                           g->diag + 19, g->st);
             })))
            return rc;
    }
    if (copy_to_host && host_raw &&
        cudaMemcpyAsync(host_raw, g->diag + 8, kEnergyRaw * sizeof(double), cudaMemcpyDeviceToHost, g->st) !=
            cudaSuccess)
        return SPE_ECUDA;
    return SPE_OK;
}

int energy_from_raw(spe_grid *g, const double *raw, spe_energy_t *out)
{
    const double static_raw = g->static_set ? raw[17] : 0.0;
    const double eta = g->cfg.hbar_over_m;
    out->mass = raw[0] * g->dv;
    const bool has_phi = g->gravity || g->static_set;
    out->potential = has_phi ? 0.5 * (raw[1] + static_raw) * g->dv : 0.0;
    out->interaction = 0.5 * g->cfg.kappa * raw[2] * g->dv;
    out->max_abs_phi = has_phi ? raw[3] : 0.0;
    out->kinetic = 0.5 * eta * eta * g->dv * (raw[8] / g->n[0] + raw[9] / g->n[1] + raw[10] / g->n[2]);
    out->star_kinetic = g->np ? raw[11] : 0.0;
    out->total = out->kinetic + out->potential + out->interaction + out->star_kinetic;
    return SPE_OK;
}

float2 *grid_psi(spe_grid *g) { return g->psi; }
cudaStream_t grid_stream(spe_grid *g) { return g->st; }

}  // namespace spe

extern "C" {

const char *spe_strerror(int s)
{
    switch (s) {
    case SPE_OK: return "ok";
    case SPE_EINVAL: return "invalid argument or unsupported configuration";
    case SPE_ENOMEM: return "out of memory or workspace too small";
    case SPE_ECUDA: return "CUDA runtime error";
    case SPE_ECFL: return "time step above the CFL bound";
    case SPE_ENONFINITE: return "field mass is not finite";
    case SPE_ETIMEOUT: return "bounded device wait timed out";
    case SPE_ESTATE: return "call out of order";
    default: return "unknown status";
    }
}

int spe_workspace_bytes(const spe_config *cfg, size_t *bytes)
{
    if (!bytes) return SPE_EINVAL;
    Layout L;
    int W, P;
    int rc = compute_layout(cfg, &L, &W, &P);
    if (rc) return rc;
    *bytes = L.total;
    return SPE_OK;
}

int spe_create_grid(const spe_config *cfg, void *workspace, size_t workspace_bytes, spe_grid **out)
{
    if (!out) return SPE_EINVAL;
    *out = nullptr;
    Layout L;
    int W, P;
    int rc = compute_layout(cfg, &L, &W, &P);
    if (rc) return rc;
    if (workspace && (workspace_bytes < L.total || ((uintptr_t)workspace & 255))) return SPE_ENOMEM;
    static bool attrs_done = false;
    if (!attrs_done) {
        if (setup_kernel_attributes() != cudaSuccess) return SPE_ECUDA;
        attrs_done = true;
    }
    spe_grid *g = new (std::nothrow) spe_grid();
    if (!g) return SPE_ENOMEM;
    g->cfg = *cfg;
    cudaGetDevice(&g->device);
    g->n[0] = cfg->nx; g->n[1] = cfg->ny; g->n[2] = cfg->nz;
    g->L[0] = cfg->Lx; g->L[1] = cfg->Ly; g->L[2] = cfg->Lz;
    for (int a = 0; a < 3; ++a) g->dx[a] = g->L[a] / g->n[a];
    g->dv = g->dx[0] * g->dx[1] * g->dx[2];
    g->ncells = (size_t)cfg->nx * cfg->ny * cfg->nz;
    g->W = W;
    g->P = P;
    g->st = (cudaStream_t)cfg->cuda_stream;
    g->gravity = !(cfg->flags & SPE_GRAVITY_OFF) && cfg->G != 0.0;
    g->profile = (cfg->flags & SPE_PROFILE) != 0;
    if (workspace) {
        g->ws = (unsigned char *)workspace;
        g->owns_ws = false;
    } else {
        if (cudaMalloc(&g->ws, L.total) != cudaSuccess) {
            cudaGetLastError();
            delete g;
            return SPE_ENOMEM;
        }
        g->owns_ws = true;
    }
    if (cudaMallocHost(&g->h_stage, ((size_t)cfg->nx * cfg->ny + 2 * cfg->nz + cfg->nx + cfg->ny) * sizeof(float4)) !=
        cudaSuccess) {
        cudaGetLastError();
        if (g->owns_ws) cudaFree(g->ws);
        delete g;
        return SPE_ENOMEM;
    }
    unsigned char *b = g->ws;
    g->psi = (float2 *)(b + L.psi);
    g->phik = (float2 *)(b + L.phik);
    g->phi = (float *)(b + L.phi);
    g->dep = cfg->max_particles ? (long long *)(b + L.dep) : nullptr;
    g->dflag = cfg->max_particles ? (unsigned char *)(b + L.dflag) : nullptr;
    const size_t pstride = align256(cfg->max_particles * sizeof(float));
    float **parr[7] = {&g->px, &g->py, &g->pz, &g->vx, &g->vy, &g->vz, &g->pm};
    for (int i = 0; i < 7; ++i) *parr[i] = (float *)(b + L.part + i * pstride);
    g->pid = (unsigned int *)(b + L.part + 7 * pstride);
    for (int i = 0; i < 7; ++i) g->alt[i] = (float *)(b + L.part + (8 + i) * pstride);
    g->alt_id = (unsigned int *)(b + L.part + 15 * pstride);
    g->skey = (int *)(b + L.part + 16 * pstride);
    g->bins = (int *)(b + L.bins);
    g->nbx = (cfg->nx + 3) / 4;
    g->nby = (cfg->ny + 3) / 4;
    g->nbins = g->nbx * g->nby * ((cfg->nz + 3) / 4);
    g->tw[0] = (float4 *)(b + L.tw);
    g->tw[1] = g->tw[0] + cfg->nx;
    g->tw[2] = g->tw[1] + cfg->ny;
    g->k2[0] = (float *)(b + L.k2);
    g->k2[1] = g->k2[0] + cfg->nx;
    g->k2[2] = g->k2[1] + cfg->ny;
    g->phib = (cfg->flags & SPE_STATIC_POTENTIAL) ? (float *)(b + L.phib) : nullptr;
    g->tc = (cfg->flags & SPE_PREC_SPLIT16) ? 1 : 0;
    g->tcw = (__half *)(b + L.tcw);
    g->status = (int *)(b + L.status);
    g->absorb = (float *)(b + L.absorb);
    g->absorbing = cfg->absorb_alpha > 0.0;
    g->dxy = (float4 *)(b + L.drift);
    g->ez = g->dxy + (size_t)cfg->nx * cfg->ny;
    g->partials = (double *)(b + L.partials);
    g->counter = (unsigned int *)(b + L.counter);
    g->diag = (double *)(b + L.diag);
    update_quantum(g);

    cudaError_t e = cudaMemsetAsync(g->ws, 0, L.total, g->st);
    // FP64-built tables: twiddles exp(-2 pi i e / N) as (hi, lo) float pairs and k^2 per axis
    const int ntot = cfg->nx + cfg->ny + cfg->nz;
    std::vector<float4> tw(ntot);
    std::vector<float> k2(ntot);
    int off = 0;
    for (int a = 0; a < 3; ++a) {
        const int n = g->n[a];
        for (int j = 0; j < n; ++j) {
            const double ang = -2.0 * kPi * (double)j / (double)n;
            tw[off + j] = split_c(cos(ang), sin(ang));
            const double k = wavenumber(j, n, g->L[a]);
            k2[off + j] = (float)(k * k);
        }
        off += n;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->tw[0], tw.data(), ntot * sizeof(float4), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->k2[0], k2.data(), ntot * sizeof(float), cudaMemcpyHostToDevice, g->st);
    // 16-point DFT as a 32 x 32 real matrix for the tensor stages, rows = outputs [Re y, Im y],
    // columns = inputs [Re x, Im x]; FP64 values split into fp16 hi + lo, stored in the
    // no-swizzle K-major core-matrix layout (element (n, k) at byte
    // (n/8)*512 + (k/8)*128 + (n%8)*16 + (k%8)*2)
    std::vector<__half> wt(4 * 1024);
    for (int d = 0; d < 2; ++d) {
        const double dir = d == 0 ? -1.0 : 1.0;
        for (int n = 0; n < 32; ++n)
            for (int k = 0; k < 32; ++k) {
                const double th = dir * 2.0 * kPi * (double)((n % 16) * (k % 16)) / 16.0;
                double w;
                if (n < 16) w = (k < 16) ? cos(th) : -sin(th);
                else w = (k < 16) ? sin(th) : cos(th);
                const __half hi = __float2half_rn((float)w);
                const __half lo = __float2half_rn((float)(w - (double)__half2float(hi)));
                const int idx = ((n >> 3) * 512 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) / 2;
                wt[(d * 2 + 0) * 1024 + idx] = hi;
                wt[(d * 2 + 1) * 1024 + idx] = lo;
            }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->tcw, wt.data(), wt.size() * sizeof(__half), cudaMemcpyHostToDevice, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) {
        spe_destroy(g);
        return SPE_ECUDA;
    }
    *out = g;
    return SPE_OK;
}

int spe_destroy(spe_grid *g)
{
    if (!g) return SPE_EINVAL;
    cudaStreamSynchronize(g->st);
    for (auto &r : g->prof) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    for (auto e : g->evfree) cudaEventDestroy(e);
    if (g->step_exec) cudaGraphExecDestroy(g->step_exec);
    if (g->cap_st) cudaStreamDestroy(g->cap_st);
    if (g->side_st) cudaStreamDestroy(g->side_st);
    if (g->fork_ev) cudaEventDestroy(g->fork_ev);
    if (g->join_ev) cudaEventDestroy(g->join_ev);
    if (g->h_stage) cudaFreeHost(g->h_stage);
    if (g->owns_ws) cudaFree(g->ws);
    delete g;
    return SPE_OK;
}

int spe_set_ic(spe_grid *g, const void *psi, size_t n, int where)
{
    if (!g || !psi || n != g->ncells || (where != SPE_HOST && where != SPE_DEVICE)) return SPE_EINVAL;
    const int rc = settle(g);   // the stars still owe the half kick
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(g->psi, psi, n * sizeof(float2),
                                    where == SPE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->st);
    if (e == cudaSuccess && where == SPE_HOST) e = cudaStreamSynchronize(g->st);
    g->phi_valid = false;
    return cuerr(e);
}

int spe_add_particles(spe_grid *g, size_t n, const float *pos3, const float *vel3, const float *mass, int where)
{
    if (!g || (n && (!pos3 || !vel3 || !mass)) || (where != SPE_HOST && where != SPE_DEVICE)) return SPE_EINVAL;
    if (n == 0) return SPE_OK;
    if (g->np + n > g->cfg.max_particles) return SPE_ENOMEM;
    if (const int rc = settle(g)) return rc;   // before the new stars join
    const size_t o = g->np;
    cudaError_t e = cudaSuccess;
    double msum = 0.0;
    if (where == SPE_HOST && 7 * n <= g->ncells) {
        // staged through the real-potential buffer (every step rewrites it before reading it), so the
        // wrap and the AoS -> SoA split run on the device
        float *stage = g->phi;
        e = cudaMemcpyAsync(stage, pos3, 3 * n * sizeof(float), cudaMemcpyHostToDevice, g->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(stage + 3 * n, vel3, 3 * n * sizeof(float), cudaMemcpyHostToDevice, g->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(stage + 6 * n, mass, n * sizeof(float), cudaMemcpyHostToDevice, g->st);
        for (size_t i = 0; i < n; ++i) msum += mass[i];
        if (e == cudaSuccess)
            e = launch_particles_to_soa(stage, stage + 3 * n, stage + 6 * n, (int)n, g->px + o, g->py + o,
                                        g->pz + o, g->vx + o, g->vy + o, g->vz + o, g->pm + o, (float)g->L[0],
                                        (float)g->L[1], (float)g->L[2], g->st);
        g->launches++;
        // the caller may reuse its arrays on return
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    } else if (where == SPE_HOST) {
        std::vector<float> soa(7 * n);
        for (size_t i = 0; i < n; ++i) {
            for (int a = 0; a < 3; ++a) {
                float x = pos3[3 * i + a];
                const float Lf = (float)g->L[a];
                soa[a * n + i] = x - Lf * floorf((x + 0.5f * Lf) / Lf);
                soa[(3 + a) * n + i] = vel3[3 * i + a];
            }
            soa[6 * n + i] = mass[i];
            msum += mass[i];
        }
        float *dst[7] = {g->px, g->py, g->pz, g->vx, g->vy, g->vz, g->pm};
        for (int k = 0; k < 7 && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(dst[k] + o, soa.data() + k * n, n * sizeof(float), cudaMemcpyHostToDevice, g->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    } else {
        std::vector<float> hm(n);
        e = cudaMemcpyAsync(hm.data(), mass, n * sizeof(float), cudaMemcpyDeviceToHost, g->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
        for (size_t i = 0; i < n; ++i) msum += hm[i];
        if (e == cudaSuccess)
            e = launch_particles_to_soa(pos3, vel3, mass, (int)n, g->px + o, g->py + o, g->pz + o, g->vx + o,
                                        g->vy + o, g->vz + o, g->pm + o, (float)g->L[0], (float)g->L[1],
                                        (float)g->L[2], g->st);
        g->launches++;
    }
    if (e == cudaSuccess) {
        e = launch_particle_ids(g->pid, (int)o, (int)n, g->st);
        g->launches++;
    }
    if (e != cudaSuccess) return SPE_ECUDA;
    g->np += n;
    g->mstar += msum;
    update_quantum(g);
    g->phi_valid = false;
    g->sort_due = true;   // new stars arrive in insertion order: reorder them at the next step
    return SPE_OK;
}

int spe_clear_particles(spe_grid *g)
{
    if (!g) return SPE_EINVAL;
    if (const int rc = settle(g)) return rc;
    g->np = 0;
    g->mstar = 0.0;
    update_quantum(g);
    g->phi_valid = false;
    return SPE_OK;
}

int spe_step(spe_grid *g, int nsteps, double dt)
{
    if (!g || nsteps < 0 || !isfinite(dt)) return SPE_EINVAL;
    if (nsteps == 0) return SPE_OK;
    if (!(g->cfg.flags & SPE_NO_CFL_CHECK)) {
        double dx = g->dx[0];
        if (g->dx[1] < dx) dx = g->dx[1];
        if (g->dx[2] < dx) dx = g->dx[2];
        const double bound = 0.5 * 4.0 / (3.0 * kPi) * dx * dx / g->cfg.hbar_over_m;
        if (fabs(dt) > bound * (1.0 + 1e-12)) return SPE_ECFL;
    }
    int rc;
    // a closing half kick still owed by the previous call joins this call's leading kick (as
    // between the steps of one call) when the step size is the same; otherwise it goes first,
    // with the tables of its own step
    if (g->kick_pending && g->pending_dt != dt && (rc = settle(g))) return rc;
    if ((rc = ensure_drift_tables(g, dt))) return rc;
    if (!g->phi_valid && (rc = compute_phi(g))) return rc;
    const bool merge = g->kick_pending;
    const double lead = merge ? g->pending_h + 0.5 * dt : 0.5 * dt;
    g->kick_pending = false;
    g->host_mass_valid = false;
    if (merge && lead == dt) {
        // the owed half kick and this call's leading one make the full kick of a step inside a call
        if ((rc = run_full_steps(g, nsteps, dt, true))) return rc;
    } else {
        if ((rc = step_body(g, lead, dt, merge))) return rc;
        g->steps_done++;
        if ((rc = run_full_steps(g, nsteps - 1, dt))) return rc;
    }
    g->kick_pending = true;
    g->pending_h = 0.5 * dt;
    g->pending_dt = dt;
    if (g->cfg.flags & SPE_ASYNC) return SPE_OK;
    double mass = 0.0;
    int st = 0;   // bounded mbarrier waits of the tile copies and tensor-core stages
    cudaError_t e = cudaMemcpyAsync(&mass, g->diag, sizeof(double), cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, g->status, sizeof(int), cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) return SPE_ECUDA;
    if (st) {
        cudaMemsetAsync(g->status, 0, sizeof(int), g->st);
        return SPE_ETIMEOUT;
    }
    if (!isfinite(mass)) return SPE_ENONFINITE;
    g->host_mass = mass;          // spe_last_mass answers from here until the next step
    g->host_mass_valid = true;
    return SPE_OK;
}

int spe_last_mass(spe_grid *g, double *mass_out)
{
    if (!g || !mass_out) return SPE_EINVAL;
    if (g->host_mass_valid) {
        *mass_out = g->host_mass * g->dv;
        return SPE_OK;
    }
    double m = 0.0;
    cudaError_t e = cudaMemcpyAsync(&m, g->diag, sizeof(double), cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) return SPE_ECUDA;
    *mass_out = m * g->dv;
    return SPE_OK;
}

int spe_mass_async(spe_grid *g, double *dst)
{
    if (!g || !dst) return SPE_EINVAL;
    return cuerr(cudaMemcpyAsync(dst, g->diag + 1, sizeof(double), cudaMemcpyDefault, g->st));
}

int spe_suggest_dt(spe_grid *g, double safety, double *dt_out)
{
    if (!g || !dt_out || !(safety > 0)) return SPE_EINVAL;
    int rc;
    if ((rc = settle(g))) return rc;
    if ((rc = potential_to_phi(g))) return rc;
    if ((rc = launch(g, KIND_DIAG, [&] {
             return launch_grid_diag(g->psi, g->phi, nullptr, 0.f, (float)g->cfg.kappa, g->dv, g->ncells,
                                     g->partials, g->counter, g->diag + 8, g->st);
         })))
        return rc;
    double raw[5];
    if ((rc = copy_out(g, raw, g->diag + 8, sizeof(raw), SPE_HOST))) return rc;
    double dx = g->dx[0];
    if (g->dx[1] < dx) dx = g->dx[1];
    if (g->dx[2] < dx) dx = g->dx[2];
    const double eta = g->cfg.hbar_over_m;
    double t = 4.0 / (3.0 * kPi) * dx * dx / eta;
    const double maxphi = (g->gravity || g->static_set) ? raw[3] : 0.0, maxrho = raw[4];
    if (maxphi > 0.0 && 2.0 * kPi * eta / maxphi < t) t = 2.0 * kPi * eta / maxphi;
    if (g->cfg.kappa != 0.0 && maxrho > 0.0) {
        const double ti = 2.0 * kPi * eta / (fabs(g->cfg.kappa) * maxrho);
        if (ti < t) t = ti;
    }
    *dt_out = safety * 0.5 * t;
    return SPE_OK;
}

int spe_density(spe_grid *g, float *out, int where)
{
    if (!g || !out || (where != SPE_HOST && where != SPE_DEVICE)) return SPE_EINVAL;
    int rc;
    if ((rc = settle(g))) return rc;
    if ((rc = deposit_only(g))) return rc;
    float *dst = (where == SPE_DEVICE) ? out : g->phi;
    if ((rc = launch(g, KIND_DIAG, [&] {
             return launch_density(g->psi, g->np ? g->dep : nullptr, (float)(g->quantum / g->dv), dst, g->ncells,
                                   g->st);
         })))
        return rc;
    if (where == SPE_HOST) return copy_out(g, out, g->phi, g->ncells * sizeof(float), SPE_HOST);
    return cuerr(cudaStreamSynchronize(g->st));
}

int spe_potential(spe_grid *g, float *out, int where)
{
    if (!g || !out || (where != SPE_HOST && where != SPE_DEVICE)) return SPE_EINVAL;
    int rc;
    if ((rc = settle(g))) return rc;
    if ((rc = potential_to_phi(g))) return rc;
    return copy_out(g, out, g->phi, g->ncells * sizeof(float), where);
}

int spe_energy(spe_grid *g, spe_energy_t *out)
{
    if (!g || !out) return SPE_EINVAL;
    double raw[spe::kEnergyRaw];
    int rc;
    if ((rc = spe::energy_issue(g, raw, false))) return rc;
    if ((rc = copy_out(g, raw, g->diag + 8, sizeof(raw), SPE_HOST))) return rc;
    return spe::energy_from_raw(g, raw, out);
}

int spe_set_static_potential(spe_grid *g, const float *phi_b, int where)
{
    if (!g || (where != SPE_HOST && where != SPE_DEVICE)) return SPE_EINVAL;
    if (!g->phib) return SPE_ESTATE;
    if (const int rc = settle(g)) return rc;   // the owed half kick feels the old potential
    if (!phi_b) {
        g->static_set = false;
        return SPE_OK;
    }
    cudaError_t e = cudaMemcpyAsync(g->phib, phi_b, g->ncells * sizeof(float),
                                    where == SPE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) return SPE_ECUDA;
    g->static_set = true;
    return SPE_OK;
}

int spe_virial(spe_grid *g, spe_virial_t *out)
{
    if (!g || !out) return SPE_EINVAL;
    int rc;
    if ((rc = settle(g))) return rc;
    if ((rc = potential_to_phi(g))) return rc;
    if ((rc = launch(g, KIND_DIAG, [&] {
             return launch_virial(g->psi, g->phi, g->n[0], g->n[1], g->n[2], (float)(0.5 / g->dx[0]),
                                  (float)(0.5 / g->dx[1]), (float)(0.5 / g->dx[2]), g->partials, g->counter,
                                  g->diag + 32, g->st);
         })))
        return rc;
    double raw[3];
    if ((rc = copy_out(g, raw, g->diag + 32, sizeof(raw), SPE_HOST))) return rc;
    const double eta = g->cfg.hbar_over_m;
    out->K = 0.5 * eta * eta * raw[0] * g->dv;
    out->Q = eta * eta * raw[1] * g->dv;
    out->V = raw[2] * g->dv;
    out->E = out->K + out->Q + out->V;
    out->virial = 2.0 * out->K + 2.0 * out->Q + out->V;
    return SPE_OK;
}

int spe_get_psi(spe_grid *g, void *out, int where)
{
    if (!g || !out || (where != SPE_HOST && where != SPE_DEVICE)) return SPE_EINVAL;
    if (const int rc = settle(g)) return rc;
    return copy_out(g, out, g->psi, g->ncells * sizeof(float2), where);
}

int spe_get_particles(spe_grid *g, float *pos3, float *vel3, int where)
{
    if (!g || (where != SPE_HOST && where != SPE_DEVICE)) return SPE_EINVAL;
    const size_t n = g->np;
    if (!n) return SPE_OK;
    if (const int rc = settle(g)) return rc;
    if (where == SPE_DEVICE) {
        int rc = launch(g, KIND_COPY, [&] {
            return launch_particles_from_soa_by_id(g->px, g->py, g->pz, g->vx, g->vy, g->vz, g->pid, (int)n, pos3,
                                                   vel3, g->st);
        });
        if (rc) return rc;
        return cuerr(cudaStreamSynchronize(g->st));
    }
    if (6 * n <= g->ncells) {
        // ordered on the device into the real-potential buffer (free between steps), then copied out
        float *stage = g->phi;
        int rc = launch(g, KIND_COPY, [&] {
            return launch_particles_from_soa_by_id(g->px, g->py, g->pz, g->vx, g->vy, g->vz, g->pid, (int)n,
                                                   pos3 ? stage : nullptr, vel3 ? stage + 3 * n : nullptr, g->st);
        });
        if (rc) return rc;
        cudaError_t e = cudaSuccess;
        if (pos3) e = cudaMemcpyAsync(pos3, stage, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, g->st);
        if (vel3 && e == cudaSuccess)
            e = cudaMemcpyAsync(vel3, stage + 3 * n, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, g->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
        return cuerr(e);
    }
    std::vector<float> soa(6 * n);
    std::vector<unsigned int> id(n);
    const float *src[6] = {g->px, g->py, g->pz, g->vx, g->vy, g->vz};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(soa.data() + k * n, src[k], n * sizeof(float), cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(id.data(), g->pid, n * sizeof(unsigned int), cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) return SPE_ECUDA;
    for (size_t i = 0; i < n; ++i) {
        const size_t o = id[i];
        if (o >= n) return SPE_ESTATE;
        for (int a = 0; a < 3; ++a) {
            if (pos3) pos3[3 * o + a] = soa[a * n + i];
            if (vel3) vel3[3 * o + a] = soa[(3 + a) * n + i];
        }
    }
    return SPE_OK;
}

int spe_particle_count(spe_grid *g, size_t *n_out)
{
    if (!g || !n_out) return SPE_EINVAL;
    *n_out = g->np;
    return SPE_OK;
}

int spe_sync(spe_grid *g)
{
    if (!g) return SPE_EINVAL;
    if (const int rc = settle(g)) return rc;
    return cuerr(cudaStreamSynchronize(g->st));
}

int spe_settle(spe_grid *g)
{
    if (!g) return SPE_EINVAL;
    return settle(g);
}

int spe_launch_count(spe_grid *g, unsigned long long *count_out, int reset)
{
    if (!g || !count_out) return SPE_EINVAL;
    *count_out = g->launches;
    if (reset) g->launches = 0;
    return SPE_OK;
}

int spe_profile_read(spe_grid *g, const char **names, unsigned long long *launches, double *ms, int cap)
{
    if (!g || cap < 0) return SPE_EINVAL;
    if (cudaStreamSynchronize(g->st) != cudaSuccess) return SPE_ECUDA;
    unsigned long long cnt[KIND_COUNT] = {0};
    double tot[KIND_COUNT] = {0};
    for (auto &r : g->prof) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.e0, r.e1) == cudaSuccess) tot[r.kind] += t;
        cnt[r.kind]++;
        g->evfree.push_back(r.e0);
        g->evfree.push_back(r.e1);
    }
    g->prof.clear();
    int w = 0;
    for (int k = 0; k < KIND_COUNT && w < cap; ++k) {
        if (names) names[w] = kKindNames[k];
        if (launches) launches[w] = cnt[k];
        if (ms) ms[w] = tot[k];
        ++w;
    }
    return w;
}

}  // extern "C"

// ======================================================================== autotuning
// The strided passes' tile width (8, 16 or 32 columns per CTA) and radix schedule are picked per
// (axis, transform length, row length nx, field) by timing every candidate on a scratch buffer the
// size of psi; choices are cached for the process.  psi's passes are timed as a forward and an
// inverse transform in one launch; the half spectrum's (rho forward, Poisson, Phi inverse) as the
// step runs them: the y forward and inverse as single transforms, the z forward transform, Poisson
// multiply and inverse transform in one launch.  Its 257 live columns at 512 points (against 512 for
// psi) and the Poisson pass's own register use can favour a narrower tile than psi's.

namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tuned;  // (axis, n, nx, field) -> (tile, plan)

int time_tile(spe_grid *g, int axis, bool half, int tile, int plan, float2 *scratch, float *ms_out)
{
    const int W = half ? g->W : g->n[0], P = half ? g->P : g->n[0];
    SParams p = axis == 1 ? base_y(g, scratch, W, P) : base_z(g, scratch, W, P);
    p.tile = tile;
    p.plan = plan;
    const int flags[2] = {half ? (axis == 1 ? S_FWD : S_FWD | S_POISSON | S_INV) : S_FWD | S_INV,
                          half && axis == 1 ? S_INV : 0};
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return SPE_ECUDA;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < 6 && e == cudaSuccess; ++r) {   // one warm-up round, then five timed
        if (r == 1) e = cudaEventRecord(a, g->st);
        for (int f = 0; f < 2 && e == cudaSuccess; ++f) {
            if (!flags[f]) continue;
            p.flags = flags[f];
            e = launch_spass(g->n[axis], p, g->st, nullptr);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, g->st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms_out, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return cuerr(e);
}

int autotune_grid(spe_grid *g, float2 *scratch)
{
    // the half spectrum (rows of P complex) must fit the psi-sized scratch
    const bool half_fits = (size_t)g->P * g->n[1] * g->n[2] <= g->ncells;
    for (int field = 0; field < 2; ++field) {
        int *tile_of = field ? g->htile : g->stile;
        int *plan_of = field ? g->hplan : g->splan;
        for (int axis = 1; axis <= 2; ++axis) {
            if (field == 1 && !half_fits) {
                tile_of[axis] = 0;   // as psi's
                plan_of[axis] = 0;
                continue;
            }
            const auto key = std::make_tuple(axis, g->n[axis], g->n[0], field);
            {
                std::lock_guard<std::mutex> lock(g_tune_mu);
                auto it = g_tuned.find(key);
                if (it != g_tuned.end()) {
                    tile_of[axis] = it->second.first;
                    plan_of[axis] = it->second.second;
                    continue;
                }
            }
            // candidates: tile widths 16, 8, 32 (32 only where it fits in shared memory) x the default
            // and the alternative radix schedules (lengths that have them)
            float best_ms = 0.f;
            int best_tile = 16, best_plan = 0, rc;
            bool first = true;
            for (int plan = 0; plan < plan_count_n(g->n[axis]); ++plan) {
                for (int tile : {16, 8, 32}) {
                    if (!spass_tile_ok(g->n[axis], tile)) continue;
                    float ms = 0.f;
                    if ((rc = time_tile(g, axis, field == 1, tile, plan, scratch, &ms))) return rc;
                    if (first || ms < best_ms) {
                        best_tile = tile;
                        best_plan = plan;
                        best_ms = ms;
                        first = false;
                    }
                }
            }
            tile_of[axis] = best_tile;
            plan_of[axis] = best_plan;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tuned[key] = std::make_pair(best_tile, best_plan);
        }
    }
    return SPE_OK;
}

}  // namespace

extern "C" int spe_autotune(spe_grid *g, int *tiles_out)
{
    if (!g) return SPE_EINVAL;
    float2 *scratch = nullptr;
    if (cudaMalloc(&scratch, g->ncells * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        return SPE_ENOMEM;
    }
    cudaMemsetAsync(scratch, 0, g->ncells * sizeof(float2), g->st);
    int rc = autotune_grid(g, scratch);
    cudaStreamSynchronize(g->st);
    cudaFree(scratch);
    if (!rc && tiles_out) {
        tiles_out[0] = g->stile[1];
        tiles_out[1] = g->stile[2];
    }
    return rc;
}

extern "C" int spe_set_schedule(spe_grid *g, const int *tiles, const int *plans)
{
    if (!g || !tiles || !plans) return SPE_EINVAL;
    for (int a = 0; a < 2; ++a) {
        const int n = g->n[a + 1];
        if (tiles[a] != 0 && !spass_tile_ok(n, tiles[a])) return SPE_EINVAL;
        if (plans[a] < 0 || plans[a] >= plan_count_n(n)) return SPE_EINVAL;
    }
    for (int a = 0; a < 2; ++a) {
        g->stile[a + 1] = tiles[a];
        g->splan[a + 1] = plans[a];
        g->htile[a + 1] = 0;   // the half spectrum's passes follow the pinned schedule
        g->hplan[a + 1] = 0;
    }
    return SPE_OK;
}

extern "C" int spe_get_schedule(spe_grid *g, int *tiles, int *plans)
{
    if (!g || !tiles || !plans) return SPE_EINVAL;
    for (int a = 0; a < 2; ++a) {
        tiles[a] = g->stile[a + 1] ? g->stile[a + 1] : spass_default_tile(g->n[a + 1]);
        plans[a] = g->splan[a + 1];
    }
    return SPE_OK;
}

extern "C" int spe_get_schedule_half(spe_grid *g, int *tiles, int *plans)
{
    if (!g || !tiles || !plans) return SPE_EINVAL;
    for (int a = 0; a < 2; ++a) {
        const bool own = g->htile[a + 1] != 0;
        const int t = own ? g->htile[a + 1] : g->stile[a + 1];
        tiles[a] = t ? t : spass_default_tile(g->n[a + 1]);
        plans[a] = own ? g->hplan[a + 1] : g->splan[a + 1];
    }
    return SPE_OK;
}

// ======================================================================== batches
// Independent grids of any supported sizes stepped together: every member runs
// on its own stream, and the members' full steps are captured as the parallel
// branches of one CUDA graph replayed on the batch stream, so small grids
// overlap on the GPU instead of each paying its own launch latency.

struct spe_batch {
    std::vector<spe_grid *> g;
    std::vector<cudaStream_t> ms;
    std::vector<cudaEvent_t> ev;
    cudaStream_t st;
    cudaStream_t cap;
    cudaEvent_t fork;
    cudaGraphExec_t exec;
    std::vector<double> key_dt;
    std::vector<size_t> key_np;
    std::vector<int> key_tiles;
    std::vector<unsigned long long> nodes;  // kernel launches per member in one captured step
    // one persistent launch per step (batch_persist.cu)
    bool persist;                           // use it when every member qualifies
    long long wait_limit;                   // barrier polls before a wait gives up
    int pblocks;                            // co-resident CTAs of the persistent kernel
    spe::BatchMember *d_mem;                // [2][count]: the first step of a call, then full steps
    int *d_offs;                            // kBatchPhases x (count + 1) work-list prefix sums
    unsigned int *d_bar;                    // barrier counter
    int *d_status;                          // timeout bit
    cudaGraphExec_t pexec;                  // memset of the counter + the launch of one full step
    std::vector<double> pkey_dt;
    std::vector<size_t> pkey_np;
    unsigned long long plaunches;           // persistent launches (kernel launches outside the members)
};

namespace {

constexpr long long kBatchWaitLimit = 1ll << 22;   // ~0.5 s of polling per barrier

// the persistent kernel carries code for gravitating cubic members of 64, 96, 128 or 192 points without
// a static potential, an absorbing layer or tensor-core stages
bool persist_member_ok(const spe_grid *g)
{
    return g->n[0] == g->n[1] && g->n[1] == g->n[2] && spe::batch_persist_n_ok(g->n[0]) && g->gravity && !g->tc &&
           !g->static_set && !g->absorbing && !(g->cfg.flags & SPE_PROFILE);
}

bool persist_ok(const spe_batch *b)
{
    if (!b->persist) return false;
    for (auto g : b->g)
        if (!persist_member_ok(g)) return false;
    return true;
}

// A member's passes for one step with leading kick dtk (the first step of a call) or dt (full
// steps), as step_body issues them for such a grid.
spe::BatchMember persist_member(spe_grid *g, double dtk, double dt)
{
    spe::BatchMember m;
    memset(&m, 0, sizeof(m));
    const bool parts = g->np > 0;
    const bool skick = parts && stars_kicked(g);
    m.xk = base_x(g);
    m.xk.flags = X_FFT | X_KICK | X_HAS_PHI | (skick ? X_WRITE_PHI : 0);
    m.xk.kick_scale = (float)(dtk / g->cfg.hbar_over_m);
    m.xd = base_x(g);
    m.xd.flags = X_IFFT | X_MASS | X_R2C | (parts ? X_DEP : 0);
    auto strided = [](SParams q, int flags) {
        q.flags = flags;
        q.tile = spe::kBatchTile;
        q.plan = 0;
        q.tma = 0;
        q.tc = 0;
        return q;
    };
    m.yf = strided(base_y(g, g->psi, g->n[0], g->n[0]), S_FWD);
    m.zd = strided(base_z(g, g->psi, g->n[0], g->n[0]), S_FWD | S_DRIFT | S_INV);
    m.yi = strided(base_y(g, g->psi, g->n[0], g->n[0]), S_INV);
    m.rf = strided(base_y(g, g->phik, g->W, g->P), S_FWD);
    m.rp = strided(base_z(g, g->phik, g->W, g->P), S_FWD | S_POISSON | S_INV);
    m.ri = strided(base_y(g, g->phik, g->W, g->P), S_INV);
    if (parts) {
        m.pp = base_p(g);
        m.pp.flags = PK_DRIFT | (skick ? PK_KICK : 0) | PK_DEPOSIT;
        m.pp.kick = (float)dtk;
        m.pp.drift = (float)dt;
    }
    m.n = g->n[0];
    m.xtiles = (g->n[1] * g->n[2] + 15) / 16;
    m.cols_psi = (g->n[0] + spe::kBatchTile - 1) / spe::kBatchTile;
    m.cols_rho = (g->W + spe::kBatchTile - 1) / spe::kBatchTile;
    m.pblocks = parts ? (int)((g->np + 255) / 256) : 0;
    return m;
}

// every member stream waits for the batch stream
int batch_fork(spe_batch *b)
{
    if (cudaEventRecord(b->fork, b->st) != cudaSuccess) return SPE_ECUDA;
    for (auto s : b->ms)
        if (cudaStreamWaitEvent(s, b->fork, 0) != cudaSuccess) return SPE_ECUDA;
    return SPE_OK;
}

// the batch stream waits for every member stream
int batch_join(spe_batch *b)
{
    for (size_t i = 0; i < b->ms.size(); ++i) {
        if (cudaEventRecord(b->ev[i], b->ms[i]) != cudaSuccess) return SPE_ECUDA;
        if (cudaStreamWaitEvent(b->st, b->ev[i], 0) != cudaSuccess) return SPE_ECUDA;
    }
    return SPE_OK;
}

int batch_graph(spe_batch *b, const double *dts)
{
    const size_t n = b->g.size();
    bool same = b->exec && b->key_dt.size() == n;
    for (size_t i = 0; same && i < n; ++i)
        same = b->key_dt[i] == dts[i] && b->key_np[i] == b->g[i]->np &&
               b->key_tiles[i] == schedule_key(b->g[i]) && !b->g[i]->static_set;
    if (same) return SPE_OK;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    std::vector<unsigned long long> before(n);
    for (size_t i = 0; i < n; ++i) before[i] = b->g[i]->launches;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    int rc = SPE_OK;
    if (e == cudaSuccess) {
        e = cudaEventRecord(b->fork, b->cap);
        for (size_t i = 0; i < n && e == cudaSuccess && !rc; ++i) {
            spe_grid *g = b->g[i];
            e = cudaStreamWaitEvent(b->ms[i], b->fork, 0);
            g->capturing = true;
            if (e == cudaSuccess) rc = step_body(g, dts[i], dts[i], true);
            g->capturing = false;
            if (e == cudaSuccess && !rc) e = cudaEventRecord(b->ev[i], b->ms[i]);
            if (e == cudaSuccess && !rc) e = cudaStreamWaitEvent(b->cap, b->ev[i], 0);
        }
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    b->nodes.resize(n);
    for (size_t i = 0; i < n; ++i) {
        b->nodes[i] = b->g[i]->launches - before[i];  // captured, not run: counted per replay instead
        b->g[i]->launches = before[i];
    }
    if (rc || e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc ? rc : SPE_ECUDA;
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        cudaGetLastError();
        return SPE_ECUDA;
    }
    b->key_dt.assign(dts, dts + n);
    b->key_np.resize(n);
    b->key_tiles.resize(n);
    for (size_t i = 0; i < n; ++i) {
        b->key_np[i] = b->g[i]->np;
        b->key_tiles[i] = schedule_key(b->g[i]);
    }
    return SPE_OK;
}

// One step of every member as one launch: the work lists of the step's phases (prefix sums per
// member) and the members' pass parameters go to the device; the barrier counter is cleared first.
int persist_launch(spe_batch *b, const spe::BatchMember *d_set)
{
    spe::BatchLaunch L;
    L.m = d_set;
    L.count = (int)b->g.size();
    L.offs = b->d_offs;
    L.bar = b->d_bar;
    L.status = b->d_status;
    L.wait_limit = b->wait_limit;
    if (cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned int), b->st) != cudaSuccess) return SPE_ECUDA;
    return cuerr(spe::launch_batch_persist(L, b->pblocks, b->st));
}

int persist_setup(spe_batch *b)
{
    if (b->d_mem) return SPE_OK;
    const size_t n = b->g.size();
    if (cuerr(spe::batch_persist_setup(&b->pblocks))) return SPE_ECUDA;
    if (cudaMalloc(&b->d_mem, 2 * n * sizeof(spe::BatchMember)) != cudaSuccess ||
        cudaMalloc(&b->d_offs, spe::kBatchPhases * (n + 1) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_bar, 256) != cudaSuccess || cudaMalloc(&b->d_status, 256) != cudaSuccess) {
        cudaGetLastError();
        return SPE_ENOMEM;
    }
    if (cudaMemsetAsync(b->d_status, 0, sizeof(int), b->st) != cudaSuccess) return SPE_ECUDA;
    return SPE_OK;
}

int persist_step(spe_batch *b, int nsteps, const double *dts)
{
    const size_t n = b->g.size();
    int rc;
    if ((rc = persist_setup(b))) return rc;
    // the batch stream takes over: it waits for the members' earlier work, and every member operation
    // of this call (tables, Phi(0), star reordering) goes onto it
    if ((rc = batch_join(b))) return rc;
    std::vector<cudaStream_t> own(n);
    for (size_t i = 0; i < n; ++i) {
        own[i] = b->g[i]->st;
        b->g[i]->st = b->st;
    }
    auto restore = [&](int code) {
        for (size_t i = 0; i < n; ++i) b->g[i]->st = own[i];
        const int f = batch_fork(b);
        return code ? code : f;
    };
    std::vector<spe::BatchMember> h(2 * n);
    std::vector<int> offs(spe::kBatchPhases * (n + 1), 0);
    for (size_t i = 0; i < n; ++i) {
        spe_grid *g = b->g[i];
        if ((rc = ensure_drift_tables(g, dts[i]))) return restore(rc);
        if (!g->phi_valid && (rc = compute_phi(g))) return restore(rc);
        const double lead = g->kick_pending ? g->pending_h + 0.5 * dts[i] : 0.5 * dts[i];
        g->kick_pending = false;
        h[i] = persist_member(g, lead, dts[i]);
        h[n + i] = persist_member(g, dts[i], dts[i]);
        const spe::BatchMember &m = h[i];
        const int items[spe::kBatchPhases] = {m.xtiles, m.cols_psi * m.n + m.pblocks, m.cols_psi * m.n,
                                              m.cols_psi * m.n, m.xtiles, m.cols_rho * m.n, m.cols_rho * m.n,
                                              m.cols_rho * m.n};
        for (int ph = 0; ph < spe::kBatchPhases; ++ph) offs[ph * (n + 1) + i + 1] = offs[ph * (n + 1) + i] + items[ph];
    }
    if (cudaMemcpyAsync(b->d_mem, h.data(), h.size() * sizeof(spe::BatchMember), cudaMemcpyHostToDevice, b->st) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_offs, offs.data(), offs.size() * sizeof(int), cudaMemcpyHostToDevice, b->st) !=
            cudaSuccess)
        return restore(SPE_ECUDA);
    // the full-step launch as a graph, captured again when dt or a star count changes
    bool same = b->pexec && b->pkey_dt.size() == n;
    for (size_t i = 0; same && i < n; ++i) same = b->pkey_dt[i] == dts[i] && b->pkey_np[i] == b->g[i]->np;
    if (nsteps > 1 && !same) {
        if (b->pexec) {
            cudaGraphExecDestroy(b->pexec);
            b->pexec = nullptr;
        }
        cudaStream_t keep = b->st;
        b->st = b->cap;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        int lrc = (e == cudaSuccess) ? persist_launch(b, b->d_mem + n) : SPE_ECUDA;
        const cudaError_t e2 = (e == cudaSuccess) ? cudaStreamEndCapture(b->cap, &graph) : e;
        b->st = keep;
        if (!lrc && e2 == cudaSuccess && cudaGraphInstantiate(&b->pexec, graph, 0) == cudaSuccess) {
            b->pkey_dt.assign(dts, dts + n);
            b->pkey_np.resize(n);
            for (size_t i = 0; i < n; ++i) b->pkey_np[i] = b->g[i]->np;
        } else {
            b->pexec = nullptr;   // the steps go out as direct launches
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
    }
    for (int s = 0; s < nsteps; ++s) {
        for (size_t i = 0; i < n; ++i) {
            spe_grid *g = b->g[i];
            if (g->np && (g->sort_due || g->steps_done % kSortEvery == 0) && (rc = sort_particles(g)))
                return restore(rc);
        }
        if (s > 0 && b->pexec) rc = cuerr(cudaGraphLaunch(b->pexec, b->st));
        else rc = persist_launch(b, b->d_mem + (s == 0 ? 0 : n));
        if (rc) return restore(rc);
        b->plaunches++;
        for (auto g : b->g) g->steps_done++;
    }
    for (size_t i = 0; i < n; ++i) {
        spe_grid *g = b->g[i];
        g->kick_pending = true;
        g->pending_h = 0.5 * dts[i];
        g->pending_dt = dts[i];
    }
    int status = 0;
    if (cudaMemcpyAsync(&status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->st) != cudaSuccess ||
        cudaStreamSynchronize(b->st) != cudaSuccess)
        return restore(SPE_ECUDA);
    if (status) {
        // the launch stopped part way: clear what a partial step leaves behind (star deposits, row
        // marks, reduction tickets) so that setting the state again starts from clean buffers
        if (cudaMemsetAsync(b->d_status, 0, sizeof(int), b->st) != cudaSuccess) return restore(SPE_ECUDA);
        for (auto g : b->g) {
            if (g->dep && cudaMemsetAsync(g->dep, 0, g->ncells * sizeof(long long), b->st) != cudaSuccess)
                return restore(SPE_ECUDA);
            if (g->dflag && cudaMemsetAsync(g->dflag, 0, (size_t)g->n[1] * g->n[2], b->st) != cudaSuccess)
                return restore(SPE_ECUDA);
            if (cudaMemsetAsync(g->counter, 0, sizeof(unsigned int), b->st) != cudaSuccess) return restore(SPE_ECUDA);
            g->phi_valid = false;
        }
        if (cudaStreamSynchronize(b->st) != cudaSuccess) return restore(SPE_ECUDA);
        return restore(SPE_ETIMEOUT);
    }
    return restore(SPE_OK);
}

}  // namespace

extern "C" {

int spe_batch_destroy(spe_batch *b)
{
    if (!b) return SPE_EINVAL;
    cudaStreamSynchronize(b->st);
    for (auto g : b->g) spe_destroy(g);
    for (auto s : b->ms) cudaStreamDestroy(s);
    for (auto e : b->ev) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->pexec) cudaGraphExecDestroy(b->pexec);
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaFree(b->d_mem);
    cudaFree(b->d_offs);
    cudaFree(b->d_bar);
    cudaFree(b->d_status);
    delete b;
    return SPE_OK;
}

int spe_batch_create(const spe_config *cfgs, int count, spe_batch **out)
{
    if (!cfgs || count <= 0 || !out) return SPE_EINVAL;
    *out = nullptr;
    spe_batch *b = new (std::nothrow) spe_batch();
    if (!b) return SPE_ENOMEM;
    b->persist = false;   // the graph of per-member branches measured faster (the persistent form is opt-in)
    b->wait_limit = kBatchWaitLimit;
    b->st = (cudaStream_t)cfgs[0].cuda_stream;
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        spe_batch_destroy(b);
        return SPE_ECUDA;
    }
    for (int i = 0; i < count; ++i) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            spe_batch_destroy(b);
            return SPE_ECUDA;
        }
        b->ms.push_back(s);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            spe_batch_destroy(b);
            return SPE_ECUDA;
        }
        b->ev.push_back(e);
        spe_config c = cfgs[i];
        c.cuda_stream = s;
        c.flags = (c.flags | SPE_NO_GRAPH) & ~SPE_PROFILE;
        spe_grid *g = nullptr;
        int rc = spe_create_grid(&c, nullptr, 0, &g);
        if (rc) {
            spe_batch_destroy(b);
            return rc;
        }
        b->g.push_back(g);
    }
    *out = b;
    return SPE_OK;
}

int spe_batch_grid(spe_batch *b, int i, spe_grid **out)
{
    if (!b || !out || i < 0 || i >= (int)b->g.size()) return SPE_EINVAL;
    *out = b->g[i];
    return SPE_OK;
}

int spe_batch_autotune(spe_batch *b)
{
    if (!b) return SPE_EINVAL;
    for (auto g : b->g) {
        int rc = spe_autotune(g, nullptr);
        if (rc) return rc;
    }
    return SPE_OK;
}

int spe_batch_step(spe_batch *b, int nsteps, const double *dts)
{
    if (!b || nsteps < 0 || !dts) return SPE_EINVAL;
    if (nsteps == 0) return SPE_OK;
    const size_t n = b->g.size();
    int rc;
    for (size_t i = 0; i < n; ++i) {
        spe_grid *g = b->g[i];
        if (!isfinite(dts[i])) return SPE_EINVAL;
        if (!(g->cfg.flags & SPE_NO_CFL_CHECK)) {
            double dx = fmin(g->dx[0], fmin(g->dx[1], g->dx[2]));
            if (fabs(dts[i]) > 0.5 * 4.0 / (3.0 * kPi) * dx * dx / g->cfg.hbar_over_m * (1.0 + 1e-12)) return SPE_ECFL;
        }
    }
    // members owe their closing half kicks like lone grids (spe_step): merged into the leading
    // kick when dt is unchanged, applied first otherwise
    for (size_t i = 0; i < n; ++i) {
        spe_grid *g = b->g[i];
        if (g->kick_pending && g->pending_dt != dts[i] && (rc = settle(g))) return rc;
        g->host_mass_valid = false;
    }
    if (persist_ok(b)) return persist_step(b, nsteps, dts);
    if ((rc = batch_fork(b))) return rc;
    for (size_t i = 0; i < n; ++i) {
        spe_grid *g = b->g[i];
        if ((rc = ensure_drift_tables(g, dts[i]))) return rc;
        if (!g->phi_valid && (rc = compute_phi(g))) return rc;
        const bool merge = g->kick_pending;
        const double lead = merge ? g->pending_h + 0.5 * dts[i] : 0.5 * dts[i];
        g->kick_pending = false;
        if ((rc = step_body(g, lead, dts[i], merge))) return rc;
        g->steps_done++;
    }
    if ((rc = batch_join(b))) return rc;
    if (nsteps > 1) {
        if ((rc = batch_graph(b, dts))) return rc;
        for (int s = 1; s < nsteps; ++s)
            if (cudaGraphLaunch(b->exec, b->st) != cudaSuccess) return SPE_ECUDA;
        for (size_t i = 0; i < n; ++i) {
            b->g[i]->steps_done += nsteps - 1;
            b->g[i]->launches += (unsigned long long)(nsteps - 1) * b->nodes[i];
        }
    }
    for (size_t i = 0; i < n; ++i) {
        spe_grid *g = b->g[i];
        g->kick_pending = true;
        g->pending_h = 0.5 * dts[i];
        g->pending_dt = dts[i];
    }
    if (cudaStreamSynchronize(b->st) != cudaSuccess) return SPE_ECUDA;
    return SPE_OK;
}

int spe_batch_settle(spe_batch *b)
{
    if (!b) return SPE_EINVAL;
    int rc;
    if ((rc = batch_fork(b))) return rc;
    for (auto g : b->g)
        if ((rc = settle(g))) return rc;
    return batch_join(b);
}

int spe_batch_launch_count(spe_batch *b, unsigned long long *count_out)
{
    if (!b || !count_out) return SPE_EINVAL;
    unsigned long long c = b->plaunches;
    for (auto g : b->g) c += g->launches;
    *count_out = c;
    return SPE_OK;
}

int spe_pair_norms(const void *a, const void *b, size_t n, int samples, double *out, void *cuda_stream)
{
    if (!a || !b || !out || n == 0 || samples <= 0) return SPE_EINVAL;
    if ((((uintptr_t)a | (uintptr_t)b | (uintptr_t)out) & 7) != 0) return SPE_EINVAL;
    return cuerr(spe::launch_pair_norms(static_cast<const float2 *>(a), static_cast<const float2 *>(b), n, samples,
                                        out, (cudaStream_t)cuda_stream));
}

int spe_batch_set_persistent(spe_batch *b, int on, long long wait_limit)
{
    if (!b || wait_limit < -1) return SPE_EINVAL;
    b->persist = on != 0;
    b->wait_limit = wait_limit < 0 ? kBatchWaitLimit : wait_limit;
    return SPE_OK;
}

int spe_batch_get_persistent(spe_batch *b, int *on_out)
{
    if (!b || !on_out) return SPE_EINVAL;
    *on_out = persist_ok(b) ? 1 : 0;
    return SPE_OK;
}

}  // extern "C"
