// The FNO surrogate's C ABI (include/spe_fno.h): parameters, buffers and the
// launch sequence of a forward pass, a backward pass and an Adam step.
//
// Forward (per layer l, after the lift has written v_0 and its x DFT):
//   y DFT  (axis over y, Efwd)      x-row buffer -> y-stage buffer
//   z DFT, mixing (R_l per mode), z IDFT (Einv, 1/n): one fused kernel per
//          (ky, kx) column, in place in the y-stage buffer (modes X_l kept
//          for training)
//   y IDFT (axis, Einv, 1/n)        -> x-row buffer
//   row kernel: x IDFT (Gx, 1/n) + W v + b, GELU, next x DFT (or projection)
// Backward runs the adjoints in reverse: an adjoint of a stage with matrix A
// is the same contraction with A^H (Efwd^H = Einv, Einv^H = Efwd, with the
// inverse's 1/n carried over).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fno_internal.cuh"
#include "spe_fno.h"

using namespace spe::fno;

// kernel kinds of the per-kernel event profile (SPE_FNO_PROFILE)
enum FnoKind {
    FK_LIFT, FK_LAYER, FK_LAST, FK_PROJ, FK_Y_FWD, FK_ZMIX, FK_Y_INV, FK_TOP_BWD, FK_START_BWD, FK_LAYER_BWD,
    FK_LIFT_BWD, FK_AXIS_BWD, FK_MIX_BWD, FK_REDUCE, FK_ADAM, FK_COUNT
};
static const char *kFnoKindNames[FK_COUNT] = {
    "fno_lift", "fno_layer", "fno_last_layer", "fno_projection", "fno_y_dft", "fno_z_mix", "fno_y_idft",
    "fno_top_bwd", "fno_start_bwd", "fno_layer_bwd", "fno_lift_bwd", "fno_axis_bwd", "fno_mix_bwd",
    "fno_reduce", "fno_adam"};

struct spe_fno {
    spe_fno_config cfg;
    int n, L, M, B;
    bool train, fp32;
    cudaStream_t st;
    Offsets off;
    size_t nparams;
    float *master, *grad, *am, *av;
    __nv_bfloat16 *w16;
    long long adam_t;
    float2 *Efwd, *Einv;
    uint4 *tcG, *tcF;
    uint4 *tcFt, *tcGt;     // backward operand images
    void *act[16];
    float2 *xrow, *ym, *Ybuf, *Xbbuf, *Xsave[8];
    float *ubar, *partials;
    double *dres;
    int *status;
    const float2 *last_psi, *last_psib;
    int last_batch;
    bool have_fwd;
    unsigned long long launches;
    std::vector<void *> allocs;
    // inference forward replayed as a CUDA graph, keyed by its buffers, batch and stream
    cudaGraphExec_t fwd_exec;
    cudaStream_t cap_st;
    const void *key_psi, *key_psib;
    void *key_out;
    int key_batch;
    cudaStream_t key_st;
    int key_seen;
    unsigned long long graph_launches;
    // per-kernel profile: event pairs recorded around each launch, read back by spe_fno_profile_read
    bool profile;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_pending;
    std::vector<cudaEvent_t> prof_free;
    unsigned long long prof_launches[FK_COUNT];
    double prof_ms[FK_COUNT];
};

namespace {

const double kPi = 3.14159265358979323846264338327950288;

bool config_ok(const spe_fno_config *c)
{
    if (!c) return false;
    if (c->n != 32 && c->n != 64) return false;
    if (c->modes != 8 && c->modes != 16) return false;
    if (c->modes > c->n / 2) return false;
    if (c->layers < 1 || c->layers > 8) return false;
    if (c->max_batch < 1 || c->max_batch > 256) return false;
    if (!std::isfinite(c->inv_A) || !std::isfinite(c->sigma) || c->sigma == 0.0) return false;
    return true;
}

Offsets make_offsets(int L, int M)
{
    Offsets o{};
    size_t off = 0;
    o.P = off; off += kC * kFin;
    o.p = off; off += kC;
    for (int l = 0; l < L; ++l) {
        o.W[l] = off; off += kC * kC;
        o.b[l] = off; off += kC;
        o.R[l] = off; off += (size_t)M * M * M * kC * kC * 2;
    }
    o.Q1 = off; off += kH * kC;
    o.q1 = off; off += kH;
    o.Q2 = off; off += kFout * kH;
    o.q2 = off; off += kFout;
    o.total = off;
    return o;
}

int signed_freq(int m, int M) { return m < M / 2 ? m : m - M; }

// float -> bfloat16 bits, round to nearest even (finite inputs)
unsigned short host_bf16(float v)
{
    uint32_t b;
    std::memcpy(&b, &v, 4);
    b += 0x7FFFu + ((b >> 16) & 1u);
    return (unsigned short)(b >> 16);
}

// byte offset of (row, k) in a no-swizzle K-major tensor-core operand with K columns
int kmaj_host(int row, int k, int K) { return (row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2; }

// BF16 operand images of the x stages for the tensor-core row kernels:
// G' [n][2M]: (Re Gx, -Im Gx) pairs; F' [2M][n]: rows (Re Fx), (Im Fx).
void build_tc_images(int n, int M, std::vector<unsigned char> &g, std::vector<unsigned char> &fimg,
                     std::vector<unsigned char> &ft, std::vector<unsigned char> &gt)
{
    const int KM = 2 * M;
    g.assign((size_t)n * KM * 2, 0);
    fimg.assign((size_t)n * KM * 2, 0);
    ft.assign((size_t)n * KM * 2, 0);
    gt.assign((size_t)n * KM * 2, 0);
    for (int x = 0; x < n; ++x)
        for (int k = 0; k < M; ++k) {
            const double th = 2.0 * kPi * (double)((long long)k * x % n) / n;
            const double w = (k == 0 ? 1.0 : 2.0) / n;
            const float gr = (float)(w * std::cos(th)), gi = (float)(w * std::sin(th));
            const float fr = (float)std::cos(th), fi = (float)-std::sin(th);
            auto put = [](std::vector<unsigned char> &v, int off, float val) {
                const unsigned short h = host_bf16(val);
                std::memcpy(v.data() + off, &h, 2);
            };
            put(g, kmaj_host(x, 2 * k, KM), gr);
            put(g, kmaj_host(x, 2 * k + 1, KM), -gi);
            put(fimg, kmaj_host(2 * k, x, n), fr);
            put(fimg, kmaj_host(2 * k + 1, x, n), fi);
            // backward: F'' [x][kk] (v bar = Re(Fx^H a bar)) and G'' [kk][x] (Bbar = Gx^H u bar)
            put(ft, kmaj_host(x, 2 * k, KM), fr);
            put(ft, kmaj_host(x, 2 * k + 1, KM), fi);
            put(gt, kmaj_host(2 * k, x, n), gr);
            put(gt, kmaj_host(2 * k + 1, x, n), -gi);
        }
}

std::mutex g_tables_mu;
bool g_tables_done[64];

// x-stage tables for n = 64 and 32 into both row-kernel translation units,
// once per device.
cudaError_t ensure_x_tables()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_tables_mu);
    if (dev < 64 && g_tables_done[dev]) return cudaSuccess;
    std::vector<float2> G[2], F[2];
    const int ns[2] = {64, 32};
    for (int s = 0; s < 2; ++s) {
        const int n = ns[s];
        G[s].resize((size_t)n * kTableM);
        F[s].resize((size_t)kTableM * n);
        for (int x = 0; x < n; ++x)
            for (int k = 0; k < kTableM; ++k) {
                const double th = 2.0 * kPi * (double)((long long)k * x % n) / n;
                const double w = (k == 0 ? 1.0 : 2.0) / n;
                G[s][(size_t)x * kTableM + k] = make_float2((float)(w * std::cos(th)), (float)(w * std::sin(th)));
                F[s][(size_t)k * n + x] = make_float2((float)std::cos(th), (float)-std::sin(th));
            }
    }
    e = upload_fwd_tables(G[0].data(), F[0].data(), G[1].data(), F[1].data());
    if (e == cudaSuccess) e = upload_bwd_tables(G[0].data(), F[0].data(), G[1].data(), F[1].data());
    if (e == cudaSuccess && dev < 64) g_tables_done[dev] = true;
    return e;
}

template <typename T>
cudaError_t dalloc(spe_fno *f, T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
    if (e != cudaSuccess) return e;
    f->allocs.push_back(q);
    *p = (T *)q;
    return cudaSuccess;
}

size_t act_bytes(const spe_fno *f) { return f->fp32 ? sizeof(float) : sizeof(__nv_bfloat16); }

void *v_buf(spe_fno *f, int l) { return f->train ? f->act[l] : f->act[l & 1]; }
void *u_buf(spe_fno *f, int l) { return f->train ? f->act[f->L + 1 + l] : nullptr; }

RowArgs base_args(spe_fno *f, int batch)
{
    RowArgs a{};
    a.rows = batch * f->n * f->n;
    a.w = f->w16;
    a.oP = f->off.P;
    a.op = f->off.p;
    a.oQ1 = f->off.Q1;
    a.oq1 = f->off.q1;
    a.oQ2 = f->off.Q2;
    a.oq2 = f->off.q2;
    a.inv_A = (float)f->cfg.inv_A;
    a.sigma = (float)f->cfg.sigma;
    a.xrow = f->xrow;
    a.ubar = f->ubar;
    a.partials = f->partials;
    a.status = f->status;
    a.tcG = f->tcG;
    a.tcF = f->tcF;
    a.tcFt = f->tcFt;
    a.tcGt = f->tcGt;
    return a;
}

int row_grid(int rows) { return rows < kRowBlocks ? rows : kRowBlocks; }

cudaEvent_t prof_event(spe_fno *f)
{
    if (!f->prof_free.empty()) {
        cudaEvent_t e = f->prof_free.back();
        f->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// one kernel launch of kind k: counted, and bracketed by events in profile mode
template <typename F>
cudaError_t run_kind(spe_fno *f, int k, F &&launch)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (f->profile) {
        e0 = prof_event(f);
        e1 = prof_event(f);
        cudaEventRecord(e0, f->st);
    }
    const cudaError_t e = launch();
    if (f->profile) {
        cudaEventRecord(e1, f->st);
        f->prof_pending.push_back({k, {e0, e1}});
    }
    ++f->launches;
    return e;
}

#define SPE_TRY(kind, expr)                                                     \
    do {                                                                        \
        if (run_kind(f, kind, [&] { return (expr); }) != cudaSuccess) return SPE_ECUDA; \
    } while (0)

// forward stages of layer l's spectral path: x-row buffer (x DFT of v_l) -> x-row buffer (y IDFT)
int spectral_fwd(spe_fno *f, int l, int batch)
{
    const int n = f->n, M = f->M;
    SPE_TRY(FK_Y_FWD, launch_axis(f->xrow, f->ym, f->Efwd, n, M, true, batch * n, M * kC, 1.f, f->st));
    SPE_TRY(FK_ZMIX, launch_zmix_fwd(n, M, f->ym, f->train ? f->Xsave[l] : nullptr, f->w16 + f->off.R[l], f->Efwd, f->Einv,
                            batch, f->st));
    SPE_TRY(FK_Y_INV, launch_axis(f->ym, f->xrow, f->Einv, n, M, false, batch * n, M * kC, 1.f / n, f->st));
    return SPE_OK;
}

// adjoint of layer l's spectral path: x-row buffer (Bbar) -> x-row buffer (abar), dL/dR_l
int spectral_bwd(spe_fno *f, int l, int batch)
{
    const int n = f->n, M = f->M;
    SPE_TRY(FK_AXIS_BWD, launch_axis(f->xrow, f->ym, f->Efwd, n, M, true, batch * n, M * kC, 1.f / n, f->st));
    SPE_TRY(FK_AXIS_BWD, launch_axis(f->ym, f->Ybuf, f->Efwd, n, M, true, batch, M * M * kC, 1.f / n, f->st));
    SPE_TRY(FK_MIX_BWD, launch_mix_bwd(M, f->Ybuf, f->Xsave[l], f->Xbbuf, f->w16 + f->off.R[l], f->grad + f->off.R[l], batch,
                           f->st));
    SPE_TRY(FK_AXIS_BWD, launch_axis(f->Xbbuf, f->ym, f->Einv, n, M, false, batch, M * M * kC, 1.f, f->st));
    SPE_TRY(FK_AXIS_BWD, launch_axis(f->ym, f->xrow, f->Einv, n, M, false, batch * n, M * kC, 1.f, f->st));
    return SPE_OK;
}

int reduce_into(spe_fno *f, int seg, int nblk, float *dst, int ndst, double *extra)
{
    SPE_TRY(FK_REDUCE, launch_reduce_partials(f->partials, seg, nblk, dst, ndst, extra, f->st));
    return SPE_OK;
}

void free_all(spe_fno *f)
{
    for (void *p : f->allocs) cudaFree(p);
    f->allocs.clear();
}

}  // namespace

extern "C" {
static int issue_forward(spe_fno *f, const void *psi, const void *psi_b, void *psi_out, int batch);
}

int spe::fno::net_n(const spe_fno *f) { return f->n; }
cudaStream_t spe::fno::net_stream(const spe_fno *f) { return f->st; }

int spe::fno::forward_direct(spe_fno *f, cudaStream_t st, const void *psi, const void *psi_b, void *psi_out,
                             int batch)
{
    if (!f || !psi || !psi_b || !psi_out || batch < 1 || batch > f->B) return SPE_EINVAL;
    const cudaStream_t keep = f->st;
    f->st = st;
    const int rc = issue_forward(f, psi, psi_b, psi_out, batch);
    f->st = keep;
    return rc;
}

int spe::fno::forward_on_stream(spe_fno *f, cudaStream_t st, const void *psi, const void *psi_b, void *psi_out,
                                int batch)
{
    const cudaStream_t keep = f->st;
    f->st = st;
    const int rc = spe_fno_forward(f, psi, psi_b, psi_out, batch);
    f->st = keep;
    return rc;
}

extern "C" {

SPE_API int spe_fno_param_count(const spe_fno_config *cfg, size_t *count)
{
    if (!config_ok(cfg) || !count) return SPE_EINVAL;
    *count = make_offsets(cfg->layers, cfg->modes).total;
    return SPE_OK;
}

SPE_API int spe_fno_create(const spe_fno_config *cfg, spe_fno **out)
{
    if (!config_ok(cfg) || !out) return SPE_EINVAL;
    *out = nullptr;
    spe_fno *f = new (std::nothrow) spe_fno();
    if (!f) return SPE_ENOMEM;
    f->cfg = *cfg;
    f->n = cfg->n;
    f->L = cfg->layers;
    f->M = cfg->modes;
    f->B = cfg->max_batch;
    f->train = (cfg->flags & SPE_FNO_TRAIN) != 0;
    f->fp32 = (cfg->flags & SPE_FNO_ACT_FP32) != 0;
    f->st = (cudaStream_t)cfg->cuda_stream;
    f->profile = (cfg->flags & SPE_FNO_PROFILE) != 0;
    f->off = make_offsets(f->L, f->M);
    f->nparams = f->off.total;
    const size_t n = f->n, M = f->M, B = f->B, cells = n * n * n;
    cudaError_t e = ensure_x_tables();
    auto ok = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    ok(dalloc(f, &f->master, f->nparams));
    ok(dalloc(f, &f->grad, f->nparams));
    ok(dalloc(f, &f->am, f->nparams));
    ok(dalloc(f, &f->av, f->nparams));
    ok(dalloc(f, &f->w16, f->nparams));
    ok(dalloc(f, &f->Efwd, M * n));
    ok(dalloc(f, &f->tcG, n * 2 * M * 2 / 16));
    ok(dalloc(f, &f->tcF, n * 2 * M * 2 / 16));
    ok(dalloc(f, &f->tcFt, n * 2 * M * 2 / 16));
    ok(dalloc(f, &f->tcGt, n * 2 * M * 2 / 16));
    ok(dalloc(f, &f->Einv, n * M));
    const int nact = f->train ? 2 * f->L : 2;
    for (int i = 0; i < nact; ++i) {
        unsigned char *p = nullptr;
        ok(dalloc(f, &p, B * cells * kC * act_bytes(f)));
        f->act[i] = p;
    }
    ok(dalloc(f, &f->xrow, B * n * n * M * kC));
    ok(dalloc(f, &f->ym, B * n * M * M * kC));
    ok(dalloc(f, &f->Ybuf, B * M * M * M * kC));
    ok(dalloc(f, &f->Xbbuf, B * M * M * M * kC));
    for (int l = 0; l < (f->train ? f->L : 0); ++l) ok(dalloc(f, &f->Xsave[l], B * M * M * M * kC));
    if (f->train) ok(dalloc(f, &f->ubar, B * cells * kC));
    ok(dalloc(f, &f->partials, (size_t)kRowBlocks * kTopSeg));
    ok(dalloc(f, &f->dres, 8));
    ok(dalloc(f, &f->status, 1));
    if (e == cudaSuccess) {
        std::vector<float2> Ef(M * n), Ei(n * M);
        for (size_t m = 0; m < M; ++m)
            for (size_t j = 0; j < n; ++j) {
                const long long fm = signed_freq((int)m, (int)M);
                const long long r = ((fm * (long long)j) % (long long)n + (long long)n) % (long long)n;
                const double th = 2.0 * kPi * (double)r / (double)n;
                Ef[m * n + j] = make_float2((float)std::cos(th), (float)-std::sin(th));
                Ei[j * M + m] = make_float2((float)std::cos(th), (float)std::sin(th));
            }
        ok(cudaMemcpy(f->Efwd, Ef.data(), Ef.size() * sizeof(float2), cudaMemcpyHostToDevice));
        ok(cudaMemcpy(f->Einv, Ei.data(), Ei.size() * sizeof(float2), cudaMemcpyHostToDevice));
        std::vector<unsigned char> gimg, fimg, ftimg, gtimg;
        build_tc_images((int)n, (int)M, gimg, fimg, ftimg, gtimg);
        ok(cudaMemcpy(f->tcG, gimg.data(), gimg.size(), cudaMemcpyHostToDevice));
        ok(cudaMemcpy(f->tcF, fimg.data(), fimg.size(), cudaMemcpyHostToDevice));
        ok(cudaMemcpy(f->tcFt, ftimg.data(), ftimg.size(), cudaMemcpyHostToDevice));
        ok(cudaMemcpy(f->tcGt, gtimg.data(), gtimg.size(), cudaMemcpyHostToDevice));
        ok(cudaMemset(f->master, 0, f->nparams * sizeof(float)));
        ok(cudaMemset(f->grad, 0, f->nparams * sizeof(float)));
        ok(cudaMemset(f->am, 0, f->nparams * sizeof(float)));
        ok(cudaMemset(f->av, 0, f->nparams * sizeof(float)));
        ok(cudaMemset(f->w16, 0, f->nparams * sizeof(__nv_bfloat16)));
        ok(cudaMemset(f->status, 0, sizeof(int)));
    }
    if (e != cudaSuccess) {
        const int rc = (e == cudaErrorMemoryAllocation) ? SPE_ENOMEM : SPE_ECUDA;
        free_all(f);
        delete f;
        return rc;
    }
    *out = f;
    return SPE_OK;
}

SPE_API int spe_fno_destroy(spe_fno *f)
{
    if (!f) return SPE_EINVAL;
    cudaStreamSynchronize(f->st);
    if (f->fwd_exec) cudaGraphExecDestroy(f->fwd_exec);
    if (f->cap_st) cudaStreamDestroy(f->cap_st);
    for (auto &p : f->prof_pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (auto e : f->prof_free) cudaEventDestroy(e);
    free_all(f);
    delete f;
    return SPE_OK;
}

SPE_API int spe_fno_set_params(spe_fno *f, const float *params, size_t count, int where)
{
    if (!f || !params || count != f->nparams || (where != SPE_HOST && where != SPE_DEVICE)) return SPE_EINVAL;
    cudaError_t e = cudaMemcpyAsync(f->master, params, count * sizeof(float),
                                    where == SPE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, f->st);
    if (e == cudaSuccess) {
        e = launch_mirror(f->master, f->w16, f->nparams, f->st);
        ++f->launches;
    }
    if (e == cudaSuccess && where == SPE_HOST) e = cudaStreamSynchronize(f->st);
    return e == cudaSuccess ? SPE_OK : SPE_ECUDA;
}

static int copy_out_vec(spe_fno *f, float *dst, const float *src, size_t count, int where)
{
    if (!f || !dst || count != f->nparams || (where != SPE_HOST && where != SPE_DEVICE)) return SPE_EINVAL;
    cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(float),
                                    where == SPE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, f->st);
    if (e == cudaSuccess && where == SPE_HOST) e = cudaStreamSynchronize(f->st);
    return e == cudaSuccess ? SPE_OK : SPE_ECUDA;
}

SPE_API int spe_fno_get_params(spe_fno *f, float *params, size_t count, int where)
{
    return copy_out_vec(f, params, f ? f->master : nullptr, count, where);
}

SPE_API int spe_fno_get_grads(spe_fno *f, float *grads, size_t count, int where)
{
    return copy_out_vec(f, grads, f ? f->grad : nullptr, count, where);
}

static int issue_forward(spe_fno *f, const void *psi, const void *psi_b, void *psi_out, int batch)
{
    const int n = f->n, M = f->M, L = f->L;
    const int rows = batch * n * n, grid = row_grid(rows);
    RowArgs a = base_args(f, batch);
    a.psi = (const float2 *)psi;
    a.psib = (const float2 *)psi_b;
    a.out = (float2 *)psi_out;
    a.vout = v_buf(f, 0);
    // BF16 activations run the row stages on the tensor cores; FP32 keeps the CUDA-core kernels
    const bool tc = !f->fp32;
    const int tiles = rows / kTcTile, tgrid = tiles < kTcBlocks ? tiles : kTcBlocks;
    if (tc)
        SPE_TRY(FK_LIFT, launch_layer_fwd_tc(n, M, 2, a, tgrid, f->st));
    else
        SPE_TRY(FK_LIFT, launch_lift_fwd(n, M, f->fp32, a, grid, f->st));
    for (int l = 0; l < L; ++l) {
        int rc = spectral_fwd(f, l, batch);
        if (rc) return rc;
        RowArgs b = base_args(f, batch);
        b.psib = (const float2 *)psi_b;
        b.out = (float2 *)psi_out;
        b.vin = v_buf(f, l);
        b.vout = v_buf(f, l + 1);
        b.uout = u_buf(f, l);
        b.store_u = (f->train && l < L - 1) ? 1 : 0;
        b.oW = f->off.W[l];
        b.ob = f->off.b[l];
        if (tc) {
            SPE_TRY(l == L - 1 ? FK_LAST : FK_LAYER, launch_layer_fwd_tc(n, M, l == L - 1 ? 1 : 0, b, tgrid, f->st));
        } else {
            SPE_TRY(l == L - 1 ? FK_LAST : FK_LAYER, launch_layer_fwd(n, M, f->fp32, l == L - 1, b, grid, f->st));
        }
    }
    if (tc) {
        RowArgs p = base_args(f, batch);
        p.vin = v_buf(f, L);
        p.psib = (const float2 *)psi_b;
        p.out = (float2 *)psi_out;
        const int cells = rows * n, ptiles = cells / 128;
        SPE_TRY(FK_PROJ, launch_proj_tc(p, cells, ptiles < kProjBlocks ? ptiles : kProjBlocks, f->st));
    }
    return SPE_OK;
}

// Capture the inference forward for these buffers once on a private stream;
// returns SPE_OK with f->fwd_exec set, or an error (nothing is left captured).
static int capture_forward(spe_fno *f, const void *psi, const void *psi_b, void *psi_out, int batch)
{
    if (!f->cap_st && cudaStreamCreateWithFlags(&f->cap_st, cudaStreamNonBlocking) != cudaSuccess) return SPE_ECUDA;
    if (f->fwd_exec) {
        cudaGraphExecDestroy(f->fwd_exec);
        f->fwd_exec = nullptr;
    }
    const cudaStream_t user = f->st;
    const unsigned long long before = f->launches;
    f->st = f->cap_st;
    cudaGraph_t graph = nullptr;
    int rc = SPE_OK;
    if (cudaStreamBeginCapture(f->cap_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = SPE_ECUDA;
    if (rc == SPE_OK) rc = issue_forward(f, psi, psi_b, psi_out, batch);
    const cudaError_t ec = cudaStreamEndCapture(f->cap_st, &graph);
    f->st = user;
    f->launches = before;
    if (rc == SPE_OK && ec != cudaSuccess) rc = SPE_ECUDA;
    if (rc == SPE_OK && cudaGraphInstantiate(&f->fwd_exec, graph, 0) != cudaSuccess) {
        f->fwd_exec = nullptr;
        rc = SPE_ECUDA;
    }
    size_t nodes = 0;
    if (graph) {
        cudaGraphGetNodes(graph, nullptr, &nodes);
        cudaGraphDestroy(graph);
    }
    f->graph_launches = nodes;
    return rc;
}

SPE_API int spe_fno_forward(spe_fno *f, const void *psi, const void *psi_b, void *psi_out, int batch)
{
    if (!f || !psi || !psi_b || !psi_out || batch < 1 || batch > f->B) return SPE_EINVAL;
    int rc;
    const bool same = f->key_psi == psi && f->key_psib == psi_b && f->key_out == psi_out &&
                      f->key_batch == batch && f->key_st == f->st;
    if (f->train || f->profile || (f->cfg.flags & SPE_FNO_NO_GRAPH)) {
        if ((rc = issue_forward(f, psi, psi_b, psi_out, batch))) return rc;
    } else if (same && f->key_seen >= 1) {
        // a repeated call: replay (capturing it on its second occurrence)
        if (!f->fwd_exec || f->key_seen == 1) {
            if ((rc = capture_forward(f, psi, psi_b, psi_out, batch))) return rc;
            f->key_seen = 2;
        }
        if (cudaGraphLaunch(f->fwd_exec, f->st) != cudaSuccess) return SPE_ECUDA;
        f->launches += f->graph_launches;
    } else {
        f->key_psi = psi;
        f->key_psib = psi_b;
        f->key_out = psi_out;
        f->key_batch = batch;
        f->key_st = f->st;
        f->key_seen = 1;
        if ((rc = issue_forward(f, psi, psi_b, psi_out, batch))) return rc;
    }
    f->last_psi = (const float2 *)psi;
    f->last_psib = (const float2 *)psi_b;
    f->last_batch = batch;
    f->have_fwd = f->train && psi_out != psi_b;
    return SPE_OK;
}

SPE_API int spe_fno_backward(spe_fno *f, const void *psi_target, double *loss_out)
{
    if (!f || !psi_target) return SPE_EINVAL;
    if (!f->train || !f->have_fwd) return SPE_ESTATE;
    const int n = f->n, M = f->M, L = f->L, batch = f->last_batch;
    const int rows = batch * n * n, grid = row_grid(rows);
    RowArgs a = base_args(f, batch);
    a.psi = f->last_psi;
    a.psib = f->last_psib;
    a.target = (const float2 *)psi_target;
    a.vin = v_buf(f, L);
    a.loss_scale = (float)(2.0 / (f->cfg.sigma * (double)batch * (double)n * n * n));
    // BF16 activations: the row kernels on the tensor cores, one partial per CTA of their grids
    const bool tc = !f->fp32;
    const int pcells = rows * n, ptiles = pcells / 128, pgrid_top = ptiles < kRowBlocks ? ptiles : kRowBlocks;
    if (tc) SPE_TRY(FK_TOP_BWD, launch_proj_bwd_tc(a, pcells, pgrid_top, f->st));
    else SPE_TRY(FK_TOP_BWD, launch_top_bwd(n, f->fp32, a, grid, f->st));
    int rc = reduce_into(f, kTopSeg, tc ? pgrid_top : grid, f->grad + f->off.Q1, kTopSeg - 1, f->dres);
    if (rc) return rc;
    a.vin = v_buf(f, L - 1);
    const int tiles = rows / kTcTile, tgrid = tiles < kRowBlocks ? tiles : kRowBlocks;
    const int pgrid = tc ? tgrid : grid;
    if (tc) SPE_TRY(FK_START_BWD, launch_layer_bwd_tc(n, M, kTcBwdStart, a, tgrid, f->st));
    else SPE_TRY(FK_START_BWD, launch_grad_start(n, M, f->fp32, a, grid, f->st));
    if ((rc = reduce_into(f, kLayerSeg, pgrid, f->grad + f->off.W[L - 1], kLayerSeg, nullptr))) return rc;
    for (int l = L - 1; l >= 0; --l) {
        if ((rc = spectral_bwd(f, l, batch))) return rc;
        RowArgs b = base_args(f, batch);
        b.psi = f->last_psi;
        b.psib = f->last_psib;
        b.oW = f->off.W[l];
        if (l >= 1) {
            b.vin = v_buf(f, l - 1);
            b.upre = u_buf(f, l - 1);
            if (tc) SPE_TRY(FK_LAYER_BWD, launch_layer_bwd_tc(n, M, kTcBwdLayer, b, tgrid, f->st));
            else SPE_TRY(FK_LAYER_BWD, launch_layer_bwd(n, M, f->fp32, b, grid, f->st));
            if ((rc = reduce_into(f, kLayerSeg, pgrid, f->grad + f->off.W[l - 1], kLayerSeg, nullptr))) return rc;
        } else {
            if (tc) SPE_TRY(FK_LIFT_BWD, launch_layer_bwd_tc(n, M, kTcBwdLift, b, tgrid, f->st));
            else SPE_TRY(FK_LIFT_BWD, launch_lift_bwd(n, M, f->fp32, b, grid, f->st));
            if ((rc = reduce_into(f, kLiftSeg, pgrid, f->grad + f->off.P, kLiftSeg, nullptr))) return rc;
        }
    }
    if (loss_out) {
        double s = 0.0;
        cudaError_t e = cudaMemcpyAsync(&s, f->dres, sizeof(double), cudaMemcpyDeviceToHost, f->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(f->st);
        if (e != cudaSuccess) return SPE_ECUDA;
        if ((rc = spe_fno_sync(f))) return rc;
        *loss_out = s / (f->cfg.sigma * f->cfg.sigma * (double)batch * (double)n * n * n);
    }
    return SPE_OK;
}

SPE_API int spe_fno_adam(spe_fno *f, double lr, double beta1, double beta2, double eps)
{
    if (!f || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return SPE_EINVAL;
    f->adam_t++;
    const double c1 = 1.0 / (1.0 - std::pow(beta1, (double)f->adam_t));
    const double c2 = 1.0 / (1.0 - std::pow(beta2, (double)f->adam_t));
    SPE_TRY(FK_ADAM, launch_adam(f->master, f->am, f->av, f->grad, f->w16, f->nparams, (float)lr, (float)beta1,
                        (float)beta2, (float)eps, (float)c1, (float)c2, f->st));
    return SPE_OK;
}

SPE_API int spe_fno_sync(spe_fno *f)
{
    if (!f) return SPE_EINVAL;
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, f->status, sizeof(int), cudaMemcpyDeviceToHost, f->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->st);
    if (e != cudaSuccess) return SPE_ECUDA;
    if (st) {
        cudaMemsetAsync(f->status, 0, sizeof(int), f->st);
        return SPE_ETIMEOUT;
    }
    return SPE_OK;
}

SPE_API int spe_fno_profile_read(spe_fno *f, const char **names, unsigned long long *launches, double *ms, int cap)
{
    if (!f || cap < 0 || (cap && (!names || !launches || !ms))) return SPE_EINVAL;
    if (!f->profile) return SPE_ESTATE;
    if (cudaStreamSynchronize(f->st) != cudaSuccess) return SPE_ECUDA;
    for (auto &p : f->prof_pending) {
        float t = 0.f;
        cudaEventElapsedTime(&t, p.second.first, p.second.second);
        f->prof_ms[p.first] += t;
        f->prof_launches[p.first] += 1;
        f->prof_free.push_back(p.second.first);
        f->prof_free.push_back(p.second.second);
    }
    f->prof_pending.clear();
    const int n = cap < FK_COUNT ? cap : FK_COUNT;
    for (int k = 0; k < n; ++k) {
        names[k] = kFnoKindNames[k];
        launches[k] = f->prof_launches[k];
        ms[k] = f->prof_ms[k];
        f->prof_launches[k] = 0;
        f->prof_ms[k] = 0.0;
    }
    return FK_COUNT;
}

SPE_API int spe_fno_launch_count(spe_fno *f, unsigned long long *count_out, int reset)
{
    if (!f || !count_out) return SPE_EINVAL;
    *count_out = f->launches;
    if (reset) f->launches = 0;
    return SPE_OK;
}

}  // extern "C"
