/*
 * libspe -- GB300-native pseudo-spectral split-step solver for the
 * Schroedinger-Poisson equation coupled to star particles.
 *
 * The method (Meng & Dong 2026, "WaveDM.jl"):
 *   i eta psi_t = -(eta^2/2) lap psi + (Phi + kappa|psi|^2) psi,
 *   lap Phi = 4 pi G (|psi|^2 + rho_*),
 * advanced per step of size dt as
 *   (a) psi <- exp(-i (Phi + kappa|psi|^2) dt/2 / eta) psi        Sec. 3.1 Eq. (SPE_solver_KDK) (a)
 *   (b) psi <- F^-1{ exp(-i eta k^2 dt / 2) F{psi} }                 step (b), Algorithm 1
 *   (c) Phi <- F^-1{ -4 pi G F{|psi|^2 + rho_*} / k^2 }, k=0 -> 0   step (c), Sec. 3.2.1
 *   (d) psi <- exp(-i (Phi + kappa|psi|^2) dt/2 / eta) psi        step (d)
 * with eta = hbar/m (Sec. 2.2, Eqs. (GPE), (Poisson), (SPE_dimensionless)),
 * kappa the local self-interaction of Sec. 2.2 / Sec. 2.4, and rho_* the
 * cloud-in-cell deposit of star particles that move by a kick-drift-kick
 * leapfrog in the same potential (Sec. 3.2.2, dynamic particle mode), their
 * acceleration the CIC interpolation of the second-order central-difference
 * gradient of Phi (Sec. 3.1, finite differences).
 *
 * Grid: periodic, nx x ny x nz nodes, node (i,j,k) at
 * (-Lx/2 + i Lx/nx, -Ly/2 + j Ly/ny, -Lz/2 + k Lz/nz).  Field arrays are
 * [z][y][x] with x fastest.  Complex values are complex64: interleaved
 * (re, im) float pairs, 8 bytes per node.  Particle arrays are n x 3 floats
 * (x, y, z per particle) plus n floats of mass.
 *
 * Every entry point returns SPE_OK (0) or a negative status; nothing aborts
 * the process and no C++ exception crosses this interface.  "where" selects
 * whether a caller buffer is host memory (SPE_HOST, pageable or pinned) or
 * device memory on the grid's device (SPE_DEVICE).  Caller buffers are only
 * borrowed for the duration of the call.
 *
 * Streams: all device work of a grid is ordered on cfg.cuda_stream (NULL =
 * the legacy default stream).  Calls that return data to the host, or that
 * report device-side status, synchronise that stream first.
 */
#ifndef SPE_H
#define SPE_H

#include <stddef.h>

#if defined(__GNUC__)
#define SPE_API __attribute__((visibility("default")))
#else
#define SPE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SPE_OK            0
#define SPE_EINVAL       -1   /* bad argument (size, pointer, unsupported shape) */
#define SPE_ENOMEM       -2   /* workspace too small or device allocation failed */
#define SPE_ECUDA        -3   /* a CUDA runtime call failed */
#define SPE_ECFL         -4   /* |dt| above the Sec. 3.5 CFL bound (unless SPE_NO_CFL_CHECK) */
#define SPE_ENONFINITE   -5   /* the field's mass became NaN or infinite */
#define SPE_ETIMEOUT     -6   /* a bounded device-side wait gave up */
#define SPE_ESTATE       -7   /* call out of order (e.g. no initial condition set) */

/* ---- where a caller buffer lives ---- */
#define SPE_HOST   0
#define SPE_DEVICE 1

/* ---- spe_config.flags ---- */
#define SPE_GRAVITY_OFF   (1 << 0)  /* G treated as 0: no Poisson solve */
#define SPE_NO_CFL_CHECK  (1 << 1)  /* spe_step does not reject dt above the kinetic CFL bound */
#define SPE_ASYNC         (1 << 2)  /* spe_step returns after enqueueing; no status check */
#define SPE_PROFILE       (1 << 3)  /* time every kernel launch with CUDA events (spe_profile_read);
                                       launches go directly, not through CUDA graphs */
#define SPE_NO_GRAPH      (1 << 4)  /* launch the per-step kernels directly, never through a CUDA graph */
#define SPE_STATIC_POTENTIAL (1 << 5) /* reserve a static external potential (spe_set_static_potential) */
#define SPE_PREC_SPLIT16  (1 << 6)  /* axes of 256 or 512 points: radix-16 DFT stages on the tensor cores,
                                       split FP16 (hi + lo) operands, FP32 accumulation */
#define SPE_NO_TMA        (1 << 7)  /* the strided (y, z) passes stage their tiles with per-thread
                                       asynchronous copies instead of TMA bulk-tensor copies */

typedef struct spe_grid spe_grid;   /* opaque */

typedef struct {
    int nx, ny, nz;          /* nodes per axis: each in {4,6,8,12,16,24,32,48,64,96,128,192,256,384,512,768,1024} */
    double Lx, Ly, Lz;       /* box side lengths */
    double hbar_over_m;      /* eta > 0 */
    double G;                /* gravitational constant in code units */
    double kappa;            /* local self-interaction strength (0 = none) */
    size_t max_particles;    /* particle capacity (0 = field only) */
    int flags;               /* SPE_* flags above */
    void *cuda_stream;       /* cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream; NULL = default */
    double absorb_alpha;     /* absorbing layer of Sec. 3.1 (alpha; 0 = off; the paper's default is 10) */
    int absorb_nb;           /* its transition parameter N_b (the paper's default is 50) */
} spe_config;

typedef struct {
    double mass;          /* sum |psi|^2 dV */
    double kinetic;       /* (eta^2/2) sum_k k^2 |F{psi}_k|^2 dV / Ncells (spectral) */
    double potential;     /* 1/2 sum (|psi|^2 + rho_*) Phi dV */
    double interaction;   /* kappa/2 sum |psi|^4 dV */
    double star_kinetic;  /* 1/2 sum m_p |v_p|^2 */
    double total;         /* kinetic + potential + interaction + star_kinetic */
    double max_abs_phi;   /* max |Phi| over the nodes */
} spe_energy_t;

/* The paper's overall energy terms (Sec. 3.6), gradients by second-order
 * central differences (Sec. 3.1), eta^2 restoring the prefactor the paper
 * absorbs:  K = 1/2 sum (rho v)^2/rho dV with rho v = eta Im(conj(psi) grad psi),
 * Q = eta^2 sum |grad sqrt(rho)|^2 dV, V = sum |psi|^2 Phi dV (Phi total). */
typedef struct {
    double K, Q, V;
    double E;        /* K + Q + V */
    double virial;   /* 2K + 2Q + V (zero at virial equilibrium in the paper's statement) */
} spe_virial_t;

/* Device bytes a grid with this configuration needs (field buffers, the
 * half-spectrum potential buffer, particle arrays, tables and reduction
 * scratch).  Returns SPE_EINVAL for an unsupported configuration. */
SPE_API int spe_workspace_bytes(const spe_config *cfg, size_t *bytes);

/* Create a grid.  workspace: a device buffer of at least
 * spe_workspace_bytes() bytes, 256-byte aligned, owned by the caller and
 * kept alive until spe_destroy (e.g. a torch uint8 tensor); or NULL, in
 * which case the library allocates it with cudaMalloc and frees it in
 * spe_destroy.  The configuration is copied.  psi starts at zero. */
SPE_API int spe_create_grid(const spe_config *cfg, void *workspace, size_t workspace_bytes, spe_grid **out);

/* Release the grid (and its workspace if the library allocated it). */
SPE_API int spe_destroy(spe_grid *g);

/* Copy the initial field in: n must equal nx*ny*nz complex64 values. */
SPE_API int spe_set_ic(spe_grid *g, const void *psi_c64, size_t n, int where);

/* Append n star particles (pos3, vel3: n x 3 floats; mass: n floats).
 * Positions are wrapped into the box.  Fails with SPE_ENOMEM if the total
 * exceeds cfg.max_particles. */
SPE_API int spe_add_particles(spe_grid *g, size_t n, const float *pos3, const float *vel3, const float *mass, int where);

/* Remove all particles. */
SPE_API int spe_clear_particles(spe_grid *g);

/* Advance nsteps kick-drift-kick steps of size dt (dt may be negative).
 * The half kicks of consecutive steps are applied as one full kick, also
 * across calls: the closing half kick of a call is deferred, and the next
 * spe_step with the same dt applies it together with its own leading half
 * kick, so that a run of single-step calls does the work of one call.  Every
 * function that reads or changes the state (spe_get_psi, spe_get_particles,
 * spe_energy, spe_set_ic, ..., spe_sync, spe_settle) applies a deferred kick
 * first, so psi and the particles are always observed synchronised;
 * spe_last_mass needs no kick (the mass is measured inside the step).
 * Unless SPE_ASYNC is set, the call waits for the work and returns
 * SPE_ETIMEOUT if a bounded device-side wait of a tile copy or a tensor-core
 * stage gave up during the call (the state is then undefined and must be set
 * again), else SPE_ENONFINITE if the field's mass stopped being finite. */
SPE_API int spe_step(spe_grid *g, int nsteps, double dt);

/* Apply a deferred closing half kick now (queued on the grid's stream, no
 * wait).  A no-op when none is owed. */
SPE_API int spe_settle(spe_grid *g);

/* Sec. 3.5: dt = safety * 0.5 * min{4/(3 pi) dx^2/eta, 2 pi eta/max|Phi|,
 * 2 pi eta/(|kappa| max|psi|^2)}, dx the smallest cell edge. */
SPE_API int spe_suggest_dt(spe_grid *g, double safety, double *dt_out);

/* rho_psi + rho_* on the nodes: nx*ny*nz floats. */
SPE_API int spe_density(spe_grid *g, float *out, int where);

/* Phi on the nodes (zero mode removed): nx*ny*nz floats. */
SPE_API int spe_potential(spe_grid *g, float *out, int where);

/* Static external potential Phi_b (Sec. 3.2.2, static particle mode): added
 * to Phi_total for the kick, the star accelerations, spe_potential and the
 * energy (where it counts once, not halved).  nx*ny*nz floats; NULL removes
 * it.  Needs SPE_STATIC_POTENTIAL at creation (else SPE_ESTATE). */
SPE_API int spe_set_static_potential(spe_grid *g, const float *phi_b, int where);

/* K, Q, V of Sec. 3.6 (FP64 accumulation on the device). */
SPE_API int spe_virial(spe_grid *g, spe_virial_t *out);

/* Mass and energy terms (FP64 accumulation on the device). */
SPE_API int spe_energy(spe_grid *g, spe_energy_t *out);

/* Mass of the field as computed inside the last step (no extra pass). */
SPE_API int spe_last_mass(spe_grid *g, double *mass_out);

/* Queue a copy of the same mass (one double, cell volume applied) to dst on
 * the grid's stream and return without waiting: dst in pinned host memory or
 * device memory (pageable host memory works but makes the copy wait).  The
 * value lands when the stream reaches this point, so a loop of SPE_ASYNC
 * spe_step calls can read every step's mass back without stalling the GPU. */
SPE_API int spe_mass_async(spe_grid *g, double *dst);

/* Copy psi out: nx*ny*nz complex64 values. */
SPE_API int spe_get_psi(spe_grid *g, void *out, int where);

/* Copy the particles out in the order they were added (pos3, vel3: n x 3
 * floats; either may be NULL). */
SPE_API int spe_get_particles(spe_grid *g, float *pos3, float *vel3, int where);

/* Number of particles currently held. */
SPE_API int spe_particle_count(spe_grid *g, size_t *n_out);

/* Apply a deferred closing half kick (spe_settle), then wait for all work
 * queued on the grid's stream. */
SPE_API int spe_sync(spe_grid *g);

/* Kernel launches issued by this grid since creation (or the last reset). */
SPE_API int spe_launch_count(spe_grid *g, unsigned long long *count_out, int reset);

/* With SPE_PROFILE: per kernel kind, the launches and the summed device
 * time (ms) measured by CUDA events on the grid's stream since the last
 * read; resets the record.  names[i] points at static strings.  Returns the
 * number of kinds written (at most cap) or a negative status. */
SPE_API int spe_profile_read(spe_grid *g, const char **names, unsigned long long *launches, double *ms, int cap);

/* ---- field energy without any device allocation ----
 * Not part of the paper's method (the paper has no counterpart); it serves
 * callers that may not allocate device memory where they need the number:
 * code running inside another framework's memory pool, a loop with a fixed
 * memory budget, or a process that must not grow its device footprint after
 * start-up.
 *
 * Computes, for n complex64 values psi_c64 already in device memory (not
 * read after return; the caller keeps ownership):
 *   out2[0] = cell_volume * sum |psi|^2                (spe_energy's mass)
 *   out2[1] = kappa / 2 * cell_volume * sum |psi|^4   (spe_energy's interaction)
 * where = SPE_HOST: out2 is host memory, filled before return;
 * where = SPE_DEVICE: out2 is two doubles of device memory, written on the
 * stream.  cuda_stream: cudaStream_t or NULL.  The call waits for its work.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * is one fixed array of SPE_NOALLOC_SCRATCH_DOUBLES doubles inside the
 * library, resident on every GPU that loads libspe until the process exits.
 * Every call shares that array, so calls that overlap on the GPU race and
 * must be serialised by the caller.  The first call on each device finds the
 * array's device address (with that device current) and remembers it; make
 * that first call before any stream capture.  The remembered address does not
 * survive cudaDeviceReset: do not call this again on a device that was reset.
 * Returns SPE_EINVAL for n == 0, n > SPE_NOALLOC_MAX_CELLS, a non-positive
 * cell volume, a NULL pointer, psi_c64 not 8-byte aligned, or (SPE_DEVICE)
 * out2 not 8-byte aligned. */
#define SPE_NOALLOC_MAX_CELLS ((size_t)1 << 30)
#define SPE_NOALLOC_SCRATCH_DOUBLES 2064
SPE_API int spe_field_energy_noalloc(const void *psi_c64, size_t n, double cell_volume, double kappa,
                                     double *out2, int where, void *cuda_stream);

/* ---- tuning and batches (beyond the paper, which steps one grid) ----------
 * spe_autotune: time the strided (y, z) passes on a scratch field of the
 * grid's size (allocated and freed inside the call) over tile widths 8, 16
 * and 32 columns (32 where it fits in shared memory) and every radix schedule
 * of the length (see spe_set_schedule), and keep the fastest per axis, once
 * for psi's passes and once for the half spectrum's (the density's forward
 * transforms, the Poisson pass and the potential's inverse transforms, timed
 * as the step runs them); choices are cached per (axis, length, nx, field) for
 * the process.  tiles_out (optional): psi's y and z widths chosen
 * (spe_get_schedule also gives the radix schedules, spe_get_schedule_half the
 * half spectrum's). */
SPE_API int spe_autotune(spe_grid *g, int *tiles_out);

/* Pin the strided passes' schedule (psi's and the half spectrum's): tiles[0..1] = tile width of the y and z
 * passes (8, 16 or 32 columns; 0 = the default for the length) and plans[0..1]
 * = radix schedule (0 = default; 1 = the first alternative, for 32, 48, 64,
 * 96, 128, 192, 256, 384, 512, 768 and 1024; 2 = the two-stage [16, 32]
 * schedule, for 512).  Tile widths only
 * regroup independent lines (results bitwise unchanged); a radix schedule
 * changes the FP32 rounding of the transform.  SPE_EINVAL for an unusable
 * choice.  spe_get_schedule reports the schedule in use. */
SPE_API int spe_set_schedule(spe_grid *g, const int *tiles, const int *plans);
SPE_API int spe_get_schedule(spe_grid *g, int *tiles, int *plans);
/* The schedule of the half spectrum's strided passes in use: psi's unless
 * spe_autotune chose one of its own (spe_set_schedule pins both). */
SPE_API int spe_get_schedule_half(spe_grid *g, int *tiles, int *plans);

/* A batch of independent grids (sizes, parameters and particle counts may
 * all differ), stepped together on the batch stream cfgs[0].cuda_stream.
 * Members allocate their own workspaces; use spe_batch_grid to reach a member
 * for spe_set_ic, spe_add_particles, spe_get_psi, spe_energy, ... (not
 * spe_destroy).
 * Two ways to run a step.  By default each member runs its kernels on its own
 * stream and the members' full steps are the parallel branches of one CUDA
 * graph.  With spe_batch_set_persistent(b, 1, ...), when every member is a
 * gravitating cube of 64, 96, 128 or 192 points without a static potential,
 * an absorbing layer, tensor-core stages or SPE_PROFILE, one cooperative
 * kernel launch per step walks eight phases (the passes of the step), each a
 * work list of every member's tiles, with a grid-wide barrier between phases;
 * full steps replay that launch as a CUDA graph.  Both give every member
 * bitwise the result of the same grid stepped alone. */
typedef struct spe_batch spe_batch;
SPE_API int spe_batch_create(const spe_config *cfgs, int count, spe_batch **out);
SPE_API int spe_batch_grid(spe_batch *b, int index, spe_grid **out);
/* spe_autotune for every member */
SPE_API int spe_batch_autotune(spe_batch *b);
/* nsteps KDK steps of every member, dts[i] for member i; returns after the work
 * completes.  Each member's closing half kick is deferred as in spe_step. */
SPE_API int spe_batch_step(spe_batch *b, int nsteps, const double *dts);
/* Apply every member's deferred closing half kick: queued on the member
 * streams and joined into the batch stream (no wait). */
SPE_API int spe_batch_settle(spe_batch *b);
/* kernel launches of all members since creation (graph replays counted per node) */
SPE_API int spe_batch_launch_count(spe_batch *b, unsigned long long *count_out);
/* Choose the persistent launch (on = 1, used where the members qualify) or the
 * graph of per-member branches (on = 0).  wait_limit: polls of a grid-wide
 * barrier before the kernel gives up (-1: the default, about half a second);
 * a wait that gives up makes spe_batch_step return SPE_ETIMEOUT without
 * hanging, and leaves the members' state undefined (set it again).  A limit
 * of 0 makes every barrier give up unless it is already complete (a way to
 * exercise that path).  spe_batch_get_persistent: 1 when the next step will
 * use the persistent launch. */
SPE_API int spe_batch_set_persistent(spe_batch *b, int on, long long wait_limit);
SPE_API int spe_batch_get_persistent(spe_batch *b, int *on_out);
SPE_API int spe_batch_destroy(spe_batch *b);

/* Per-sample squared norms, for the surrogate's output scale and its relative
 * errors against the solver (the paper has no counterpart): a and b hold
 * `samples` fields of n complex64 values each in device memory, sample after
 * sample (a may equal b); out is 2 * samples doubles of device memory and
 * receives out[2s] = sum_i |a_si - b_si|^2 and out[2s + 1] = sum_i |b_si|^2,
 * accumulated in FP64 in a fixed order (bitwise reproducible).  Asynchronous
 * on cuda_stream (cudaStream_t or NULL); the caller keeps all three buffers.
 * SPE_EINVAL for a NULL pointer, n == 0, samples <= 0 or a pointer that is not
 * 8-byte aligned. */
SPE_API int spe_pair_norms(const void *a, const void *b, size_t n, int samples, double *out, void *cuda_stream);

/* Human-readable text for a status code (static storage). */
SPE_API const char *spe_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* SPE_H */
