/*
 * Plain FP64 CPU oracle for the Schroedinger-Poisson split-step method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or
 * calls this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library; it has its own FFT, its own tables and its own CIC.
 *
 * What it computes (Meng & Dong 2026, "WaveDM.jl"):
 *   - the dimensionless SPE, Sec. 2.2 Eq. (SPE_dimensionless), with the
 *     hbar/m factor kept as a parameter (Sec. 2.2 Eqs. (GPE), (Poisson)),
 *     and the optional local self-interaction kappa|psi|^2 of Sec. 2.2 /
 *     Sec. 2.4 (local interactions);
 *   - the kick-drift-kick split step, Sec. 3.1 Eq. (SPE_solver_KDK) steps
 *     (a)-(d) and Algorithm 1, executed literally in that order every step
 *     (no fusion of the two half kicks of consecutive steps);
 *   - the periodic FFT Poisson solve with the zero mode removed,
 *     Sec. 3.2.1 (equivalent to subtracting <rho>);
 *   - star particles coupled through the same potential (Sec. 3.2.2,
 *     ":particles_dynamic"): a cloud-in-cell deposit into the Poisson
 *     source and a CIC interpolation of the second-order central
 *     difference gradient of Sec. 3.1 (finite differences), advanced by a
 *     KDK leapfrog in lock step with the field;
 *   - the CFL time step bound of Sec. 3.5;
 *   - mass and the conserved energy (spectral kinetic term).
 *
 * Readings taken where the paper is silent or inconsistent (all listed in
 * the design notes):
 *   - periodic grid: dx = L/N, node i at x_i = -L/2 + i dx, i < N
 *     (Sec. 3.1 writes L/(N-1), which does not close on a periodic box);
 *   - Poisson prefactor -4 pi G / k^2 with G a parameter (Sec. 3.1 step (c)
 *     has -4pi/k^2, Sec. 3.2.1 writes -1/k^2);
 *   - kick phase (Phi + kappa|psi|^2) dt / (hbar/m), drift phase
 *     (hbar/m) k^2 dt / 2;
 *   - Phi at n = 0 is computed from psi(0) and the particles before the
 *     first kick (Algorithm 1 does not say where Phi comes from at n = 0);
 *   - CIC: node-centred, u = (x + L/2)/dx, i0 = floor(u), f = u - i0,
 *     weights (1-f, f) per axis, periodic indices; the same weights deposit
 *     mass and interpolate the node gradient;
 *   - particle positions wrap into [-L/2, L/2).
 *
 * Layout: psi[z][y][x], x fastest, complex stored as interleaved
 * (re, im) doubles.  Particles: pos/vel as n x 3 doubles, mass n doubles.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* FFT: recursive decimation in time over the smallest prime factor.        */
/*                                                                          */
/*   X[k] = sum_{n<N} x[n] exp(sign * 2 pi i n k / N)                        */
/*                                                                          */
/* N = p*m: split x into p interleaved subsequences x[r + p j] (r < p),      */
/* transform each (length m), then                                          */
/*   X[k + q m] = sum_{r<p} exp(sign 2 pi i r (k + q m) / N) S_r[k].          */
/* tw[e] = exp(sign 2 pi i e / Ntop); the sub-length n uses                  */
/* exp(sign 2 pi i e / n) = tw[(e * (Ntop/n)) mod Ntop].                     */
/* ------------------------------------------------------------------------ */

static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

static void fft_rec(const cplx *in, size_t stride, cplx *out, int n,
                    const cplx *tw, int ntop, cplx *tmp)
{
    if (n == 1) { out[0] = in[0]; return; }
    int p = smallest_factor(n);
    int m = n / p;
    for (int r = 0; r < p; ++r)
        fft_rec(in + (size_t)r * stride, stride * (size_t)p, out + (size_t)r * m, m, tw, ntop, tmp);
    int step = ntop / n;
    for (int k = 0; k < m; ++k) {
        for (int r = 0; r < p; ++r) tmp[r] = out[(size_t)r * m + k];
        for (int q = 0; q < p; ++q) {
            cplx acc = 0.0;
            for (int r = 0; r < p; ++r) {
                long e = ((long)r * (long)(k + q * m)) % n;
                acc += tw[(e * step) % ntop] * tmp[r];
            }
            out[(size_t)q * m + k] = acc;
        }
    }
}

static cplx *make_twiddles(int n, int sign)
{
    cplx *tw = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    for (int e = 0; e < n; ++e) {
        double a = sign * 2.0 * PI * (double)e / (double)n;
        tw[e] = cos(a) + I * sin(a);
    }
    return tw;
}

/* Transform every line along one axis of a (nx, ny, nz) array in place.
 * axis 0 = x (stride 1), 1 = y (stride nx), 2 = z (stride nx*ny).
 * sign = -1: forward, unnormalised.  sign = +1: inverse, divided by n. */
static void fft_axis(cplx *a, int nx, int ny, int nz, int axis, int sign)
{
    int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    if (n == 1) return;
    size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)nx : (size_t)nx * ny);
    long nlines = (long)nx * ny * nz / n;
    cplx *tw = make_twiddles(n, sign);
    double scale = sign > 0 ? 1.0 / n : 1.0;
    #pragma omp parallel
    {
        cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *res = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *tmp = (cplx *)malloc(sizeof(cplx) * (size_t)(n + 1));
        #pragma omp for schedule(static)
        for (long l = 0; l < nlines; ++l) {
            /* line l: the index with the transformed axis removed */
            size_t base;
            if (axis == 0) base = (size_t)l * nx;
            else if (axis == 1) base = (size_t)(l % nx) + (size_t)(l / nx) * nx * ny;
            else base = (size_t)l;
            for (int i = 0; i < n; ++i) line[i] = a[base + i * stride];
            fft_rec(line, 1, res, n, tw, n, tmp);
            for (int i = 0; i < n; ++i) a[base + i * stride] = res[i] * scale;
        }
        free(line); free(res); free(tmp);
    }
    free(tw);
}

static void fft3(cplx *a, int nx, int ny, int nz, int sign)
{
    fft_axis(a, nx, ny, nz, 0, sign);
    fft_axis(a, nx, ny, nz, 1, sign);
    fft_axis(a, nx, ny, nz, 2, sign);
}

/* Exported FFT entry points for the pin tests. data: interleaved (re, im). */
void oracle_fft1(int n, double *data, int sign)
{
    fft_axis((cplx *)data, n, 1, 1, 0, sign);
}

void oracle_fft3(int nx, int ny, int nz, double *data, int sign)
{
    fft3((cplx *)data, nx, ny, nz, sign);
}

/* ------------------------------------------------------------------------ */
/* State                                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;
    double L[3];
    double eta;      /* hbar / m */
    double G;
    double kappa;
    cplx *psi;
    double *phi;     /* Phi_total on the nodes */
    double *rho_star;
    int phi_valid;
    size_t np;
    double *pos, *vel, *mass;  /* n x 3, n x 3, n */
    double *phi_b;             /* static external potential (Sec. 3.2.2 static mode), or NULL */
    double absorb_alpha;       /* absorbing layer (Sec. 3.1): alpha, 0 = off */
    int absorb_nb;             /* N_b */
} oracle_t;

static size_t ncells(const oracle_t *o) { return (size_t)o->nx * o->ny * o->nz; }
static double cell_volume(const oracle_t *o)
{
    return (o->L[0] / o->nx) * (o->L[1] / o->ny) * (o->L[2] / o->nz);
}

/* Angular wavenumber of FFT mode index j on an axis of n points and length L:
 * k = 2 pi j / L for j < n/2, else 2 pi (j - n) / L (Sec. 3.1, "k: wavenumber"). */
static double wavenumber(int j, int n, double L)
{
    int s = (2 * j < n) ? j : j - n;
    return 2.0 * PI * (double)s / L;
}

oracle_t *oracle_create(int nx, int ny, int nz, double Lx, double Ly, double Lz,
                        double hbar_over_m, double G, double kappa)
{
    oracle_t *o = (oracle_t *)calloc(1, sizeof(oracle_t));
    o->nx = nx; o->ny = ny; o->nz = nz;
    o->L[0] = Lx; o->L[1] = Ly; o->L[2] = Lz;
    o->eta = hbar_over_m; o->G = G; o->kappa = kappa;
    size_t n = ncells(o);
    o->psi = (cplx *)calloc(n, sizeof(cplx));
    o->phi = (double *)calloc(n, sizeof(double));
    o->rho_star = (double *)calloc(n, sizeof(double));
    return o;
}

void oracle_destroy(oracle_t *o)
{
    if (!o) return;
    free(o->psi); free(o->phi); free(o->rho_star);
    free(o->pos); free(o->vel); free(o->mass);
    free(o->phi_b);
    free(o);
}

void oracle_set_psi(oracle_t *o, const double *psi)
{
    memcpy(o->psi, psi, sizeof(cplx) * ncells(o));
    o->phi_valid = 0;
}

void oracle_get_psi(const oracle_t *o, double *out)
{
    memcpy(out, o->psi, sizeof(cplx) * ncells(o));
}

void oracle_set_particles(oracle_t *o, size_t n, const double *pos, const double *vel,
                          const double *mass)
{
    free(o->pos); free(o->vel); free(o->mass);
    o->np = n;
    o->pos = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
    o->vel = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
    o->mass = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (n) {
        memcpy(o->pos, pos, sizeof(double) * 3 * n);
        memcpy(o->vel, vel, sizeof(double) * 3 * n);
        memcpy(o->mass, mass, sizeof(double) * n);
    }
    o->phi_valid = 0;
}

void oracle_get_particles(const oracle_t *o, double *pos, double *vel)
{
    if (!o->np) return;
    memcpy(pos, o->pos, sizeof(double) * 3 * o->np);
    memcpy(vel, o->vel, sizeof(double) * 3 * o->np);
}

/* Test hook: impose a potential on the nodes (used by the CIC force pins). */
void oracle_set_phi(oracle_t *o, const double *phi)
{
    memcpy(o->phi, phi, sizeof(double) * ncells(o));
    o->phi_valid = 1;
}

/* ------------------------------------------------------------------------ */
/* Cloud in cell                                                            */
/* ------------------------------------------------------------------------ */

/* Node-centred CIC: the lower node index (periodic) and the fraction f in
 * [0, 1) toward the upper node, along one axis. */
static void cic_axis(double x, double L, int n, int *i0, double *f)
{
    double dx = L / n;
    double u = (x + 0.5 * L) / dx;
    double fl = floor(u);
    long i = (long)fl % n;
    if (i < 0) i += n;
    *i0 = (int)i;
    *f = u - fl;
}

static size_t node(const oracle_t *o, int i, int j, int k)
{
    i = ((i % o->nx) + o->nx) % o->nx;
    j = ((j % o->ny) + o->ny) % o->ny;
    k = ((k % o->nz) + o->nz) % o->nz;
    return (size_t)i + (size_t)o->nx * ((size_t)j + (size_t)o->ny * (size_t)k);
}

/* rho_* on the nodes: each particle spreads m_p over its 8 surrounding
 * nodes with the trilinear CIC weights; divided by the cell volume. */
static void deposit(oracle_t *o)
{
    size_t n = ncells(o);
    memset(o->rho_star, 0, sizeof(double) * n);
    double inv_dv = 1.0 / cell_volume(o);
    for (size_t p = 0; p < o->np; ++p) {
        int i0[3]; double f[3];
        for (int a = 0; a < 3; ++a)
            cic_axis(o->pos[3 * p + a], o->L[a], a == 0 ? o->nx : (a == 1 ? o->ny : o->nz), &i0[a], &f[a]);
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    double w = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1]) * (c ? f[2] : 1.0 - f[2]);
                    o->rho_star[node(o, i0[0] + a, i0[1] + b, i0[2] + c)] += o->mass[p] * w * inv_dv;
                }
    }
}

/* -dPhi/dx_axis at a node by the second-order central difference (Sec. 3.1). */
static double node_accel(const oracle_t *o, int i, int j, int k, int axis)
{
    double h = o->L[axis] / (axis == 0 ? o->nx : (axis == 1 ? o->ny : o->nz));
    size_t up, dn;
    if (axis == 0) { up = node(o, i + 1, j, k); dn = node(o, i - 1, j, k); }
    else if (axis == 1) { up = node(o, i, j + 1, k); dn = node(o, i, j - 1, k); }
    else { up = node(o, i, j, k + 1); dn = node(o, i, j, k - 1); }
    return -(o->phi[up] - o->phi[dn]) / (2.0 * h);
}

/* Acceleration at each particle: the node gradients interpolated with the
 * same CIC weights as the deposit. g: n x 3. */
static void interp_accel(const oracle_t *o, double *g)
{
    #pragma omp parallel for schedule(static)
    for (long p = 0; p < (long)o->np; ++p) {
        int i0[3]; double f[3];
        for (int a = 0; a < 3; ++a)
            cic_axis(o->pos[3 * p + a], o->L[a], a == 0 ? o->nx : (a == 1 ? o->ny : o->nz), &i0[a], &f[a]);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    double w = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1]) * (c ? f[2] : 1.0 - f[2]);
                    for (int ax = 0; ax < 3; ++ax)
                        acc[ax] += w * node_accel(o, i0[0] + a, i0[1] + b, i0[2] + c, ax);
                }
        for (int ax = 0; ax < 3; ++ax) g[3 * p + ax] = acc[ax];
    }
}

void oracle_accel(const oracle_t *o, double *g) { interp_accel(o, g); }

void oracle_deposit(oracle_t *o, double *rho_star)
{
    deposit(o);
    memcpy(rho_star, o->rho_star, sizeof(double) * ncells(o));
}

/* ------------------------------------------------------------------------ */
/* The split-step operators                                                 */
/* ------------------------------------------------------------------------ */

/* Sec. 3.2.1 and Sec. 3.1 step (c): rho = |psi|^2 + rho_*;
 * Phi = F^-1{ -4 pi G F{rho} / k^2 }, with the k = 0 mode set to zero
 * (the same as subtracting <rho>). */
static void compute_phi(oracle_t *o)
{
    size_t n = ncells(o);
    deposit(o);
    cplx *w = (cplx *)malloc(sizeof(cplx) * n);
    #pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)n; ++c) {
        double r = creal(o->psi[c]) * creal(o->psi[c]) + cimag(o->psi[c]) * cimag(o->psi[c]);
        w[c] = r + o->rho_star[c];
    }
    fft3(w, o->nx, o->ny, o->nz, -1);
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                double kx = wavenumber(i, o->nx, o->L[0]);
                double ky = wavenumber(j, o->ny, o->L[1]);
                double kz = wavenumber((int)k, o->nz, o->L[2]);
                double k2 = kx * kx + ky * ky + kz * kz;
                size_t c = (size_t)i + (size_t)o->nx * ((size_t)j + (size_t)o->ny * (size_t)k);
                w[c] = (k2 == 0.0) ? 0.0 : w[c] * (-4.0 * PI * o->G / k2);
            }
    fft3(w, o->nx, o->ny, o->nz, +1);
    #pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)n; ++c) o->phi[c] = creal(w[c]) + (o->phi_b ? o->phi_b[c] : 0.0);
    free(w);
    o->phi_valid = 1;
}

/* Sec. 3.1 steps (a) and (d): psi <- exp(-i V h / eta) psi with
 * V = Phi + kappa |psi|^2 (Sec. 2.4, local interaction). |psi| is unchanged. */
static void kick(oracle_t *o, double h)
{
    size_t n = ncells(o);
    #pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)n; ++c) {
        double a2 = creal(o->psi[c]) * creal(o->psi[c]) + cimag(o->psi[c]) * cimag(o->psi[c]);
        double v = o->phi[c] + o->kappa * a2;
        o->psi[c] *= cexp(-I * v * h / o->eta);
    }
}

/* Sec. 3.1 step (b): psi <- F^-1{ exp(-i eta k^2 dt / 2) F{psi} }. */
static void drift(oracle_t *o, double dt)
{
    fft3(o->psi, o->nx, o->ny, o->nz, -1);
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                double kx = wavenumber(i, o->nx, o->L[0]);
                double ky = wavenumber(j, o->ny, o->L[1]);
                double kz = wavenumber((int)k, o->nz, o->L[2]);
                double k2 = kx * kx + ky * ky + kz * kz;
                size_t c = (size_t)i + (size_t)o->nx * ((size_t)j + (size_t)o->ny * (size_t)k);
                o->psi[c] *= cexp(-I * o->eta * k2 * dt / 2.0);
            }
    fft3(o->psi, o->nx, o->ny, o->nz, +1);
}

static void particles_kick(oracle_t *o, double h)
{
    if (!o->np) return;
    double *g = (double *)malloc(sizeof(double) * 3 * o->np);
    interp_accel(o, g);
    for (size_t q = 0; q < 3 * o->np; ++q) o->vel[q] += g[q] * h;
    free(g);
}

static void particles_drift(oracle_t *o, double dt)
{
    for (size_t p = 0; p < o->np; ++p)
        for (int a = 0; a < 3; ++a) {
            double L = o->L[a];
            double x = o->pos[3 * p + a] + o->vel[3 * p + a] * dt;
            o->pos[3 * p + a] = x - L * floor((x + 0.5 * L) / L);
        }
}

/* Sec. 3.1 absorbing layer, applied after the second half kick (Algorithm 1):
 * B = exp(-alpha dt (6 - sum_a [tanh((x_a + L_a/2)/(L_a/N_b)) - tanh((x_a - L_a/2)/(L_a/N_b))])),
 * reading the trailing dt of the printed formula as multiplying the exponent. */
static double absorb_factor(const oracle_t *o, int i, int j, int k, double dt)
{
    int idx[3] = {i, j, k};
    int nn[3] = {o->nx, o->ny, o->nz};
    double sum = 0.0;
    for (int a = 0; a < 3; ++a) {
        double L = o->L[a];
        double x = -0.5 * L + idx[a] * (L / nn[a]);
        double w = L / o->absorb_nb;
        sum += tanh((x + 0.5 * L) / w) - tanh((x - 0.5 * L) / w);
    }
    return exp(-o->absorb_alpha * dt * (6.0 - sum));
}

static void absorb(oracle_t *o, double dt)
{
    if (o->absorb_alpha == 0.0 || o->absorb_nb <= 0) return;
    #pragma omp parallel for schedule(static)
    for (long k = 0; k < o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i)
                o->psi[(size_t)i + (size_t)o->nx * ((size_t)j + (size_t)o->ny * (size_t)k)] *=
                    absorb_factor(o, i, j, (int)k, dt);
}

void oracle_set_absorb(oracle_t *o, double alpha, int nb)
{
    o->absorb_alpha = alpha;
    o->absorb_nb = nb;
}

/* Static external potential added to Phi_total (NULL removes it). */
void oracle_set_static_phi(oracle_t *o, const double *phi_b)
{
    free(o->phi_b);
    o->phi_b = NULL;
    if (phi_b) {
        o->phi_b = (double *)malloc(sizeof(double) * ncells(o));
        memcpy(o->phi_b, phi_b, sizeof(double) * ncells(o));
    }
    o->phi_valid = 0;
}

/* nsteps kick-drift-kick steps of size dt (Sec. 3.1 Eq. (SPE_solver_KDK),
 * Algorithm 1), with the star particles advanced by a KDK leapfrog using the
 * same Phi_total (Sec. 3.2.2, dynamic mode). */
void oracle_step(oracle_t *o, int nsteps, double dt)
{
    if (!o->phi_valid) compute_phi(o);
    for (int s = 0; s < nsteps; ++s) {
        kick(o, 0.5 * dt);              /* (a) */
        particles_kick(o, 0.5 * dt);
        drift(o, dt);                   /* (b) */
        particles_drift(o, dt);
        compute_phi(o);                 /* (c) */
        kick(o, 0.5 * dt);              /* (d) */
        particles_kick(o, 0.5 * dt);
        absorb(o, dt);                  /* absorbing layer (Algorithm 1) */
    }
}

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                              */
/* ------------------------------------------------------------------------ */

void oracle_potential(oracle_t *o, double *out)
{
    if (!o->phi_valid) compute_phi(o);
    memcpy(out, o->phi, sizeof(double) * ncells(o));
}

/* rho_psi + rho_* on the nodes. */
void oracle_density(oracle_t *o, double *out)
{
    deposit(o);
    size_t n = ncells(o);
    for (size_t c = 0; c < n; ++c)
        out[c] = creal(o->psi[c]) * creal(o->psi[c]) + cimag(o->psi[c]) * cimag(o->psi[c]) + o->rho_star[c];
}

/* out = {mass, kinetic, potential, interaction, star_kinetic, total, max|Phi|}.
 *   mass        = sum |psi|^2 dV
 *   kinetic     = (eta^2 / 2) sum_k k^2 |F{psi}_k|^2 dV / Ncells
 *   potential   = 1/2 sum (|psi|^2 + rho_*) Phi dV
 *   interaction = kappa / 2 sum |psi|^4 dV
 *   star KE     = 1/2 sum m_p |v_p|^2
 * The sum of the last four is the energy the split step conserves to
 * O(dt^2) (Hamiltonian of Sec. 2.2 with Sec. 2.4's local term). */
void oracle_energy(oracle_t *o, double *out)
{
    if (!o->phi_valid) compute_phi(o);
    deposit(o);
    size_t n = ncells(o);
    double dv = cell_volume(o);
    double mass = 0.0, pot = 0.0, inter = 0.0, maxphi = 0.0;
    for (size_t c = 0; c < n; ++c) {
        double a2 = creal(o->psi[c]) * creal(o->psi[c]) + cimag(o->psi[c]) * cimag(o->psi[c]);
        mass += a2 * dv;
        /* self gravity counted once (the 1/2), a static external potential in full */
        pot += 0.5 * (a2 + o->rho_star[c]) * (o->phi[c] + (o->phi_b ? o->phi_b[c] : 0.0)) * dv;
        inter += 0.5 * o->kappa * a2 * a2 * dv;
        if (fabs(o->phi[c]) > maxphi) maxphi = fabs(o->phi[c]);
    }
    cplx *w = (cplx *)malloc(sizeof(cplx) * n);
    memcpy(w, o->psi, sizeof(cplx) * n);
    fft3(w, o->nx, o->ny, o->nz, -1);
    double kin = 0.0;
    for (int k = 0; k < o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                double kx = wavenumber(i, o->nx, o->L[0]);
                double ky = wavenumber(j, o->ny, o->L[1]);
                double kz = wavenumber(k, o->nz, o->L[2]);
                size_t c = (size_t)i + (size_t)o->nx * ((size_t)j + (size_t)o->ny * (size_t)k);
                double a2 = creal(w[c]) * creal(w[c]) + cimag(w[c]) * cimag(w[c]);
                kin += (kx * kx + ky * ky + kz * kz) * a2;
            }
    free(w);
    kin *= 0.5 * o->eta * o->eta * dv / (double)n;
    double skin = 0.0;
    for (size_t p = 0; p < o->np; ++p)
        skin += 0.5 * o->mass[p] * (o->vel[3 * p] * o->vel[3 * p] + o->vel[3 * p + 1] * o->vel[3 * p + 1] +
                                    o->vel[3 * p + 2] * o->vel[3 * p + 2]);
    out[0] = mass;
    out[1] = kin;
    out[2] = pot;
    out[3] = inter;
    out[4] = skin;
    out[5] = kin + pot + inter + skin;
    out[6] = maxphi;
}

/* Sec. 3.6 overall energy terms, with the second-order central differences of
 * Sec. 3.1 for the gradients (periodic), eta^2 restoring the dimensional
 * prefactor the paper absorbs (eta = 1 gives the paper's expressions):
 *   K = 1/2 sum (rho v)^2 / rho dV, rho v = eta Im(conj(psi) grad psi)
 *   Q = eta^2 sum |grad sqrt(rho)|^2 dV
 *   V = sum rho Phi_total dV         (rho = |psi|^2)
 * out = {K, Q, V, K + Q + V, 2K + 2Q + V}. */
void oracle_virial(oracle_t *o, double *out)
{
    if (!o->phi_valid) compute_phi(o);
    double dv = cell_volume(o);
    double h[3] = {o->L[0] / o->nx, o->L[1] / o->ny, o->L[2] / o->nz};
    double K = 0.0, Q = 0.0, V = 0.0;
    for (int k = 0; k < o->nz; ++k)
        for (int j = 0; j < o->ny; ++j)
            for (int i = 0; i < o->nx; ++i) {
                size_t c = node(o, i, j, k);
                cplx p = o->psi[c];
                double rho = creal(p) * creal(p) + cimag(p) * cimag(p);
                V += rho * o->phi[c] * dv;
                size_t up[3] = {node(o, i + 1, j, k), node(o, i, j + 1, k), node(o, i, j, k + 1)};
                size_t dn[3] = {node(o, i - 1, j, k), node(o, i, j - 1, k), node(o, i, j, k - 1)};
                double j2 = 0.0, g2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    cplx d = (o->psi[up[a]] - o->psi[dn[a]]) / (2.0 * h[a]);
                    double jj = o->eta * cimag(conj(p) * d);
                    j2 += jj * jj;
                    double su = cabs(o->psi[up[a]]), sd = cabs(o->psi[dn[a]]);
                    double gs = (su - sd) / (2.0 * h[a]);
                    g2 += gs * gs;
                }
                if (rho > 0.0) K += 0.5 * j2 / rho * dv;
                Q += o->eta * o->eta * g2 * dv;
            }
    out[0] = K;
    out[1] = Q;
    out[2] = V;
    out[3] = K + Q + V;
    out[4] = 2.0 * K + 2.0 * Q + V;
}

/* Sec. 3.5: dt_max = 0.5 min{ 4/(3 pi) dx^2 / eta, 2 pi eta / max|Phi|,
 * 2 pi eta / (|kappa| max|psi|^2) }, dt = safety * dt_max, dx the smallest
 * cell edge.  Terms whose denominator is zero are left out. */
double oracle_suggest_dt(oracle_t *o, double safety)
{
    if (!o->phi_valid) compute_phi(o);
    double dx = o->L[0] / o->nx;
    if (o->L[1] / o->ny < dx) dx = o->L[1] / o->ny;
    if (o->L[2] / o->nz < dx) dx = o->L[2] / o->nz;
    double t = 4.0 / (3.0 * PI) * dx * dx / o->eta;
    size_t n = ncells(o);
    double maxphi = 0.0, maxrho = 0.0;
    for (size_t c = 0; c < n; ++c) {
        if (fabs(o->phi[c]) > maxphi) maxphi = fabs(o->phi[c]);
        double a2 = creal(o->psi[c]) * creal(o->psi[c]) + cimag(o->psi[c]) * cimag(o->psi[c]);
        if (a2 > maxrho) maxrho = a2;
    }
    if (maxphi > 0.0 && 2.0 * PI * o->eta / maxphi < t) t = 2.0 * PI * o->eta / maxphi;
    if (o->kappa != 0.0 && maxrho > 0.0) {
        double ti = 2.0 * PI * o->eta / (fabs(o->kappa) * maxrho);
        if (ti < t) t = ti;
    }
    return safety * 0.5 * t;
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
