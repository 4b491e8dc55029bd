// Internal declarations shared by the libspe translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace spe {

// Supported axis lengths (each instantiates its own FFT kernels).
#define SPE_FOR_EACH_N(X) \
    X(4) X(6) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)

bool supported_n(int n);
bool spass_tile_ok(int n, int tile);      // strided-pass tile width 8, 16 or 32 usable at length n
int spass_default_tile(int n);            // the width used when none is chosen
bool has_alt_plan_n(int n);               // length n has an alternative radix schedule
int plan_count_n(int n);                  // radix schedules available at length n (1, 2 or 3)

// ---------------------------------------------------------------- x passes
// Lines along x are contiguous rows of nx complex values; rows = ny * nz.
// The half-spectrum buffer holds W = nx/2 + 1 complex values per row at a
// row pitch of P (P = W rounded up to a multiple of 4 complex = 32 bytes).

enum XFlags : int {
    X_HAS_PHI = 1 << 0,    // rebuild Phi on the row from the half spectrum (C2R)
    X_WRITE_PHI = 1 << 1,  // store Phi (real) to phi_out
    X_KICK = 1 << 2,       // psi *= exp(-i (Phi + kappa|psi|^2) kick_scale)
    X_FFT = 1 << 3,        // forward x transform of psi after the kick
    X_IFFT = 1 << 4,       // inverse x transform of psi before the density
    X_DEP = 1 << 5,        // add the fixed-point star deposit to rho and clear it
    X_MASS = 1 << 6,       // reduce sum |psi|^2 into diag[0] (deterministic)
    X_R2C = 1 << 7,        // forward real-to-complex x transform of rho into the half spectrum
    X_KIN = 1 << 8,        // reduce sum_k kx^2 |psi_hat|^2 (energy diagnostic), no store
    X_ABSORB = 1 << 9,     // psi *= absorbing-layer factor absorb_x[x] absorb_y[y] absorb_z[z]
    X_STATIC = 1 << 10,    // add the static potential phib to Phi (kick and phi_out)
};

struct XParams {
    float2 *psi;              // rows of nx complex
    float2 *phik;             // rows of P complex (half spectrum)
    float *phi_out;           // rows of nx floats (X_WRITE_PHI)
    long long *dep;           // fixed-point star mass per node (X_DEP)
    unsigned char *dflag;     // per row: nonzero when the row's deposit may be nonzero (X_DEP)
    const float4 *tw;         // nx twiddles, (hi, lo) float pairs
    const float *k2;          // nx values of kx^2 (X_KIN)
    int rows;                 // ny * nz
    int P;                    // half-spectrum row pitch (complex)
    float kick_scale;         // dt_kick / eta
    float kappa;
    float dep_scale;          // mass quantum / cell volume
    double *partials;         // per-block partial sums
    unsigned int *counter;    // last-block ticket (returns to 0 after use)
    double *result;           // where the final reduction goes (X_MASS: the sum, then the sum times mass_scale)
    double mass_scale;        // cell volume (X_MASS)
    int *status;              // device status word (bit 0: non-finite mass)
    const float *absorb_x, *absorb_y, *absorb_z;  // per-axis absorbing-layer factors (X_ABSORB)
    const float *phib;        // static external potential, nodes (X_STATIC)
    int ny;                   // rows are y + ny z
    int tc;                   // radix-16 stages on the tensor cores (split FP16), N = 256 and 512
    const void *tcw;          // the 32 x 32 DFT operands for them (fp16 hi / lo, both directions)
    int flags;
};

// ---------------------------------------------------------------- strided passes
// Lines along y or z: point n of column c in batch b sits at
//   data[b * bstride + c + n * S]     (complex units), c < W.

enum SFlags : int {
    S_FWD = 1 << 0,
    S_INV = 1 << 1,
    S_DRIFT = 1 << 2,     // multiply by dxy[b * dxy_pitch + c] * ez[n] ((hi, lo) complex tables)
    S_POISSON = 1 << 3,   // multiply by -4 pi G norm / (colk2[c] + batchk2[b] + linek2[n]), 0 at k = 0
    S_KIN = 1 << 4,       // reduce sum_k linek2[n] |X|^2 after the forward transform, no store
};

struct SParams {
    float2 *data;
    long long S;          // element stride along the line
    long long bstride;    // batch stride
    int W;                // live columns
    int batches;
    const float4 *tw;     // N twiddles, (hi, lo) float pairs
    const float4 *dxy;    // drift factor per (column, batch), normalisation folded in, (hi, lo)
    const float4 *ez;     // drift factor per line point, (hi, lo)
    int dxy_pitch;
    const float *colk2, *batchk2, *linek2; // k^2 tables
    float norm;           // 1 / (nx ny nz) folded into the Poisson multiply
    float poisson;        // -4 pi G
    double *partials;
    unsigned int *counter;
    double *result;
    int tile;             // columns per CTA: 8, 16 or 32 (0 = the per-length default)
    int plan;             // radix schedule: 0 default, 1 and 2 the alternatives (lengths that have them)
    int tc;               // radix-16 stages on the tensor cores (split FP16), N = 256 and 512
    const void *tcw;
    int *status;          // device status word (tensor-stage and tile-copy timeouts)
    int tma;              // stage the tiles with TMA bulk-tensor copies where the shape allows
    int flags;
};

// ---------------------------------------------------------------- particles

struct PParams {
    float *x, *y, *z, *vx, *vy, *vz;
    const float *m;
    const float *phi;        // nodes, x fastest
    long long *dep;          // fixed-point deposit (PK_DEPOSIT)
    unsigned char *dflag;    // set to 1 for every row (y + ny z) that receives deposit
    int n;
    int nx, ny, nz;
    float Lx, Ly, Lz;
    float inv_dx, inv_dy, inv_dz;      // 1/dx
    float gx_scale, gy_scale, gz_scale; // 1/(2 dx)
    float kick;              // dt for the velocity update (0 = none)
    float drift;             // dt for the position update (0 = none)
    float inv_quantum;       // 1 / mass quantum of the deposit
    int flags;
};

enum PFlags : int {
    PK_KICK = 1 << 0,
    PK_DRIFT = 1 << 1,
    PK_DEPOSIT = 1 << 2,
};

struct SortParams {
    float *src[7], *dst[7];        // x, y, z, vx, vy, vz, m
    unsigned int *src_id, *dst_id;
    int *key;                      // per star
    int *count;                    // nbins counters / offsets
    int *totals;                   // ceil(nbins / 2048) span totals of the scan
    int n, nbins;
    int nx, ny, nz, nbx, nby;
    float Lx, Ly, Lz, inv_dx, inv_dy, inv_dz;
};

// ---------------------------------------------------------------- batch: one persistent launch per step
// (batch_persist.cu).  A member's passes with their parameters, and the launch's work lists.

constexpr int kBatchThreads = 256;   // threads per CTA of the persistent kernel
constexpr int kBatchTile = 16;       // strided-pass tile width in it
constexpr int kBatchPhases = 8;

struct BatchMember {
    XParams xk, xd;                    // x kick pass, x density pass
    SParams yf, zd, yi;                // psi: forward y, z drift, inverse y
    SParams rf, rp, ri;                // half spectrum: forward y, z Poisson, inverse y
    PParams pp;                        // stars (n = 0: none)
    int n;                             // axis length (members are cubes)
    int xtiles;                        // x-pass tiles (16 rows each)
    int cols_psi, cols_rho;            // strided column tiles of psi and of the half spectrum
    int pblocks;                       // star blocks (256 stars each)
};

struct BatchLaunch {
    const BatchMember *m;
    int count;
    const int *offs;                   // kBatchPhases rows of count + 1 prefix sums: items per phase
    unsigned int *bar;                 // grid-barrier counter, 0 at launch
    int *status;                       // bit 1 set when a barrier wait gave up
    long long wait_limit;              // polls of a barrier before it gives up
};

bool batch_persist_n_ok(int n);
size_t batch_persist_smem();
cudaError_t batch_persist_setup(int *blocks_out);   // grid size of a co-resident launch
cudaError_t launch_batch_persist(const BatchLaunch &L, int blocks, cudaStream_t st);

// ---------------------------------------------------------------- launchers
// Each returns cudaGetLastError() after the launch.  blocks_out (if given)
// receives the grid size, for the reductions' partial counts.

cudaError_t launch_xpass(int nx, const XParams &p, cudaStream_t st, int *blocks_out);
cudaError_t launch_spass(int n, const SParams &p, cudaStream_t st, int *blocks_out);
size_t xpass_rows_per_block(int nx);
cudaError_t setup_kernel_attributes();

cudaError_t launch_particles(const PParams &p, cudaStream_t st);
cudaError_t launch_particles_to_soa(const float *pos3, const float *vel3, const float *mass, int n,
                                    float *x, float *y, float *z, float *vx, float *vy, float *vz, float *m,
                                    float Lx, float Ly, float Lz, cudaStream_t st);
cudaError_t launch_particles_from_soa(const float *x, const float *y, const float *z, const float *vx,
                                      const float *vy, const float *vz, int n, float *pos3, float *vel3,
                                      cudaStream_t st);

cudaError_t launch_particle_sort(const SortParams &s, cudaStream_t st, int *launches);
cudaError_t launch_particle_ids(unsigned int *id, int first, int n, cudaStream_t st);
cudaError_t launch_particles_from_soa_by_id(const float *x, const float *y, const float *z, const float *vx,
                                            const float *vy, const float *vz, const unsigned int *id, int n,
                                            float *pos3, float *vel3, cudaStream_t st);

// Grid diagnostics (raw sums): out[0] = sum |psi|^2, out[1] = sum (|psi|^2 + rho_*) phi,
// out[2] = sum |psi|^4, out[3] = max |phi|, out[4] = max |psi|^2; clears dep if given.
// Deterministic (fixed-order) FP64 accumulation.
cudaError_t launch_grid_diag(const float2 *psi, const float *phi, long long *dep, float dep_scale, float kappa,
                             double dv, size_t ncells, double *partials, unsigned int *counter, double *out,
                             cudaStream_t st);
// Raw sums of the Sec. 3.6 terms: out[0] = sum |Im(conj psi D psi)|^2/|psi|^2, out[1] = sum |D|psi||^2,
// out[2] = sum |psi|^2 phi, D the central difference (ihx = 1/(2 dx), ...).
cudaError_t launch_virial(const float2 *psi, const float *phi, int nx, int ny, int nz, float ihx, float ihy,
                          float ihz, double *partials, unsigned int *counter, double *out, cudaStream_t st);
// out[0] = 1/2 sum m v^2
cudaError_t launch_particle_ke(const float *vx, const float *vy, const float *vz, const float *m, int n,
                               double *partials, unsigned int *counter, double *out, cudaStream_t st);
// dens[i] = |psi_i|^2 + dep_i * dep_scale; clears dep if given.
cudaError_t launch_density(const float2 *psi, long long *dep, float dep_scale, float *dens, size_t ncells,
                           cudaStream_t st);

// out[2 s] = sum |a - b|^2, out[2 s + 1] = sum |b|^2 over sample s of n complex values (FP64).
cudaError_t launch_pair_norms(const float2 *a, const float2 *b, size_t n, int samples, double *out, cudaStream_t st);

// Maximum number of partial-sum slots any reduction uses.
constexpr int kMaxPartials = 1 << 17;
constexpr int kReduceBlocks = 1024;

}  // namespace spe
