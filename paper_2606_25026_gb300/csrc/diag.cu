// Diagnostics off the per-step path: mass / potential / interaction energy
// and the maxima the CFL bound needs (Sec. 3.5), the stars' kinetic energy,
// and the density field.  FP32 data, FP64 accumulation, fixed-order
// (deterministic) grid reductions.
#include "reduce.cuh"
#include "spe_internal.cuh"

namespace spe {

constexpr int kDiagNT = 256;

// Raw sums: out[0] = sum |psi|^2, out[1] = sum (|psi|^2 + rho_*) Phi, out[2] = sum |psi|^4,
// out[3] = max |Phi|, out[4] = max |psi|^2 (the caller scales by dV, 1/2, kappa/2).
__global__ void __launch_bounds__(kDiagNT) grid_diag_kernel(const float2 *__restrict__ psi,
                                                            const float *__restrict__ phi, long long *dep,
                                                            float dep_scale, float kappa, double dv, size_t n,
                                                            double *partials, unsigned int *counter, double *out)
{
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)kDiagNT + threadIdx.x; i < n; i += (size_t)gridDim.x * kDiagNT) {
        const float2 v = psi[i];
        const double a2 = (double)v.x * v.x + (double)v.y * v.y;
        double rs = 0.0;
        if (dep) {
            rs = (double)dep[i] * dep_scale;
            dep[i] = 0;
        }
        const double f = phi ? (double)phi[i] : 0.0;
        acc[0] += a2;
        acc[1] += (a2 + rs) * f;
        acc[2] += a2 * a2;
        acc[3] = fmax(acc[3], fabs(f));
        acc[4] = fmax(acc[4], a2);
    }
    grid_reduce<5, kDiagNT>(acc, (1 << 3) | (1 << 4), partials, counter, out);
}

// Per-sample squared norms: one block per sample, a fixed per-thread stride and a fixed shuffle
// tree, so the sums do not depend on scheduling.  out[2 s] = sum |a - b|^2, out[2 s + 1] = sum |b|^2.
__global__ void __launch_bounds__(kDiagNT) pair_norms_kernel(const float2 *__restrict__ a,
                                                             const float2 *__restrict__ b, size_t n, double *out)
{
    __shared__ double sh[2 * (kDiagNT / 32)];
    const size_t base = (size_t)blockIdx.x * n;
    double acc[2] = {0.0, 0.0};
    for (size_t i = threadIdx.x; i < n; i += kDiagNT) {
        const float2 x = a[base + i], y = b[base + i];
        const double dr = (double)x.x - y.x, di = (double)x.y - y.y;
        acc[0] += dr * dr + di * di;
        acc[1] += (double)y.x * y.x + (double)y.y * y.y;
    }
    block_reduce<2, kDiagNT>(acc, 0, sh);
    if (threadIdx.x == 0) {
        out[2 * (size_t)blockIdx.x] = acc[0];
        out[2 * (size_t)blockIdx.x + 1] = acc[1];
    }
}

cudaError_t launch_pair_norms(const float2 *a, const float2 *b, size_t n, int samples, double *out, cudaStream_t st)
{
    pair_norms_kernel<<<samples, kDiagNT, 0, st>>>(a, b, n, out);
    return cudaGetLastError();
}

cudaError_t launch_grid_diag(const float2 *psi, const float *phi, long long *dep, float dep_scale, float kappa,
                             double dv, size_t ncells, double *partials, unsigned int *counter, double *out,
                             cudaStream_t st)
{
    size_t blocks = (ncells + kDiagNT - 1) / kDiagNT;
    if (blocks > (size_t)kReduceBlocks) blocks = kReduceBlocks;
    grid_diag_kernel<<<(unsigned)blocks, kDiagNT, 0, st>>>(psi, phi, dep, dep_scale, kappa, dv, ncells, partials,
                                                           counter, out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kDiagNT) particle_ke_kernel(const float *vx, const float *vy, const float *vz,
                                                              const float *m, int n, double *partials,
                                                              unsigned int *counter, double *out)
{
    double acc[1] = {0.0};
    for (int i = blockIdx.x * kDiagNT + threadIdx.x; i < n; i += gridDim.x * kDiagNT) {
        const double v2 = (double)vx[i] * vx[i] + (double)vy[i] * vy[i] + (double)vz[i] * vz[i];
        acc[0] += 0.5 * (double)m[i] * v2;
    }
    grid_reduce<1, kDiagNT>(acc, 0, partials, counter, out);
}

cudaError_t launch_particle_ke(const float *vx, const float *vy, const float *vz, const float *m, int n,
                               double *partials, unsigned int *counter, double *out, cudaStream_t st)
{
    int blocks = (n + kDiagNT - 1) / kDiagNT;
    if (blocks < 1) blocks = 1;
    if (blocks > kReduceBlocks) blocks = kReduceBlocks;
    particle_ke_kernel<<<blocks, kDiagNT, 0, st>>>(vx, vy, vz, m, n, partials, counter, out);
    return cudaGetLastError();
}

__global__ void density_kernel(const float2 *__restrict__ psi, long long *dep, float dep_scale, float *dens,
                               size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = psi[i];
        float r = v.x * v.x + v.y * v.y;
        if (dep) {
            r += (float)dep[i] * dep_scale;
            dep[i] = 0;
        }
        dens[i] = r;
    }
}

cudaError_t launch_density(const float2 *psi, long long *dep, float dep_scale, float *dens, size_t ncells,
                           cudaStream_t st)
{
    size_t blocks = (ncells + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    density_kernel<<<(unsigned)blocks, 256, 0, st>>>(psi, dep, dep_scale, dens, ncells);
    return cudaGetLastError();
}

}  // namespace spe

namespace spe {

// Raw sums of the Sec. 3.6 energy terms with second-order central differences
// (Sec. 3.1), periodic: out[0] = sum |Im(conj psi D psi)|^2 / |psi|^2,
// out[1] = sum |D |psi||^2, out[2] = sum |psi|^2 Phi (the caller scales).
__global__ void __launch_bounds__(kDiagNT) virial_kernel(const float2 *__restrict__ psi,
                                                         const float *__restrict__ phi, int nx, int ny, int nz,
                                                         float ihx, float ihy, float ihz, double *partials,
                                                         unsigned int *counter, double *out)
{
    const size_t n = (size_t)nx * ny * nz;
    double acc[3] = {0.0, 0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)kDiagNT + threadIdx.x; i < n; i += (size_t)gridDim.x * kDiagNT) {
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = (int)(i / ((size_t)nx * ny));
        const float2 p = psi[i];
        const double rho = (double)p.x * p.x + (double)p.y * p.y;
        const size_t sx = 1, sy = nx, sz = (size_t)nx * ny;
        size_t u[3], d[3];
        u[0] = (x + 1 == nx) ? i - (size_t)(nx - 1) : i + sx;
        d[0] = (x == 0) ? i + (size_t)(nx - 1) : i - sx;
        u[1] = (y + 1 == ny) ? i - (size_t)(ny - 1) * sy : i + sy;
        d[1] = (y == 0) ? i + (size_t)(ny - 1) * sy : i - sy;
        u[2] = (z + 1 == nz) ? i - (size_t)(nz - 1) * sz : i + sz;
        d[2] = (z == 0) ? i + (size_t)(nz - 1) * sz : i - sz;
        const float ih[3] = {ihx, ihy, ihz};
        double j2 = 0.0, g2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float2 pu = psi[u[a]], pd = psi[d[a]];
            const double dre = ((double)pu.x - pd.x) * ih[a], dim = ((double)pu.y - pd.y) * ih[a];
            const double j = (double)p.x * dim - (double)p.y * dre;
            j2 += j * j;
            const double gs = (sqrt((double)pu.x * pu.x + (double)pu.y * pu.y) -
                               sqrt((double)pd.x * pd.x + (double)pd.y * pd.y)) * ih[a];
            g2 += gs * gs;
        }
        if (rho > 0.0) acc[0] += j2 / rho;
        acc[1] += g2;
        acc[2] += rho * (phi ? (double)phi[i] : 0.0);
    }
    grid_reduce<3, kDiagNT>(acc, 0, partials, counter, out);
}

cudaError_t launch_virial(const float2 *psi, const float *phi, int nx, int ny, int nz, float ihx, float ihy,
                          float ihz, double *partials, unsigned int *counter, double *out, cudaStream_t st)
{
    const size_t n = (size_t)nx * ny * nz;
    size_t blocks = (n + kDiagNT - 1) / kDiagNT;
    if (blocks > (size_t)kReduceBlocks) blocks = kReduceBlocks;
    virial_kernel<<<(unsigned)blocks, kDiagNT, 0, st>>>(psi, phi, nx, ny, nz, ihx, ihy, ihz, partials, counter, out);
    return cudaGetLastError();
}

}  // namespace spe
