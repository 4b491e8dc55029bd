// Star particles: cloud-in-cell coupling to the field's potential and a
// kick-drift-kick leapfrog in lock step with the field (Sec. 3.2.2, dynamic
// mode: particles add their mass to the Poisson source, and the potential's
// acceleration is interpolated back to the particles).
//
// CIC convention: node i of an axis at x_i = -L/2 + i dx; a particle at x
// has u = (x + L/2)/dx, lower node i0 = floor(u) (periodic), fraction
// f = u - i0 and weights (1 - f, f).  The acceleration at a node is the
// second-order central difference -(Phi_{i+1} - Phi_{i-1}) / (2 dx) of
// Sec. 3.1, interpolated with the same weights as the deposit.
//
// Deposit: every particle adds round(m w / q) to a 64-bit integer per node,
// q a mass quantum (total star mass / 2^50).  Integer addition is
// associative, so the deposited field does not depend on the order in
// which threads run: the step stays bitwise reproducible.
#include "spe_internal.cuh"

namespace spe {

struct Cic {
    int i0, i1;
    float w0, w1;
};

__device__ __forceinline__ Cic cic_axis(float x, float halfL, float inv_dx, int n)
{
    const float u = (x + halfL) * inv_dx;
    const float fl = floorf(u);
    int i = (int)fl;
    i %= n;
    if (i < 0) i += n;
    Cic c;
    c.i0 = i;
    c.i1 = (i + 1 == n) ? 0 : i + 1;
    c.w1 = u - fl;
    c.w0 = 1.f - c.w1;
    return c;
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ float wrap_pos(float x, float L)
{
    return x - L * floorf((x + 0.5f * L) / L);
}

__global__ void particles_kernel(PParams p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    float x = p.x[i], y = p.y[i], z = p.z[i];
    float vx = p.vx[i], vy = p.vy[i], vz = p.vz[i];
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    if (p.flags & PK_KICK) {
        const Cic cx = cic_axis(x, 0.5f * p.Lx, p.inv_dx, nx);
        const Cic cy = cic_axis(y, 0.5f * p.Ly, p.inv_dy, ny);
        const Cic cz = cic_axis(z, 0.5f * p.Lz, p.inv_dz, nz);
        float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int k = c ? cz.i1 : cz.i0;
            const float wz = c ? cz.w1 : cz.w0;
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                const int j = bb ? cy.i1 : cy.i0;
                const float wy = bb ? cy.w1 : cy.w0;
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int ii = a ? cx.i1 : cx.i0;
                    const float w = (a ? cx.w1 : cx.w0) * wy * wz;
                    const size_t plane = (size_t)k * ny;
                    const float *row = p.phi + (plane + j) * nx;
                    const float dphix = __ldg(&row[wrapi(ii + 1, nx)]) - __ldg(&row[wrapi(ii - 1, nx)]);
                    const float dphiy = __ldg(&p.phi[(plane + wrapi(j + 1, ny)) * nx + ii]) -
                                        __ldg(&p.phi[(plane + wrapi(j - 1, ny)) * nx + ii]);
                    const float dphiz = __ldg(&p.phi[((size_t)wrapi(k + 1, nz) * ny + j) * nx + ii]) -
                                        __ldg(&p.phi[((size_t)wrapi(k - 1, nz) * ny + j) * nx + ii]);
                    gx -= w * dphix;
                    gy -= w * dphiy;
                    gz -= w * dphiz;
                }
            }
        }
        vx += p.kick * gx * p.gx_scale;
        vy += p.kick * gy * p.gy_scale;
        vz += p.kick * gz * p.gz_scale;
        p.vx[i] = vx;
        p.vy[i] = vy;
        p.vz[i] = vz;
    }
    if (p.flags & PK_DRIFT) {
        x = wrap_pos(x + vx * p.drift, p.Lx);
        y = wrap_pos(y + vy * p.drift, p.Ly);
        z = wrap_pos(z + vz * p.drift, p.Lz);
        p.x[i] = x;
        p.y[i] = y;
        p.z[i] = z;
    }
    if (p.flags & PK_DEPOSIT) {
        const Cic cx = cic_axis(x, 0.5f * p.Lx, p.inv_dx, nx);
        const Cic cy = cic_axis(y, 0.5f * p.Ly, p.inv_dy, ny);
        const Cic cz = cic_axis(z, 0.5f * p.Lz, p.inv_dz, nz);
        const float mq = p.m[i] * p.inv_quantum;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int k = c ? cz.i1 : cz.i0;
            const float wz = c ? cz.w1 : cz.w0;
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                const int j = bb ? cy.i1 : cy.i0;
                const float wyz = (bb ? cy.w1 : cy.w0) * wz;
                unsigned long long *row =
                    reinterpret_cast<unsigned long long *>(p.dep) + ((size_t)k * ny + j) * nx;
                const long long q0 = llrintf(mq * cx.w0 * wyz);
                const long long q1 = llrintf(mq * cx.w1 * wyz);
                if (q0) atomicAdd(&row[cx.i0], (unsigned long long)q0);
                if (q1) atomicAdd(&row[cx.i1], (unsigned long long)q1);
            }
        }
    }
}

cudaError_t launch_particles(const PParams &p, cudaStream_t st)
{
    if (p.n <= 0) return cudaSuccess;
    const int nt = 256;
    particles_kernel<<<(p.n + nt - 1) / nt, nt, 0, st>>>(p);
    return cudaGetLastError();
}

__global__ void to_soa_kernel(const float *pos3, const float *vel3, const float *mass, int n, float *x, float *y,
                              float *z, float *vx, float *vy, float *vz, float *m, float Lx, float Ly, float Lz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = wrap_pos(pos3[3 * i + 0], Lx);
    y[i] = wrap_pos(pos3[3 * i + 1], Ly);
    z[i] = wrap_pos(pos3[3 * i + 2], Lz);
    vx[i] = vel3[3 * i + 0];
    vy[i] = vel3[3 * i + 1];
    vz[i] = vel3[3 * i + 2];
    m[i] = mass[i];
}

__global__ void from_soa_kernel(const float *x, const float *y, const float *z, const float *vx, const float *vy,
                                const float *vz, int n, float *pos3, float *vel3)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (pos3) {
        pos3[3 * i + 0] = x[i];
        pos3[3 * i + 1] = y[i];
        pos3[3 * i + 2] = z[i];
    }
    if (vel3) {
        vel3[3 * i + 0] = vx[i];
        vel3[3 * i + 1] = vy[i];
        vel3[3 * i + 2] = vz[i];
    }
}

cudaError_t launch_particles_to_soa(const float *pos3, const float *vel3, const float *mass, int n, float *x,
                                    float *y, float *z, float *vx, float *vy, float *vz, float *m, float Lx,
                                    float Ly, float Lz, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    to_soa_kernel<<<(n + 255) / 256, 256, 0, st>>>(pos3, vel3, mass, n, x, y, z, vx, vy, vz, m, Lx, Ly, Lz);
    return cudaGetLastError();
}

cudaError_t launch_particles_from_soa(const float *x, const float *y, const float *z, const float *vx,
                                      const float *vy, const float *vz, int n, float *pos3, float *vel3,
                                      cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    from_soa_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, y, z, vx, vy, vz, n, pos3, vel3);
    return cudaGetLastError();
}

}  // namespace spe
