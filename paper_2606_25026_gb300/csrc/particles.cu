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
// which threads run: the step stays bitwise reproducible.  Every row (y, z)
// that receives mass is also marked in a byte array, so that the density
// pass reads and clears only the rows that can hold deposits.
#include "spe_internal.cuh"

#include <climits>

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
    if ((unsigned)i >= (unsigned)n) {   // positions are kept in the box: only u = n after rounding lands here
        i %= n;
        if (i < 0) i += n;
    }
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

// Shared-memory boxes of the tiled path: the Phi nodes the block's kick
// stencils touch, or the deposit nodes of its stars.  Stars are kept sorted by
// 4^3 cell blocks, so a block of 256 consecutive stars usually covers one or
// two cell blocks and its box is small; a block whose box does not fit (stars
// spread out, or on both sides of the periodic boundary) uses global memory.
constexpr int kPartThreads = 256;
constexpr int kBoxBytes = 16384;
constexpr int kBoxPhi = kBoxBytes / 4;     // floats
constexpr int kBoxDep = kBoxBytes / 8;     // 64-bit counters

// Exact v / d for 0 <= v, d < 2^16, d >= 2, with m = div_magic(d): the product's error v (m - 2^32/d)
// / 2^32 < v / 2^32 < 1/d cannot carry v/d past the next integer.
__device__ __forceinline__ unsigned div_magic(unsigned d) { return 0xffffffffu / d + 1u; }
__device__ __forceinline__ int div_small(int v, unsigned m) { return (int)__umulhi((unsigned)v, m); }

// Block-wide min and max of three integers over the live threads; results
// in out[0..2] (min) and out[3..5] (max).  All threads of the block call it.
__device__ __forceinline__ void block_minmax3(int a, int b, int c, bool live, int (*red)[kPartThreads / 32],
                                              int *out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int v[6] = {live ? a : INT_MAX, live ? b : INT_MAX, live ? c : INT_MAX,
                live ? a : INT_MIN, live ? b : INT_MIN, live ? c : INT_MIN};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        v[q] = __reduce_min_sync(0xffffffffu, v[q]);
        v[q + 3] = __reduce_max_sync(0xffffffffu, v[q + 3]);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 6; ++q) red[q][warp] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int q = threadIdx.x;
        int r = red[q][0];
        for (int w = 1; w < kPartThreads / 32; ++w) r = q < 3 ? min(r, red[q][w]) : max(r, red[q][w]);
        out[q] = r;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kPartThreads, 4) particles_kernel(PParams p)
{
    __shared__ __align__(16) unsigned char box_raw[kBoxBytes];
    __shared__ int red[6][kPartThreads / 32];
    __shared__ int bb[6];
    float *sphi = reinterpret_cast<float *>(box_raw);
    unsigned long long *sdep = reinterpret_cast<unsigned long long *>(box_raw);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < p.n;
    float x = 0.f, y = 0.f, z = 0.f, vx = 0.f, vy = 0.f, vz = 0.f;
    if (live) {
        x = p.x[i];
        y = p.y[i];
        z = p.z[i];
        vx = p.vx[i];
        vy = p.vy[i];
        vz = p.vz[i];
    }
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    if (p.flags & PK_KICK) {
        const Cic cx = cic_axis(x, 0.5f * p.Lx, p.inv_dx, nx);
        const Cic cy = cic_axis(y, 0.5f * p.Ly, p.inv_dy, ny);
        const Cic cz = cic_axis(z, 0.5f * p.Lz, p.inv_dz, nz);
        // the stencil of a star spans nodes i0 - 1 .. i0 + 2 on each axis
        block_minmax3(cx.i0, cy.i0, cz.i0, live, red, bb);
        const int ox = bb[0] - 1, oy = bb[1] - 1, oz = bb[2] - 1;
        const int ex = bb[3] - bb[0] + 4, ey = bb[4] - bb[1] + 4, ez = bb[5] - bb[2] + 4;
        const bool tiled = (long long)ex * ey * ez <= kBoxPhi;
        if (tiled) {
            const unsigned mx = div_magic(ex), my = div_magic(ey);
            for (int v = threadIdx.x; v < ex * ey * ez; v += kPartThreads) {
                const int r = div_small(v, mx), c = div_small(r, my);
                const int a = v - r * ex, b = r - c * ey;
                sphi[v] = __ldg(&p.phi[((size_t)wrapi(oz + c, nz) * ny + wrapi(oy + b, ny)) * nx + wrapi(ox + a, nx)]);
            }
            __syncthreads();
        }
        float gx = 0.f, gy = 0.f, gz = 0.f;
        if (live && tiled) {
            // the eight corners' central differences read 32 distinct nodes: the four x nodes
            // i0-1 .. i0+2 of the corner rows, and the rows j0-1, j0+2 and planes k0-1, k0+2
            const int sz = ex * ey;
            const float *q0 = sphi + ((cz.i0 - oz) * ey + (cy.i0 - oy)) * ex + (cx.i0 - ox);
            float r[2][2][4];
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int b2 = 0; b2 < 2; ++b2)
#pragma unroll
                    for (int a4 = 0; a4 < 4; ++a4) r[c][b2][a4] = q0[c * sz + b2 * ex + a4 - 1];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float wz = c ? cz.w1 : cz.w0;
#pragma unroll
                for (int b2 = 0; b2 < 2; ++b2) {
                    const float wy = b2 ? cy.w1 : cy.w0;
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        const float w = (a ? cx.w1 : cx.w0) * wy * wz;
                        const float dphix = r[c][b2][a + 2] - r[c][b2][a];
                        const float yp = b2 ? q0[c * sz + 2 * ex + a] : r[c][1][a + 1];
                        const float ym = b2 ? r[c][0][a + 1] : q0[c * sz - ex + a];
                        const float zp = c ? q0[2 * sz + b2 * ex + a] : r[1][b2][a + 1];
                        const float zm = c ? r[0][b2][a + 1] : q0[-sz + b2 * ex + a];
                        gx -= w * dphix;
                        gy -= w * (yp - ym);
                        gz -= w * (zp - zm);
                    }
                }
            }
        } else if (live) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int k = c ? cz.i1 : cz.i0;
                const float wz = c ? cz.w1 : cz.w0;
#pragma unroll
                for (int b2 = 0; b2 < 2; ++b2) {
                    const int j = b2 ? cy.i1 : cy.i0;
                    const float wy = b2 ? cy.w1 : cy.w0;
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
        }
        if (live) {
            vx += p.kick * gx * p.gx_scale;
            vy += p.kick * gy * p.gy_scale;
            vz += p.kick * gz * p.gz_scale;
            p.vx[i] = vx;
            p.vy[i] = vy;
            p.vz[i] = vz;
        }
        __syncthreads();   // the box is reused below
    }
    if ((p.flags & PK_DRIFT) && live) {
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
        // a star deposits to nodes i0 .. i0 + 1 on each axis
        block_minmax3(cx.i0, cy.i0, cz.i0, live, red, bb);
        const int ox = bb[0], oy = bb[1], oz = bb[2];
        const int ex = bb[3] - bb[0] + 2, ey = bb[4] - bb[1] + 2, ez = bb[5] - bb[2] + 2;
        const int vol = ex * ey * ez;
        const bool tiled = (long long)ex * ey * ez <= kBoxDep;
        if (tiled) {
            for (int v = threadIdx.x; v < vol; v += kPartThreads) sdep[v] = 0ull;
            __syncthreads();
        }
        if (live) {
            const float mq = p.m[i] * p.inv_quantum;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int k = c ? cz.i1 : cz.i0;
                const float wz = c ? cz.w1 : cz.w0;
#pragma unroll
                for (int b2 = 0; b2 < 2; ++b2) {
                    const int j = b2 ? cy.i1 : cy.i0;
                    const float wyz = (b2 ? cy.w1 : cy.w0) * wz;
                    const long long q0 = llrintf(mq * cx.w0 * wyz);
                    const long long q1 = llrintf(mq * cx.w1 * wyz);
                    if (tiled) {
                        unsigned long long *srow =
                            sdep + ((cz.i0 + c - oz) * ey + (cy.i0 + b2 - oy)) * ex + (cx.i0 - ox);
                        if (q0) atomicAdd(&srow[0], (unsigned long long)q0);
                        if (q1) atomicAdd(&srow[1], (unsigned long long)q1);
                    } else {
                        unsigned long long *row =
                            reinterpret_cast<unsigned long long *>(p.dep) + ((size_t)k * ny + j) * nx;
                        if (q0) atomicAdd(&row[cx.i0], (unsigned long long)q0);
                        if (q1) atomicAdd(&row[cx.i1], (unsigned long long)q1);
                        if (q0 | q1) p.dflag[(size_t)k * ny + j] = 1;
                    }
                }
            }
        }
        if (tiled) {
            __syncthreads();
            unsigned long long *dep = reinterpret_cast<unsigned long long *>(p.dep);
            const unsigned mx = div_magic(ex), my = div_magic(ey);
            for (int v = threadIdx.x; v < vol; v += kPartThreads) {
                const unsigned long long q = sdep[v];
                if (q) {
                    const int r = div_small(v, mx), c = div_small(r, my);
                    const int a = v - r * ex, b = r - c * ey;
                    const size_t row = (size_t)wrapi(oz + c, nz) * ny + wrapi(oy + b, ny);
                    atomicAdd(&dep[row * nx + wrapi(ox + a, nx)], q);
                    p.dflag[row] = 1;   // every writer stores the same byte
                }
            }
        }
    }
}

cudaError_t launch_particles(const PParams &p, cudaStream_t st)
{
    if (p.n <= 0) return cudaSuccess;
    particles_kernel<<<(p.n + kPartThreads - 1) / kPartThreads, kPartThreads, 0, st>>>(p);
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

// ---------------------------------------------------------------- reordering by cell block
// Stars are kept in memory grouped by coarse cell blocks (4 x 4 x 4 grid
// cells) so that a warp's Phi gathers and deposit atomics land on few L2
// lines.  Counting sort: histogram of block keys, exclusive scan, scatter.
// The order inside a block depends on atomic arrival and is not
// reproducible, but every per-star update is independent of memory order
// and the deposit is an integer sum, so the physics stays bitwise
// reproducible; the id array maps memory slots back to insertion order.

namespace spe {

__device__ __forceinline__ int block_key(float x, float y, float z, const SortParams &s)
{
    const Cic cx = cic_axis(x, 0.5f * s.Lx, s.inv_dx, s.nx);
    const Cic cy = cic_axis(y, 0.5f * s.Ly, s.inv_dy, s.ny);
    const Cic cz = cic_axis(z, 0.5f * s.Lz, s.inv_dz, s.nz);
    return ((cz.i0 >> 2) * s.nby + (cy.i0 >> 2)) * s.nbx + (cx.i0 >> 2);
}

// Lanes of a warp that share a key add to its counter with one atomic (the
// Plummer core puts most stars in a few blocks, so per-lane atomics would
// serialise on those counters).  Returns this lane's slot: base + its rank
// among the lanes with the same key.
__device__ __forceinline__ int warp_aggregated_add(int *counter, int key, bool active)
{
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (!active) return 0;
    const unsigned same = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(same) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&counter[key], __popc(same));
    base = __shfl_sync(same, base, leader);
    return base + __popc(same & ((1u << lane) - 1u));
}

__global__ void sort_hist_kernel(SortParams s)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < s.n;
    int k = 0;
    if (active) {
        k = block_key(s.src[0][i], s.src[1][i], s.src[2][i], s);
        s.key[i] = k;
    }
    warp_aggregated_add(s.count, k, active);
}

// Exclusive scan of count[0..nbins) in place, in three launches: each CTA of 256 threads
// totals a span of kScanSpan bins (8 consecutive bins per thread), one CTA scans those totals,
// and each CTA then scans its span again with its total's offset.  Integer sums, so the result
// is exact and independent of scheduling.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanSpan = kScanThreads * kScanPer;

// inclusive block scan of one int per thread (kScanThreads threads); returns this thread's
// inclusive prefix, total in *block_total
__device__ __forceinline__ int block_scan_incl(int v, int *sh, int *block_total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kScanThreads / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        if (lane < kScanThreads / 32) sh[lane] = w;
    }
    __syncthreads();
    const int r = v + (warp ? sh[warp - 1] : 0);
    *block_total = sh[kScanThreads / 32 - 1];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) sort_span_totals_kernel(const int *count, int nbins, int *totals)
{
    __shared__ int sh[kScanThreads / 32];
    const int b0 = blockIdx.x * kScanSpan + threadIdx.x * kScanPer;
    int sum = 0;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q)
        if (b0 + q < nbins) sum += count[b0 + q];
    int total;
    block_scan_incl(sum, sh, &total);
    if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

// exclusive scan of the span totals in place, one CTA of 1024 threads, contiguous chunks
__global__ void __launch_bounds__(1024) sort_scan_totals_kernel(int *totals, int nspans)
{
    __shared__ int part[1024];
    const int chunk = (nspans + 1023) / 1024;
    const int s0 = threadIdx.x * chunk;
    const int s1 = min(s0 + chunk, nspans);
    int sum = 0;
    for (int k = s0; k < s1; ++k) sum += totals[k];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - sum;
    for (int k = s0; k < s1; ++k) {
        const int c = totals[k];
        totals[k] = run;
        run += c;
    }
}

__global__ void __launch_bounds__(kScanThreads) sort_span_scan_kernel(int *count, int nbins, const int *offsets)
{
    __shared__ int sh[kScanThreads / 32];
    const int b0 = blockIdx.x * kScanSpan + threadIdx.x * kScanPer;
    int c[kScanPer];
    int sum = 0;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        c[q] = b0 + q < nbins ? count[b0 + q] : 0;
        sum += c[q];
    }
    int total;
    int run = block_scan_incl(sum, sh, &total) - sum + offsets[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        if (b0 + q < nbins) count[b0 + q] = run;
        run += c[q];
    }
}

__global__ void sort_scatter_kernel(SortParams s)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < s.n;
    const int dst = warp_aggregated_add(s.count, active ? s.key[i] : 0, active);
    if (!active) return;
#pragma unroll
    for (int a = 0; a < 7; ++a) s.dst[a][dst] = s.src[a][i];
    s.dst_id[dst] = s.src_id[i];
}

cudaError_t launch_particle_sort(const SortParams &s, cudaStream_t st, int *launches)
{
    if (s.n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(s.count, 0, sizeof(int) * (size_t)s.nbins, st);
    if (e != cudaSuccess) return e;
    const int nb = (s.n + 255) / 256;
    const int nspans = (s.nbins + kScanSpan - 1) / kScanSpan;
    sort_hist_kernel<<<nb, 256, 0, st>>>(s);
    sort_span_totals_kernel<<<nspans, kScanThreads, 0, st>>>(s.count, s.nbins, s.totals);
    sort_scan_totals_kernel<<<1, 1024, 0, st>>>(s.totals, nspans);
    sort_span_scan_kernel<<<nspans, kScanThreads, 0, st>>>(s.count, s.nbins, s.totals);
    sort_scatter_kernel<<<nb, 256, 0, st>>>(s);
    if (launches) *launches += 5;
    return cudaGetLastError();
}

__global__ void ids_kernel(unsigned int *id, int first, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) id[i] = (unsigned int)(first + i);
}

cudaError_t launch_particle_ids(unsigned int *id, int first, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    ids_kernel<<<(n + 255) / 256, 256, 0, st>>>(id + first, first, n);
    return cudaGetLastError();
}

// AoS output in insertion order: slot i holds the star with id[i].
__global__ void from_soa_by_id_kernel(const float *x, const float *y, const float *z, const float *vx,
                                      const float *vy, const float *vz, const unsigned int *id, int n,
                                      float *pos3, float *vel3)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned int o = id[i];
    if (pos3) {
        pos3[3 * o + 0] = x[i];
        pos3[3 * o + 1] = y[i];
        pos3[3 * o + 2] = z[i];
    }
    if (vel3) {
        vel3[3 * o + 0] = vx[i];
        vel3[3 * o + 1] = vy[i];
        vel3[3 * o + 2] = vz[i];
    }
}

cudaError_t launch_particles_from_soa_by_id(const float *x, const float *y, const float *z, const float *vx,
                                            const float *vy, const float *vz, const unsigned int *id, int n,
                                            float *pos3, float *vel3, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    from_soa_by_id_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, y, z, vx, vy, vz, id, n, pos3, vel3);
    return cudaGetLastError();
}

}  // namespace spe
