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
#include "particles_impl.cuh"

namespace spe {

__global__ void __launch_bounds__(kPartThreads, 4) particles_kernel(PParams p)
{
    __shared__ __align__(16) unsigned char box_raw[kBoxBytes];
    particles_body(p, blockIdx.x, box_raw);
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
