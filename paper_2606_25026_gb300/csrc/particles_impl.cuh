// Star-particle device code shared by the stand-alone star kernel (particles.cu) and the batch's
// persistent kernel: the CIC helpers and the per-block kick-drift-deposit body.
#pragma once
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

// The stars of block `block` (kPartThreads of them, one per thread); box_raw is kBoxBytes of
// 16-byte-aligned shared memory.  The kernel below runs one block of stars per CTA, a persistent
// kernel any block from any CTA.
__device__ __forceinline__ void particles_body(const PParams &p, int block, unsigned char *box_raw)
{
    __shared__ int red[6][kPartThreads / 32];
    __shared__ int bb[6];
    float *sphi = reinterpret_cast<float *>(box_raw);
    unsigned long long *sdep = reinterpret_cast<unsigned long long *>(box_raw);
    const int i = block * kPartThreads + threadIdx.x;
    const bool live = i < p.n;
    float x = 0.f, y = 0.f, z = 0.f, vx = 0.f, vy = 0.f, vz = 0.f, m = 0.f;
    if (live) {
        if (p.flags & PK_DEPOSIT) m = p.m[i];   // with the other loads: the deposit would wait on it
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
            // four nodes per thread in flight before their stores: the box fill waits on L2 once per
            // four nodes instead of once per node
            const unsigned mx = div_magic(ex), my = div_magic(ey);
            const int vol = ex * ey * ez;
            for (int v0 = threadIdx.x; v0 < vol; v0 += 4 * kPartThreads) {
                float f[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int v = v0 + u * kPartThreads;
                    if (v < vol) {
                        const int r = div_small(v, mx), c = div_small(r, my);
                        const int a = v - r * ex, b = r - c * ey;
                        f[u] = __ldg(&p.phi[((size_t)wrapi(oz + c, nz) * ny + wrapi(oy + b, ny)) * nx + wrapi(ox + a, nx)]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (v0 + u * kPartThreads < vol) sphi[v0 + u * kPartThreads] = f[u];
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
        const float mq = live ? m * p.inv_quantum : 0.f;
        // The block's box counts in two 32-bit halves, q = hi 2^21 + lo (lo < 2^21): while every
        // share q < 2^41 (a star below 2^-9 of the total star mass), 256 stars cannot carry either
        // half's sum past 2^29, and the flush joins them into the exact 64-bit sum.  32-bit shared
        // atomics run about twice as fast as 64-bit ones here (76 -> 60 us per launch for 1e6
        // Plummer stars at 256^3); heavier stars take the 64-bit box.
        unsigned *slo = reinterpret_cast<unsigned *>(box_raw), *shi = slo + kBoxDep;
        const bool split = __syncthreads_and(mq < 0x1p41f) != 0;
        if (tiled) {
            if (split) {
                for (int v = threadIdx.x; v < vol; v += kPartThreads) slo[v] = shi[v] = 0u;
            } else {
                for (int v = threadIdx.x; v < vol; v += kPartThreads) sdep[v] = 0ull;
            }
            __syncthreads();
        }
        if (live) {
            if (tiled && split) {
                const int rot = threadIdx.x & 7;
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const int cc = (kk + rot) & 7;
                    const int a = cc & 1, b2 = (cc >> 1) & 1, c = cc >> 2;
                    const float wyz = (b2 ? cy.w1 : cy.w0) * (c ? cz.w1 : cz.w0);
                    const long long q = llrintf(mq * (a ? cx.w1 : cx.w0) * wyz);
                    if (q) {
                        const int v = ((cz.i0 + c - oz) * ey + (cy.i0 + b2 - oy)) * ex + (cx.i0 + a - ox);
                        atomicAdd(&slo[v], (unsigned)(q & 0x1FFFFF));
                        const unsigned h = (unsigned)(q >> 21);
                        if (h) atomicAdd(&shi[v], h);
                    }
                }
            } else if (tiled) {
                // lane l visits its corners starting at corner l mod 8: where a warp's stars share a
                // cell (a dense cluster), the lanes of one atomic spread over the eight corner nodes
                // instead of all meeting on one.  The quantised values are the ones of the loop below.
                const int rot = threadIdx.x & 7;
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const int cc = (kk + rot) & 7;
                    const int a = cc & 1, b2 = (cc >> 1) & 1, c = cc >> 2;
                    const float wyz = (b2 ? cy.w1 : cy.w0) * (c ? cz.w1 : cz.w0);
                    const long long q = llrintf(mq * (a ? cx.w1 : cx.w0) * wyz);
                    if (q)
                        atomicAdd(&sdep[((cz.i0 + c - oz) * ey + (cy.i0 + b2 - oy)) * ex + (cx.i0 + a - ox)],
                                  (unsigned long long)q);
                }
            } else {
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
                const unsigned long long q = split ? ((unsigned long long)shi[v] << 21) + slo[v] : sdep[v];
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

}  // namespace spe
