// Warp-per-line x passes for lines of 256 and 512 points (FP32, no shared
// memory, no block-wide barriers).  One warp owns a pair of rows (2m, 2m+1).
// A line of N = 32 R points lives in the warp's registers, R per lane, in one
// of two layouts:
//   layout A: lane a holds points a + 32 r,          r = 0..R-1
//   layout B: lane l holds points r + R bitrev5(l),  r = 0..R-1 (R contiguous)
// With n = a + 32 r and k = k2 + R k1 the DFT factors as
//   X[k2 + R k1] = sum_a W32^{a k1} [ W_N^{a k2} sum_r x[a + 32 r] W_R^{r k2} ],
// so A -> B is an R-point DFT in registers, a twiddle, and a radix-2
// decimation-in-frequency network across lanes (shuffles; its output comes
// out bit-reversed, which is layout B); B -> A runs the reverse sequence
// (decimation-in-time across lanes from bit-reversed input, twiddle, register
// DFT).  The inverse transforms go A -> B, the forward ones B -> A, so that
//   kick pass   : Phi (the inverse of the packed half-spectrum rows) comes out
//                 in layout B, psi is loaded in layout B (R contiguous points
//                 per lane), kicked, transformed forward into layout A and
//                 stored coalesced;
//   density pass: psi-hat is loaded in layout A (coalesced), transformed back
//                 into layout B and stored, |psi|^2 (+ the star deposit) packed
//                 as one complex line per row pair, transformed forward into
//                 layout A and separated into the two rows' half spectra with
//                 the mirror value of each point fetched across lanes.
// Twiddles come from the grid's FP64-built (hi, lo) table with the same
// compensated multiply as the shared-memory passes.
#include "fft_tile.cuh"
#include "reduce.cuh"
#include "spe_internal.cuh"

namespace spe {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kXwThreads = 256;      // 8 warps, 8 row pairs, 16 rows per block

__device__ __forceinline__ int brev5(int l) { return (int)(__brev((unsigned)l) >> 27); }

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m)
{
    return make_float2(__shfl_xor_sync(kFull, v.x, m), __shfl_xor_sync(kFull, v.y, m));
}

__device__ __forceinline__ float2 shfl2(float2 v, int src)
{
    return make_float2(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src));
}

// e^{DIR 2 pi i m / N} from the table of e^{-2 pi i m / N} as (hi, lo)
template <int DIR>
__device__ __forceinline__ void twiddle(const float4 *__restrict__ tw, int m, float2 &hi, float2 &lo)
{
    const float4 w = __ldg(&tw[m]);
    hi = make_float2(w.x, DIR > 0 ? -w.y : w.y);
    lo = make_float2(w.z, DIR > 0 ? -w.w : w.w);
}

// layout A -> layout B
template <int N, int DIR>
__device__ __forceinline__ void fft_ab(float2 (&v)[N / 32], const float4 *__restrict__ tw)
{
    constexpr int R = N / 32;
    const int a = threadIdx.x & 31;
    Dft<R, DIR>::run(v);
#pragma unroll
    for (int k = 1; k < R; ++k) {
        float2 hi, lo;
        twiddle<DIR>(tw, a * k, hi, lo);
        v[k] = cmul_comp(v[k], hi, lo);
    }
#pragma unroll
    for (int span = 16; span >= 1; span >>= 1) {
        const bool up = (a & span) != 0;
        float2 hi, lo;
        twiddle<DIR>(tw, (a & (span - 1)) * (N / (2 * span)), hi, lo);
        if (!up) {
            hi = make_float2(1.f, 0.f);
            lo = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 p = shfl_xor2(v[r], span);
            const float2 s = up ? csub(p, v[r]) : cadd(v[r], p);
            v[r] = cmul_comp(s, hi, lo);
        }
    }
}

// layout B -> layout A
template <int N, int DIR>
__device__ __forceinline__ void fft_ba(float2 (&v)[N / 32], const float4 *__restrict__ tw)
{
    constexpr int R = N / 32;
    const int a = threadIdx.x & 31;
#pragma unroll
    for (int span = 1; span <= 16; span <<= 1) {
        const bool up = (a & span) != 0;
        float2 hi, lo;
        twiddle<DIR>(tw, (a & (span - 1)) * (N / (2 * span)), hi, lo);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 p = shfl_xor2(v[r], span);
            // lower lane: v + w p, upper lane: p - w v
            const float2 t = cmul_comp(up ? v[r] : p, hi, lo);
            const float2 o = up ? p : v[r];
            v[r] = up ? csub(o, t) : cadd(o, t);
        }
    }
#pragma unroll
    for (int k = 1; k < R; ++k) {
        float2 hi, lo;
        twiddle<DIR>(tw, a * k, hi, lo);
        v[k] = cmul_comp(v[k], hi, lo);
    }
    Dft<R, DIR>::run(v);
}

constexpr int kKickFlags = X_HAS_PHI | X_WRITE_PHI | X_KICK | X_FFT | X_STATIC | X_ABSORB;
constexpr int kDensityFlags = X_IFFT | X_MASS | X_R2C | X_DEP;

template <int N>
__global__ void __launch_bounds__(kXwThreads) xwarp_kick_kernel(XParams p)
{
    constexpr int R = N / 32, H = N / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ra = 2 * (blockIdx.x * (kXwThreads / 32) + warp);
    if (ra >= p.rows) return;    // whole warps; this kernel has no block-level synchronisation
    const int flags = p.flags;
    const int nb = R * brev5(lane);  // first point of this lane in layout B
    float pa[R], pb[R];
#pragma unroll
    for (int r = 0; r < R; ++r) pa[r] = pb[r] = 0.f;

    if (flags & X_HAS_PHI) {
        // packed line Z = A + iB of the two rows' Hermitian half spectra, layout A
        float2 z[R];
        const bool has_b = ra + 1 < p.rows;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int n = lane + 32 * r;
            const int kk = (n <= H) ? n : N - n;
            float2 A = __ldg(&p.phik[(size_t)ra * p.P + kk]);
            float2 B = has_b ? __ldg(&p.phik[(size_t)(ra + 1) * p.P + kk]) : make_float2(0.f, 0.f);
            if (n > H) {
                A.y = -A.y;
                B.y = -B.y;
            }
            if (n == 0 || n == H) {
                A.y = 0.f;
                B.y = 0.f;
            }
            z[r] = make_float2(A.x - B.y, A.y + B.x);
        }
        fft_ab<N, +1>(z, p.tw);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            pa[r] = z[r].x;
            pb[r] = z[r].y;
        }
        if ((flags & X_WRITE_PHI) && has_b) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float za = pa[r], zb = pb[r];
                if (flags & X_STATIC) {
                    za += __ldg(&p.phib[(size_t)ra * N + nb + r]);
                    zb += __ldg(&p.phib[(size_t)(ra + 1) * N + nb + r]);
                }
                p.phi_out[(size_t)ra * N + nb + r] = za;
                p.phi_out[(size_t)(ra + 1) * N + nb + r] = zb;
            }
        }
    }

    if (flags & (X_KICK | X_FFT)) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = ra + h;
            if (row >= p.rows) break;
            float2 v[R];
            const float4 *src = reinterpret_cast<const float4 *>(p.psi + (size_t)row * N + nb);
#pragma unroll
            for (int q = 0; q < R / 2; ++q) {
                const float4 w = src[q];
                v[2 * q] = make_float2(w.x, w.y);
                v[2 * q + 1] = make_float2(w.z, w.w);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int n = nb + r;
                if (flags & X_KICK) {
                    const float a2 = v[r].x * v[r].x + v[r].y * v[r].y;
                    float phi = (flags & X_HAS_PHI) ? (h ? pb[r] : pa[r]) : 0.f;
                    if (flags & X_STATIC) {
                        const float pbv = __ldg(&p.phib[(size_t)row * N + n]);
                        phi += pbv;
                        if ((flags & X_WRITE_PHI) && !(flags & X_HAS_PHI)) p.phi_out[(size_t)row * N + n] = pbv;
                    }
                    // v * exp(-i ph) = v + v (cos ph - 1 - i sin ph), cos ph - 1 = -2 sin^2(ph/2)
                    float sh, ch;
                    sincosf(0.5f * ((phi + p.kappa * a2) * p.kick_scale), &sh, &ch);
                    const float cm1 = -2.f * sh * sh, sn = 2.f * sh * ch;
                    v[r] = make_float2(fmaf(v[r].x, cm1, fmaf(v[r].y, sn, v[r].x)),
                                       fmaf(v[r].y, cm1, fmaf(-v[r].x, sn, v[r].y)));
                }
                if (flags & X_ABSORB) {
                    const float b = __ldg(&p.absorb_x[n]) * __ldg(&p.absorb_y[row % p.ny]) *
                                    __ldg(&p.absorb_z[row / p.ny]);
                    v[r] = make_float2(v[r].x * b, v[r].y * b);
                }
            }
            if (flags & X_FFT) {
                fft_ba<N, -1>(v, p.tw);
#pragma unroll
                for (int r = 0; r < R; ++r) p.psi[(size_t)row * N + lane + 32 * r] = v[r];
            } else {
                float4 *dst = reinterpret_cast<float4 *>(p.psi + (size_t)row * N + nb);
#pragma unroll
                for (int q = 0; q < R / 2; ++q)
                    dst[q] = make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
            }
        }
    }
}

template <int N>
__global__ void __launch_bounds__(kXwThreads) xwarp_density_kernel(XParams p)
{
    constexpr int R = N / 32, H = N / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ra = 2 * (blockIdx.x * (kXwThreads / 32) + warp);
    const bool live = ra < p.rows;       // every thread reaches the grid reduction
    const int flags = p.flags;
    const int nb = R * brev5(lane);
    float msum = 0.f;
    float rho[2][R];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int row = ra + h;
        const bool ok = live && row < p.rows;
        float2 v[R];
        if (flags & X_IFFT) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                v[r] = ok ? p.psi[(size_t)row * N + lane + 32 * r] : make_float2(0.f, 0.f);
            fft_ab<N, +1>(v, p.tw);
            if (ok) {
                float4 *dst = reinterpret_cast<float4 *>(p.psi + (size_t)row * N + nb);
#pragma unroll
                for (int q = 0; q < R / 2; ++q)
                    dst[q] = make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
            }
        } else {
            const float4 *src = reinterpret_cast<const float4 *>(p.psi + (size_t)row * N + nb);
#pragma unroll
            for (int q = 0; q < R / 2; ++q) {
                const float4 w = ok ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                v[2 * q] = make_float2(w.x, w.y);
                v[2 * q + 1] = make_float2(w.z, w.w);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float a2 = v[r].x * v[r].x + v[r].y * v[r].y;
            msum += a2;
            rho[h][r] = a2;
        }
        if ((flags & X_DEP) && ok) {
            long long *dep = p.dep + (size_t)row * N + nb;
            long long d[R];
#pragma unroll
            for (int r = 0; r < R; ++r) d[r] = __ldcs(&dep[r]);
#pragma unroll
            for (int r = 0; r < R; ++r) rho[h][r] += (float)d[r] * p.dep_scale;
            // every value of this lane's run has been read: clear it for the next step
#pragma unroll
            for (int r = 0; r < R; ++r) __stcs(&dep[r], 0ll);
        }
    }
    if (flags & X_R2C) {
        float2 z[R];
#pragma unroll
        for (int r = 0; r < R; ++r) z[r] = make_float2(rho[0][r], rho[1][r]);
        fft_ba<N, -1>(z, p.tw);
        // separate the two real rows: A_k = (Z_k + conj Z_{N-k}) / 2, B_k = (Z_k - conj Z_{N-k}) / (2i);
        // N - k of k = a + 32 r is (32 - a) + 32 (R - 1 - r) for a > 0 and 32 (R - r) for a = 0
        const int src = (32 - lane) & 31;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 zp = shfl2(z[R - 1 - r], src);
            if (lane == 0) zp = z[(R - r) % R];
            const float2 zc = make_float2(zp.x, -zp.y);
            const float2 A = make_float2(0.5f * (z[r].x + zc.x), 0.5f * (z[r].y + zc.y));
            const float2 D = csub(z[r], zc);
            const float2 B = make_float2(0.5f * D.y, -0.5f * D.x);
            const int k = lane + 32 * r;
            if (live && k <= H && ra + 1 < p.rows) {
                p.phik[(size_t)ra * p.P + k] = A;
                p.phik[(size_t)(ra + 1) * p.P + k] = B;
            }
        }
    }
    if (flags & X_MASS) {
        double v[1] = {(double)msum};
        grid_reduce<1, kXwThreads>(v, 0, p.partials, p.counter, p.result);
    }
}

template <int N>
cudaError_t launch_xw(const XParams &p, cudaStream_t st, int *blocks_out)
{
    const int blocks = (p.rows + 15) / 16;
    if (blocks_out) *blocks_out = blocks;
    if ((p.flags & ~kKickFlags) == 0)
        xwarp_kick_kernel<N><<<blocks, kXwThreads, 0, st>>>(p);
    else
        xwarp_density_kernel<N><<<blocks, kXwThreads, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

// The warp-per-line form of the x pass where it applies (lines of 256 or 512,
// an even row count, the kick or the density flag sets); cudaErrorNotSupported
// otherwise, and the caller runs the shared-memory kernel.
cudaError_t launch_xwarp(int nx, const XParams &p, cudaStream_t st, int *blocks_out)
{
    const bool kick = (p.flags & ~kKickFlags) == 0;
    const bool dens = (p.flags & ~kDensityFlags) == 0;
    if (p.tc || (p.rows & 1) || !(kick || dens)) return cudaErrorNotSupported;
    if (nx == 256) return launch_xw<256>(p, st, blocks_out);
    if (nx == 512) return launch_xw<512>(p, st, blocks_out);
    return cudaErrorNotSupported;
}

}  // namespace spe
