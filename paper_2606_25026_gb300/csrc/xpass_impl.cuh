// x-axis passes: lines along x are contiguous rows of the field.
//
// One CTA owns T = 16 consecutive rows.  Rows are staged in shared memory
// element-major (tile[n * (T+1) + t], the +1 pad keeps both the row-wise
// global<->shared copies and the FFT stages free of bank conflicts).  What a
// launch does is selected by XParams::flags; the step uses two combinations:
//
//   kick pass     (X_HAS_PHI | X_KICK | X_FFT [| X_WRITE_PHI]):
//       Phi rows rebuilt from the x half spectrum (inverse real transform,
//       two rows packed as one complex line), psi *= exp(-i (Phi +
//       kappa|psi|^2) dt_k / eta)  [Sec. 3.1 steps (a)/(d), Algorithm 1],
//       then the forward x transform of psi  [step (b), first axis].
//   density pass  (X_IFFT | X_MASS | X_R2C [| X_DEP]):
//       inverse x transform of psi  [step (b), last axis], rho = |psi|^2 +
//       rho_*  [step (c)], the mass reduced on the fly, and the forward real
//       x transform of rho into the half spectrum  [step (c), first axis].
#pragma once
#include "fft_tile.cuh"
#include "reduce.cuh"
#include "spe_internal.cuh"
#include "tc16.cuh"

namespace spe {

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

// sin h and cos h of a kick half-angle.  A kick turns the phase by a small angle (|h| well below
// 1/2 at any stable time step), where the Maclaurin series of sine to h^11 and of cosine to h^10
// are exact to under 1e-12 relative (the first omitted terms are h^13/13! and h^12/12!), so the
// only error is the FP32 rounding of the Horner evaluation; larger angles take sincosf.  For
// |h| <= 2^-6 (the common case: about 1e-4 at a CFL-limited step of a 512^3 halo) the series to h^5
// and h^4 already stay under 1e-12 relative (h^6/7! < 3e-15, h^6/6! < 2e-14).
__device__ __forceinline__ void half_angle_sincos(float h, float &sh, float &ch)
{
    if (fabsf(h) <= 0.015625f) {
        const float s2 = h * h;
        sh = fmaf(h * s2, fmaf(s2, 1.f / 120.f, -1.f / 6.f), h);
        ch = fmaf(s2, fmaf(s2, 1.f / 24.f, -0.5f), 1.f);
    } else if (fabsf(h) <= 0.5f) {
        const float s2 = h * h;
        float ps = -1.f / 39916800.f;
        ps = fmaf(ps, s2, 1.f / 362880.f);
        ps = fmaf(ps, s2, -1.f / 5040.f);
        ps = fmaf(ps, s2, 1.f / 120.f);
        ps = fmaf(ps, s2, -1.f / 6.f);
        sh = fmaf(h * s2, ps, h);
        float pc = -1.f / 3628800.f;
        pc = fmaf(pc, s2, 1.f / 40320.f);
        pc = fmaf(pc, s2, -1.f / 720.f);
        pc = fmaf(pc, s2, 1.f / 24.f);
        pc = fmaf(pc, s2, -0.5f);
        ch = fmaf(s2, pc, 1.f);
    } else {
        sincosf(h, &sh, &ch);
    }
}

template <int N, bool TC = false> struct XCfg {
    static constexpr int T = 16;
    static constexpr int TP = T + 1;
    static constexpr int HP = T / 2 + 1;   // pitch of the packed Phi lines
    static constexpr int NT = (N >= 512 && !TC) ? 512 : ((N * T / 8 >= 256) ? 256 : ((N * T / 8 >= 128) ? 128 : 64));
    // tile + aux; aux holds T real rows, the T half-spectrum rows of N/2 + 1 complex while staging,
    // or the T/2 packed complex Phi lines (pitch HP) while they are transformed
    static constexpr size_t aux_bytes = cmax(cmax(sizeof(float2) * T * (N / 2 + 1), sizeof(float2) * N * HP),
                                             sizeof(float) * T * N);
    static constexpr size_t base = sizeof(float2) * N * TP + aux_bytes;
    static constexpr size_t tc_off = (base + 127) & ~(size_t)127;
    static constexpr size_t smem = TC ? tc_off + sizeof(TcSmem) : base;
};

// all transforms of a tile: FP32 Stockham, or with the radix-16 stages on the tensor cores
template <int N, int T, int TP, int NT, int DIR, bool TC>
__device__ __forceinline__ void tfft(float2 *s, const float4 *tw, TcSmem *c, int *status)
{
    if constexpr (TC) tile_fft_tc<N, T, TP, NT, DIR>(s, tw, *c, status);
    else tile_fft<N, T, TP, NT, DIR>(s, tw);
}

template <int N, bool TC>
__global__ void __launch_bounds__(XCfg<N, TC>::NT) xpass_kernel(XParams p)
{
    constexpr int T = XCfg<N, TC>::T, TP = XCfg<N, TC>::TP, NT = XCfg<N, TC>::NT, H = N / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *tile = reinterpret_cast<float2 *>(smem_raw);
    float *aux = reinterpret_cast<float *>(tile + N * TP);  // aux[t * N + n]: real row t (or Phi work area)
    const int row0 = blockIdx.x * T;
    const int tid = threadIdx.x;
    const int flags = p.flags;
    TcSmem *tcs = nullptr;
    if constexpr (TC) {
        tcs = reinterpret_cast<TcSmem *>(smem_raw + XCfg<N, TC>::tc_off);
        tc_setup(*tcs, static_cast<const __half *>(p.tcw), NT);
    }

    // psi rows of a kick pass stream into the tile from the start; the Phi work below runs in aux
    const bool psi_early = (flags & X_HAS_PHI) && (flags & (X_KICK | X_FFT));

    // ---- Phi rows from the half spectrum: rows (2m, 2m+1) as one complex line, all in aux
    if (flags & X_HAS_PHI) {
        constexpr int HP = XCfg<N, TC>::HP;
        constexpr int PV = (T / 2) * N;               // packed values of the tile
        constexpr int PB = (PV + NT - 1) / NT;        // per thread
        float2 *stage = reinterpret_cast<float2 *>(aux);
        float2 *pk = reinterpret_cast<float2 *>(aux);   // packed lines [n][HP]
        for (int idx = tid; idx < T * (H + 1); idx += NT) {
            const int t = idx / (H + 1), k = idx % (H + 1);
            const int row = row0 + t;
            if (row < p.rows) cp_async8(&stage[idx], &p.phik[(size_t)row * p.P + k]);
            else stage[idx] = make_float2(0.f, 0.f);
        }
        cp_async_commit();
        if (psi_early) {
            for (int idx = tid; idx < T * N; idx += NT) {
                const int n = idx % N, t = idx / N;
                const int row = row0 + t;
                if (row < p.rows) cp_async8(&tile[n * TP + t], &p.psi[(size_t)row * N + n]);
                else tile[n * TP + t] = make_float2(0.f, 0.f);
            }
            cp_async_commit();
            cp_async_wait_group<1>();   // the half-spectrum rows; psi may still be in flight
        } else {
            cp_async_wait_group<0>();
        }
        __syncthreads();
        // build the packed lines Z = A + iB (Hermitian extension of both rows) through registers,
        // since they overwrite the staged rows
        float2 z[PB];
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            const int idx = tid + q * NT;
            if (idx >= PV) break;
            const int n = idx % N, m = idx / N;
            const int kk = (n <= H) ? n : N - n;
            float2 A = stage[(2 * m) * (H + 1) + kk], B = stage[(2 * m + 1) * (H + 1) + kk];
            if (n > H) { A.y = -A.y; B.y = -B.y; }
            if (n == 0 || n == H) { A.y = 0.f; B.y = 0.f; }
            z[q] = make_float2(A.x - B.y, A.y + B.x);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            const int idx = tid + q * NT;
            if (idx < PV) pk[(idx % N) * HP + idx / N] = z[q];
        }
        __syncthreads();
        tfft<N, T / 2, HP, NT, +1, TC>(pk, p.tw, tcs, p.status);
        // real rows into aux (again through registers: they overwrite the packed lines)
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            const int idx = tid + q * NT;
            if (idx < PV) z[q] = pk[(idx % N) * HP + idx / N];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            const int idx = tid + q * NT;
            if (idx >= PV) break;
            const int n = idx % N, m = idx / N;
            aux[(2 * m) * N + n] = z[q].x;
            aux[(2 * m + 1) * N + n] = z[q].y;
            const int ra = row0 + 2 * m;
            if ((flags & X_WRITE_PHI) && ra + 1 < p.rows) {
                float za = z[q].x, zb = z[q].y;
                if (flags & X_STATIC) {
                    za += __ldg(&p.phib[(size_t)ra * N + n]);
                    zb += __ldg(&p.phib[(size_t)(ra + 1) * N + n]);
                }
                p.phi_out[(size_t)ra * N + n] = za;
                p.phi_out[(size_t)(ra + 1) * N + n] = zb;
            }
        }
        __syncthreads();
    }

    // ---- kick and forward x transform of psi
    if (flags & (X_KICK | X_FFT)) {
        const bool fft = flags & X_FFT;
        if (!psi_early) {
            for (int idx = tid; idx < T * N; idx += NT) {
                const int n = idx % N, t = idx / N;
                const int row = row0 + t;
                if (row < p.rows) cp_async8(&tile[n * TP + t], &p.psi[(size_t)row * N + n]);
                else tile[n * TP + t] = make_float2(0.f, 0.f);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        for (int idx = tid; idx < T * N; idx += NT) {
            const int n = idx % N, t = idx / N;
            const int row = row0 + t;
            float2 v = tile[n * TP + t];
            if (flags & X_KICK) {
                // v * exp(-i ph) = v + v * (cos ph - 1 - i sin ph), with cos ph - 1 = -2 sin^2(ph/2):
                // the factor's modulus error is O(ph^2 eps) instead of the O(eps) of a rounded cos ph,
                // which would otherwise recur identically step after step while Phi changes slowly.
                const float a2 = v.x * v.x + v.y * v.y;
                float phi = (flags & X_HAS_PHI) ? aux[t * N + n] : 0.f;
                if ((flags & X_STATIC) && row < p.rows) {
                    const float pb = __ldg(&p.phib[(size_t)row * N + n]);
                    phi += pb;
                    if ((flags & X_WRITE_PHI) && !(flags & X_HAS_PHI)) p.phi_out[(size_t)row * N + n] = pb;
                }
                float sh, ch;
                half_angle_sincos(0.5f * ((phi + p.kappa * a2) * p.kick_scale), sh, ch);
                const float cm1 = -2.f * sh * sh, sn = 2.f * sh * ch;
                v = make_float2(fmaf(v.x, cm1, fmaf(v.y, sn, v.x)), fmaf(v.y, cm1, fmaf(-v.x, sn, v.y)));
            }
            if ((flags & X_ABSORB) && row < p.rows) {
                // absorbing layer of the step that just ended (Sec. 3.1, Algorithm 1): a real
                // pointwise factor, so it commutes with the kick it is fused with
                const float b = __ldg(&p.absorb_x[n]) * __ldg(&p.absorb_y[row % p.ny]) * __ldg(&p.absorb_z[row / p.ny]);
                v = make_float2(v.x * b, v.y * b);
            }
            if (fft) tile[n * TP + t] = v;
            else if (row < p.rows) p.psi[(size_t)row * N + n] = v;
        }
        if (fft) {
            __syncthreads();
            tfft<N, T, TP, NT, -1, TC>(tile, p.tw, tcs, p.status);
            for (int idx = tid; idx < T * N; idx += NT) {
                const int n = idx % N, t = idx / N;
                const int row = row0 + t;
                if (row < p.rows) p.psi[(size_t)row * N + n] = tile[n * TP + t];
            }
        }
    }

    // ---- inverse x transform, density, mass, real-to-complex x transform of rho
    if (flags & (X_R2C | X_MASS | X_IFFT)) {
        const bool ifft = flags & X_IFFT;
        // psi (transformed or not) streams into the tile asynchronously while the star
        // deposit of the same rows is read, converted and cleared into aux
        for (int idx = tid; idx < T * N; idx += NT) {
            const int n = idx % N, t = idx / N;
            const int row = row0 + t;
            if (row < p.rows) cp_async8(&tile[n * TP + t], &p.psi[(size_t)row * N + n]);
            else tile[n * TP + t] = make_float2(0.f, 0.f);
        }
        // rows the star kernel did not mark hold no deposit: neither read nor cleared
        unsigned live_rows = 0;   // bit t: row row0 + t is marked
        if (flags & X_DEP) {
            const uint4 f = __ldg(reinterpret_cast<const uint4 *>(p.dflag + row0));
            const unsigned w[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
            for (int t = 0; t < T; ++t)
                if (((w[t >> 2] >> (8 * (t & 3))) & 0xffu) && row0 + t < p.rows) live_rows |= 1u << t;
        }
        if (flags & X_DEP) {
            // loads only: a zero store to an address whose load is still in flight has to wait
            // for that load, which serialises the loop on memory latency (measured 4x slower)
            const long long *__restrict__ dep = p.dep + (size_t)row0 * N;
#pragma unroll 4
            for (int idx = tid; idx < T * N; idx += NT)
                aux[idx] = ((live_rows >> (idx / N)) & 1u) ? (float)__ldcs(&dep[idx]) * p.dep_scale : 0.f;
        }
        cp_async_wait_all();
        __syncthreads();
        if (flags & X_DEP) {
            // every deposit value of the tile has been consumed by now: clear for the next step
            long long *__restrict__ dep = p.dep + (size_t)row0 * N;
            for (int idx = tid; idx < T * N; idx += NT)
                if ((live_rows >> (idx / N)) & 1u) __stcs(&dep[idx], 0ll);
            if (tid < T && ((live_rows >> tid) & 1u)) p.dflag[row0 + tid] = 0;
        }
        if (ifft) tfft<N, T, TP, NT, +1, TC>(tile, p.tw, tcs, p.status);
        float msum = 0.f;
        if constexpr (NT == N && N <= 256) {
            // one thread per point n: it alone reads and writes column n of the tile (and its
            // deposit values in aux), so rho goes from registers straight into the packed lines
            // Z_m[n] = rho[2m][n] + i rho[2m+1][n], with no pass through aux and no barrier between
            // (at 512 points the sixteen extra registers cost more than the pass saves)
            const int n = tid;
            float r[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const float2 v = tile[n * TP + t];
                if (ifft && row0 + t < p.rows) p.psi[(size_t)(row0 + t) * N + n] = v;
                r[t] = v.x * v.x + v.y * v.y;
                msum += r[t];
                if (flags & X_DEP) r[t] += aux[t * N + n];
            }
            if (flags & X_R2C) {
#pragma unroll
                for (int m = 0; m < T / 2; ++m) tile[n * TP + m] = make_float2(r[2 * m], r[2 * m + 1]);
            }
        } else {
            for (int idx = tid; idx < T * N; idx += NT) {
                const int n = idx % N, t = idx / N;
                const int row = row0 + t;
                const float2 v = tile[n * TP + t];
                if (ifft && row < p.rows) p.psi[(size_t)row * N + n] = v;
                float r = v.x * v.x + v.y * v.y;
                msum += r;
                if (flags & X_DEP) r += aux[t * N + n];
                aux[t * N + n] = r;
            }
            __syncthreads();
            if (flags & X_R2C) {
                for (int idx = tid; idx < (T / 2) * N; idx += NT) {
                    const int n = idx % N, m = idx / N;
                    tile[n * TP + m] = make_float2(aux[(2 * m) * N + n], aux[(2 * m + 1) * N + n]);
                }
            }
        }
        if (flags & X_R2C) {
            __syncthreads();
            tfft<N, T / 2, TP, NT, -1, TC>(tile, p.tw, tcs, p.status);
            // separate the two real rows: A_k = (Z_k + conj Z_{N-k}) / 2, B_k = (Z_k - conj Z_{N-k}) / (2i)
            for (int idx = tid; idx < (T / 2) * (H + 1); idx += NT) {
                const int k = idx % (H + 1), m = idx / (H + 1);
                const int ra = row0 + 2 * m;
                const float2 Z = tile[k * TP + m];
                const float2 Zc = cconj(tile[((N - k) % N) * TP + m]);
                const float2 A = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
                const float2 D = csub(Z, Zc);
                const float2 B = make_float2(0.5f * D.y, -0.5f * D.x);
                if (ra + 1 < p.rows) {
                    p.phik[(size_t)ra * p.P + k] = A;
                    p.phik[(size_t)(ra + 1) * p.P + k] = B;
                }
            }
        }
        if (flags & X_MASS) {
            double v[1] = {(double)msum};
            grid_reduce<1, NT>(v, 0, p.partials, p.counter, p.result, p.result + 1, p.mass_scale);
        }
    }

    // ---- kinetic-energy diagnostic along x: sum_k kx^2 |F_x psi|^2 (no store)
    if (flags & X_KIN) {
        for (int idx = tid; idx < T * N; idx += NT) {
            const int n = idx % N, t = idx / N;
            const int row = row0 + t;
            if (row < p.rows) cp_async8(&tile[n * TP + t], &p.psi[(size_t)row * N + n]);
            else tile[n * TP + t] = make_float2(0.f, 0.f);
        }
        cp_async_wait_all();
        __syncthreads();
        tfft<N, T, TP, NT, -1, TC>(tile, p.tw, tcs, p.status);
        double acc = 0.0;
        for (int idx = tid; idx < T * N; idx += NT) {
            const int n = idx % N, t = idx / N;
            const float2 v = tile[n * TP + t];
            acc += (double)(__ldg(&p.k2[n]) * (v.x * v.x + v.y * v.y));
        }
        double v[1] = {acc};
        grid_reduce<1, NT>(v, 0, p.partials, p.counter, p.result);
    }
    if constexpr (TC) tc_teardown(*tcs);
}

}  // namespace spe
