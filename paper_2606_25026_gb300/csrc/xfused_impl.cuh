// Fused x passes of the production step (FP32 Stockham path, gravitating grid).
//
// The generic x pass (xpass_impl.cuh) selects its work with runtime flags and
// moves every intermediate through shared memory.  These two kernels serve the
// two flag sets every step uses, with the flags known at compile time and the
// boundaries between transforms fused into register-resident steps:
//
//   kick pass (Sec. 3.1 steps (a)/(d) and the first axis of step (b)):
//     the first inverse stage of the packed Phi lines reads the staged half
//     spectrum and unpacks it (Hermitian extension of two real rows as one
//     complex line) on the way; the last inverse stage of Phi is in place per
//     butterfly (its outputs are its inputs' points), so the thread that owns
//     it kicks psi at exactly those points of the two rows of the packed line:
//     psi *= exp(-i (Phi + kappa |psi|^2) dt_k / eta); then the forward
//     transform of psi.
//   density pass (last axis of step (b), step (c) and the first axis of the
//     Poisson transform): the last inverse stage of psi is in place per
//     butterfly, so its owner forms rho = |psi|^2 (+ rho_*) of the two rows of
//     a packed line at those points, reduces the mass, and takes the first
//     stage of the real forward transform of rho with the radix plan reversed
//     (its first radix is the inverse plan's last, so its butterfly reads the
//     same points).
//
// Every Stockham stage otherwise follows fft_tile.cuh (lanes over lines, tile
// element-major with pitch TP = T + 1, compensated (hi, lo) twiddles); a
// transform's last stage skips the barrier between its loads and stores, since
// each thread writes back the points it read.
#pragma once
#include "tma.cuh"
#include "xpass_impl.cuh"

namespace spe {

template <class L> struct MiddleOf {
    using type = typename SplitFirst<typename SplitLast<L>::init>::rest;
};

// The last stage of a transform (Ns = N / R): butterfly j of line t reads and writes the points
// j + r N/R, so no barrier separates its loads from its stores.  Ends with a barrier.
template <int N, int T, int TP, int NT, int DIR, int R, class TW>
__device__ __forceinline__ void xf_last_stage(float2 *s, TW tw)
{
    constexpr int B = N / R;
    constexpr int TOTAL = B * T;
    constexpr int PER = (TOTAL + NT - 1) / NT;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int t = idx % T, j = idx / T;
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s[(j + r * B) * TP + t];
            if (B > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = tw_mul<DIR>(v[r], tw, j * r);
            }
            Dft<R, DIR>::run(v);
#pragma unroll
            for (int r = 0; r < R; ++r) s[(j + r * B) * TP + t] = v[r];
        }
    }
    __syncthreads();
}

// The last stage of a transform straight to the global rows: lanes over the butterflies j of a
// line (the tile reads stay conflict free at the odd pitch TP, and each warp stores whole row
// segments), so the tile is not walked again for a separate copy-out.  No barrier at the end.
template <int N, int T, int TP, int NT, int DIR, int R, class TW>
__device__ __forceinline__ void xf_last_stage_to_rows(const float2 *s, TW tw, float2 *__restrict__ dst, int row0,
                                                      int rows)
{
    constexpr int B = N / R;
    constexpr int TOTAL = B * T;
    constexpr int PER = (TOTAL + NT - 1) / NT;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int j = idx % B, t = idx / B;
            float2 v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s[(j + r * B) * TP + t];
            if (B > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = tw_mul<DIR>(v[r], tw, j * r);
            }
            Dft<R, DIR>::run(v);
            const int row = row0 + t;
            if (row < rows) {
                float2 *d = dst + (size_t)row * N + j;
#pragma unroll
                for (int r = 0; r < R; ++r) d[r * B] = v[r];
            }
        }
    }
}

// The stages of a plan that ends the transform (Ns * R = N at its last radix): fft_stage for all
// but the last, xf_last_stage for the last.
template <int N, int T, int TP, int NT, int DIR, int Ns, class TW, int R>
__device__ __forceinline__ void xf_stages(float2 *s, TW tw, RList<R>)
{
    static_assert(Ns * R == N, "plan does not cover the length");
    xf_last_stage<N, T, TP, NT, DIR, R>(s, tw);
}
template <int N, int T, int TP, int NT, int DIR, int Ns, class TW, int R0, int R1, int... Rs>
__device__ __forceinline__ void xf_stages(float2 *s, TW tw, RList<R0, R1, Rs...>)
{
    fft_stage<N, T, TP, NT, DIR, Ns, R0>(s, tw);
    xf_stages<N, T, TP, NT, DIR, Ns * R0>(s, tw, RList<R1, Rs...>{});
}

// Packed lines (M = 8 of them, lanes over the line first): element n of line m at aux[n * 8 + m].
// A half-warp then holds 8 lines x 2 consecutive butterflies; at pitch 8 the points j + r B of two
// consecutive butterflies fall in opposite halves of the banks, so every stage but the first is
// conflict free.  The first stage (Ns = 1) writes points j R + r, of equal parity for both
// butterflies: odd butterflies write their outputs in the order r ^ 1, which puts them in the
// other half.
template <int R, int HP>
__device__ __forceinline__ void xf_store_first_stage(float2 *aux, const float2 (&v)[R], int j, int m)
{
    if constexpr (R % 2 == 0) {
        const bool odd = j & 1;
#pragma unroll
        for (int r = 0; r < R; ++r) aux[(j * R + (r ^ (int)odd)) * HP + m] = odd ? v[r ^ 1] : v[r];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) aux[(j * R + r) * HP + m] = v[r];
    }
}

// rows t of the tile from global rows row0 + t (zeros past the last row), asynchronously; one warp
// per row, lanes over the points (coalesced reads, conflict-free element-major writes)
template <int N, int T, int TP, int NT>
__device__ __forceinline__ void xf_rows_in(float2 *tile, const float2 *__restrict__ src, int row0, int rows)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = warp; t < T; t += NT / 32) {
        const int row = row0 + t;
        if (row < rows) {
            const float2 *r = src + (size_t)row * N;
            for (int n = lane; n < N; n += 32) cp_async8(&tile[n * TP + t], r + n);
        } else {
            for (int n = lane; n < N; n += 32) tile[n * TP + t] = make_float2(0.f, 0.f);
        }
    }
}

template <int N, int T, int TP, int NT>
__device__ __forceinline__ void xf_rows_out(const float2 *tile, float2 *__restrict__ dst, int row0, int rows)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = warp; t < T; t += NT / 32) {
        const int row = row0 + t;
        if (row < rows) {
            float2 *r = dst + (size_t)row * N;
            for (int n = lane; n < N; n += 32) r[n] = tile[n * TP + t];
        }
    }
}

// Resident CTAs per SM the register allocation is held to: as many as the tile's shared memory
// allows, up to 1024 threads per SM (64 registers a thread).  The 256-point density pass holds
// 32 complex values across its fused radix-16 step and keeps three CTAs (85 registers) instead of
// spilling at 64.
// Threads of the density pass's CTA: 256 at 512 points (four butterflies per thread and up to 128
// registers instead of two at 64: 762 -> 735 us per launch at 512^3, the same shared memory and
// residency), else the x passes' XCfg count.
template <int N> __host__ __device__ constexpr int xdens_nt() { return N == 512 ? 256 : XCfg<N>::NT; }

template <int N, bool DENS> struct XFMinBlocks {
    static constexpr int by_smem = (int)((227 * 1024) / (XCfg<N>::smem + 1024));
    static constexpr int by_threads = 1024 / (DENS ? xdens_nt<N>() : XCfg<N>::NT);
    static constexpr int fit = by_smem < by_threads ? by_smem : by_threads;
    static constexpr int value = (DENS && N == 256 && fit > 3) ? 3 : (fit < 1 ? 1 : fit);
};

// v exp(-i (phi + kappa |v|^2) ks) = v + v (cos th - 1 - i sin th), cos th - 1 = -2 sin^2(th / 2)
__device__ __forceinline__ float2 xf_kick(float2 v, float phi, float kap, float ks)
{
    const float a2 = v.x * v.x + v.y * v.y;
    float sh, ch;
    half_angle_sincos(0.5f * ((phi + kap * a2) * ks), sh, ch);
    const float cm1 = -2.f * sh * sh, sn = 2.f * sh * ch;
    return make_float2(fmaf(v.x, cm1, fmaf(v.y, sn, v.x)), fmaf(v.y, cm1, fmaf(-v.x, sn, v.y)));
}

template <int N> constexpr bool xfused_ok() { return N >= 32 && Length<typename Plan<N>::type>::value >= 2; }

// Row t of a tile staged row-major in the tile's space by bulk copies: t N + 2 (t / 2) complex (16-byte
// aligned; rows 2m and 2m + 1 shifted by 2m, so that a half-warp reading point j, j + 1 of the eight
// packed lines' rows hits sixteen different bank pairs when N is a multiple of 16).  The last row ends at
// 16 N + 14 <= 17 N = the element-major tile.
template <int N> __device__ __forceinline__ int xf_row_off(int t) { return t * N + 2 * (t >> 1); }

// The kick pass's half-spectrum rows staged by bulk copies: H + 2 complex a row (a multiple of 16 bytes;
// the element past H lies inside the row pitch P, a multiple of 4), row t at t SPB + 2 (t / 2) with SPB a
// multiple of 16, so that the first stage's reads of rows 2m (and 2m + 1) for eight m and two
// consecutive points hit sixteen different bank pairs.
template <int N> __host__ __device__ constexpr int xf_spec_copy() { return N / 2 + 2; }
template <int N> __host__ __device__ constexpr int xf_spec_pitch() { return (xf_spec_copy<N>() + 15) & ~15; }
template <int N> __device__ __forceinline__ int xf_spec_off(int t) { return t * xf_spec_pitch<N>() + 2 * (t >> 1); }

// The density pass's psi rows staged by bulk copies: row t at t (N + 16) + 2 (t mod 8), so that eight
// consecutive rows at two consecutive points hit sixteen different bank pairs (N a multiple of 16); the
// last row ends at 16 N + 254, inside the element-major tile for N >= 254.
template <int N> __device__ __forceinline__ int xd_row_off(int t) { return t * (N + 16) + 2 * (t & 7); }

// First stage (Ns = 1) of the density pass's inverse transform, reading the rows staged at xd_row_off and
// writing the element-major tile over them: all loads, one barrier, then the radix-R DFTs and the stores
// (the same outputs and positions as fft_stage at Ns = 1).  Lanes run over pairs of butterflies, then
// the 16 lines: a half-warp reads 8 lines x 2 points and, for R <= 8, stores conflict free at pitch 17.
template <int N, int T, int TP, int NT, int R>
__device__ __forceinline__ void xd_first_stage_from_rows(float2 *s)
{
    constexpr int B = N / R, TOTAL = B * T, PER = (TOTAL + NT - 1) / NT;
    static_assert(T == 16 && B % 2 == 0, "16 lines, an even number of butterflies");
    float2 v[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int t = (idx >> 1) & 15, j = ((idx >> 5) << 1) | (idx & 1);
            const float2 *row = s + xd_row_off<N>(t);
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = row[j + r * B];
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int t = (idx >> 1) & 15, j = ((idx >> 5) << 1) | (idx & 1);
            Dft<R, +1>::run(v[p]);
#pragma unroll
            for (int r = 0; r < R; ++r) s[(j * R + r) * TP + t] = v[p][r];
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- kick pass
// flags X_HAS_PHI | X_KICK | X_FFT, plus X_WRITE_PHI when WPHI (stars interpolate the real Phi).
// The body works on tile `tile` (rows 16 tile .. 16 tile + 15) with NT threads and XCfg<N>::smem
// bytes of shared memory at smem_raw; the kernel below runs one tile per block, a persistent kernel
// any tile from any block.
// BULK: the psi rows arrive by one bulk copy per row onto an mbarrier (thread 0 issues them; the wait is
// bounded and a timeout sets the status bit), staged row-major at xf_row_off, instead of per-thread
// 8-byte copies into the element-major tile.  Only the fused last-stage branch (last radix <= 8) reads
// the staged rows; the persistent batch kernel, which runs many tiles per block, keeps the copies.
template <int N, int NT, bool WPHI, bool BULK = false>
__device__ __forceinline__ void xkick_fused_body(const XParams &p, int tile, unsigned char *smem_raw)
{
    using C = XCfg<N>;
    constexpr int T = C::T, TP = C::TP, H = N / 2, M = T / 2, HP = M, SP = H + 1;
    using PP = typename Plan<N>::type;      // Phi, inverse: R_1 .. R_m
    using PS = typename Reverse<PP>::type;  // psi, forward: R_m .. R_1
    constexpr int R1 = SplitFirst<PP>::first, RL = SplitLast<PP>::last;
    float2 *tile_s = reinterpret_cast<float2 *>(smem_raw);
    float2 *aux = tile_s + N * TP;   // staged half-spectrum rows [t * SP + k], then packed lines [n * HP + m]
    const int row0 = tile * T, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    // the staged psi rows end at 16 N + 14 <= 17 N; the staged half-spectrum rows must fit the aux area
    // (N = 384, 512, 768), else only the psi rows go by bulk copies
    constexpr bool kBulk = BULK && RL <= 8;
    constexpr bool kBulkPhi =
        kBulk && (size_t)(15 * xf_spec_pitch<N>() + 14 + xf_spec_copy<N>()) * sizeof(float2) <= C::aux_bytes;
    __shared__ __align__(8) unsigned long long phi_bar, rows_bar;

    if constexpr (kBulk) {
        // half-spectrum rows of Phi first, then psi, all in flight at once (one thread issues them)
        const int live = min(T, p.rows - row0);
        if (tid == 0) {
            if constexpr (kBulkPhi) mbar_init(&phi_bar, 1);
            mbar_init(&rows_bar, 1);
            fence_mbar_init();
            if constexpr (kBulkPhi) {
                mbar_expect_tx(&phi_bar, (uint32_t)(live * xf_spec_copy<N>() * sizeof(float2)));
                for (int t = 0; t < live; ++t)
                    bulk_load(aux + xf_spec_off<N>(t), p.phik + (size_t)(row0 + t) * p.P,
                              xf_spec_copy<N>() * sizeof(float2), &phi_bar);
            }
            mbar_expect_tx(&rows_bar, (uint32_t)(live * N * sizeof(float2)));
            for (int t = 0; t < live; ++t)
                bulk_load(tile_s + xf_row_off<N>(t), p.psi + (size_t)(row0 + t) * N, N * sizeof(float2), &rows_bar);
        }
        for (int idx = live * N + tid; idx < T * N; idx += NT) tile_s[xf_row_off<N>(idx / N) + idx % N] = make_float2(0.f, 0.f);
        if constexpr (kBulkPhi) {
            for (int idx = live * SP + tid; idx < T * SP; idx += NT)
                aux[xf_spec_off<N>(idx / SP) + idx % SP] = make_float2(0.f, 0.f);
        } else {
            for (int t = warp; t < T; t += NT / 32) {
                const int row = row0 + t;
                if (row < p.rows) {
                    const float2 *r = p.phik + (size_t)row * p.P;
                    for (int k = lane; k < SP; k += 32) cp_async8(&aux[t * SP + k], r + k);
                } else {
                    for (int k = lane; k < SP; k += 32) aux[t * SP + k] = make_float2(0.f, 0.f);
                }
            }
            cp_async_commit();
            cp_async_wait_group<0>();
        }
    } else {
        // half-spectrum rows of Phi first, then psi, all in flight at once
        for (int t = warp; t < T; t += NT / 32) {
            const int row = row0 + t;
            if (row < p.rows) {
                const float2 *r = p.phik + (size_t)row * p.P;
                for (int k = lane; k < SP; k += 32) cp_async8(&aux[t * SP + k], r + k);
            } else {
                for (int k = lane; k < SP; k += 32) aux[t * SP + k] = make_float2(0.f, 0.f);
            }
        }
        cp_async_commit();
        xf_rows_in<N, T, TP, NT>(tile_s, p.psi, row0, p.rows);
        cp_async_commit();
        cp_async_wait_group<1>();
    }
    __syncthreads();   // also publishes thread 0's mbarrier initialisation: no thread waits on them before
    if constexpr (kBulkPhi) {
        if (!mbar_wait(&phi_bar, 0) && lane == 0) atomicOr(p.status, kTcStatusTimeout);
    }

    // first inverse stage of the packed lines Z_m = A + i B (A, B the rows 2m, 2m + 1), with the
    // Hermitian extension A_{N-n} = conj A_n read straight from the staged rows
    {
        constexpr int B = N / R1, TOTAL = B * M, PER = (TOTAL + NT - 1) / NT;
        float2 v[PER][R1];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int idx = tid + q * NT;
            if (TOTAL % NT == 0 || idx < TOTAL) {
                const int m = idx % M, j = idx / M;
                const float2 *ra = kBulkPhi ? aux + xf_spec_off<N>(2 * m) : aux + (2 * m) * SP;
                const float2 *rb = kBulkPhi ? aux + xf_spec_off<N>(2 * m + 1) : ra + SP;
#pragma unroll
                for (int r = 0; r < R1; ++r) {
                    const int n = j + r * B;
                    float2 A, Bv;
                    if (n <= H) {
                        A = ra[n];
                        Bv = rb[n];
                        if (n == 0 || n == H) {
                            A.y = 0.f;
                            Bv.y = 0.f;
                        }
                    } else {
                        A = cconj(ra[N - n]);
                        Bv = cconj(rb[N - n]);
                    }
                    v[q][r] = make_float2(A.x - Bv.y, A.y + Bv.x);
                }
            }
        }
        __syncthreads();   // the packed lines overwrite the staged rows
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int idx = tid + q * NT;
            if (TOTAL % NT == 0 || idx < TOTAL) {
                const int m = idx % M, j = idx / M;
                Dft<R1, +1>::run(v[q]);
                xf_store_first_stage<R1, HP>(aux, v[q], j, m);
            }
        }
        if constexpr (!kBulk) cp_async_wait_group<0>();
        __syncthreads();
    }
    // the inverse stages between the first and the last
    fft_stages<N, M, HP, NT, +1, R1>(aux, PlainTw{p.tw}, typename MiddleOf<PP>::type{});

    if constexpr (RL <= 8) {
        // last inverse stage of Phi, the kick of both psi rows at its points and psi's first forward
        // stage in registers: the reversed plan starts with radix RL, so that stage's butterfly j reads
        // the points j + r N/RL the Phi butterfly j produced.  Loads, one barrier, then the first
        // stage's outputs (which land on points other threads read).
        constexpr int B = N / RL, TOTAL = B * M, PER = (TOTAL + NT - 1) / NT;
        const float ks = p.kick_scale, kap = p.kappa;
        float2 f[PER][RL], va[PER][RL], vb[PER][RL];
        if constexpr (kBulk) {
            if (!mbar_wait(&rows_bar, 0) && lane == 0) atomicOr(p.status, kTcStatusTimeout);
        }
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int idx = tid + q * NT;
            if (TOTAL % NT == 0 || idx < TOTAL) {
                const int m = idx % M, j = idx / M;
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    const int n = j + r * B;
                    f[q][r] = aux[n * HP + m];
                    if constexpr (kBulk) {
                        va[q][r] = tile_s[xf_row_off<N>(2 * m) + n];
                        vb[q][r] = tile_s[xf_row_off<N>(2 * m + 1) + n];
                    } else {
                        va[q][r] = tile_s[n * TP + 2 * m];
                        vb[q][r] = tile_s[n * TP + 2 * m + 1];
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int idx = tid + q * NT;
            if (TOTAL % NT == 0 || idx < TOTAL) {
                const int m = idx % M, j = idx / M;
                if (B > 1) {
#pragma unroll
                    for (int r = 1; r < RL; ++r) f[q][r] = tw_mul<+1>(f[q][r], PlainTw{p.tw}, j * r);
                }
                Dft<RL, +1>::run(f[q]);
                // f[r] = Phi(row 2m, point j + r B) + i Phi(row 2m + 1, point j + r B)
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    va[q][r] = xf_kick(va[q][r], f[q][r].x, kap, ks);
                    vb[q][r] = xf_kick(vb[q][r], f[q][r].y, kap, ks);
                    if (WPHI) {
                        const int n = j + r * B, ra = row0 + 2 * m;
                        if (ra < p.rows) p.phi_out[(size_t)ra * N + n] = f[q][r].x;
                        if (ra + 1 < p.rows) p.phi_out[(size_t)(ra + 1) * N + n] = f[q][r].y;
                    }
                }
                Dft<RL, -1>::run(va[q]);
                Dft<RL, -1>::run(vb[q]);
                // outputs at points j RL + r; odd butterflies store their second row first, which puts
                // a half-warp's two butterflies in opposite halves of the banks
                const bool odd = j & 1;
#pragma unroll
                for (int r = 0; r < RL; ++r) {
                    float2 *d = tile_s + (j * RL + r) * TP + 2 * m;
                    d[odd ? 1 : 0] = odd ? vb[q][r] : va[q][r];
                    d[odd ? 0 : 1] = odd ? va[q][r] : vb[q][r];
                }
            }
        }
        __syncthreads();
        // the remaining forward stages of psi (from Ns = RL)
        using Rest = typename SplitFirst<PS>::rest;
        if constexpr (SplitLast<PS>::last <= 8) {
            fft_stages<N, T, TP, NT, -1, RL>(tile_s, p.tw, typename SplitLast<Rest>::init{});
            xf_last_stage_to_rows<N, T, TP, NT, -1, SplitLast<PS>::last>(tile_s, p.tw, p.psi, row0, p.rows);
        } else {
            xf_stages<N, T, TP, NT, -1, RL>(tile_s, p.tw, Rest{});
            xf_rows_out<N, T, TP, NT>(tile_s, p.psi, row0, p.rows);
        }
    } else {
        // last inverse stage of Phi (in place per butterfly) and the kick of psi at its points
        {
            constexpr int B = N / RL, TOTAL = B * M, PER = (TOTAL + NT - 1) / NT;
            const float ks = p.kick_scale, kap = p.kappa;
    #pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int idx = tid + q * NT;
                if (TOTAL % NT == 0 || idx < TOTAL) {
                    const int m = idx % M, j = idx / M;
                    float2 f[RL];
    #pragma unroll
                    for (int r = 0; r < RL; ++r) f[r] = aux[(j + r * B) * HP + m];
                    if (B > 1) {
    #pragma unroll
                        for (int r = 1; r < RL; ++r) f[r] = tw_mul<+1>(f[r], PlainTw{p.tw}, j * r);
                    }
                    Dft<RL, +1>::run(f);
                    // f[r] = Phi(row 2m, point j + r B) + i Phi(row 2m + 1, point j + r B)
    #pragma unroll
                    for (int r = 0; r < RL; ++r) {
                        const int n = j + r * B;
    #pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int t = 2 * m + h;
                            const float phi = h ? f[r].y : f[r].x;
                            float2 v = tile_s[n * TP + t];
                            // v exp(-i ph) = v + v (cos ph - 1 - i sin ph), cos ph - 1 = -2 sin^2(ph / 2)
                            const float a2 = v.x * v.x + v.y * v.y;
                            float sh, ch;
                            half_angle_sincos(0.5f * ((phi + kap * a2) * ks), sh, ch);
                            const float cm1 = -2.f * sh * sh, sn = 2.f * sh * ch;
                            v = make_float2(fmaf(v.x, cm1, fmaf(v.y, sn, v.x)), fmaf(v.y, cm1, fmaf(-v.x, sn, v.y)));
                            tile_s[n * TP + t] = v;
                            if (WPHI && row0 + t < p.rows) p.phi_out[(size_t)(row0 + t) * N + n] = phi;
                        }
                    }
                }
            }
            __syncthreads();
        }

        // forward transform of psi with the reversed plan; a last stage of radix 8 or less stores the rows
        // itself (with lanes over the butterflies each lane loads its own twiddles, which costs more than
        // the copy-out it saves once the stage has 15 of them)
        if constexpr (SplitLast<PS>::last <= 8) {
            fft_stages<N, T, TP, NT, -1, 1>(tile_s, p.tw, typename SplitLast<PS>::init{});
            xf_last_stage_to_rows<N, T, TP, NT, -1, SplitLast<PS>::last>(tile_s, p.tw, p.psi, row0, p.rows);
        } else {
            xf_stages<N, T, TP, NT, -1, 1>(tile_s, p.tw, PS{});
            xf_rows_out<N, T, TP, NT>(tile_s, p.psi, row0, p.rows);
        }

    }
}

template <int N, bool WPHI>
__global__ void __launch_bounds__(XCfg<N>::NT, XFMinBlocks<N, false>::value) xkick_fused_kernel(XParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    xkick_fused_body<N, XCfg<N>::NT, WPHI, true>(p, blockIdx.x, smem_raw);
}

// ---------------------------------------------------------------- density pass
// flags X_IFFT | X_MASS | X_R2C, plus X_DEP when DEP (the stars' fixed-point deposit).
// The body works on tile `tile` of the ntiles tiles of the pass (the mass reduction counts them).
// BULK: the psi rows arrive by one bulk copy per row onto an mbarrier, staged at xd_row_off (bounded
// wait, timeout status bit), and the first inverse stage reads them from there; the persistent batch
// kernel keeps the per-thread copies.
template <int N, int NT, bool DEP, bool BULK = false>
__device__ __forceinline__ void xdens_fused_body(const XParams &p, int tile, int ntiles, unsigned char *smem_raw)
{
    using C = XCfg<N>;
    constexpr int T = C::T, TP = C::TP, H = N / 2, M = T / 2, HP = M, DP = N + 2;
    using PI = typename Plan<N>::type;      // psi, inverse: R_1 .. R_m
    using PR = typename Reverse<PI>::type;  // packed rho, forward: R_m .. R_1
    constexpr int RL = SplitLast<PI>::last;
    static_assert((size_t)T * DP * sizeof(float) <= C::aux_bytes && (size_t)N * HP * sizeof(float2) <= C::aux_bytes,
                  "aux area too small");
    float2 *tile_s = reinterpret_cast<float2 *>(smem_raw);
    float2 *aux = tile_s + N * TP;                // packed rho lines [n * HP + m]
    float *auxf = reinterpret_cast<float *>(aux);  // before them: deposit rows [t * DP + n]
    const int row0 = tile * T, tid = threadIdx.x;
    using PInit = typename SplitLast<PI>::init;   // the inverse stages but the last
    constexpr int R1 = SplitFirst<PI>::first;
    constexpr bool kBulk = BULK && N % 16 == 0 && 16 * N + 254 <= N * TP && (N / R1) % 2 == 0;
    __shared__ __align__(8) unsigned long long rows_bar;

    if constexpr (kBulk) {
        const int live = min(T, p.rows - row0);
        if (tid == 0) {
            mbar_init(&rows_bar, 1);
            fence_mbar_init();
            mbar_expect_tx(&rows_bar, (uint32_t)(live * N * sizeof(float2)));
            for (int t = 0; t < live; ++t)
                bulk_load(tile_s + xd_row_off<N>(t), p.psi + (size_t)(row0 + t) * N, N * sizeof(float2), &rows_bar);
        }
        for (int idx = live * N + tid; idx < T * N; idx += NT) tile_s[xd_row_off<N>(idx / N) + idx % N] = make_float2(0.f, 0.f);
    } else {
        xf_rows_in<N, T, TP, NT>(tile_s, p.psi, row0, p.rows);
    }
    cp_async_commit();
    unsigned live_rows = 0;   // bit t: row row0 + t holds deposit (marked by the star kernel)
    if (DEP) {
        const uint4 f = __ldg(reinterpret_cast<const uint4 *>(p.dflag + row0));
        const unsigned w[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
        for (int t = 0; t < T; ++t)
            if (((w[t >> 2] >> (8 * (t & 3))) & 0xffu) && row0 + t < p.rows) live_rows |= 1u << t;
        // loads only here: a zero store to an address whose load is still in flight would wait for it
        const long long *__restrict__ dep = p.dep + (size_t)row0 * N;
#pragma unroll 4
        // rows at pitch N + 2: the fused step below reads 8 rows x 4 points per warp, conflict free
        for (int idx = tid; idx < T * N; idx += NT) {
            const int t = idx / N;
            auxf[t * DP + (idx - t * N)] = ((live_rows >> t) & 1u) ? (float)__ldcs(&dep[idx]) * p.dep_scale : 0.f;
        }
    }
    cp_async_wait_group<0>();
    __syncthreads();   // also publishes thread 0's mbarrier initialisation: no thread waits on it before
    if constexpr (kBulk) {
        if (!mbar_wait(&rows_bar, 0) && (tid & 31) == 0) atomicOr(p.status, kTcStatusTimeout);
    }
    if (DEP) {
        long long *__restrict__ dep = p.dep + (size_t)row0 * N;
        for (int idx = tid; idx < T * N; idx += NT)
            if ((live_rows >> (idx / N)) & 1u) __stcs(&dep[idx], 0ll);
        if (tid < T && ((live_rows >> tid) & 1u)) p.dflag[row0 + tid] = 0;
    }

    // inverse stages of psi but the last
    if constexpr (kBulk) {
        xd_first_stage_from_rows<N, T, TP, NT, R1>(tile_s);
        fft_stages<N, T, TP, NT, +1, R1>(tile_s, p.tw, typename SplitFirst<PInit>::rest{});
    } else {
        fft_stages<N, T, TP, NT, +1, 1>(tile_s, p.tw, PInit{});
    }

    // last inverse stage of psi (in place per butterfly) for the rows 2m, 2m + 1, rho at its points,
    // and the first forward stage of the packed line Z_m = rho_2m + i rho_2m+1
    float msum = 0.f;
    {
        constexpr int B = N / RL, TOTAL = B * M, PER = (TOTAL + NT - 1) / NT;
        float2 z[PER][RL];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int idx = tid + q * NT;
            if (TOTAL % NT == 0 || idx < TOTAL) {
                const int m = idx % M, j = idx / M;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int t = 2 * m + h;
                    float2 v[RL];
#pragma unroll
                    for (int r = 0; r < RL; ++r) v[r] = tile_s[(j + r * B) * TP + t];
                    if (B > 1) {
#pragma unroll
                        for (int r = 1; r < RL; ++r) {
                            const float4 w = __ldg(&p.tw[j * r]);
                            v[r] = cmul_comp(v[r], make_float2(w.x, -w.y), make_float2(w.z, -w.w));
                        }
                    }
                    Dft<RL, +1>::run(v);
#pragma unroll
                    for (int r = 0; r < RL; ++r) {
                        tile_s[(j + r * B) * TP + t] = v[r];
                        float rho = v[r].x * v[r].x + v[r].y * v[r].y;
                        msum += rho;
                        if (DEP) rho += auxf[t * DP + j + r * B];
                        if (h) z[q][r].y = rho;
                        else z[q][r].x = rho;
                    }
                }
            }
        }
        __syncthreads();   // the deposit rows in aux are all read; the packed lines overwrite them
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int idx = tid + q * NT;
            if (TOTAL % NT == 0 || idx < TOTAL) {
                const int m = idx % M, j = idx / M;
                Dft<RL, -1>::run(z[q]);
                xf_store_first_stage<RL, HP>(aux, z[q], j, m);
            }
        }
        __syncthreads();
    }
    xf_rows_out<N, T, TP, NT>(tile_s, p.psi, row0, p.rows);
    // the remaining forward stages of the packed lines
    xf_stages<N, M, HP, NT, -1, RL>(aux, PlainTw{p.tw}, typename SplitFirst<PR>::rest{});
    // separate the two real rows: A_k = (Z_k + conj Z_{N-k}) / 2, B_k = (Z_k - conj Z_{N-k}) / (2i)
    for (int idx = tid; idx < M * (H + 1); idx += NT) {
        const int m = idx % M, k = idx / M;
        const int ra = row0 + 2 * m;
        const float2 Z = aux[k * HP + m];
        const float2 Zc = cconj(aux[((N - k) % N) * HP + m]);
        const float2 A = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y + Zc.y));
        const float2 D = csub(Z, Zc);
        const float2 Bk = make_float2(0.5f * D.y, -0.5f * D.x);
        if (ra < p.rows) p.phik[(size_t)ra * p.P + k] = A;
        if (ra + 1 < p.rows) p.phik[(size_t)(ra + 1) * p.P + k] = Bk;
    }
    double v[1] = {(double)msum};
    tile_reduce<1, NT>(v, 0, p.partials, p.counter, p.result, p.result + 1, p.mass_scale, (unsigned)tile,
                       (unsigned)ntiles);
}

template <int N, bool DEP>
__global__ void __launch_bounds__(xdens_nt<N>(), XFMinBlocks<N, true>::value) xdens_fused_kernel(XParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    xdens_fused_body<N, xdens_nt<N>(), DEP, true>(p, blockIdx.x, gridDim.x, smem_raw);
}

}  // namespace spe
