// Shared-memory tile FFT core for sm_103a.
//
// A tile holds T independent lines of N complex64 points, laid out
// element-major: s[n * TP + t] is point n of line t (TP >= T is the row
// pitch).  Lanes of a warp run over t first, so every stage reads and writes
// whole 128-byte rows of the tile: with TP = T (strided passes) or TP = T + 1
// (x passes, whose global loads run lanes over n) there are no bank conflicts
// for T >= 16.
//
// Each stage is one radix-R pass of the Stockham autosort FFT (natural order
// in, natural order out): with Ns the product of the radices already done,
// butterfly j (0 <= j < N/R) of a line reads points j + r N/R (r < R),
// multiplies point r by W_{Ns R}^{(j mod Ns) r}, takes an R-point DFT and
// writes output q to (j div Ns) Ns R + (j mod Ns) + q Ns.  Twiddles come
// from an N-entry table tw[e] = exp(-2 pi i e / N) built in FP64 on the host
// (W_{Ns R}^{m} = tw[m N / (Ns R)]); DIR = +1 (inverse) uses conjugates.
// Transforms are unnormalised.
//
// Precision: each table entry holds the FP64 value split into two floats,
// hi = fl(w) and lo = fl(w - hi), and every twiddle product is formed as
// v*hi + v*lo with FMAs, so the effective twiddle is exact to ~1e-15 and the
// only FP32 error is the data-dependent rounding of the result.  With plain
// FP32 twiddles (|fl(w)| != 1) the same rounding error recurs in every
// transform and adds up coherently over the thousands of transforms of a run;
// the radix-8 and radix-3 butterfly constants (1/sqrt 2, sqrt 3 / 2) are
// applied the same way for the same reason.
#pragma once
#include <cuda_runtime.h>

namespace spe {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// v * (hi + lo): the small correction v*lo first, then the main products
// folded in with FMAs (one rounding per component at the end).
__device__ __forceinline__ float2 cmul_comp(float2 v, float2 hi, float2 lo)
{
    const float cr = fmaf(v.x, lo.x, -v.y * lo.y);
    const float ci = fmaf(v.x, lo.y, v.y * lo.x);
    return make_float2(fmaf(v.x, hi.x, fmaf(-v.y, hi.y, cr)), fmaf(v.x, hi.y, fmaf(v.y, hi.x, ci)));
}
// x * (hi + lo) for a real constant split in two floats
__device__ __forceinline__ float mul_comp(float x, float hi, float lo) { return fmaf(x, hi, x * lo); }

// 1/sqrt(2) and sqrt(3)/2 as hi + lo float pairs (split at compile time in double)
constexpr double kRsqrt2 = 0.70710678118654752440084436210485;
constexpr double kSqrt3h2 = 0.86602540378443864676372317075294;
constexpr float kRsqrt2Hi = (float)kRsqrt2;
constexpr float kRsqrt2Lo = (float)(kRsqrt2 - (double)kRsqrt2Hi);
constexpr float kSqrt3h2Hi = (float)kSqrt3h2;
constexpr float kSqrt3h2Lo = (float)(kSqrt3h2 - (double)kSqrt3h2Hi);
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (DIR < 0) or +i (DIR > 0): the R = 4 rotation in direction DIR
template <int DIR>
__device__ __forceinline__ float2 rot90(float2 a)
{
    return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// ---- small DFTs in registers: v[q] <- sum_r v[r] exp(DIR 2 pi i r q / R) ----

template <int R, int DIR> struct Dft;

template <int DIR> struct Dft<2, DIR> {
    __device__ __forceinline__ static void run(float2 *v)
    {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int DIR> struct Dft<3, DIR> {
    __device__ __forceinline__ static void run(float2 *v)
    {
        // W = exp(DIR 2 pi i / 3) = -1/2 + DIR i sqrt(3)/2
        float2 a = v[0], b = v[1], c = v[2];
        float2 sum = cadd(b, c), dif = csub(b, c);
        float2 m = make_float2(fmaf(-0.5f, sum.x, a.x), fmaf(-0.5f, sum.y, a.y));
        // DIR i s (b - c)
        const float sx = mul_comp(dif.x, kSqrt3h2Hi, kSqrt3h2Lo), sy = mul_comp(dif.y, kSqrt3h2Hi, kSqrt3h2Lo);
        float2 r = DIR < 0 ? make_float2(sy, -sx) : make_float2(-sy, sx);
        v[0] = cadd(a, sum);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};

template <int DIR> struct Dft<4, DIR> {
    __device__ __forceinline__ static void run(float2 *v)
    {
        float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        float2 s13 = cadd(v[1], v[3]), d13 = rot90<DIR>(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    }
};

template <int DIR> struct Dft<8, DIR> {
    __device__ __forceinline__ static void run(float2 *v)
    {
        // split into even / odd 4-point DFTs, combine with W8^q = exp(DIR 2 pi i q / 8)
        float2 e[4] = {v[0], v[2], v[4], v[6]};
        float2 o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, DIR>::run(e);
        Dft<4, DIR>::run(o);
        // o1 * W8^1, o2 * W8^2, o3 * W8^3 with W8 = exp(DIR i pi / 4) = (1 + DIR i) / sqrt 2
        const float hi = kRsqrt2Hi, lo = kRsqrt2Lo;
        float2 o1 = DIR < 0 ? make_float2(mul_comp(o[1].x + o[1].y, hi, lo), mul_comp(o[1].y - o[1].x, hi, lo))
                            : make_float2(mul_comp(o[1].x - o[1].y, hi, lo), mul_comp(o[1].y + o[1].x, hi, lo));
        float2 o2 = rot90<DIR>(o[2]);
        float2 o3 = DIR < 0 ? make_float2(mul_comp(o[3].y - o[3].x, hi, lo), -mul_comp(o[3].x + o[3].y, hi, lo))
                            : make_float2(-mul_comp(o[3].x + o[3].y, hi, lo), mul_comp(o[3].x - o[3].y, hi, lo));
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

// ---- radix plans per transform length ----

template <int... R> struct RList {};
template <int N> struct Plan;
template <> struct Plan<2> { using type = RList<2>; };
template <> struct Plan<4> { using type = RList<4>; };
template <> struct Plan<6> { using type = RList<3, 2>; };
template <> struct Plan<8> { using type = RList<8>; };
template <> struct Plan<12> { using type = RList<3, 4>; };
template <> struct Plan<16> { using type = RList<4, 4>; };
template <> struct Plan<24> { using type = RList<3, 8>; };
template <> struct Plan<32> { using type = RList<8, 4>; };
template <> struct Plan<48> { using type = RList<3, 4, 4>; };
template <> struct Plan<64> { using type = RList<8, 8>; };
template <> struct Plan<96> { using type = RList<3, 4, 8>; };
template <> struct Plan<128> { using type = RList<8, 4, 4>; };
template <> struct Plan<192> { using type = RList<3, 8, 8>; };
template <> struct Plan<256> { using type = RList<4, 8, 8>; };
template <> struct Plan<384> { using type = RList<3, 4, 4, 8>; };
template <> struct Plan<512> { using type = RList<8, 8, 8>; };
template <> struct Plan<768> { using type = RList<3, 4, 8, 8>; };
template <> struct Plan<1024> { using type = RList<4, 4, 8, 8>; };

// One Stockham stage over all T lines of the tile, in place through registers.
template <int N, int T, int TP, int NT, int DIR, int Ns, int R>
__device__ __forceinline__ void fft_stage(float2 *s, const float4 *__restrict__ tw)
{
    constexpr int B = N / R;
    constexpr int TOTAL = B * T;
    constexpr int PER = (TOTAL + NT - 1) / NT;
    float2 v[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int t = idx % T, j = idx / T;
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = s[(j + r * B) * TP + t];
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int t = idx % T, j = idx / T;
            const int k = j % Ns;
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float4 w = __ldg(&tw[k * r * (N / (Ns * R))]);
                    const float2 hi = make_float2(w.x, DIR > 0 ? -w.y : w.y);
                    const float2 lo = make_float2(w.z, DIR > 0 ? -w.w : w.w);
                    v[p][r] = cmul_comp(v[p][r], hi, lo);
                }
            }
            Dft<R, DIR>::run(v[p]);
            const int base = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) s[(base + r * Ns) * TP + t] = v[p][r];
        }
    }
    __syncthreads();
}

template <int N, int T, int TP, int NT, int DIR, int Ns>
__device__ __forceinline__ void fft_stages(float2 *, const float4 *, RList<>) {}

template <int N, int T, int TP, int NT, int DIR, int Ns, int R, int... Rest>
__device__ __forceinline__ void fft_stages(float2 *s, const float4 *tw, RList<R, Rest...>)
{
    fft_stage<N, T, TP, NT, DIR, Ns, R>(s, tw);
    fft_stages<N, T, TP, NT, DIR, Ns * R>(s, tw, RList<Rest...>{});
}

// Transform all T lines of the tile.  Callers __syncthreads() before (the
// tile must be complete); the last stage ends with a barrier.
template <int N, int T, int TP, int NT, int DIR>
__device__ __forceinline__ void tile_fft(float2 *s, const float4 *tw)
{
    fft_stages<N, T, TP, NT, DIR, 1>(s, tw, typename Plan<N>::type{});
}

}  // namespace spe
