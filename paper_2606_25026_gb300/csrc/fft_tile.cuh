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
// cos(pi/8), sin(pi/8) for the radix-16 butterfly
constexpr double kCos8 = 0.92387953251128675612818318939678829;
constexpr double kSin8 = 0.38268343236508977172845998403039887;
constexpr float kCos8Hi = (float)kCos8;
constexpr float kCos8Lo = (float)(kCos8 - (double)kCos8Hi);
constexpr float kSin8Hi = (float)kSin8;
constexpr float kSin8Lo = (float)(kSin8 - (double)kSin8Hi);
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (DIR < 0) or +i (DIR > 0): the R = 4 rotation in direction DIR
template <int DIR>
__device__ __forceinline__ float2 rot90(float2 a)
{
    return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// ---- twiddle products.  A table pointer gives the compensated product with the entry's (hi, lo)
// pair; PlainTw the plain FP32 product with hi alone, for the transforms of the potential (the
// density's real transform and Phi's inverse): Phi is recomputed every step and reaches psi only
// through the kick's phase, a small angle, so a fixed relative error of 1e-7 in Phi moves psi's
// phase by about 1e-7 of that angle per step instead of compounding like an error in psi's own
// transforms.
struct PlainTw {
    const float4 *p;
};
template <int DIR>
__device__ __forceinline__ float2 tw_mul(float2 v, const float4 *__restrict__ tw, int i)
{
    const float4 w = __ldg(&tw[i]);
    return cmul_comp(v, make_float2(w.x, DIR > 0 ? -w.y : w.y), make_float2(w.z, DIR > 0 ? -w.w : w.w));
}
template <int DIR>
__device__ __forceinline__ float2 tw_mul(float2 v, PlainTw tw, int i)
{
    const float2 w = __ldg(reinterpret_cast<const float2 *>(tw.p + i));
    return cmul(v, make_float2(w.x, DIR > 0 ? -w.y : w.y));
}

// ---- asynchronous global -> shared copies (all of a tile's loads in flight at once)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N committed groups of this thread are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

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

template <int DIR> struct Dft<16, DIR> {
    // 16 = 4 x 4: with n = 4a + b and k = c + 4d,
    // X[c + 4d] = sum_b W4^{bd} W16^{bc} sum_a x[4a + b] W4^{ac}.
    __device__ __forceinline__ static void rot(float2 &v, int e)
    {
        // v *= W16^e, W16 = exp(DIR 2 pi i / 16), e in {1, 2, 3, 4, 6, 9}
        const float2 c8h = make_float2(kCos8Hi, DIR * kSin8Hi), c8l = make_float2(kCos8Lo, DIR * kSin8Lo);
        const float2 s8h = make_float2(kSin8Hi, DIR * kCos8Hi), s8l = make_float2(kSin8Lo, DIR * kCos8Lo);
        switch (e) {
        case 1: v = cmul_comp(v, c8h, c8l); break;                                     // exp(DIR i pi/8)
        case 2: {                                                                      // exp(DIR i pi/4)
            const float a = DIR < 0 ? v.x + v.y : v.x - v.y, b = DIR < 0 ? v.y - v.x : v.y + v.x;
            v = make_float2(mul_comp(a, kRsqrt2Hi, kRsqrt2Lo), mul_comp(b, kRsqrt2Hi, kRsqrt2Lo));
            break;
        }
        case 3: v = cmul_comp(v, s8h, s8l); break;                                     // exp(DIR i 3pi/8)
        case 4: v = rot90<DIR>(v); break;                                              // exp(DIR i pi/2)
        case 6: {                                                                      // exp(DIR i 3pi/4)
            const float a = DIR < 0 ? v.y - v.x : -v.x - v.y, b = DIR < 0 ? -v.x - v.y : v.x - v.y;
            v = make_float2(mul_comp(a, kRsqrt2Hi, kRsqrt2Lo), mul_comp(b, kRsqrt2Hi, kRsqrt2Lo));
            break;
        }
        case 9: v = cmul_comp(v, make_float2(-c8h.x, -c8h.y), make_float2(-c8l.x, -c8l.y)); break;  // -W16^1
        default: break;
        }
    }
    __device__ __forceinline__ static void run(float2 *v)
    {
        float2 u[4][4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            float2 t[4] = {v[b], v[4 + b], v[8 + b], v[12 + b]};
            Dft<4, DIR>::run(t);
#pragma unroll
            for (int c = 0; c < 4; ++c) u[b][c] = t[c];
        }
#pragma unroll
        for (int b = 1; b < 4; ++b)
#pragma unroll
            for (int c = 1; c < 4; ++c) rot(u[b][c], b * c);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float2 t[4] = {u[0][c], u[1][c], u[2][c], u[3][c]};
            Dft<4, DIR>::run(t);
#pragma unroll
            for (int d = 0; d < 4; ++d) v[c + 4 * d] = t[d];
        }
    }
};

// cos(k pi / 16), k = 0..16, for the radix-32 butterfly (textbook values to 35 digits)
constexpr double kCos16[17] = {
    1.0,
    0.98078528040323044912618223613424,
    0.92387953251128675612818318939679,
    0.83146961230254523707878837761791,
    0.70710678118654752440084436210485,
    0.55557023301960222474283081394853,
    0.38268343236508977172845998403040,
    0.19509032201612826784828486847702,
    0.0,
    -0.19509032201612826784828486847702,
    -0.38268343236508977172845998403040,
    -0.55557023301960222474283081394853,
    -0.70710678118654752440084436210485,
    -0.83146961230254523707878837761791,
    -0.92387953251128675612818318939679,
    -0.98078528040323044912618223613424,
    -1.0};
// cos and sin of e pi / 16 for any integer e
__host__ __device__ constexpr double cos16(int e) { return kCos16[(e & 31) <= 16 ? (e & 31) : 32 - (e & 31)]; }
__host__ __device__ constexpr double sin16(int e) { return cos16(e - 8); }

template <int DIR> struct Dft<32, DIR> {
    // 32 = 4 x 8: with n = 8a + b and k = c + 4d,
    // X[c + 4d] = sum_b W8^{bd} W32^{bc} sum_a x[8a + b] W4^{ac}.
    template <int E>
    __device__ __forceinline__ static void rot(float2 &v)
    {
        // v *= W32^E = exp(DIR i pi E / 16), the constant split into (hi, lo) float pairs
        if constexpr (E % 32 == 0) {
        } else if constexpr (E % 32 == 8) {
            v = rot90<DIR>(v);
        } else {
            constexpr double c = cos16(E), sn = DIR * sin16(E);
            constexpr float ch = (float)c, sh = (float)sn;
            constexpr float cl = (float)(c - (double)ch), sl = (float)(sn - (double)sh);
            v = cmul_comp(v, make_float2(ch, sh), make_float2(cl, sl));
        }
    }
    template <int B, int C>
    __device__ __forceinline__ static void rot_bc(float2 (&u)[8][4])
    {
        rot<B * C>(u[B][C]);
    }
    __device__ __forceinline__ static void run(float2 *v)
    {
        float2 u[8][4];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            float2 t[4] = {v[b], v[8 + b], v[16 + b], v[24 + b]};
            Dft<4, DIR>::run(t);
#pragma unroll
            for (int c = 0; c < 4; ++c) u[b][c] = t[c];
        }
        rot_bc<1, 1>(u); rot_bc<1, 2>(u); rot_bc<1, 3>(u);
        rot_bc<2, 1>(u); rot_bc<2, 2>(u); rot_bc<2, 3>(u);
        rot_bc<3, 1>(u); rot_bc<3, 2>(u); rot_bc<3, 3>(u);
        rot_bc<4, 1>(u); rot_bc<4, 2>(u); rot_bc<4, 3>(u);
        rot_bc<5, 1>(u); rot_bc<5, 2>(u); rot_bc<5, 3>(u);
        rot_bc<6, 1>(u); rot_bc<6, 2>(u); rot_bc<6, 3>(u);
        rot_bc<7, 1>(u); rot_bc<7, 2>(u); rot_bc<7, 3>(u);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float2 t[8] = {u[0][c], u[1][c], u[2][c], u[3][c], u[4][c], u[5][c], u[6][c], u[7][c]};
            Dft<8, DIR>::run(t);
#pragma unroll
            for (int d = 0; d < 8; ++d) v[c + 4 * d] = t[d];
        }
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
template <> struct Plan<16> { using type = RList<16>; };
template <> struct Plan<24> { using type = RList<3, 8>; };
template <> struct Plan<32> { using type = RList<8, 4>; };
template <> struct Plan<48> { using type = RList<3, 4, 4>; };
template <> struct Plan<64> { using type = RList<8, 8>; };
template <> struct Plan<96> { using type = RList<3, 4, 8>; };
template <> struct Plan<128> { using type = RList<8, 4, 4>; };
template <> struct Plan<192> { using type = RList<3, 8, 8>; };
template <> struct Plan<256> { using type = RList<16, 16>; };
template <> struct Plan<384> { using type = RList<3, 4, 4, 8>; };
template <> struct Plan<512> { using type = RList<8, 8, 8>; };
template <> struct Plan<768> { using type = RList<3, 4, 8, 8>; };
template <> struct Plan<1024> { using type = RList<4, 16, 16>; };

// Alternative radix schedules the autotuner may pick for the strided passes
// (PL = 1); lengths without one use the default plan.
template <int N, int PL> struct PlanSel { using type = typename Plan<N>::type; };
template <> struct PlanSel<32, 1> { using type = RList<2, 16>; };
template <> struct PlanSel<48, 1> { using type = RList<3, 16>; };
template <> struct PlanSel<64, 1> { using type = RList<4, 16>; };
template <> struct PlanSel<96, 1> { using type = RList<3, 2, 16>; };
template <> struct PlanSel<128, 1> { using type = RList<16, 8>; };
template <> struct PlanSel<192, 1> { using type = RList<3, 4, 16>; };
template <> struct PlanSel<256, 1> { using type = RList<4, 8, 8>; };
template <> struct PlanSel<384, 1> { using type = RList<3, 8, 16>; };
template <> struct PlanSel<512, 1> { using type = RList<16, 16, 2>; };
template <> struct PlanSel<768, 1> { using type = RList<3, 16, 16>; };
template <> struct PlanSel<1024, 1> { using type = RList<8, 8, 16>; };
// A third schedule (PL = 2) where a radix-32 last stage saves a pass through shared memory.
template <> struct PlanSel<512, 2> { using type = RList<16, 32>; };
template <int N> constexpr bool has_plan2() { return N == 512; }
template <int N> constexpr bool has_alt_plan()
{
    return N == 32 || N == 48 || N == 64 || N == 96 || N == 128 || N == 192 || N == 256 || N == 384 || N == 512 ||
           N == 768 || N == 1024;
}

// One Stockham stage over all T lines of the tile, in place through registers.
template <int N, int T, int TP, int NT, int DIR, int Ns, int R, class TW>
__device__ __forceinline__ void fft_stage(float2 *s, TW tw)
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
    // the last stage of a transform (Ns R = N) writes back exactly the points each thread read
    if constexpr (Ns * R != N) __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int t = idx % T, j = idx / T;
            const int k = j % Ns;
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[p][r] = tw_mul<DIR>(v[p][r], tw, k * r * (N / (Ns * R)));
            }
            Dft<R, DIR>::run(v[p]);
            const int base = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) s[(base + r * Ns) * TP + t] = v[p][r];
        }
    }
    __syncthreads();
}

template <int N, int T, int TP, int NT, int DIR, int Ns, class TW>
__device__ __forceinline__ void fft_stages(float2 *, TW, RList<>) {}

template <int N, int T, int TP, int NT, int DIR, int Ns, class TW, int R, int... Rest>
__device__ __forceinline__ void fft_stages(float2 *s, TW tw, RList<R, Rest...>)
{
    fft_stage<N, T, TP, NT, DIR, Ns, R>(s, tw);
    fft_stages<N, T, TP, NT, DIR, Ns * R>(s, tw, RList<Rest...>{});
}

// Transform all T lines of the tile.  Callers __syncthreads() before (the
// tile must be complete); the last stage ends with a barrier.
template <int N, int T, int TP, int NT, int DIR, int PL = 0>
__device__ __forceinline__ void tile_fft(float2 *s, const float4 *tw)
{
    fft_stages<N, T, TP, NT, DIR, 1>(s, tw, typename PlanSel<N, PL>::type{});
}

// ---- plan utilities: the last radix, the plan without it, a reversed plan
template <int R, class L> struct Prepend;
template <int R, int... Rs> struct Prepend<R, RList<Rs...>> { using type = RList<R, Rs...>; };
template <class L> struct SplitLast;
template <int R> struct SplitLast<RList<R>> {
    static constexpr int last = R;
    using init = RList<>;
};
template <int R0, int R1, int... Rs> struct SplitLast<RList<R0, R1, Rs...>> {
    static constexpr int last = SplitLast<RList<R1, Rs...>>::last;
    using init = typename Prepend<R0, typename SplitLast<RList<R1, Rs...>>::init>::type;
};
template <class L, class Acc = RList<>> struct Reverse;
template <class Acc> struct Reverse<RList<>, Acc> { using type = Acc; };
template <int R, int... Rs, int... As> struct Reverse<RList<R, Rs...>, RList<As...>> {
    using type = typename Reverse<RList<Rs...>, RList<R, As...>>::type;
};

// Forward transform, a pointwise op in k space, inverse transform, with the
// last forward stage, the op and the first inverse stage done in registers.
// With the plan R_1..R_m the last forward stage (Ns = N / R_m) reads and
// writes the same index group {j + q N/R_m} of butterfly j, and so does a
// first inverse stage of radix R_m (Ns = 1, no twiddles); the inverse then
// continues with R_{m-1}..R_1.  op(v, n, t) gets the value of frequency n of
// line t and returns it multiplied.
template <int N, int T, int TP, int NT, class Op, int PL = 0, class TW = const float4 *>
__device__ __forceinline__ void tile_fft_fwd_op_inv(float2 *s, TW tw, const Op &op)
{
    using Full = typename PlanSel<N, PL>::type;
    constexpr int R = SplitLast<Full>::last;
    using Init = typename SplitLast<Full>::init;
    constexpr int B = N / R;
    fft_stages<N, T, TP, NT, -1, 1>(s, tw, Init{});
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
            if (B > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) v[p][r] = tw_mul<-1>(v[p][r], tw, j * r);
            }
            Dft<R, -1>::run(v[p]);
#pragma unroll
            for (int q = 0; q < R; ++q) v[p][q] = op(v[p][q], j + q * B, t);
            Dft<R, +1>::run(v[p]);
#pragma unroll
            for (int q = 0; q < R; ++q) s[(j * R + q) * TP + t] = v[p][q];
        }
    }
    __syncthreads();
    fft_stages<N, T, TP, NT, +1, R>(s, tw, typename Reverse<Init>::type{});
}

// ---- one transform whose first stage reads global memory and whose last stage writes it
//
// The first Stockham stage (Ns = 1, no twiddles) of butterfly j reads points j + r N/R_1; with
// lanes over t and then j, each of those loads covers whole rows of the tile's columns, so the
// thread can load them from global memory straight into registers; the last stage writes points
// j + q N/R_m (Ns = N/R_m) straight back.  Against staging the tile in shared memory first and
// copying it out last, this saves one shared-memory write and read per element on each side.
// ld(n, t) returns point n of line t; st(n, t, v) stores it.

template <class L> struct Length;
template <int... Rs> struct Length<RList<Rs...>> { static constexpr int value = sizeof...(Rs); };
template <class L> struct SplitFirst;
template <int R, int... Rs> struct SplitFirst<RList<R, Rs...>> {
    static constexpr int first = R;
    using rest = RList<Rs...>;
};

template <int N, int T, int TP, int NT, int DIR, int R, class Ld>
__device__ __forceinline__ void fft_stage_from(float2 *s, const Ld &ld)
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
            for (int r = 0; r < R; ++r) v[p][r] = ld(j + r * B, t);
        }
    }
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int t = idx % T, j = idx / T;
            Dft<R, DIR>::run(v[p]);
#pragma unroll
            for (int r = 0; r < R; ++r) s[(j * R + r) * TP + t] = v[p][r];
        }
    }
    __syncthreads();
}

template <int N, int T, int TP, int NT, int DIR, int R, class St>
__device__ __forceinline__ void fft_stage_to(const float2 *s, const float4 *__restrict__ tw, const St &st)
{
    constexpr int B = N / R;   // = Ns of the last stage
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
    // as in fft_stage, a barrier between the tile reads and the twiddle loads (without it the
    // compiler hoists the twiddle loads above the reads and runs out of registers)
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int idx = threadIdx.x + p * NT;
        if (TOTAL % NT == 0 || idx < TOTAL) {
            const int t = idx % T, j = idx / T;
            if (B > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const float4 w = __ldg(&tw[j * r]);
                    const float2 hi = make_float2(w.x, DIR > 0 ? -w.y : w.y);
                    const float2 lo = make_float2(w.z, DIR > 0 ? -w.w : w.w);
                    v[p][r] = cmul_comp(v[p][r], hi, lo);
                }
            }
            Dft<R, DIR>::run(v[p]);
#pragma unroll
            for (int q = 0; q < R; ++q) st(j + q * B, t, v[p][q]);
        }
    }
}

// one transform of all T lines from ld to st, for plans of two stages or more
template <int N, int T, int TP, int NT, int DIR, int PL, class Ld, class St>
__device__ __forceinline__ void tile_fft_direct(float2 *s, const float4 *tw, const Ld &ld, const St &st)
{
    using Full = typename PlanSel<N, PL>::type;
    constexpr int R1 = SplitFirst<Full>::first;
    using Init = typename SplitLast<Full>::init;       // R_1 .. R_{m-1}
    fft_stage_from<N, T, TP, NT, DIR, R1>(s, ld);
    fft_stages<N, T, TP, NT, DIR, R1>(s, tw, typename SplitFirst<Init>::rest{});
    fft_stage_to<N, T, TP, NT, DIR, SplitLast<Full>::last>(s, tw, st);
}

}  // namespace spe
