// vp_line.cuh -- the PFC update of one line held in registers (Sec. 2.1 of
// Yoshikawa, Yoshida & Umemura 2013), for lines of compile-time length N.
//
// Slope corrector in saturating form.  With a = 2 f_j, F = 2 f_inf (f_inf
// the line maximum) and the one-sided differences d+ = f_{j+1} - f_j,
// d- = f_j - f_{j-1}, the corrected differences of Filbet, Sonnendruecker &
// Bertrand (2001) are
//   E+ = clamp(d+, -(F - a), a) = a - F sat((3 f_j - f_{j+1}) / F)
//   E- = clamp(d-, -a, F - a)   = -a + F sat((3 f_j - f_{j-1}) / F)
// where sat(x) = min(max(x, 0), 1) is the free saturation of an FMA.  With
// the scaled values h_j = -f_j / F and r3 = 3 / F the two arguments are
// single FMAs: s1 = sat(r3 f_j + h_{j+1}), s2 = sat(r3 f_j + h_{j-1}).
// The partial flux phi_j = c0 f_j + c1 E+ + c2 E- (u > 0) then becomes
//   phi_j = K0 f_j + A1 s1 + A2 s2,
//   K0 = c0 + 2 (c1 - c2),  A1 = -c1 F,  A2 = c2 F.
// For u < 0 the mirrored line gives phi_j = c0 f_j - c2 E+ - c1 E- with the
// same s1, s2: K0 is unchanged, A1 = c2 F, A2 = -c1 F, and the update takes
// its inflow from the right neighbour.  phi_j <= f_j is enforced (it holds
// in exact arithmetic) so that the update never goes negative; phi_j >= 0
// holds in floating point as well because every term is bounded below by
// the exact-arithmetic margin beta f_j / 3.
#pragma once

#include <cuda_runtime.h>

#include "vp_device.cuh"

namespace vpline {

// ---------------------------------------------------------------------------
// small vector abstraction: float2 (two lines packed, f32x2 instructions) or
// a scalar float/double (one line)
// ---------------------------------------------------------------------------
// sat(a b + c) with one rounding
__device__ __forceinline__ float fmasat(float a, float b, float c)
{
    float r;
    asm("fma.rn.ftz.sat.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double fmasat(double a, double b, double c)
{
    // the clamp to [0, 1] on the bits (the integer pipes, not the FP64
    // one): a non-negative double orders like its bit pattern; u <= 0 and
    // NaN give 0, as the f32 .sat form
    const double u = ::fma(a, b, c);
    const long long k = __double_as_longlong(u);
    return k <= 0 ? 0.0 : (k >= 0x3ff0000000000000LL ? (k > 0x7ff0000000000000LL ? 0.0 : 1.0) : u);
}
__device__ __forceinline__ float max3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double max3(double a, double b, double c) { return ::vmax(a, ::vmax(b, c)); }

template <typename V>
struct VOps;

template <>
struct VOps<float2> {
    typedef float S;
    static constexpr int W = 2;
    __device__ __forceinline__ static float2 splat(float a) { return make_float2(a, a); }
    __device__ __forceinline__ static float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    __device__ __forceinline__ static float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    __device__ __forceinline__ static float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    // a - b as fma(b, -1, a)
    __device__ __forceinline__ static float2 sub(float2 a, float2 b)
    {
        return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
    }
    __device__ __forceinline__ static float2 fsat(float2 a, float2 b, float2 c)
    {
        return make_float2(fmasat(a.x, b.x, c.x), fmasat(a.y, b.y, c.y));
    }
    __device__ __forceinline__ static float2 vmin(float2 a, float2 b)
    {
        return make_float2(fminf(a.x, b.x), fminf(a.y, b.y));
    }
    __device__ __forceinline__ static float2 zero() { return make_float2(0.f, 0.f); }
};

template <>
struct VOps<float> {
    typedef float S;
    static constexpr int W = 1;
    __device__ __forceinline__ static float splat(float a) { return a; }
    __device__ __forceinline__ static float fma(float a, float b, float c) { return fmaf(a, b, c); }
    __device__ __forceinline__ static float mul(float a, float b) { return a * b; }
    __device__ __forceinline__ static float add(float a, float b) { return a + b; }
    __device__ __forceinline__ static float sub(float a, float b) { return a - b; }
    __device__ __forceinline__ static float fsat(float a, float b, float c) { return fmasat(a, b, c); }
    __device__ __forceinline__ static float vmin(float a, float b) { return fminf(a, b); }
    __device__ __forceinline__ static float zero() { return 0.f; }
};

template <>
struct VOps<double> {
    typedef double S;
    static constexpr int W = 1;
    __device__ __forceinline__ static double splat(double a) { return a; }
    __device__ __forceinline__ static double fma(double a, double b, double c) { return ::fma(a, b, c); }
    __device__ __forceinline__ static double mul(double a, double b) { return a * b; }
    __device__ __forceinline__ static double add(double a, double b) { return a + b; }
    __device__ __forceinline__ static double sub(double a, double b) { return a - b; }
    __device__ __forceinline__ static double fsat(double a, double b, double c) { return fmasat(a, b, c); }
    __device__ __forceinline__ static double vmin(double a, double b) { return ::vmin(a, b); }
    __device__ __forceinline__ static double zero() { return 0.0; }
};

// per-line weights of the saturating form
template <typename V>
struct LineW {
    V K0, A1, A2, ninvF;   // ninvF = -1/F (0 when the line is empty)
};

// component-wise line maximum
template <int N>
__device__ __forceinline__ float tree_max(const float (&v)[N]);

template <int N>
__device__ __forceinline__ float line_max(const float (&x)[N])
{
    return fmaxf(tree_max<N>(x), 0.f);
}
template <int N>
__device__ __forceinline__ double line_max(const double (&x)[N])
{
    double m = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) m = ::vmax(m, x[j]);
    return m;
}
// tree of 3-input maxima (short dependency chain)
template <int N>
__device__ __forceinline__ float tree_max(const float (&v)[N])
{
    if constexpr (N == 1) {
        return v[0];
    } else if constexpr (N == 2) {
        return fmaxf(v[0], v[1]);
    } else {
        constexpr int M = (N + 2) / 3;
        float w[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int a = 3 * i;
            if (a + 2 < N) w[i] = max3(v[a], v[a + 1], v[a + 2]);
            else if (a + 1 < N) w[i] = fmaxf(v[a], v[a + 1]);
            else w[i] = v[a];
        }
        return tree_max<M>(w);
    }
}

template <int N>
__device__ __forceinline__ float2 line_max(const float2 (&x)[N])
{
    float vx[N], vy[N];
#pragma unroll
    for (int j = 0; j < N; ++j) { vx[j] = x[j].x; vy[j] = x[j].y; }
    return make_float2(fmaxf(tree_max<N>(vx), 0.f), fmaxf(tree_max<N>(vy), 0.f));
}

__device__ __forceinline__ float recip(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double recip(double a) { return __drcp_rn(a); }

// weights from (c0, c1, c2), direction and the line maximum, one component
template <typename S>
__device__ __forceinline__ void weights1(S c0, S c1, S c2, int neg, S finf, S &K0, S &A1, S &A2,
                                         S &ninvF)
{
    const S F = finf + finf;
    K0 = c0 + S(2) * (c1 - c2);
    A1 = neg ? c2 * F : -c1 * F;
    A2 = neg ? -c1 * F : c2 * F;
    ninvF = F > S(0) ? -recip(F) : S(0);
}

// phi of one cell from its own value and the scaled values h = -f / F of its
// left and right neighbours (r3 = 3 / F)
template <typename V>
__device__ __forceinline__ V flux(V f0, V hm, V hp, const LineW<V> &w, V r3)
{
    typedef VOps<V> O;
    const V s1 = O::fsat(f0, r3, hp);         // sat((3 f_j - f_{j+1}) / F)
    const V s2 = O::fsat(f0, r3, hm);         // sat((3 f_j - f_{j-1}) / F)
    V ph = O::mul(w.K0, f0);
    ph = O::fma(w.A1, s1, ph);
    ph = O::fma(w.A2, s2, ph);
    return O::vmin(ph, f0);
}

// In-place PFC update of the line x (zero shift, |alpha| < 1).  Returns the
// amount that left through the outflow end (0 for periodic lines).  Every
// value is read before it is overwritten: the update is a stencil of the old
// line, and each cell's scaled value h is formed once, as it first becomes a
// right (u > 0) or left (u < 0) neighbour.
template <typename V, int N, bool PERIODIC>
__device__ __forceinline__ V update_line(V (&x)[N], const LineW<V> &w, bool neg)
{
    typedef VOps<V> O;
    const V z = O::zero();
    const V r3 = O::mul(w.ninvF, O::splat(typename O::S(-3)));
    if (!neg) {
        V hm = z, phprev = z;
        V hc = O::mul(x[0], w.ninvF);
        const V h0 = hc;
        if (PERIODIC) {
            const V hl = O::mul(x[N - 1], w.ninvF);
            const V hl2 = N >= 2 ? O::mul(x[N >= 2 ? N - 2 : 0], w.ninvF) : hl;
            phprev = flux(x[N - 1], hl2, h0, w, r3);
            hm = hl;
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const V fc = x[i];
            const V hp = (i + 1 < N) ? O::mul(x[i + 1 < N ? i + 1 : 0], w.ninvF) : (PERIODIC ? h0 : z);
            const V ph = flux(fc, hm, hp, w, r3);
            x[i] = O::add(O::sub(fc, ph), phprev);
            phprev = ph;
            hm = hc;
            hc = hp;
        }
        return PERIODIC ? z : phprev;
    } else {
        V hp = z, phnext = z;
        V hc = O::mul(x[N - 1], w.ninvF);
        const V hl = hc;
        if (PERIODIC) {
            const V h0 = O::mul(x[0], w.ninvF);
            const V h1 = N >= 2 ? O::mul(x[N >= 2 ? 1 : 0], w.ninvF) : h0;
            phnext = flux(x[0], hl, h1, w, r3);
            hp = h0;
        }
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            const V fc = x[i];
            const V hm = (i >= 1) ? O::mul(x[i >= 1 ? i - 1 : 0], w.ninvF) : (PERIODIC ? hl : z);
            const V ph = flux(fc, hm, hp, w, r3);
            x[i] = O::add(O::sub(fc, ph), phnext);
            phnext = ph;
            hp = hc;
            hc = hm;
        }
        return PERIODIC ? z : phnext;
    }
}

// FP64 line update in the saturating form for any line maximum.  For a line
// whose maximum lies below 2^-968 (subnormal or barely normal) the reciprocal
// -1/F and the weights A1, A2 would overflow or lose their significant bits;
// such a line is swept scaled by 2^968 and scaled back.  The PFC update is
// positively homogeneous of degree one (scaling the line scales every face
// flux), and a power of two scales without rounding, so the scaled sweep is
// the same update; only the final scaling back rounds, into the subnormal
// range, as the store of the unscaled result would.
template <int N, bool PERIODIC>
__device__ __forceinline__ double update_line_f64(double (&x)[N], double c0, double c1, double c2,
                                                  int neg)
{
    constexpr double UP = 0x1p+968, DOWN = 0x1p-968;
    double finf = line_max(x);
    const bool tiny = finf > 0.0 && finf < DOWN;
    if (tiny) {
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] *= UP;
        finf *= UP;
    }
    LineW<double> w;
    weights1<double>(c0, c1, c2, neg, finf, w.K0, w.A1, w.A2, w.ninvF);
    double lost = update_line<double, N, PERIODIC>(x, w, neg);
    if (tiny) {
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] *= DOWN;
        lost *= DOWN;
    }
    return lost;
}

}  // namespace vpline
