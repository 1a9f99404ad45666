// vp_line.cuh -- the PFC update of one line held in registers (Sec. 2.1 of
// Yoshikawa, Yoshida & Umemura 2013), for lines of compile-time length N.
//
// Slope corrector in saturating-multiply form.  With a = 2 f_j,
// F = 2 f_inf (f_inf the line maximum) and the one-sided differences
// d+ = f_{j+1} - f_j, d- = f_j - f_{j-1}, the corrected differences of
// Filbet, Sonnendruecker & Bertrand (2001) are
//   E+ = clamp(d+, -(F - a), a) = a - F sat((3 f_j - f_{j+1}) / F)
//   E- = clamp(d-, -a, F - a)   = -a + F sat((3 f_j - f_{j-1}) / F)
// where sat(x) = min(max(x, 0), 1) is the free saturation of a multiply.
// The partial flux phi_j = c0 f_j + c1 E+ + c2 E- (u > 0) then becomes
//   phi_j = K0 f_j + A1 s1 + A2 s2,   s1 = sat((3 f_j - f_{j+1}) / F),
//                                     s2 = sat((3 f_j - f_{j-1}) / F),
//   K0 = c0 + 2 (c1 - c2),  A1 = -c1 F,  A2 = c2 F.
// For u < 0 the mirrored line gives phi_j = c0 f_j - c2 E+ - c1 E- with the
// same s1, s2: K0 is unchanged, A1 = c2 F, A2 = -c1 F, and the update takes
// its inflow from the right neighbour.  phi_j <= f_j is enforced (it holds
// in exact arithmetic) so that the update never goes negative; phi_j >= 0
// holds in floating point as well because every term is bounded below by
// the exact-arithmetic margin beta f_j / 3.
#pragma once

#include <cuda_runtime.h>

namespace vpline {

// ---------------------------------------------------------------------------
// small vector abstraction: float2 (two lines packed, f32x2 instructions) or
// a scalar float/double (one line)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mulsat(float a, float b)
{
    float r;
    asm("mul.rn.sat.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ double mulsat(double a, double b)
{
    return fmin(fmax(a * b, 0.0), 1.0);       // NaN -> 0, as the f32 .sat form
}
__device__ __forceinline__ float max3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double max3(double a, double b, double c) { return fmax(a, fmax(b, c)); }

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
    __device__ __forceinline__ static float2 msat(float2 a, float2 b)
    {
        return make_float2(mulsat(a.x, b.x), mulsat(a.y, b.y));
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
    __device__ __forceinline__ static float msat(float a, float b) { return mulsat(a, b); }
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
    __device__ __forceinline__ static double msat(double a, double b) { return mulsat(a, b); }
    __device__ __forceinline__ static double vmin(double a, double b) { return fmin(a, b); }
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
    for (int j = 0; j < N; ++j) m = fmax(m, x[j]);
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

// phi of one cell from its left, own and right values
template <typename V>
__device__ __forceinline__ V flux(V fm, V f0, V fp, const LineW<V> &w)
{
    typedef VOps<V> O;
    const V m3 = O::splat(typename O::S(-3));
    const V u1 = O::fma(f0, m3, fp);          // f_{j+1} - 3 f_j
    const V u2 = O::fma(f0, m3, fm);          // f_{j-1} - 3 f_j
    const V s1 = O::msat(u1, w.ninvF);        // sat((3 f_j - f_{j+1}) / F)
    const V s2 = O::msat(u2, w.ninvF);
    V ph = O::mul(w.K0, f0);
    ph = O::fma(w.A1, s1, ph);
    ph = O::fma(w.A2, s2, ph);
    return O::vmin(ph, f0);
}

// In-place PFC update of the line x (zero shift, |alpha| < 1).  Returns the
// amount that left through the outflow end (0 for periodic lines).
template <typename V, int N, bool PERIODIC>
__device__ __forceinline__ V update_line(V (&x)[N], const LineW<V> &w, bool neg)
{
    typedef VOps<V> O;
    if (!neg) {
        V fm, phprev;
        const V x0 = x[0];
        if (PERIODIC) {
            fm = x[N - 1];
            phprev = flux(N >= 2 ? x[N - 2] : x[0], x[N - 1], x[0], w);
        } else {
            fm = O::zero();
            phprev = O::zero();
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const V fc = x[i];
            const V fp = (i + 1 < N) ? x[i + 1] : (PERIODIC ? x0 : O::zero());
            const V ph = flux(fm, fc, fp, w);
            x[i] = O::add(O::sub(fc, ph), phprev);
            phprev = ph;
            fm = fc;
        }
        return PERIODIC ? O::zero() : phprev;
    } else {
        V fp, phnext;
        const V xl = x[N - 1];
        if (PERIODIC) {
            fp = x[0];
            phnext = flux(x[N - 1], x[0], N >= 2 ? x[1] : x[0], w);
        } else {
            fp = O::zero();
            phnext = O::zero();
        }
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            const V fc = x[i];
            const V fm = (i >= 1) ? x[i - 1] : (PERIODIC ? xl : O::zero());
            const V ph = flux(fm, fc, fp, w);
            x[i] = O::add(O::sub(fc, ph), phnext);
            phnext = ph;
            fp = fc;
        }
        return PERIODIC ? O::zero() : phnext;
    }
}

}  // namespace vpline
