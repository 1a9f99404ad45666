// vp_device.cuh -- device helpers: the PFC flux of one cell, compensated
// accumulators and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "vp_internal.cuh"

// ---------------------------------------------------------------------------
// FP64 minimum and maximum on the integer pipes: GB300 issues FP64
// instructions at a small fraction of its integer rate, and a comparison of
// two doubles is exact on a key of their bits that orders every non-NaN
// double as its value (-0 below +0).  vmin/vmax: these for double, the FP32
// instructions for float.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long dkey(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double vmin(double a, double b) { return dkey(b) < dkey(a) ? b : a; }
__device__ __forceinline__ double vmax(double a, double b) { return dkey(b) > dkey(a) ? b : a; }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }

// ---------------------------------------------------------------------------
// PFC partial flux of cell j (Sec. 2.1): the integral of the third-order
// reconstruction over the fraction beta of cell j that crosses its downwind
// face, in units of the cell average.  The slope corrector of Filbet,
// Sonnendruecker & Bertrand (2001) is written as clamps of the one-sided
// differences:
//   E+ = clamp(f_{j+1} - f_j, -2 (finf - f_j), 2 f_j)
//   E- = clamp(f_j - f_{j-1}, -2 f_j, 2 (finf - f_j))
//   phi_j = c0 f_j + c1 E+ + c2 E-,
// with finf the maximum of f over the line.  In exact arithmetic 0 <= phi_j
// <= f_j; the final clamp only removes rounding excursions, so that the
// update (f_j - phi_j) + phi_{j-1} is never negative.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T pfc_flux(T fm, T f0, T fp, T finf, T c0, T c1, T c2)
{
    const T a = f0 + f0;
    const T b = (finf - f0) * T(2);
    const T ep = vmin(vmax(fp - f0, -b), a);
    const T em = vmin(vmax(f0 - fm, -a), b);
    T phi = c0 * f0 + c1 * ep + c2 * em;
    return vmin(vmax(phi, T(0)), f0);
}

// ---------------------------------------------------------------------------
// compensated accumulation.  float: a double-float pair (s, e) built with
// Knuth's TwoSum; the inputs are exact floats, so the pair carries about 48
// bits.  double: Neumaier's compensated sum.
// ---------------------------------------------------------------------------
template <typename T>
struct Acc;

template <>
struct Acc<float> {
    float s = 0.f, e = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = s + x;
        const float bb = t - s;
        const float err = (s - (t - bb)) + (x - bb);
        s = t;
        e += err;
    }
    __device__ __forceinline__ void merge(const Acc<float> &o)
    {
        const float t = s + o.s;
        const float bb = t - s;
        const float err = (s - (t - bb)) + (o.s - bb);
        s = t;
        e += o.e + err;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)e; }
    __device__ __forceinline__ void shfl_merge(int delta)
    {
        Acc<float> o;
        o.s = __shfl_xor_sync(0xffffffffu, s, delta);
        o.e = __shfl_xor_sync(0xffffffffu, e, delta);
        merge(o);
    }
};

template <>
struct Acc<double> {
    double s = 0.0, c = 0.0;
    __device__ __forceinline__ void add(double x)
    {
        const double t = s + x;
        if (fabs(s) >= fabs(x))
            c += (s - t) + x;
        else
            c += (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ void merge(const Acc<double> &o)
    {
        add(o.s);
        c += o.c;
    }
    __device__ __forceinline__ double value() const { return s + c; }
    __device__ __forceinline__ void shfl_merge(int delta)
    {
        Acc<double> o;
        o.s = __shfl_xor_sync(0xffffffffu, s, delta);
        o.c = __shfl_xor_sync(0xffffffffu, c, delta);
        merge(o);
    }
};

// Block-wide merge of Acc values; the result is valid in thread 0.
// `scratch` must hold 32 entries of Acc<T>.
template <typename T>
__device__ __forceinline__ Acc<T> block_merge(Acc<T> a, Acc<T> *scratch)
{
    for (int d = 16; d > 0; d >>= 1) a.shfl_merge(d);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) scratch[warp] = a;
    __syncthreads();
    if (warp == 0) {
        Acc<T> b;
        if (lane < nwarps) b = scratch[lane];
        for (int d = 16; d > 0; d >>= 1) b.shfl_merge(d);
        a = b;
    }
    return a;
}

// Block-wide sum of a double (result in thread 0).  scratch: 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *scratch)
{
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nwarps ? scratch[lane] : 0.0;
        for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    }
    return v;
}

__device__ __forceinline__ double block_max(double v, double *scratch)
{
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, d));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nwarps ? scratch[lane] : 0.0;
        for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, d));
    }
    return v;
}

// Shift alpha = u tau / h as LineCoef (FP64 in, the storage type out).
template <typename T>
__device__ __forceinline__ LineCoef<T> make_line_coef(double alpha)
{
    LineCoef<T> c;
    const int neg = alpha < 0.0;
    double a = fabs(alpha);
    if (!(a < 1.0e8)) a = 1.0e8;          // also catches NaN: no motion past this
    const double s = floor(a);
    const double b = a - s;
    c.code = 2 * (int)s + neg;
    c.c0 = (T)b;
    c.c1 = (T)(b * (1.0 - b) * (2.0 - b) / 6.0);
    c.c2 = (T)(b * (1.0 - b) * (1.0 + b) / 6.0);
    return c;
}
