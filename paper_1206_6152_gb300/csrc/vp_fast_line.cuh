// vp_fast_line.cuh -- line helpers of the register kernels, shared by
// the forward sweeps (vp_sweep_fast.cu) and by the adjoint kernels that
// recompute a forward sweep (vp_adjoint_fast.cu), so that a recomputed
// sweep input is bitwise the one the forward pass produced.
#pragma once

#include <cuda_runtime.h>

#include "vp_device.cuh"
#include "vp_internal.cuh"
#include "vp_line.cuh"

namespace vpline {

__device__ __forceinline__ LineW<float2> weights_pair(const LineCoef<float> &cf, float2 finf)
{
    LineW<float2> w;
    const int neg = cf.code & 1;
    weights1<float>(cf.c0, cf.c1, cf.c2, neg, finf.x, w.K0.x, w.A1.x, w.A2.x, w.ninvF.x);
    weights1<float>(cf.c0, cf.c1, cf.c2, neg, finf.y, w.K0.y, w.A1.y, w.A2.y, w.ninvF.y);
    return w;
}

__device__ __forceinline__ LineW<float2> weights_pair2(const LineCoef<float> &ca,
                                                        const LineCoef<float> &cb, float2 finf)
{
    LineW<float2> w;
    weights1<float>(ca.c0, ca.c1, ca.c2, ca.code & 1, finf.x, w.K0.x, w.A1.x, w.A2.x, w.ninvF.x);
    weights1<float>(cb.c0, cb.c1, cb.c2, cb.code & 1, finf.y, w.K0.y, w.A1.y, w.A2.y, w.ninvF.y);
    return w;
}

template <typename S>
__device__ __forceinline__ LineW<S> weights_one(const LineCoef<S> &cf, S finf)
{
    LineW<S> w;
    weights1<S>(cf.c0, cf.c1, cf.c2, cf.code & 1, finf, w.K0, w.A1, w.A2, w.ninvF);
    return w;
}

// zero-shift update of two packed lines (PERIODIC or outflow); a pair whose
// lines travel in opposite directions is done as two scalar lines
template <int N, bool PERIODIC>
__device__ __forceinline__ float drift_pair(float2 (&x)[N], const LineCoef<float> &ca,
                                            const LineCoef<float> &cb)
{
    if ((ca.code & 1) == (cb.code & 1)) {
        const LineW<float2> w = weights_pair2(ca, cb, line_max(x));
        const float2 out = update_line<float2, N, PERIODIC>(x, w, ca.code & 1);
        return out.x + out.y;
    }
    float y0[N], y1[N];
#pragma unroll
    for (int j = 0; j < N; ++j) { y0[j] = x[j].x; y1[j] = x[j].y; }
    const LineW<float> w0 = weights_one<float>(ca, line_max(y0));
    const LineW<float> w1 = weights_one<float>(cb, line_max(y1));
    float lost = update_line<float, N, PERIODIC>(y0, w0, ca.code & 1);
    lost += update_line<float, N, PERIODIC>(y1, w1, cb.code & 1);
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = make_float2(y0[j], y1[j]);
    return lost;
}

__device__ __forceinline__ int upos(int j, int n, int neg) { return neg ? n - 1 - j : j; }

// generic in-place line update in shared memory (any whole-cell shift,
// outflow boundaries); used only for cube-sweeps with |alpha| >= 1
template <typename T>
__device__ __noinline__ T kick_line_shifted(T *L, int st, int n, const LineCoef<T> cf)
{
    const int s = cf.code >> 1, neg = cf.code & 1;
    const T c0 = cf.c0, c1 = cf.c1, c2 = cf.c2;
    T finf = T(0);
    for (int j = 0; j < n; ++j) finf = vmax(finf, L[j * st]);
    T lost = T(0);
    for (int j = (n - s > 0 ? n - s : 0); j < n; ++j) lost += L[upos(j, n, neg) * st];
    const int jtop = n - 1 - s;
    if (jtop < 0) {
        for (int i = 0; i < n; ++i) L[i * st] = T(0);
        return lost;
    }
    auto fget = [&](int j) -> T { return (j >= 0 && j < n) ? L[upos(j, n, neg) * st] : T(0); };
    T f0 = fget(jtop), fm = fget(jtop - 1);
    T ph = pfc_flux(fm, f0, fget(jtop + 1), finf, c0, c1, c2);
    lost += ph;
    for (int i = n - 1; i >= 0; --i) {
        const int j = i - s;
        if (j < 0) {
            L[upos(i, n, neg) * st] = T(0);
            continue;
        }
        const T fmm = fget(j - 2);
        const T phm = (j >= 1) ? pfc_flux(fmm, fm, f0, finf, c0, c1, c2) : T(0);
        L[upos(i, n, neg) * st] = (f0 - ph) + phm;
        f0 = fm;
        fm = fmm;
        ph = phm;
    }
    return lost;
}

// one sweep of the owned lines held in registers
template <int N>
__device__ __forceinline__ float sweep_pairs(float2 (&x)[N], const LineCoef<float> &cf)
{
    const LineW<float2> w = weights_pair(cf, line_max(x));
    const float2 out = update_line<float2, N, false>(x, w, cf.code & 1);
    return out.x + out.y;
}


}  // namespace vpline
