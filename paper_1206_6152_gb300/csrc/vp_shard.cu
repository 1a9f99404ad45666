// vp_shard.cu -- the pieces of the split step that change when position
// space is cut into slabs along x, one slab per GPU (the decomposition of
// Sec. 2.3): the x drift of a slab whose lines continue into ghost planes
// of the neighbouring slabs, the per-line maxima along x of a slab (reduced
// over the slabs by the caller, since f_inf is the maximum of the whole
// line), and a context that only solves for the field of a density it is
// given (the FFT stays whole on every GPU: the density is gathered).  The
// slab-local parts of the step run in the same fused passes as the
// single-context step: the half kicks (one, or K2^n and K1^{n+1} together)
// and the z then y drift.
#include <cuda_runtime.h>
#include <math.h>

#include "vp_device.cuh"
#include "vp_fast_line.cuh"
#include "vp_internal.cuh"
#include "vp_line.cuh"

using namespace vpline;

int vp_sm_count();

namespace {

// per (y, z, velocity) line of the slab: the maximum over its x planes (at
// least 0, as the line maximum of the sweeps)
template <typename T>
__global__ void k_line_max_x(const T *__restrict__ f, T *__restrict__ out, long long nl, int nx)
{
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < nl;
         l += (long long)gridDim.x * blockDim.x) {
        T m = T(0);
        for (int i = 0; i < nx; ++i) m = vmax(m, f[(long long)i * nl + l]);
        out[l] = m;
    }
}

// The x drift of the slab, in place, one thread per line (y, z, velocity):
// the line is read in its upwind order p in [-G, nx + G) with the ghost
// planes glo (p < 0) and ghi (p >= nx) beyond the slab, and updated from
// its last cell down, so that every read lies at least two cells behind the
// last write (Sec. 2.1: f_i <- f_{i-s} - phi_{i-s} + phi_{i-s-1} with the
// corrected partial fluxes of the clamp form and the line maximum finf of
// the whole line).
template <typename T>
__global__ void k_drift_x_ghosted(T *__restrict__ f, const T *__restrict__ glo,
                                  const T *__restrict__ ghi, const LineCoef<T> *__restrict__ coef,
                                  const T *__restrict__ lmax, long long nl, int nx, int G,
                                  long long nvc, int nvyz)
{
    for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < nl;
         l += (long long)gridDim.x * blockDim.x) {
        const LineCoef<T> cf = coef[(int)((l % nvc) / nvyz)];
        const int s = cf.code >> 1, neg = cf.code & 1;
        const T finf = lmax[l];
        auto get = [&](int p) -> T {
            const int r = neg ? nx - 1 - p : p;
            if (r < 0) return glo[(long long)(G + r) * nl + l];
            if (r >= nx) return ghi[(long long)(r - nx) * nl + l];
            return f[(long long)r * nl + l];
        };
        int j = nx - 1 - s;
        T f0 = get(j), fm = get(j - 1);
        T ph = pfc_flux(fm, f0, get(j + 1), finf, cf.c0, cf.c1, cf.c2);
        for (int i = nx - 1; i >= 0; --i) {
            j = i - s;
            const T fmm = get(j - 2);
            const T phm = pfc_flux(fmm, fm, f0, finf, cf.c0, cf.c1, cf.c2);
            const int r = neg ? nx - 1 - i : i;
            f[(long long)r * nl + l] = (f0 - ph) + phm;
            f0 = fm;
            fm = fmm;
            ph = phm;
        }
    }
}

// The zero-shift update of the slab's part x[0, NX) of a line pair (array
// order, packed) in the saturating form of the single-context kernels, the
// line continued by ghost values: for u > 0 gm2 = f_{-2}, gm1 = f_{-1}
// upwind and gp = f_{NX} downwind; for u < 0 gm2 = f_{NX+1}, gm1 = f_{NX}
// upwind and gp = f_{-1}.  Cell for cell the arithmetic of the periodic
// whole-line update of the register-line x drift (a slab's line with its
// neighbours' planes is a stretch of the whole line), so where the whole box
// runs that kernel the slabs' x drift equals it bit for bit.
template <int NX>
__device__ __forceinline__ void update_ghosted(float2 (&x)[NX], float2 gm2, float2 gm1, float2 gp,
                                               const LineW<float2> &w, bool neg)
{
    typedef VOps<float2> O;
    const float2 r3 = O::mul(w.ninvF, O::splat(-3.f));
    if (!neg) {
        float2 phprev = flux(gm1, O::mul(gm2, w.ninvF), O::mul(x[0], w.ninvF), w, r3);   // phi_{-1}
        float2 hm = O::mul(gm1, w.ninvF), hc = O::mul(x[0], w.ninvF);
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            const float2 fc = x[i];
            const float2 hp = O::mul(i + 1 < NX ? x[i + 1 < NX ? i + 1 : 0] : gp, w.ninvF);
            const float2 ph = flux(fc, hm, hp, w, r3);
            x[i] = O::add(O::sub(fc, ph), phprev);
            phprev = ph;
            hm = hc;
            hc = hp;
        }
    } else {
        float2 phnext = flux(gm1, O::mul(x[NX - 1], w.ninvF), O::mul(gm2, w.ninvF), w, r3);   // phi_{NX}
        float2 hp = O::mul(gm1, w.ninvF), hc = O::mul(x[NX - 1], w.ninvF);
#pragma unroll
        for (int i = NX - 1; i >= 0; --i) {
            const float2 fc = x[i];
            const float2 hm = O::mul(i >= 1 ? x[i >= 1 ? i - 1 : 0] : gp, w.ninvF);
            const float2 ph = flux(fc, hm, hp, w, r3);
            x[i] = O::add(O::sub(fc, ph), phnext);
            phnext = ph;
            hp = hc;
            hc = hm;
        }
    }
}

// The x drift of the slab for zero-shift steps (FP32): two lines per thread
// (adjacent velocity cells, the same v_x), the slab's NX planes and the
// three ghost values in registers, loaded before any arithmetic (a warp
// reads 256 contiguous bytes per load).
template <int NX>
__global__ void __launch_bounds__(128) k_drift_x_ghosted_pairs(
    float *__restrict__ f, const float *__restrict__ glo, const float *__restrict__ ghi,
    const LineCoef<float> *__restrict__ coef, const float *__restrict__ lmax, long long nl, int G,
    long long nvc, int nvyz)
{
    const long long npair = nl / 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < npair;
         q += (long long)gridDim.x * blockDim.x) {
        const long long l = 2 * q;
        const LineCoef<float> cf = coef[(int)((l % nvc) / nvyz)];
        const bool neg = cf.code & 1;
        float2 x[NX];
#pragma unroll
        for (int k = 0; k < NX; ++k) x[k] = *reinterpret_cast<const float2 *>(f + k * nl + l);
        const float2 *gl = reinterpret_cast<const float2 *>(glo + l);
        const float2 *gh = reinterpret_cast<const float2 *>(ghi + l);
        const long long st = nl / 2;          // one plane in float2 units
        float2 gm2, gm1, gp;
        if (!neg) {
            gm2 = gl[(G - 2) * st];
            gm1 = gl[(G - 1) * st];
            gp = gh[0];
        } else {
            gm2 = gh[st];
            gm1 = gh[0];
            gp = gl[(G - 1) * st];
        }
        const float2 finf = *reinterpret_cast<const float2 *>(lmax + l);
        update_ghosted<NX>(x, gm2, gm1, gp, weights_pair2(cf, cf, finf), neg);
#pragma unroll
        for (int k = 0; k < NX; ++k) *reinterpret_cast<float2 *>(f + k * nl + l) = x[k];
    }
}

unsigned grid_for(long long n, int threads)
{
    long long g = (n + threads - 1) / threads;
    const long long cap = 16LL * vp_sm_count();
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

__global__ void k_set_tau(double *p, double v) { *p = v; }

}  // namespace

extern "C" {

int vp_line_max_x(vp_ctx *c, void *lmax_dev)
{
    if (!c || !lmax_dev) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    const long long nl = c->ncells / c->n[0];
    if (c->isdouble)
        k_line_max_x<double><<<grid_for(nl, 256), 256, 0, c->stream>>>((const double *)c->f,
                                                                      (double *)lmax_dev, nl, c->n[0]);
    else
        k_line_max_x<float><<<grid_for(nl, 256), 256, 0, c->stream>>>((const float *)c->f,
                                                                     (float *)lmax_dev, nl, c->n[0]);
    VP_CUDA_TRY(cudaGetLastError());
    return VP_OK;
}

int vp_drift_x_ghosted(vp_ctx *c, double tau, const void *ghost_lo, const void *ghost_hi,
                       int nghost, const void *lmax_dev)
{
    if (!c || !ghost_lo || !ghost_hi || !lmax_dev || !isfinite(tau) || nghost < 2) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    // every line's whole-cell shift plus the stencil must lie inside the ghosts
    const double amax = vp_drift_alpha_bound(c, fabs(tau));
    if (!(amax < 1.0e6) || (double)nghost < floor(amax) + 2.0) return VP_ERR_ARG;
    double *tau_ptr = &c->sc->pad[0];
    k_set_tau<<<1, 1, 0, c->stream>>>(tau_ptr, tau);
    VP_CUDA_TRY(cudaGetLastError());
    VP_CUDA_TRY(launch_coef_drift(c, tau_ptr, 1.0, c->coef_drift));
    const long long nl = c->ncells / c->n[0];
    const int nvyz = c->nv[1] * c->nv[2];
    if (!c->isdouble && amax < 1.0 && nvyz % 2 == 0) {
        // zero-shift steps: the register-line kernel for the common slab
        // thicknesses
        const unsigned grid = grid_for(nl / 2, 128);
        float *fp = (float *)c->f;
        const float *lo = (const float *)ghost_lo, *hi = (const float *)ghost_hi;
        const LineCoef<float> *cf = (const LineCoef<float> *)c->coef_drift;
        const float *lm = (const float *)lmax_dev;
        bool done = true;
        switch (c->n[0]) {
#define VP_GHOSTED(NX)                                                                       \
    case NX:                                                                                 \
        k_drift_x_ghosted_pairs<NX><<<grid, 128, 0, c->stream>>>(fp, lo, hi, cf, lm, nl, nghost, \
                                                                 c->nvc, nvyz);              \
        break;
            VP_GHOSTED(2) VP_GHOSTED(4) VP_GHOSTED(6) VP_GHOSTED(8) VP_GHOSTED(12)
            VP_GHOSTED(16) VP_GHOSTED(24) VP_GHOSTED(32)
#undef VP_GHOSTED
        default:
            done = false;
        }
        if (done) {
            VP_CUDA_TRY(cudaGetLastError());
            return VP_OK;
        }
    }
    if (c->isdouble)
        k_drift_x_ghosted<double><<<grid_for(nl, 128), 128, 0, c->stream>>>(
            (double *)c->f, (const double *)ghost_lo, (const double *)ghost_hi,
            (const LineCoef<double> *)c->coef_drift, (const double *)lmax_dev, nl, c->n[0], nghost,
            c->nvc, nvyz);
    else
        k_drift_x_ghosted<float><<<grid_for(nl, 128), 128, 0, c->stream>>>(
            (float *)c->f, (const float *)ghost_lo, (const float *)ghost_hi,
            (const LineCoef<float> *)c->coef_drift, (const float *)lmax_dev, nl, c->n[0], nghost,
            c->nvc, nvyz);
    VP_CUDA_TRY(cudaGetLastError());
    return VP_OK;
}

int vp_kick(vp_ctx *c, double tau1, double tau2)
{
    if (!c || !isfinite(tau1) || !isfinite(tau2)) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    double *t1 = &c->sc->pad[4], *t2 = &c->sc->pad[5];
    k_set_tau<<<1, 1, 0, c->stream>>>(t1, tau1);
    VP_CUDA_TRY(cudaGetLastError());
    VP_CUDA_TRY(launch_coef_kick(c, c->g, t1, 1.0, c->coef_kick2));
    if (tau2 == 0.0) {
        VP_CUDA_TRY(launch_kick(c, c->f, c->coef_kick2, nullptr, 3, 0));
        return VP_OK;
    }
    k_set_tau<<<1, 1, 0, c->stream>>>(t2, tau2);
    VP_CUDA_TRY(cudaGetLastError());
    VP_CUDA_TRY(launch_coef_kick(c, c->g, t2, 1.0, c->coef_kick1));
    VP_CUDA_TRY(launch_kick(c, c->f, c->coef_kick2, c->coef_kick1, 6, 0));
    return VP_OK;
}

int vp_drift_yz(vp_ctx *c, double tau)
{
    if (!c || !isfinite(tau)) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    double *tp = &c->sc->pad[4];
    k_set_tau<<<1, 1, 0, c->stream>>>(tp, tau);
    VP_CUDA_TRY(cudaGetLastError());
    VP_CUDA_TRY(launch_coef_drift(c, tp, 1.0, c->coef_drift));
    const double amax = vp_drift_alpha_bound(c, fabs(tau));
    if (amax < 1.0 && vp_drift_yz_ok(c)) {
        VP_CUDA_TRY(launch_drift_yz(c, c->f, c->coef_drift, c->f));
    } else {
        VP_CUDA_TRY(launch_drift(c, c->f, 2, c->coef_drift, amax, nullptr));
        VP_CUDA_TRY(launch_drift(c, c->f, 1, c->coef_drift, amax, nullptr));
    }
    return VP_OK;
}

int vp_field_solve(vp_ctx *c, const double *rho_dev, double *g_dev, double *dt_out)
{
    if (!c || !rho_dev) return VP_ERR_ARG;
    VP_CUDA_TRY(launch_field_solve(c, rho_dev, c->g));
    if (g_dev)
        VP_CUDA_TRY(cudaMemcpyAsync(g_dev, c->g, sizeof(double) * 3 * c->np,
                                    cudaMemcpyDeviceToDevice, c->stream));
    if (dt_out) {
        VP_CUDA_TRY(launch_dt(c, c->g));
        VP_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                                    c->stream));
        VP_CUDA_TRY(cudaStreamSynchronize(c->stream));
        *dt_out = c->sc_host->dt;
        if (!isfinite(*dt_out)) return VP_ERR_NONFINITE;
    }
    return VP_OK;
}

}  // extern "C"
