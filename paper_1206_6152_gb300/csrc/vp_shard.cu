// vp_shard.cu -- the pieces of the split step that change when position
// space is cut into slabs along x, one slab per GPU (the decomposition of
// Sec. 2.3): the x drift of a slab whose lines continue into ghost planes
// of the neighbouring slabs, the per-line maxima along x of a slab (reduced
// over the slabs by the caller, since f_inf is the maximum of the whole
// line), and a context that only solves for the field of a density it is
// given (the FFT stays whole on every GPU: the density is gathered).
#include <cuda_runtime.h>
#include <math.h>

#include "vp_device.cuh"
#include "vp_internal.cuh"

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
        for (int i = 0; i < nx; ++i) m = fmax(m, f[(long long)i * nl + l]);
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
