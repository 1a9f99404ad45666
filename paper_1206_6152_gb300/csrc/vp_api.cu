// vp_api.cu -- the C ABI of include/vp.h: context set-up, the split step as
// CUDA graphs, diagnostics and the host-buffer entry point.
//
// Split step (Sec. 2.1, Eq. integration, Poisson after the drifts, Sec. 2.2):
//   dt^n = C min(dt_p, dt_v(g^n))                               (Sec. 2.4)
//   K1: T_vx, T_vy, T_vz (dt^n / 2, g^n)
//   D : T_z, T_y, T_x (dt^n)
//   rho, phi, g^{n+1}
//   K2: T_vx, T_vy, T_vz (dt^n / 2, g^{n+1})
// Between two steps K2^n and K1^{n+1} use the same g^{n+1}; they run as one
// 6-sweep pass over each velocity cube (one read and one write of f instead
// of two).  The graphs are:
//   prologue: dt, tables, K1 (3 sweeps)
//   body    : D, rho, field, K2 table, t += dt, dt, tables, K2+K1 (6 sweeps)
//   tail    : D, rho, field, K2 table, t += dt, K2 (3 sweeps)
// and vp_step(n) replays prologue, (n - 1) x body, tail.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include <atomic>

#include "vp_device.cuh"
#include "vp_internal.cuh"

namespace {

thread_local char g_last_error[512];

__global__ void k_set_scalar(double *p, double v) { *p = v; }

// counts of the cells of f that are not finite (cnt[0]) and below zero (cnt[1])
template <typename T>
__global__ void k_check(const T *__restrict__ f, long long n, unsigned long long *cnt)
{
    unsigned long long bad = 0, neg = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const T v = f[i];
        if (!isfinite(v)) ++bad;
        else if (v < T(0)) ++neg;
    }
    for (int d = 16; d > 0; d >>= 1) {
        bad += __shfl_xor_sync(0xffffffffu, bad, d);
        neg += __shfl_xor_sync(0xffffffffu, neg, d);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicAdd(cnt, bad);
        if (neg) atomicAdd(cnt + 1, neg);
    }
}
__global__ void k_zero_lost(DevScalars *sc, double t0) { sc->lost = 0.0; sc->t = t0; sc->dt = 0.0; }

template <typename T>
size_t coef_size() { return sizeof(LineCoef<T>); }

void free_ctx(vp_ctx *c)
{
    if (!c) return;
    cudaGraphExec_t gs[] = {c->g_first, c->g_middle, c->g_last, c->g_single};
    for (auto g : gs)
        if (g) cudaGraphExecDestroy(g);
    void *bufs[] = {c->rho, c->phi, c->g, c->cbuf, c->ghat, c->coef_kick1, c->coef_kick2,
                    c->coef_drift, c->vc[0], c->vc[1], c->vc[2], c->red, c->rho2, c->rho_part, c->sc,
                    c->ax[0].tw, c->ax[1].tw, c->ax[2].tw, c->adj_f, c->adj_g, c->adj_lg,
                    c->adj_tmp, c->adj_flag};
    for (void *b : bufs)
        if (b) cudaFree(b);
    vp_free_adjoint_states(c);
    if (c->sc_host) cudaFreeHost(c->sc_host);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
}

// fault injection for tests: the k-th allocation after vp_debug_fail_alloc(k)
// fails (0: off)
std::atomic<int> g_fail_alloc{0};

int dalloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1) return VP_ERR_OOM;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return VP_ERR_OOM;
    }
    return VP_OK;
}

#define TRY(x)                   \
    do {                         \
        int _r = (x);            \
        if (_r != VP_OK) return _r; \
    } while (0)

// host-side FFT used only to build the isolated Green's function at set-up
int build_twiddles(vp_ctx *c)
{
    for (int a = 0; a < 3; ++a) {
        const int n = c->fn[a];
        TRY(vp_fft_plan_axis(&c->ax[a], n));
        std::vector<double2> tw(n);
        for (int k = 0; k < n; ++k) {
            const double ang = -2.0 * M_PI * (double)k / (double)n;
            tw[k] = make_double2(cos(ang), sin(ang));
        }
        TRY(dalloc((void **)&c->ax[a].tw, sizeof(double2) * n));
        VP_CUDA_TRY(cudaMemcpy(c->ax[a].tw, tw.data(), sizeof(double2) * n,
                               cudaMemcpyHostToDevice));
    }
    return VP_OK;
}

// G(k) of the 7-point Laplacian (periodic), or the transformed doubled
// kernel -G/r (isolated); both scaled by the inverse transform's 1/N.
int build_green(vp_ctx *c)
{
    const long long nf = c->nfft;
    std::vector<double> gh(nf);
    const int f0 = c->fn[0], f1 = c->fn[1], f2 = c->fn[2];
    if (!c->isolated) {
        std::vector<double> s0(f0), s1(f1), s2(f2);
        for (int i = 0; i < f0; ++i) { const double s = sin(M_PI * i / f0); s0[i] = s * s / (c->dx[0] * c->dx[0]); }
        for (int i = 0; i < f1; ++i) { const double s = sin(M_PI * i / f1); s1[i] = s * s / (c->dx[1] * c->dx[1]); }
        for (int i = 0; i < f2; ++i) { const double s = sin(M_PI * i / f2); s2[i] = s * s / (c->dx[2] * c->dx[2]); }
        for (int i = 0; i < f0; ++i)
            for (int j = 0; j < f1; ++j)
                for (int k = 0; k < f2; ++k) {
                    const double den = s0[i] + s1[j] + s2[k];
                    const long long t = ((long long)i * f1 + j) * f2 + k;
                    gh[t] = den > 0.0 ? -M_PI * c->cfg.G / den / (double)nf : 0.0;
                }
    } else {
        // real-space doubled kernel, transformed with the library's own FFT
        const double d = c->dx[0];
        const double self = -c->cfg.G * (3.0 * log(2.0 + sqrt(3.0)) - 0.5 * M_PI) / d;
        std::vector<double2> ker(nf);
        for (int i = 0; i < f0; ++i) {
            const double xi = (double)(i <= f0 - i ? i : f0 - i) * c->dx[0];
            for (int j = 0; j < f1; ++j) {
                const double yj = (double)(j <= f1 - j ? j : f1 - j) * c->dx[1];
                for (int k = 0; k < f2; ++k) {
                    const double zk = (double)(k <= f2 - k ? k : f2 - k) * c->dx[2];
                    const double r = sqrt(xi * xi + yj * yj + zk * zk);
                    const long long t = ((long long)i * f1 + j) * f2 + k;
                    ker[t] = make_double2(r > 0.0 ? -c->cfg.G / r : self, 0.0);
                }
            }
        }
        VP_CUDA_TRY(cudaMemcpyAsync(c->cbuf, ker.data(), sizeof(double2) * nf,
                                    cudaMemcpyHostToDevice, c->stream));
        for (int a = 2; a >= 0; --a) VP_CUDA_TRY(launch_fft(c, c->cbuf, a, 0));
        VP_CUDA_TRY(cudaMemcpyAsync(ker.data(), c->cbuf, sizeof(double2) * nf,
                                    cudaMemcpyDeviceToHost, c->stream));
        VP_CUDA_TRY(cudaStreamSynchronize(c->stream));
        for (long long t = 0; t < nf; ++t) gh[t] = ker[t].x * c->dvol_x / (double)nf;
    }
    VP_CUDA_TRY(cudaMemcpy(c->ghat, gh.data(), sizeof(double) * nf, cudaMemcpyHostToDevice));
    return VP_OK;
}

int check_config(const vp_config *cfg)
{
    for (int a = 0; a < 3; ++a) {
        if (cfg->n[a] < 1 || cfg->nv[a] < 1) return VP_ERR_CONFIG;
        if (!(cfg->box_hi[a] > cfg->box_lo[a])) return VP_ERR_CONFIG;
        if (!(cfg->vhi[a] > cfg->vlo[a])) return VP_ERR_CONFIG;
    }
    if (!(cfg->courant > 0.0) && !(cfg->dt_fixed > 0.0)) return VP_ERR_CONFIG;
    if (!isfinite(cfg->G) || !isfinite(cfg->dt_fixed)) return VP_ERR_CONFIG;
    if (cfg->space_bc != 0 && cfg->space_bc != 1) return VP_ERR_CONFIG;
    if (cfg->poisson_bc != 0 && cfg->poisson_bc != 1) return VP_ERR_CONFIG;
    if (cfg->dtype != 0 && cfg->dtype != 1) return VP_ERR_CONFIG;
    return VP_OK;
}

}  // namespace

// host bound of |v tau / dx| over the drift tables: for the step, tau = dt,
// which is either fixed or at most C dx_a / V^max_a on every axis (tau <= 0)
double vp_drift_alpha_bound(const vp_ctx *c, double tau)
{
    double m = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double vmax = fmax(fabs(c->cfg.vlo[a] + 0.5 * c->dv[a]),
                                 fabs(c->cfg.vhi[a] - 0.5 * c->dv[a]));
        double alpha;
        if (tau > 0.0) {
            alpha = vmax * tau / c->dx[a];
        } else {            // adaptive dt of the step
            const double vbox = fmax(fabs(c->cfg.vlo[a]), fabs(c->cfg.vhi[a]));
            alpha = c->cfg.courant * vmax / vbox;
        }
        m = fmax(m, alpha);
    }
    return m;
}

namespace {

double step_alpha_bound(const vp_ctx *c)
{
    return vp_drift_alpha_bound(c, c->cfg.dt_fixed > 0.0 ? c->cfg.dt_fixed : -1.0);
}

int field_from_f(vp_ctx *c)
{
    VP_CUDA_TRY(launch_density(c, c->f, c->rho));
    VP_CUDA_TRY(launch_field_solve(c, c->rho, c->g));
    return VP_OK;
}

// ---------------------------------------------------------------------------
// step segments (enqueued on c->stream; captured into graphs)
// ---------------------------------------------------------------------------
int enqueue_prologue(vp_ctx *c)
{
    VP_CUDA_TRY(launch_dt(c, c->g));
    VP_CUDA_TRY(launch_coef_kick(c, c->g, &c->sc->dt, 0.5, c->coef_kick1));
    VP_CUDA_TRY(launch_coef_drift(c, &c->sc->dt, 1.0, c->coef_drift));
    VP_CUDA_TRY(launch_kick(c, c->f, c->coef_kick1, nullptr, 3, 0));
    return VP_OK;
}

// drift z, y, x and the density of the result
int enqueue_drift_density(vp_ctx *c)
{
    const double amax = step_alpha_bound(c);
    if (amax < 1.0 && vp_drift_yz_ok(c)) {
        VP_CUDA_TRY(launch_drift_yz(c, c->f, c->coef_drift, c->f));
    } else {
        VP_CUDA_TRY(launch_drift(c, c->f, 2, c->coef_drift, amax, nullptr));
        VP_CUDA_TRY(launch_drift(c, c->f, 1, c->coef_drift, amax, nullptr));
    }
    if (c->rho_part && vp_rho_fuse_ok(c) && amax < 1.0) {
        VP_CUDA_TRY(launch_drift(c, c->f, 0, c->coef_drift, amax, c->rho_part));
        VP_CUDA_TRY(launch_rho_finish(c, c->rho_part, c->rho_nparts, c->rho));
    } else {
        VP_CUDA_TRY(launch_drift(c, c->f, 0, c->coef_drift, amax, nullptr));
        VP_CUDA_TRY(launch_density(c, c->f, c->rho));
    }
    return VP_OK;
}

int enqueue_body(vp_ctx *c, int last)
{
    TRY(enqueue_drift_density(c));
    VP_CUDA_TRY(launch_field_solve(c, c->rho, c->g));
    VP_CUDA_TRY(launch_coef_kick(c, c->g, &c->sc->dt, 0.5, c->coef_kick2));
    VP_CUDA_TRY(launch_advance_time(c));
    if (last) {
        VP_CUDA_TRY(launch_kick(c, c->f, c->coef_kick2, nullptr, 3, 0));
    } else {
        VP_CUDA_TRY(launch_dt(c, c->g));
        VP_CUDA_TRY(launch_coef_kick(c, c->g, &c->sc->dt, 0.5, c->coef_kick1));
        VP_CUDA_TRY(launch_coef_drift(c, &c->sc->dt, 1.0, c->coef_drift));
        VP_CUDA_TRY(launch_kick(c, c->f, c->coef_kick2, c->coef_kick1, 6, 0));
    }
    return VP_OK;
}

int capture(vp_ctx *c, int which, cudaGraphExec_t *out, long long *nkernels)
{
    cudaStream_t user = c->stream;
    c->stream = c->cap;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        c->stream = user;
        vp_note_cuda_error(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
        return VP_ERR_CUDA;
    }
    int r = which == 0 ? enqueue_prologue(c) : enqueue_body(c, which == 2);
    e = cudaStreamEndCapture(c->cap, &graph);
    c->stream = user;
    if (r != VP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return r;
    }
    if (e != cudaSuccess) {
        vp_note_cuda_error(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        return VP_ERR_CUDA;
    }
    size_t nn = 0;
    *nkernels = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
            for (size_t i = 0; i < nn; ++i) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                    ++*nkernels;
            }
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        vp_note_cuda_error(e, "cudaGraphInstantiate", __FILE__, __LINE__);
        return VP_ERR_CUDA;
    }
    return VP_OK;
}

int ensure_graphs(vp_ctx *c)
{
    if (c->graphs_ready) return VP_OK;
    TRY(capture(c, 0, &c->g_first, &c->nk_first));
    TRY(capture(c, 1, &c->g_middle, &c->nk_middle));
    TRY(capture(c, 2, &c->g_last, &c->nk_last));
    c->graphs_ready = 1;
    return VP_OK;
}

void drop_graphs(vp_ctx *c)
{
    cudaGraphExec_t *gs[] = {&c->g_first, &c->g_middle, &c->g_last};
    for (auto g : gs)
        if (*g) { cudaGraphExecDestroy(*g); *g = nullptr; }
    c->graphs_ready = 0;
}

}  // namespace

void vp_note_cuda_error(cudaError_t e, const char *expr, const char *file, int line)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", cudaGetErrorString(e), expr,
             file, line);
}

extern "C" {

const char *vp_error_string(int code)
{
    switch (code) {
    case VP_OK: return "ok";
    case VP_ERR_CONFIG: return "invalid configuration";
    case VP_ERR_OOM: return "device allocation failed";
    case VP_ERR_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case VP_ERR_NONFINITE: return "non-finite value detected";
    case VP_ERR_ARG: return "invalid argument";
    case VP_ERR_STATE: return "invalid state";
    case VP_ERR_UNSUPPORTED: return "unsupported grid size";
    default: return "unknown error";
    }
}

}  // extern "C"

namespace {

// the context of vp_init; without f (f_dev == nullptr) only what the field
// solve needs is used and no field is computed
int init_ctx(const vp_config *cfg, void *f_dev, void *cuda_stream, vp_ctx **out)
{
    if (!cfg || !out) return VP_ERR_ARG;
    *out = nullptr;
    TRY(check_config(cfg));
    vp_ctx *c = new (std::nothrow) vp_ctx();
    if (!c) return VP_ERR_OOM;
    memset((void *)c, 0, sizeof(*c));
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cuda_stream;
    c->f = f_dev;
    c->isdouble = cfg->dtype == 1;
    c->esize = c->isdouble ? sizeof(double) : sizeof(float);
    c->np = 1;
    c->nvc = 1;
    c->maxnv = 0;
    for (int a = 0; a < 3; ++a) {
        c->n[a] = cfg->n[a];
        c->nv[a] = cfg->nv[a];
        c->np *= cfg->n[a];
        c->nvc *= cfg->nv[a];
        c->dx[a] = (cfg->box_hi[a] - cfg->box_lo[a]) / cfg->n[a];
        c->dv[a] = (cfg->vhi[a] - cfg->vlo[a]) / cfg->nv[a];
        if (cfg->nv[a] > c->maxnv) c->maxnv = cfg->nv[a];
    }
    c->ncells = c->np * c->nvc;
    c->dvol_x = c->dx[0] * c->dx[1] * c->dx[2];
    c->dvol_v = c->dv[0] * c->dv[1] * c->dv[2];
    c->periodic_space = cfg->space_bc == 0;
    c->isolated = cfg->poisson_bc == 1;
    int r = VP_OK;
    auto fail = [&](int code) {
        free_ctx(c);
        return code;
    };
    // size limits of the kernels
    {
        // drift tiles N_l x C and per-axis kick tiles N^v_l x (C + 1); cubes
        // above the shared-memory size are kicked one axis per pass
        for (int a = 0; a < 3; ++a) {
            const size_t tile = (size_t)c->n[a] * (c->isdouble ? 128 : 256) * c->esize;
            const size_t ktile = (size_t)c->nv[a] * (c->isdouble ? 129 : 257) * c->esize;
            if (tile > 220 * 1024 || ktile > 220 * 1024) return fail(VP_ERR_UNSUPPORTED);
        }
        if (c->nvc > 0x7fffffffLL || c->np / c->n[0] > 65535 || c->np / c->n[1] > 65535 ||
            c->np / c->n[2] > 65535 || c->np > 0x7fffffffLL)
            return fail(VP_ERR_UNSUPPORTED);
    }
    if (c->isolated) {
        const double d = c->dx[0];
        if (fabs(c->dx[1] - d) > 1e-12 * d || fabs(c->dx[2] - d) > 1e-12 * d)
            return fail(VP_ERR_CONFIG);
    }
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) { vp_note_cuda_error(e, "cudaGetDevice", __FILE__, __LINE__); return fail(VP_ERR_CUDA); }
    e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) { vp_note_cuda_error(e, "cudaStreamCreate", __FILE__, __LINE__); return fail(VP_ERR_CUDA); }
    c->nfft = 1;
    for (int a = 0; a < 3; ++a) {
        c->fn[a] = c->isolated ? 2 * c->n[a] : c->n[a];
        if (c->isolated && c->n[a] == 1) c->fn[a] = 1;
        c->nfft *= c->fn[a];
        if (c->fn[a] > 2048) return fail(VP_ERR_UNSUPPORTED);
    }
    const size_t cs = c->isdouble ? coef_size<double>() : coef_size<float>();
    if ((r = dalloc((void **)&c->rho, sizeof(double) * c->np)) ||
        (r = dalloc((void **)&c->rho2, sizeof(double) * c->np)) ||
        (r = dalloc((void **)&c->phi, sizeof(double) * c->nfft)) ||
        (r = dalloc((void **)&c->g, sizeof(double) * 3 * c->np)) ||
        (r = dalloc((void **)&c->cbuf, sizeof(double2) * c->nfft)) ||
        (r = dalloc((void **)&c->ghat, sizeof(double) * c->nfft)) ||
        (r = dalloc(&c->coef_kick1, cs * 3 * c->np)) ||
        (r = dalloc(&c->coef_kick2, cs * 3 * c->np)) ||
        (r = dalloc(&c->coef_drift, cs * 3 * c->maxnv)) ||
        (r = dalloc((void **)&c->red, sizeof(double) * (2 * c->np + 64))) ||
        (r = dalloc((void **)&c->sc, sizeof(DevScalars))))
        return fail(r);
    if (vp_rho_fuse_ok(c)) {
        c->rho_nparts = vp_rho_parts(c);
        if ((r = dalloc((void **)&c->rho_part, sizeof(double) * c->np * c->rho_nparts)))
            return fail(r);
    }
    for (int a = 0; a < 3; ++a) {
        if ((r = dalloc((void **)&c->vc[a], sizeof(double) * c->nv[a]))) return fail(r);
        std::vector<double> vc(c->nv[a]);
        for (int j = 0; j < c->nv[a]; ++j) vc[j] = cfg->vlo[a] + (j + 0.5) * c->dv[a];
        e = cudaMemcpy(c->vc[a], vc.data(), sizeof(double) * c->nv[a], cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { vp_note_cuda_error(e, "cudaMemcpy", __FILE__, __LINE__); return fail(VP_ERR_CUDA); }
    }
    e = cudaMallocHost((void **)&c->sc_host, sizeof(DevScalars));
    if (e != cudaSuccess) { cudaGetLastError(); c->sc_host = nullptr; return fail(VP_ERR_OOM); }
    if ((r = build_twiddles(c))) return fail(r);
    if ((r = build_green(c))) return fail(r);
    k_zero_lost<<<1, 1, 0, c->stream>>>(c->sc, 0.0);
    if (c->f && (r = field_from_f(c))) return fail(r);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { vp_note_cuda_error(e, "vp_init sync", __FILE__, __LINE__); return fail(VP_ERR_CUDA); }
    *out = c;
    return VP_OK;
}

}  // namespace

extern "C" {

int vp_init(const vp_config *cfg, void *f_dev, void *cuda_stream, vp_ctx **out)
{
    if (!f_dev) {
        if (out) *out = nullptr;
        return VP_ERR_ARG;
    }
    return init_ctx(cfg, f_dev, cuda_stream, out);
}

int vp_field_init(const vp_config *cfg, void *cuda_stream, vp_ctx **out)
{
    return init_ctx(cfg, nullptr, cuda_stream, out);
}

int vp_refresh_field(vp_ctx *c)
{
    if (!c) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    return field_from_f(c);
}

int vp_set_distribution(vp_ctx *c, void *f_dev)
{
    if (!c || !f_dev) return VP_ERR_ARG;
    if (f_dev != c->f) {
        c->f = f_dev;
        drop_graphs(c);
    }
    return field_from_f(c);
}

int vp_step(vp_ctx *c, int nsteps, double *t_out)
{
    if (!c || nsteps < 0) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    if (nsteps > 0) {
        TRY(ensure_graphs(c));
        VP_CUDA_TRY(cudaGraphLaunch(c->g_first, c->stream));
        for (int i = 0; i < nsteps - 1; ++i) VP_CUDA_TRY(cudaGraphLaunch(c->g_middle, c->stream));
        VP_CUDA_TRY(cudaGraphLaunch(c->g_last, c->stream));
        c->kernels_launched += c->nk_first + (nsteps - 1) * c->nk_middle + c->nk_last;
    }
    if (t_out) {
        VP_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                                    c->stream));
        VP_CUDA_TRY(cudaStreamSynchronize(c->stream));
        *t_out = c->sc_host->t;
        if (!isfinite(c->sc_host->dt)) return VP_ERR_NONFINITE;
    }
    return VP_OK;
}

int vp_sweep(vp_ctx *c, int axis, double tau)
{
    if (!c || axis < 0 || axis > 5 || !isfinite(tau)) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    double *tau_ptr = &c->sc->pad[0];
    k_set_scalar<<<1, 1, 0, c->stream>>>(tau_ptr, tau);
    VP_CUDA_TRY(cudaGetLastError());
    if (axis < 3) {
        VP_CUDA_TRY(launch_coef_drift(c, tau_ptr, 1.0, c->coef_drift));
        VP_CUDA_TRY(launch_drift(c, c->f, axis, c->coef_drift, vp_drift_alpha_bound(c, fabs(tau)),
                                 nullptr));
    } else {
        VP_CUDA_TRY(launch_coef_kick(c, c->g, tau_ptr, 1.0, c->coef_kick1));
        VP_CUDA_TRY(launch_kick(c, c->f, c->coef_kick1, nullptr, 1, axis - 3));
    }
    return VP_OK;
}

int vp_moments(vp_ctx *c, double *rho_dev)
{
    if (!c || !rho_dev) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    VP_CUDA_TRY(launch_density(c, c->f, rho_dev));
    return VP_OK;
}

int vp_get_field(vp_ctx *c, double *rho_dev, double *phi_dev, double *g_dev)
{
    if (!c) return VP_ERR_ARG;
    if (rho_dev)
        VP_CUDA_TRY(cudaMemcpyAsync(rho_dev, c->rho, sizeof(double) * c->np,
                                    cudaMemcpyDeviceToDevice, c->stream));
    if (phi_dev) VP_CUDA_TRY(launch_copy_phi_box(c, phi_dev));
    if (g_dev)
        VP_CUDA_TRY(cudaMemcpyAsync(g_dev, c->g, sizeof(double) * 3 * c->np,
                                    cudaMemcpyDeviceToDevice, c->stream));
    return VP_OK;
}

int vp_set_accel(vp_ctx *c, const double *g_dev)
{
    if (!c || !g_dev) return VP_ERR_ARG;
    VP_CUDA_TRY(cudaMemcpyAsync(c->g, g_dev, sizeof(double) * 3 * c->np,
                                cudaMemcpyDeviceToDevice, c->stream));
    return VP_OK;
}

int vp_energy(vp_ctx *c, double out[5])
{
    if (!c || !out) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    // M and K: per-cell partials, then a compensated reduction
    VP_CUDA_TRY(launch_energy_partials(c, c->f, c->red));
    double *sums = c->red + 2 * c->np;
    VP_CUDA_TRY(launch_reduce_strided(c, c->red, c->np, 2, sums));
    // U: the potential of the current f
    VP_CUDA_TRY(launch_density(c, c->f, c->rho2));
    VP_CUDA_TRY(launch_field_solve(c, c->rho2, nullptr));
    VP_CUDA_TRY(launch_dot_rho_phi(c, c->rho2, sums + 2));
    double h[3];
    VP_CUDA_TRY(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    VP_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                                c->stream));
    VP_CUDA_TRY(cudaStreamSynchronize(c->stream));
    const double dV = c->dvol_x * c->dvol_v;
    out[0] = h[0] * dV;
    out[1] = 0.5 * h[1] * dV;
    out[2] = 0.5 * h[2] * c->dvol_x;
    out[3] = out[1] + out[2];
    out[4] = c->sc_host->lost * dV;
    for (int i = 0; i < 5; ++i)
        if (!isfinite(out[i])) return VP_ERR_NONFINITE;
    return VP_OK;
}

int vp_time(vp_ctx *c, double *t, double *dt_last)
{
    if (!c) return VP_ERR_ARG;
    VP_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                                c->stream));
    VP_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (t) *t = c->sc_host->t;
    if (dt_last) *dt_last = c->sc_host->dt;
    return VP_OK;
}

int vp_step_host(vp_ctx *c, const void *f_host_in, void *f_host_out, int nsteps, double *t_out,
                 double *diag_out)
{
    if (!c || !f_host_in || nsteps < 0) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    const size_t bytes = (size_t)c->ncells * c->esize;
    VP_CUDA_TRY(cudaMemcpyAsync(c->f, f_host_in, bytes, cudaMemcpyHostToDevice, c->stream));
    TRY(field_from_f(c));
    TRY(vp_step(c, nsteps, nullptr));
    if (diag_out) TRY(vp_energy(c, diag_out));
    if (f_host_out)
        VP_CUDA_TRY(cudaMemcpyAsync(f_host_out, c->f, bytes, cudaMemcpyDeviceToHost, c->stream));
    VP_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                                c->stream));
    VP_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (t_out) *t_out = c->sc_host->t;
    return VP_OK;
}

int vp_check(vp_ctx *c, long long *counts)
{
    if (!c) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(c->red);
    VP_CUDA_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), c->stream));
    const unsigned grid = (unsigned)(vp_sm_count() * 8);
    if (c->isdouble)
        k_check<double><<<grid, 256, 0, c->stream>>>((const double *)c->f, c->ncells, cnt);
    else
        k_check<float><<<grid, 256, 0, c->stream>>>((const float *)c->f, c->ncells, cnt);
    VP_CUDA_TRY(cudaGetLastError());
    unsigned long long h[2];
    VP_CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    VP_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (counts) {
        counts[0] = (long long)h[0];
        counts[1] = (long long)h[1];
    }
    return (h[0] || h[1]) ? VP_ERR_NONFINITE : VP_OK;
}

int vp_debug_fail_alloc(int k)
{
    if (k < 0) return VP_ERR_ARG;
    g_fail_alloc.store(k);
    return VP_OK;
}

int vp_stats(vp_ctx *c, long long *kernels_launched)
{
    if (!c || !kernels_launched) return VP_ERR_ARG;
    *kernels_launched = c->kernels_launched;
    return VP_OK;
}

int vp_profile_step(vp_ctx *c, double *ms_out)
{
    if (!c || !ms_out) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    cudaEvent_t ev[12];
    for (int i = 0; i < 12; ++i) VP_CUDA_TRY(cudaEventCreate(&ev[i]));
    for (int i = 8; i < 11; ++i) ms_out[i] = 0.0;
    const bool big_kick = vp_kick_big_ok(c) != 0;      // the fused kick runs as three passes
    int r = VP_OK;
    auto rec = [&](int i) { return cudaEventRecord(ev[i], c->stream); };
#define PROF(x)                                                              \
    do {                                                                     \
        cudaError_t _e = (x);                                                \
        if (_e != cudaSuccess) {                                             \
            vp_note_cuda_error(_e, #x, __FILE__, __LINE__);                  \
            r = VP_ERR_CUDA;                                                 \
            goto done;                                                       \
        }                                                                    \
    } while (0)
    // state entering the body: K1 of this step already applied, as after
    // the prologue of vp_step; run the prologue first, untimed
    if ((r = enqueue_prologue(c)) != VP_OK) goto done;
    {
        const double amax = step_alpha_bound(c);
        const bool fuse = c->rho_part && vp_rho_fuse_ok(c) && amax < 1.0;
        PROF(rec(0));
        if (amax < 1.0 && vp_drift_yz_ok(c)) {
            PROF(launch_drift_yz(c, c->f, c->coef_drift, c->f));
            PROF(rec(1));
        } else {
            PROF(launch_drift(c, c->f, 2, c->coef_drift, amax, nullptr));
            PROF(rec(1));
            PROF(launch_drift(c, c->f, 1, c->coef_drift, amax, nullptr));
        }
        PROF(rec(2));
        PROF(launch_drift(c, c->f, 0, c->coef_drift, amax, fuse ? c->rho_part : nullptr));
        PROF(rec(3));
        if (fuse) PROF(launch_rho_finish(c, c->rho_part, c->rho_nparts, c->rho));
        else PROF(launch_density(c, c->f, c->rho));
        PROF(rec(4));
    }
    PROF(launch_field_solve(c, c->rho, c->g));
    PROF(rec(5));
    PROF(launch_coef_kick(c, c->g, &c->sc->dt, 0.5, c->coef_kick2));
    PROF(launch_advance_time(c));
    PROF(launch_dt(c, c->g));
    PROF(launch_coef_kick(c, c->g, &c->sc->dt, 0.5, c->coef_kick1));
    PROF(launch_coef_drift(c, &c->sc->dt, 1.0, c->coef_drift));
    PROF(rec(6));
    if (big_kick) c->kick_pass_ev = ev + 8;
    {
        const cudaError_t ek = launch_kick(c, c->f, c->coef_kick2, c->coef_kick1, 6, 0);
        c->kick_pass_ev = nullptr;
        PROF(ek);
    }
    PROF(rec(7));
    // close the step: drift, field and the final half kick, untimed
    if ((r = enqueue_body(c, 1)) != VP_OK) goto done;
    PROF(cudaStreamSynchronize(c->stream));
    {
        float ms;
        const int fam[7][2] = {{6, 7}, {0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}, {5, 6}};
        for (int i = 0; i < 7; ++i) {
            PROF(cudaEventElapsedTime(&ms, ev[fam[i][0]], ev[fam[i][1]]));
            ms_out[i] = ms;
        }
        PROF(cudaEventElapsedTime(&ms, ev[0], ev[7]));
        ms_out[7] = ms;
        if (big_kick)
            for (int i = 0; i < 3; ++i) {
                PROF(cudaEventElapsedTime(&ms, ev[8 + i], ev[9 + i]));
                ms_out[8 + i] = ms;
            }
    }
#undef PROF
done:
    for (int i = 0; i < 12; ++i) cudaEventDestroy(ev[i]);
    return r;
}

void vp_destroy(vp_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
}

}  // extern "C"
