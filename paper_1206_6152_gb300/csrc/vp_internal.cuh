// vp_internal.cuh -- context and device helpers shared by the CUDA sources of
// the GB300 Vlasov--Poisson library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vp.h"

#define VP_CUDA_TRY(expr)                                        \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) {                                 \
            vp_note_cuda_error(_e, #expr, __FILE__, __LINE__);   \
            return VP_ERR_CUDA;                                  \
        }                                                        \
    } while (0)

void vp_note_cuda_error(cudaError_t e, const char *expr, const char *file, int line);

// One advection line's shift alpha = u tau / h written as |alpha| = s + beta
// with the direction of travel.  The PFC partial-flux weights of Sec. 2.1
// (third-order reconstruction): c0 = beta, c1 = beta(1-beta)(2-beta)/6,
// c2 = beta(1-beta)(1+beta)/6.  code = 2 s + (alpha < 0).
template <typename T>
struct __align__(16) LineCoef {
    int code;
    T c0, c1, c2;
};

// Device-resident scalars of a context.
struct DevScalars {
    double dt;          // dt of the current step
    double t;           // simulated time
    double lost;        // phase-space sum of f that left (unscaled)
    double amax;        // max_l,x |g_l| / dv_l of the last dt evaluation
    double pad[6];      // per-call scalars of the entry points (stream-ordered)
};

struct FFTAxis {
    int n;              // length
    int nrad;           // number of radix stages
    int rad[24];        // radices, applied in order
    double2 *tw;        // twiddles W_n^k = exp(-2 pi i k / n), k < n (device)
};

struct vp_ctx {
    vp_config cfg;
    int device;
    cudaStream_t stream;        // caller's stream
    cudaStream_t cap;           // internal stream used to capture graphs
    void *f;                    // borrowed distribution function
    int isdouble;
    size_t esize;
    int n[3], nv[3];
    long long np, nvc, ncells;  // spatial cells, velocity cells, total
    double dx[3], dv[3];
    double dvol_x, dvol_v;
    int periodic_space;
    int isolated;

    // fields (device, owned)
    double *rho;                // np
    double *phi;                // nfft (real potential on the FFT grid)
    double *g;                  // 3 np
    double2 *cbuf;              // nfft complex work buffer
    double *ghat;               // nfft real Green's function in k space / nfft
    int fn[3];                  // FFT grid (n or 2n)
    long long nfft;
    FFTAxis ax[3];

    // tables (device, owned)
    void *coef_kick1;           // LineCoef<T>[np][3] for the first half kick
    void *coef_kick2;           // LineCoef<T>[np][3] for the second half kick
    void *coef_drift;           // LineCoef<T>[3][maxnv]
    int maxnv;
    double *vc[3];              // velocity cell centres (device)
    double *red;                // reduction scratch (2 np + 64 doubles)
    double *rho2;               // density of the current f for diagnostics
    double *rho_part;           // density partials of the fused x drift
    int rho_nparts;
    DevScalars *sc;             // device scalars
    DevScalars *sc_host;        // pinned mirror for read-back

    // CUDA graphs (built lazily) and their kernel-node counts
    cudaGraphExec_t g_first, g_middle, g_last, g_single;
    int graphs_ready;
    long long nk_first, nk_middle, nk_last;
    long long kernels_launched;

    // adjoint scratch (lazily allocated)
    void *adj_f;                // one state in f's dtype
    double *adj_g;              // 3 np
    double *adj_lg;             // 3 np
    double *adj_tmp;            // nfft
    int *adj_flag;              // set when the register adjoint skipped a line
    void **adj_states;          // sweep inputs (f's dtype): nine slots (those the path
                                // reads; some may share a buffer), or two to recompute into
    int adj_nstates;
    int adj_mode;               // 0 automatic, 1 two states, 2 the kept sweep inputs

    // tracing: when set, the kick of 48^3 cubes records an event before
    // its first pass and after each pass (vp_profile_step)
    cudaEvent_t *kick_pass_ev;
};

// ---------------------------------------------------------------------------
// launch wrappers implemented in the .cu files; all return cudaError_t of the
// launch (cudaGetLastError)
// ---------------------------------------------------------------------------
cudaError_t launch_coef_drift(vp_ctx *c, const double *tau_ptr, double factor, void *out);
cudaError_t launch_coef_kick(vp_ctx *c, const double *g, const double *tau_ptr, double factor,
                             void *out);
cudaError_t launch_dt(vp_ctx *c, const double *g);
cudaError_t launch_advance_time(vp_ctx *c);
// drift along a spatial axis; max_alpha is a host-side bound of |v tau / dx|
// over the table (the register kernels need it below 1); with rho_part the
// x drift also writes density partials (returns cudaErrorNotSupported if it
// cannot)
cudaError_t launch_drift(vp_ctx *c, void *f, int axis, const void *coef, double max_alpha,
                         double *rho_part);
// nsweeps velocity sweeps over every cube; sweep k runs along axis
// (first_axis + k) % 3 with table coef_a for k < 3 and coef_b afterwards
cudaError_t launch_kick(vp_ctx *c, void *f, const void *coef_a, const void *coef_b, int nsweeps,
                        int first_axis);
cudaError_t launch_density(vp_ctx *c, const void *f, double *rho);
cudaError_t launch_field_solve(vp_ctx *c, const double *rho, double *g_out);
cudaError_t launch_energy_partials(vp_ctx *c, const void *f, double *partials);
cudaError_t launch_copy_phi_box(vp_ctx *c, double *dst);
cudaError_t launch_dot_rho_phi(vp_ctx *c, const double *rho, double *out2);
cudaError_t launch_reduce_strided(vp_ctx *c, const double *in, long long n, int stride,
                                  double *out);
int vp_sm_count();

// register-line kernels (vp_sweep_fast.cu)
int vp_kick_fast_ok(const vp_ctx *c);
int vp_drift_fast_ok(const vp_ctx *c, int axis);
int vp_rho_fuse_ok(const vp_ctx *c);
int vp_rho_parts(vp_ctx *c);
// FP32 cubes of edge 48: whole half kicks and the fused kick in passes of
// two sweeps on slabs (vp_kick_big.cu); other sweep runs one pass per vx
// sweep and per run of consecutive vy / vz sweeps, lines in registers
int vp_kick_big_ok(const vp_ctx *c);
cudaError_t launch_kick_big(vp_ctx *c, void *f, const void *ca, const void *cb, int nsweeps,
                            int first_axis, void *fo = nullptr);
cudaError_t launch_kick_big3(vp_ctx *c, float *f, const LineCoef<float> *ca,
                             const LineCoef<float> *cb, int nsweeps, int first_axis, float *fo);
// FP64 cubes of edge 16 or 32: one launch per sweep, one line per thread in
// registers (vp_sweep_f64.cu); fo: output array (nullptr: in place)
int vp_kick_f64_ok(const vp_ctx *c);
cudaError_t launch_kick_f64(vp_ctx *c, void *f, const void *ca, const void *cb, int nsweeps,
                            int first_axis, void *fo);
// fused z then y drift of the whole grid (FP32, N_y = N_z in {16, 32}; in
// place when fo == f)
int vp_drift_yz_ok(const vp_ctx *c);
cudaError_t launch_drift_yz(vp_ctx *c, const void *f, const void *coef, void *fo);
// fo: output array (nullptr: in place);
// inter0/inter1: optional copies of the cube after sweeps 0 and 1.  gate:
// if not null, nothing runs unless *gate != 0, and only cubes whose table
// entries (ca, all three axes) have a whole-cell shift are swept.
cudaError_t launch_kick_fast(vp_ctx *c, void *f, const void *ca, const void *cb, int nsweeps,
                             int first_axis, void *fo = nullptr, void *inter0 = nullptr,
                             void *inter1 = nullptr, const int *gate = nullptr);
cudaError_t launch_drift_fast(vp_ctx *c, void *f, int axis, const void *coef, double *rho_part,
                              void *fo = nullptr);
// one sweep from src into dst (dst != src), used by the adjoint's replay;
// kick tables [np][3], drift tables [3][maxnv]
cudaError_t launch_sweep_into(vp_ctx *c, const void *src, void *dst, int axis, const void *coef,
                              double drift_alpha_bound);
cudaError_t launch_rho_finish(vp_ctx *c, const double *part, int nparts, double *rho);

int vp_fft_plan_axis(FFTAxis *a, int n);
cudaError_t launch_fft(vp_ctx *c, double2 *data, int axis, int inverse);

cudaError_t launch_green_mul(vp_ctx *c);
double vp_drift_alpha_bound(const vp_ctx *c, double tau);

// adjoint (vp_adjoint.cu)
// bc (x axis only, may be null): dvol_v lam_rho per spatial cell, added to
// lam before the adjoint (the deferred density broadcast of the field adjoint)
cudaError_t launch_drift_adjoint(vp_ctx *c, const void *fin, void *lam, int axis, const void *coef,
                                 const double *bc);
cudaError_t launch_kick_adjoint(vp_ctx *c, const void *fin, void *lam, int vaxis, const void *coef,
                                double tau, double *lam_g);
// defer: leave dvol_v lam_rho in c->rho2 instead of adding it to lam_f
cudaError_t launch_field_adjoint(vp_ctx *c, const double *lam_g, void *lam_f, bool defer);
// FP32 packed register-line adjoint sweeps (line lengths 16/32/48, zero
// whole-cell shift; skipped lines set c->adj_flag)
int vp_adjoint_pairs_ok(const vp_ctx *c, int axis);
// the three velocity-sweep adjoints of a half kick in one cube pass (FP32,
// cubic 16/32 velocity grids); cubes with a whole-cell shift on any axis
// are skipped and set c->adj_flag
int vp_kick_adjoint3_ok(const vp_ctx *c);
// the y then z drift adjoints of a zero-shift step in one pass (FP32,
// N_y = N_z in {16, 32}); s3: the input of the z drift (the input of the y
// drift is recomputed from it); the grids of launch_drift_yz for those N
int vp_drift_adjoint_yz_ok(const vp_ctx *c);
// frees the adjoint's scratch states (each buffer once)
void vp_free_adjoint_states(vp_ctx *c);
cudaError_t launch_drift_adjoint_yz(vp_ctx *c, const void *s3, void *lam, const void *coef);
cudaError_t launch_kick_adjoint3(vp_ctx *c, const void *sa, const void *sb, void *lam,
                                 const void *coef, double *lam_g, double tau);
// cube3 (kick axes): skip every cube with a shift on any velocity axis and
// keep c->adj_flag as it is
cudaError_t launch_adjoint_pairs(vp_ctx *c, const void *fin, void *lam, int axis, const void *coef,
                                 double *lam_g, double scale, const double *bc, int cube3 = 0);
