/*
 * vp.h -- C ABI of the GB300 six-dimensional Vlasov--Poisson integrator.
 *
 * The library advances a distribution function f(x, v) on a uniform
 * N_x N_y N_z x N^v_x N^v_y N^v_z phase-space grid with the directionally
 * split positive-flux-conservation (PFC) scheme of Yoshikawa, Yoshida &
 * Umemura (2013), "Direct integration of the collisionless Boltzmann
 * equation in six-dimensional phase space: self-gravitating systems":
 *
 *   Sec. 2 (grid)        x in [box_lo, box_hi), v in [vlo, vhi), cell
 *                        averages at cell centres V^- + (j + 1/2) dv;
 *   Sec. 2.1             1D advection sweeps T_l with the PFC flux and the
 *                        slope corrector (line maximum f_inf), outflow in
 *                        velocity, periodic or outflow in position;
 *   Sec. 2.1, Eq. (integration)
 *                        f^{n+1} = T_vz T_vy T_vx(dt/2) T_x T_y T_z(dt)
 *                                  T_vz T_vy T_vx(dt/2) f^n;
 *   Sec. 2.2             rho = integral of f dv, Poisson by FFT convolution
 *                        (periodic discrete Green's function, or Hockney's
 *                        doubling for isolated boundaries), force by the
 *                        2-point central difference;
 *   Sec. 2.4             dt = C min(dt_p, dt_v).
 *
 * Memory layout of f (device, borrowed from the caller, never freed here):
 *   f[x][y][z][vx][vy][vz], C order, vz fastest, element type float
 *   (dtype 0) or double (dtype 1).  The velocity cube of one spatial cell
 *   is contiguous.  Size N_x N_y N_z N^v_x N^v_y N^v_z elements.
 * Spatial fields (rho, phi, g) are double, [x][y][z] C order; g is three
 * such arrays back to back (g_x, g_y, g_z), g = -grad phi.
 *
 * Threading and streams: every call is asynchronous on the stream given
 * to vp_init, except those documented as synchronising.  A context is not
 * thread safe.  No call ever spins on the host.
 *
 * Errors: every int-returning call returns VP_OK (0) or a negative code;
 * vp_error_string() names it.  No C++ exception crosses this interface.
 * After VP_ERR_CUDA the context should be destroyed.
 */
#ifndef VP_H
#define VP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VP_OK 0
#define VP_ERR_CONFIG (-1)      /* invalid vp_config                          */
#define VP_ERR_OOM (-2)         /* device allocation failed                   */
#define VP_ERR_CUDA (-3)        /* a CUDA runtime call failed                 */
#define VP_ERR_NONFINITE (-4)   /* NaN/Inf or negative f detected             */
#define VP_ERR_ARG (-5)         /* bad argument (null pointer, bad axis...)   */
#define VP_ERR_STATE (-6)       /* call not valid in the context's state      */
#define VP_ERR_UNSUPPORTED (-7) /* grid size the kernels do not support       */

/* Run parameters (Sec. 2 grid, Sec. 2.1 boundaries, Sec. 2.4 timestep). */
typedef struct vp_config {
    int n[3];            /* N_x, N_y, N_z (>= 1)                             */
    int nv[3];           /* N^v_x, N^v_y, N^v_z (>= 1)                       */
    double box_lo[3];    /* lower corner of the spatial box (-L/2)           */
    double box_hi[3];    /* upper corner (+L/2)                              */
    double vlo[3];       /* V^-                                              */
    double vhi[3];       /* V^+                                              */
    double G;            /* gravitational constant                           */
    double courant;      /* C of dt = C min(dt_p, dt_v)                      */
    double dt_fixed;     /* > 0: fixed dt; <= 0: adaptive dt                 */
    int space_bc;        /* 0 periodic, 1 outflow (position sweeps)          */
    int poisson_bc;      /* 0 periodic, 1 isolated (Hockney doubling)        */
    int dtype;           /* 0: f is float, 1: f is double                    */
} vp_config;

typedef struct vp_ctx vp_ctx;

/* Creates a context for the borrowed device array f_dev (layout above) and
 * computes the acceleration g^0 = -grad phi[rho(f^0)] that the first half
 * kick uses.  cuda_stream is a cudaStream_t (NULL: the legacy default
 * stream).  The context allocates its own fields, FFT buffers, tables and
 * scratch (all freed by vp_destroy).  Returns VP_ERR_CONFIG for invalid
 * sizes or box, VP_ERR_UNSUPPORTED when a spatial FFT length has a prime
 * factor above 13 or a line is longer than 1024 cells, VP_ERR_OOM when an
 * allocation fails.  Synchronises the stream once. */
int vp_init(const vp_config *cfg, void *f_dev, void *cuda_stream, vp_ctx **out);

/* Points the context at another f array of the same shape and dtype and
 * recomputes g from it (as vp_refresh_field). */
int vp_set_distribution(vp_ctx *ctx, void *f_dev);

/* Recomputes rho, phi and g from the current f (Sec. 2.2).  Use after
 * changing f outside the library. */
int vp_refresh_field(vp_ctx *ctx);

/* Advances f in place by nsteps split steps (Sec. 2.1, Eq. integration;
 * Poisson after the drift).  The state between steps is (f, g).  With
 * dt_fixed <= 0 each step's dt = C min(dt_p, dt_v(g^n)) is computed on the
 * device.  If t_out is not NULL the simulated time after the steps is
 * written there (this synchronises the stream). */
int vp_step(vp_ctx *ctx, int nsteps, double *t_out);

/* One sweep T_axis(tau) of f in place (Sec. 2.1).  axis 0..2: drift along
 * x, y, z with the cell-centre velocity; axis 3..5: kick along vx, vy, vz
 * with the context's current acceleration g.  tau may be negative. */
int vp_sweep(vp_ctx *ctx, int axis, double tau);

/* rho(x) = sum_v f dv_x dv_y dv_z of the current f into rho_dev
 * (N_x N_y N_z doubles, device), compensated summation (Sec. 2.2). */
int vp_moments(vp_ctx *ctx, double *rho_dev);

/* Copies the context's rho, phi (box part) and g (3 N_x N_y N_z) into
 * caller device buffers; any pointer may be NULL.  These are the fields of
 * the last field solve. */
int vp_get_field(vp_ctx *ctx, double *rho_dev, double *phi_dev, double *g_dev);

/* Replaces the context's acceleration g (3 N_x N_y N_z doubles, device). */
int vp_set_accel(vp_ctx *ctx, const double *g_dev);

/* Diagnostics of the current f (Sec. 3.1, 3.2): out[0] = M = sum f dV,
 * out[1] = K = 1/2 sum f |v|^2 dV (cell-centre v), out[2] = U = 1/2 sum
 * rho phi dV_x, out[3] = E = K + U, out[4] = mass that left through
 * outflow faces since vp_init.  Solves the Poisson equation of the
 * current f without touching g.  Synchronises the stream. */
int vp_energy(vp_ctx *ctx, double out[5]);

/* Simulated time and the dt of the last step (synchronises). */
int vp_time(vp_ctx *ctx, double *t, double *dt_last);

/* End-to-end call on host buffers: copies f_host_in (host memory, same
 * layout and dtype as f, ideally pinned) into the context's f, recomputes
 * g from it, advances nsteps split steps, writes the simulated time into
 * *t_out (host, may be NULL), the diagnostics of vp_energy into
 * diag_out[5] (host, may be NULL) and, when f_host_out is not NULL,
 * copies the result back to it.  Synchronises the stream. */
int vp_step_host(vp_ctx *ctx, const void *f_host_in, void *f_host_out, int nsteps,
                 double *t_out, double *diag_out);

/* Tracing: runs one split step (drift, density, field, tables and the
 * fused 6-sweep kick of the steady state) without CUDA graphs, with CUDA
 * events on the context's stream around each kernel family, and writes
 * the elapsed milliseconds into ms_out[VP_PROFILE_SLOTS] (host):
 *   [0] fused kick pass (6 velocity sweeps)   [1] drift z
 *   [2] drift y                                [3] drift x
 * (where the z and y drifts run as one fused pass, [1] holds that pass
 * and [2] brackets no kernel),
 *   [4] density reduction                      [5] Poisson + force
 *   [6] dt, shift tables, time                 [7] whole step
 *   [8], [9], [10] the three passes of the fused kick of 48^3 velocity
 *   cubes (vx+vy, vz+vx, vy+vz; [0] is their sum); 0 for other cubes, whose
 *   fused kick is one pass.
 * The first and last half kicks around the timed body run untimed, so f
 * advances by two split steps, exactly as vp_step(ctx, 2).  Synchronises. */
#define VP_PROFILE_SLOTS 11
int vp_profile_step(vp_ctx *ctx, double *ms_out);

/* Number of kernels vp_step has launched on the device since vp_init
 * (graph kernel nodes times replays). */
int vp_stats(vp_ctx *ctx, long long *kernels_launched);

/* Scans the current f (one read; synchronises the stream): counts[0] =
 * cells that are NaN or infinite, counts[1] = cells below zero (the scheme
 * keeps f >= 0, Sec. 2.1); counts (host, 2 entries) may be NULL.  Returns
 * VP_ERR_NONFINITE if either count is non-zero, else VP_OK. */
int vp_check(vp_ctx *ctx, long long counts[2]);

/* Fault injection for tests (not in the paper): the k-th device allocation
 * the library's context set-up makes after this call fails as if the
 * device were out of memory, so that the VP_ERR_OOM paths and their
 * clean-up can be exercised without exhausting the device; k = 0 switches
 * it off.  Process-wide; VP_ERR_ARG for k < 0. */
int vp_debug_fail_alloc(int k);

/* Discrete adjoint of one split step (not in the paper; limiter branches,
 * integer shifts and line-maximum positions frozen at the forward pass).
 * Requires dt_fixed > 0 (VP_ERR_STATE otherwise).  On first use the
 * context allocates its scratch states plus small tables: the inputs of the
 * sweeps of the replayed step that its adjoint reads (at most eight states
 * of f's size; six for FP32 velocity cubes of edge 16 or 32 with fused y+z
 * drifts) or, where they do not fit or vp_set_adjoint_states asks for it,
 * three or two states with which the inputs are recomputed from f_start in
 * partial replays (12 or 15 passes over f against the forward step's
 * six); VP_ERR_OOM if even two do not fit.
 *   f_start: the step-start f^n (device, same layout/dtype as f; read only)
 *   g_start: the step-start acceleration g^n (3 N^p doubles, device)
 *   lambda_f: in: cotangent of f^{n+1}; out: cotangent of f^n (device,
 *             same layout and dtype as f)
 *   lambda_g: in: cotangent of g^{n+1}; out: cotangent of g^n (3 N^p
 *             doubles, device)
 * The context's own f is not modified; the context's scratch is used to
 * replay the forward step. */
/* Scratch policy of vp_adjoint_step (not in the paper): 0 automatic (the
 * kept sweep inputs if they fit, else three states, else two), 1 two
 * states (the sweep inputs recomputed), 2 the kept sweep inputs, 3 three
 * states (fewer recomputed than with two).  Frees the scratch held so far;
 * VP_ERR_ARG for another mode. */
int vp_set_adjoint_states(vp_ctx *ctx, int mode);

int vp_adjoint_step(vp_ctx *ctx, const void *f_start, const double *g_start,
                    void *lambda_f, double *lambda_g);

/* Adjoint of one sweep T_axis(tau) (as vp_sweep) at the input f_in (device,
 * f layout and dtype): lambda (device, same layout and dtype) holds the
 * cotangent of the sweep output on entry and that of the input on exit.
 * For velocity axes the cotangent of the acceleration component is added
 * to lambda_g (3 N^p doubles, device; may be NULL).  The kick shifts use the
 * context's current g. */
int vp_sweep_adjoint(vp_ctx *ctx, int axis, double tau, const void *f_in, void *lambda,
                     double *lambda_g);

/* Adds to lambda_f (device, f layout and dtype) the cotangent of f that
 * flows back through g = -grad phi[rho(f)] from lambda_g (3 N^p doubles,
 * device).  Used for g^0 = field(f^0) at the start of a trajectory. */
int vp_field_adjoint(vp_ctx *ctx, const double *lambda_g, void *lambda_f);

/* Cotangent of f for a final-time functional of the current f:
 * kind 0: J = U = 1/2 sum rho phi dV_x; kind 1: J = 1/2 sum (rho -
 * target)^2 dV_x with target (N^p doubles, device).  Writes dJ/df into
 * lambda_f (device, f layout and dtype) and J into *J_out (host; this
 * synchronises). */
int vp_functional(vp_ctx *ctx, int kind, const double *target, void *lambda_f,
                  double *J_out);

/* ---------------------------------------------------------------------
 * Position space cut into slabs along x, one slab per GPU (the
 * decomposition of Sec. 2.3: position space divided among the processes,
 * velocity space kept whole).  A slab's context is made by vp_init with the
 * slab's own grid (n[0] = its planes, box_lo[0]/box_hi[0] its extent, the
 * same cell widths).  Kicks and the y and z drifts are slab-local
 * (vp_kick, vp_drift_yz); the x drift needs the neighbours' planes and the maximum of
 * every whole x line (vp_line_max_x, vp_drift_x_ghosted); the field is
 * solved from the gathered density by a field-only context of the whole
 * grid (vp_field_init, vp_field_solve) on every GPU, and the slab's part of
 * g is handed to the slab's context (vp_set_accel).  The exchanges between
 * GPUs are the caller's (paper_1206_6152_gb300/sharded.py: all-reduce of the
 * line maxima, halo planes, all-gather of the density).  Periodic position
 * space only.
 * ------------------------------------------------------------------- */

/* The velocity sweeps of a half kick, T_vx T_vy T_vz (Sec. 2.1, Eq.
 * (adv_vel)), in place, with the context's acceleration (vp_set_accel) and
 * duration tau1; with tau2 != 0 followed by a second half kick of duration
 * tau2 with the same acceleration (K2 of step n and K1 of step n+1, which
 * share g^{n+1}), in the passes over f of the step's own fused kick (one
 * pass for cubes of 16 and 32, three for 48).  Results as six vp_sweep
 * calls.  VP_ERR_ARG for a non-finite tau; asynchronous. */
int vp_kick(vp_ctx *ctx, double tau1, double tau2);

/* The z then the y drift, T_z(tau) T_y(tau) (Sec. 2.1, Eq. (adv_xpos)), in
 * place, in one pass where the fused drift kernel applies (FP32, N_y = N_z
 * in {16, 32}, no whole-cell shift), else one pass each.  Results as two
 * vp_sweep calls.  VP_ERR_ARG for a non-finite tau; asynchronous. */
int vp_drift_yz(vp_ctx *ctx, double tau);

/* Per-line maxima along x of the context's f: lmax_dev[(y, z, v)] = max(0,
 * max_i f[i][y][z][v]) over the slab's planes, laid out [ny][nz][nvx][nvy]
 * [nvz] in f's dtype (device, ny nz nvx nvy nvz elements, caller-owned).
 * The maximum of a whole line (f_inf of Sec. 2.1) is the maximum of these
 * over the slabs.  Asynchronous.  VP_ERR_STATE for a field-only context. */
int vp_line_max_x(vp_ctx *ctx, void *lmax_dev);

/* The x drift T_x(tau) (Sec. 2.1, Eq. (adv_xpos)) of the context's slab,
 * in place, for x lines that continue beyond it: ghost_lo holds the nghost
 * planes below the slab (the lower neighbour's last planes; in periodic
 * space the last planes of the whole box for the first slab), ghost_hi the
 * nghost planes above it, each laid out [nghost][ny][nz][nvx][nvy][nvz] in
 * f's dtype (device, caller-owned, read only); lmax_dev the maxima of the
 * whole lines (vp_line_max_x reduced over the slabs).  The update of a cell
 * reads up to floor(|alpha|) + 2 cells upwind and one downwind, so nghost
 * must be at least floor(max |v_x| tau / dx) + 2; else VP_ERR_ARG.
 * Asynchronous. */
int vp_drift_x_ghosted(vp_ctx *ctx, double tau, const void *ghost_lo, const void *ghost_hi,
                       int nghost, const void *lmax_dev);

/* A context for the field alone (Sec. 2.2: Poisson and force on the
 * config's grid, periodic or isolated), with no distribution function:
 * vp_field_solve, vp_get_field and vp_destroy only (the calls that need f
 * return VP_ERR_STATE).  Errors as vp_init. */
int vp_field_init(const vp_config *cfg, void *cuda_stream, vp_ctx **out);

/* phi and g = -grad phi of the density rho_dev (device, N_x N_y N_z
 * doubles) on the context's grid; g is copied to g_dev (device, 3 N_x N_y
 * N_z doubles, [axis][x][y][z]) unless NULL.  With dt_out (host), also the
 * timestep of Sec. 2.4 for that g (the fixed dt if configured); that
 * synchronises.  VP_ERR_NONFINITE for a non-finite dt. */
int vp_field_solve(vp_ctx *ctx, const double *rho_dev, double *g_dev, double *dt_out);

/* Allocation-free moments (the paper has no counterpart; this is a service
 * for callers that cannot allocate device memory when they need the
 * diagnostic -- e.g. code inside a CUDA stream capture, which an allocation
 * would break, or an application whose device memory is handed out by its
 * own allocator and fixed after start-up).  No context is needed and no
 * device memory is allocated or freed.
 *   f_dev:    distribution function (device, layout above), dtype 0 float /
 *             1 double, spatial grid n[3], velocity grid nv[3] on
 *             [vlo, vhi) (host arrays)
 *   sums_dev: output, 2 doubles on the device: sums_dev[0] = sum f and
 *             sums_dev[1] = sum f |v|^2 over all cells (cell-centre v,
 *             compensated sums; multiply by dV = dx^3 dv^3, and by 1/2 for
 *             K, to get the M and K of vp_energy)
 * Asynchronous on cuda_stream.  The per-cell partial sums live in one
 * static device array of the library sized for at most 262144 spatial cells
 * (64^3; 4 MiB, held on every GPU that loads the library until the process
 * exits); larger grids return VP_ERR_UNSUPPORTED.  f_dev and sums_dev must
 * be device memory of the current device, else VP_ERR_ARG (checked with
 * cudaPointerGetAttributes before any launch).  The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress) and
 * caches it with the id of the current CUDA context, so make the first call
 * on a device before any stream capture; after a device reset the next
 * call, made in the new context, looks the address up again (make it, too,
 * outside a capture).
 * Every call writes all the partials it reads, so no state carries over
 * between calls, but all calls share the one array: calls that overlap on
 * the GPU (different streams, or a stream and a graph) race and must be
 * serialised by the caller. */
int vp_moments_noalloc(const void *f_dev, int dtype, const int n[3], const int nv[3],
                       const double vlo[3], const double vhi[3], double *sums_dev,
                       void *cuda_stream);

/* Releases everything the context owns (not f). */
void vp_destroy(vp_ctx *ctx);

/* Static description of an error code. */
const char *vp_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* VP_H */
