/*
 * vp_oracle.c -- plain FP64 CPU oracle of the PFC Vlasov sweeps.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header or constant with the CUDA path and is deliberately slow:
 * every sweep walks every line one cell at a time, in the order and the
 * notation of Yoshikawa, Yoshida & Umemura, "Direct integration of the
 * collisionless Boltzmann equation in six-dimensional phase space:
 * self-gravitating systems", Sec. 2.1.
 *
 * Paper references (section / equation):
 *   Sec. 2.1, Eq. (1d_adv)      df/dt + u df/dx = 0 on a line of cells
 *   Sec. 2.1, cell averages     f_i = (1/dx) * integral of f over cell i
 *   Sec. 2.1, Eqs. (phi_plus), (phi_minus)
 *                               Phi^+ / Phi^-: integral of f(t^n) from the
 *                               foot of the characteristic to the right /
 *                               left face of the cell, in units of dx
 *   Sec. 2.1, update            f_i^{n+1} = f_i^n + Phi^- - Phi^+
 *   Sec. 2.1, reconstruction    third-order reconstruction with the slope
 *                               corrector of Filbet, Sonnendruecker &
 *                               Bertrand (2001); the corrector uses the
 *                               maximum of f over the whole 1D line
 *                               (Sec. 4, discussion of the line maximum)
 *   Sec. 2.1, boundaries        outflow in velocity (matter beyond V^+/-
 *                               vanishes), periodic or outflow in position
 *   Sec. 2.2, density           rho(x) = integral of f over velocity
 *
 * The slope corrector is the published one of Filbet et al. (2001), written
 * in its ratio form  eps = min(1, 2 f / (f_{j+1} - f_j))  etc.; the paper
 * cites it without printing it.
 *
 * Readings where the paper is silent:
 *   - the line maximum f_inf is the maximum of f over the in-domain cells
 *     of the line being swept, taken at t^n;
 *   - outflow ghost cells hold f = 0 and their own partial integral is
 *     evaluated with the same formula (it vanishes);
 *   - u < 0 is the mirror image of u > 0: reflect the line, advect with |u|,
 *     reflect back;
 *   - a negative result can only come from rounding (PFC is positive in
 *     exact arithmetic); it is set to 0.
 *
 * The adjoint sweeps (not in the paper) differentiate this forward code
 * with every limiter branch, the integer part of the shift and the argmax
 * of f_inf frozen at the forward input.  Rounding-only clamps are treated
 * as inactive.
 */
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* one line                                                            */
/* ------------------------------------------------------------------ */

/* Cell value with the ghost rule of Sec. 2.1: periodic wrap, or 0 beyond
 * an outflow boundary. */
static double cell(const double *f, long n, long j, int periodic)
{
    if (periodic) {
        long m = j % n;
        if (m < 0) m += n;
        return f[m];
    }
    return (j < 0 || j >= n) ? 0.0 : f[j];
}

/* Filbet's slope corrector applied to the forward difference:
 * returns eps^+_j * (f_{j+1} - f_j). */
static double eps_plus_diff(double f0, double fp, double finf)
{
    double d = fp - f0;
    double eps = 1.0;
    if (d > 0.0) {
        double r = 2.0 * f0 / d;
        if (r < eps) eps = r;
    } else if (d < 0.0) {
        double r = -2.0 * (finf - f0) / d;
        if (r < eps) eps = r;
    }
    return eps * d;
}

/* Filbet's slope corrector applied to the backward difference:
 * returns eps^-_j * (f_j - f_{j-1}). */
static double eps_minus_diff(double fm, double f0, double finf)
{
    double d = f0 - fm;
    double eps = 1.0;
    if (d > 0.0) {
        double r = 2.0 * (finf - f0) / d;
        if (r < eps) eps = r;
    } else if (d < 0.0) {
        double r = -2.0 * f0 / d;
        if (r < eps) eps = r;
    }
    return eps * d;
}

/* Integral of the corrected third-order reconstruction of f over the
 * rightmost fraction beta of cell j, divided by dx (Sec. 2.1: the
 * reconstruction with Filbet's slope corrector that the fluxes of
 * Eqs. (phi_plus), (phi_minus) integrate).  For beta in [0,1] this is the
 * piece of Phi at the right face of cell j contributed by cell j itself. */
static double partial_integral(const double *f, long n, long j, double beta,
                               double finf, int periodic)
{
    double fm = cell(f, n, j - 1, periodic);
    double f0 = cell(f, n, j, periodic);
    double fp = cell(f, n, j + 1, periodic);
    double wp = beta * (1.0 - beta) * (2.0 - beta) / 6.0;
    double wm = beta * (1.0 - beta) * (1.0 + beta) / 6.0;
    return beta * f0 + wp * eps_plus_diff(f0, fp, finf)
                     + wm * eps_minus_diff(fm, f0, finf);
}

/* Phi at the right face of cell i (i.e. at x_{i+1/2}), Eq. (phi_plus), for
 * a shift alpha = u dt / dx = s + beta >= 0: the foot of the characteristic
 * through x_{i+1/2} lies a fraction beta from the right face of cell
 * i - s, so Phi = (whole cells i-s+1 .. i) + (part of cell i-s). */
static double face_flux(const double *f, long n, long i, long s, double beta,
                        double finf, int periodic)
{
    double phi = 0.0;
    for (long k = i - s + 1; k <= i; ++k) phi += cell(f, n, k, periodic);
    phi += partial_integral(f, n, i - s, beta, finf, periodic);
    return phi;
}

/* Forward PFC update of one line with alpha >= 0 (Sec. 2.1, Eq. (conserve)
 * as f_i + Phi^- - Phi^+, the line maximum taken at t^n); a rounding-negative
 * result is set to 0. */
static void pfc_line_pos_max(const double *f, double *out, long n, double alpha,
                             int periodic, double finf)
{
    long s = (long)floor(alpha);
    double beta = alpha - (double)s;
    for (long i = 0; i < n; ++i) {
        double phi_minus = face_flux(f, n, i - 1, s, beta, finf, periodic);
        double phi_plus = face_flux(f, n, i, s, beta, finf, periodic);
        double v = f[i] + phi_minus - phi_plus;
        out[i] = v > 0.0 ? v : 0.0;
    }
}

static void pfc_line_pos(const double *f, double *out, long n, double alpha,
                         int periodic)
{
    double finf = 0.0;
    for (long j = 0; j < n; ++j) if (f[j] > finf) finf = f[j];
    pfc_line_pos_max(f, out, n, alpha, periodic, finf);
}

/* Public: one line, any sign of alpha (u < 0 as the mirror image of u > 0,
 * Sec. 2.1).  fin and fout may alias. */
void oracle_pfc_line(const double *fin, double *fout, long n, double alpha,
                     int periodic)
{
    double a[n], b[n];
    if (alpha >= 0.0) {
        memcpy(a, fin, sizeof(double) * (size_t)n);
        pfc_line_pos(a, b, n, alpha, periodic);
        memcpy(fout, b, sizeof(double) * (size_t)n);
    } else {
        for (long j = 0; j < n; ++j) a[j] = fin[n - 1 - j];
        pfc_line_pos(a, b, n, -alpha, periodic);
        for (long j = 0; j < n; ++j) fout[j] = b[n - 1 - j];
    }
}

/* Public: the update of the n cells of a piece of a longer line (the
 * decomposition of position space into slabs, Sec. 2.3).  ext holds the
 * piece with G cells of the line on each side (ext[G + j] = cell j,
 * j in [-G, n + G)), finf is the maximum of the whole line.  A cell's update
 * reads cells i - s - 2 .. i + 1 (u >= 0; mirrored for u < 0) and finf only,
 * so with G >= floor(|alpha|) + 2 it is, bit for bit, the one
 * oracle_pfc_line computes on the whole line. */
void oracle_pfc_line_ghosted(const double *ext, double *out, long n, long G, double alpha,
                             double finf)
{
    const long m = n + 2 * G;
    double a[m], b[m];
    if (alpha >= 0.0) {
        memcpy(a, ext, sizeof(double) * (size_t)m);
        pfc_line_pos_max(a, b, m, alpha, 0, finf);
        memcpy(out, b + G, sizeof(double) * (size_t)n);
    } else {
        for (long j = 0; j < m; ++j) a[j] = ext[m - 1 - j];
        pfc_line_pos_max(a, b, m, -alpha, 0, finf);
        for (long j = 0; j < n; ++j) out[j] = b[m - 1 - (G + j)];
    }
}

/* ------------------------------------------------------------------ */
/* adjoint of one line (frozen branches)                               */
/* ------------------------------------------------------------------ */

/* Adds the cotangent c of eps^+ (f_{j+1}-f_j) to lam (cells j, j+1) and
 * to *lfinf, following the branch the forward pass took. */
static void eps_plus_diff_adj(double f0, double fp, double finf, double c,
                              double *l0, double *lp, double *lfinf)
{
    double d = fp - f0;
    if (d > 0.0 && 2.0 * f0 < d) {            /* limited: 2 f_j */
        *l0 += 2.0 * c;
    } else if (d < 0.0 && -2.0 * (finf - f0) > d) {  /* -2(finf - f_j) */
        *l0 += 2.0 * c;
        *lfinf -= 2.0 * c;
    } else {                                  /* unlimited: f_{j+1}-f_j */
        *lp += c;
        *l0 -= c;
    }
}

static void eps_minus_diff_adj(double fm, double f0, double finf, double c,
                               double *lm, double *l0, double *lfinf)
{
    double d = f0 - fm;
    if (d > 0.0 && 2.0 * (finf - f0) < d) {  /* 2(finf - f_j) */
        *lfinf += 2.0 * c;
        *l0 -= 2.0 * c;
    } else if (d < 0.0 && -2.0 * f0 > d) {   /* -2 f_j */
        *l0 -= 2.0 * c;
    } else {                                  /* unlimited: f_j - f_{j-1} */
        *l0 += c;
        *lm -= c;
    }
}

/* Index of an in-domain cell after the ghost rule of Sec. 2.1, or -1 for a
 * ghost. */
static long cell_index(long n, long j, int periodic)
{
    if (periodic) {
        long m = j % n;
        if (m < 0) m += n;
        return m;
    }
    return (j < 0 || j >= n) ? -1 : j;
}

static void add_at(double *lam, long n, long j, int periodic, double v)
{
    long m = cell_index(n, j, periodic);
    if (m >= 0) lam[m] += v;
}

/* Reverse of partial_integral (the adjoint is not in the paper; the arms
 * of the corrector are frozen): cotangent psi of P_j(beta).  Returns the
 * contribution psi * dP_j/dbeta. */
static double partial_integral_adj(const double *f, long n, long j,
                                   double beta, double finf, int periodic,
                                   double psi, double *lam, double *lfinf)
{
    double fm = cell(f, n, j - 1, periodic);
    double f0 = cell(f, n, j, periodic);
    double fp = cell(f, n, j + 1, periodic);
    double wp = beta * (1.0 - beta) * (2.0 - beta) / 6.0;
    double wm = beta * (1.0 - beta) * (1.0 + beta) / 6.0;
    double dwp = (2.0 - 6.0 * beta + 3.0 * beta * beta) / 6.0;
    double dwm = (1.0 - 3.0 * beta * beta) / 6.0;
    double ep = eps_plus_diff(f0, fp, finf);
    double em = eps_minus_diff(fm, f0, finf);
    double lm = 0.0, l0 = 0.0, lp = 0.0;
    l0 += beta * psi;
    eps_plus_diff_adj(f0, fp, finf, wp * psi, &l0, &lp, lfinf);
    eps_minus_diff_adj(fm, f0, finf, wm * psi, &lm, &l0, lfinf);
    add_at(lam, n, j - 1, periodic, lm);
    add_at(lam, n, j, periodic, l0);
    add_at(lam, n, j + 1, periodic, lp);
    return psi * (f0 + dwp * ep + dwm * em);
}

/* Adjoint of pfc_line_pos (not in the paper; frozen arms, the rounding
 * guard inactive, the line-maximum cotangent to its first position):
 * lout = cotangent of out, lin = cotangent of f (overwritten).  Returns
 * dJ/dalpha. */
static double pfc_line_pos_adj(const double *f, const double *lout,
                               double *lin, long n, double alpha, int periodic)
{
    long s = (long)floor(alpha);
    double beta = alpha - (double)s;
    double finf = 0.0;
    long arg = 0;
    for (long j = 0; j < n; ++j)
        if (f[j] > finf) { finf = f[j]; arg = j; }
    double lfinf = 0.0, dbeta = 0.0;
    for (long j = 0; j < n; ++j) lin[j] = lout[j];       /* f_i term */
    /* face m+1/2 carries Phi; cell m+1 adds it (Phi^-), cell m subtracts
     * it (Phi^+) */
    long mlo = periodic ? 0 : -1;
    for (long m = mlo; m < n; ++m) {
        double psi = 0.0;
        if (periodic) {
            psi = lout[(m + 1) % n] - lout[m];
        } else {
            if (m + 1 < n) psi += lout[m + 1];
            if (m >= 0) psi -= lout[m];
        }
        if (psi == 0.0) continue;
        for (long k = m - s + 1; k <= m; ++k) add_at(lin, n, k, periodic, psi);
        dbeta += partial_integral_adj(f, n, m - s, beta, finf, periodic, psi,
                                      lin, &lfinf);
    }
    lin[arg] += lfinf;
    return dbeta;
}

/* Public: adjoint of oracle_pfc_line.  Returns dJ/dalpha. */
double oracle_pfc_line_adjoint(const double *fin, const double *lout,
                               double *lin, long n, double alpha, int periodic)
{
    double a[n], la[n], lb[n];
    double dalpha;
    if (alpha >= 0.0) {
        memcpy(a, fin, sizeof(double) * (size_t)n);
        memcpy(la, lout, sizeof(double) * (size_t)n);
        dalpha = pfc_line_pos_adj(a, la, lb, n, alpha, periodic);
        memcpy(lin, lb, sizeof(double) * (size_t)n);
    } else {
        for (long j = 0; j < n; ++j) {
            a[j] = fin[n - 1 - j];
            la[j] = lout[n - 1 - j];
        }
        dalpha = -pfc_line_pos_adj(a, la, lb, n, -alpha, periodic);
        for (long j = 0; j < n; ++j) lin[j] = lb[n - 1 - j];
    }
    return dalpha;
}

/* ------------------------------------------------------------------ */
/* sweeps over the 6D array f[x][y][z][vx][vy][vz] (last index fastest) */
/* ------------------------------------------------------------------ */

/* Line geometry of axis `axis` in a C-ordered array of 6 dims. */
static void line_geometry(const long dims[6], int axis, long *n, long *stride,
                          long *nlines)
{
    long st = 1;
    for (int a = 5; a > axis; --a) st *= dims[a];
    long total = 1;
    for (int a = 0; a < 6; ++a) total *= dims[a];
    *n = dims[axis];
    *stride = st;
    *nlines = total / dims[axis];
}

/* Start offset of line `l` and the index that selects its speed:
 * for a position axis the velocity index along the same direction
 * (u = v cell centre, Sec. 2.1 Eqs. adv_xpos..adv_zpos), for a velocity
 * axis the spatial cell (u = -dphi/dx there, Eqs. adv_xvel..adv_zvel). */
static void line_start(const long dims[6], int axis, long l, long *start,
                       long *speed_index)
{
    long idx[6];
    long rem = l;
    for (int a = 5; a >= 0; --a) {
        if (a == axis) { idx[a] = 0; continue; }
        idx[a] = rem % dims[a];
        rem /= dims[a];
    }
    long off = 0;
    for (int a = 0; a < 6; ++a) off = off * dims[a] + idx[a];
    *start = off;
    if (axis < 3)
        *speed_index = idx[3 + axis];
    else
        *speed_index = (idx[0] * dims[1] + idx[1]) * dims[2] + idx[2];
}

/* T_axis(tau), Sec. 2.1: PFC update of every line along `axis`.
 * speed: axis < 3 -> dims[3+axis] cell-centre velocities;
 *        axis >= 3 -> dims[0]*dims[1]*dims[2] accelerations.
 * Returns the sum of f (unscaled) that left through outflow faces. */
double oracle_sweep(double *f, const long dims[6], int axis,
                    const double *speed, double tau, double h, int periodic)
{
    long n, stride, nlines;
    line_geometry(dims, axis, &n, &stride, &nlines);
    double lost = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : lost)
    for (long l = 0; l < nlines; ++l) {
        long start, si;
        line_start(dims, axis, l, &start, &si);
        double a[n];
        double before = 0.0, after = 0.0;
        for (long j = 0; j < n; ++j) {
            a[j] = f[start + j * stride];
            before += a[j];
        }
        double alpha = speed[si] * tau / h;
        oracle_pfc_line(a, a, n, alpha, periodic);
        for (long j = 0; j < n; ++j) {
            f[start + j * stride] = a[j];
            after += a[j];
        }
        if (!periodic) lost += before - after;
    }
    return lost;
}

/* The x sweep of a slab of nx = dims[0] position planes (Sec. 2.3's
 * decomposition): every x line continues into G planes below (glo) and
 * above (ghi) the slab, each laid out as [G][ny][nz][nv...], and has the
 * maximum lmax[(y, z, v)] over the whole line.  out receives the slab's
 * updated planes.  speed: the dims[3] cell-centre velocities along x. */
void oracle_sweep_x_ghosted(const double *f, const double *glo, const double *ghi,
                            double *out, const long dims[6], long G, const double *speed,
                            double tau, double h, const double *lmax)
{
    const long nx = dims[0];
    long nl = 1;
    for (int a = 1; a < 6; ++a) nl *= dims[a];
    const long nvc = dims[3] * dims[4] * dims[5];
#pragma omp parallel for schedule(static)
    for (long l = 0; l < nl; ++l) {
        double ext[nx + 2 * G], res[nx];
        for (long j = 0; j < G; ++j) {
            ext[j] = glo[j * nl + l];
            ext[G + nx + j] = ghi[j * nl + l];
        }
        for (long i = 0; i < nx; ++i) ext[G + i] = f[i * nl + l];
        const long vx = (l % nvc) / (dims[4] * dims[5]);
        const double alpha = speed[vx] * tau / h;
        oracle_pfc_line_ghosted(ext, res, nx, G, alpha, lmax[l]);
        for (long i = 0; i < nx; ++i) out[i * nl + l] = res[i];
    }
}

/* Adjoint of oracle_sweep at input fin (not in the paper; frozen arms).
 * lam: cotangent of the output on entry, of the input on exit.  dspeed (may
 * be NULL) accumulates dJ/du. */
void oracle_sweep_adjoint(const double *fin, double *lam, const long dims[6],
                          int axis, const double *speed, double tau, double h,
                          int periodic, double *dspeed)
{
    long n, stride, nlines;
    line_geometry(dims, axis, &n, &stride, &nlines);
    double *dline = (double *)calloc((size_t)nlines, sizeof(double));
    long *sidx = (long *)malloc(sizeof(long) * (size_t)nlines);
#pragma omp parallel for schedule(static)
    for (long l = 0; l < nlines; ++l) {
        long start, si;
        line_start(dims, axis, l, &start, &si);
        sidx[l] = si;
        double a[n], lo[n], li[n];
        for (long j = 0; j < n; ++j) {
            a[j] = fin[start + j * stride];
            lo[j] = lam[start + j * stride];
        }
        double alpha = speed[si] * tau / h;
        double dalpha = oracle_pfc_line_adjoint(a, lo, li, n, alpha, periodic);
        for (long j = 0; j < n; ++j) lam[start + j * stride] = li[j];
        dline[l] = dalpha * tau / h;
    }
    if (dspeed)
        for (long l = 0; l < nlines; ++l) dspeed[sidx[l]] += dline[l];
    free(dline);
    free(sidx);
}

/* ------------------------------------------------------------------ */
/* reductions (Neumaier compensated summation)                         */
/* ------------------------------------------------------------------ */

static void neumaier_add(double *s, double *c, double x)
{
    double t = *s + x;
    if (fabs(*s) >= fabs(x))
        *c += (*s - t) + x;
    else
        *c += (x - t) + *s;
    *s = t;
}

/* rho(x) = sum over the velocity cells at x of f, times dvol (Sec. 2.2). */
void oracle_density(const double *f, long np, long nv, double dvol,
                    double *rho)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < np; ++p) {
        double s = 0.0, c = 0.0;
        const double *q = f + p * nv;
        for (long v = 0; v < nv; ++v) neumaier_add(&s, &c, q[v]);
        rho[p] = (s + c) * dvol;
    }
}

/* Sums of f and of f |v|^2 over the whole array (unscaled; the M and K of
 * Sec. 3.1, Eqs. (total_mass), (kinetic_energy), before the volume
 * factors); v2[v] is |v|^2 at the cell centre of velocity cell v.
 * out[0] = sum f, out[1] = sum f v^2. */
void oracle_moments(const double *f, long np, long nv, const double *v2,
                    double *out)
{
    double s0 = 0.0, c0 = 0.0, s2 = 0.0, c2 = 0.0;
    for (long p = 0; p < np; ++p) {
        const double *q = f + p * nv;
        for (long v = 0; v < nv; ++v) {
            neumaier_add(&s0, &c0, q[v]);
            neumaier_add(&s2, &c2, q[v] * v2[v]);
        }
    }
    out[0] = s0 + c0;
    out[1] = s2 + c2;
}

/* Number of threads the OpenMP loops above run on (for reporting). */
int oracle_threads(void) { return omp_get_max_threads(); }
