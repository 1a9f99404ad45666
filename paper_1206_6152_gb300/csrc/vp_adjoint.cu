// vp_adjoint.cu -- discrete adjoint of the split step (not in the paper).
//
// The forward sweep of one line is, in its upwind frame with shift
// |alpha| = s + beta,
//   out_i = f_{i-s} - phi_{i-s} + phi_{i-s-1},
//   phi_j = c0 f_j + c1 E+_j + c2 E-_j,
//   E+_j  = clamp(f_{j+1} - f_j, -2 (finf - f_j), 2 f_j),
//   E-_j  = clamp(f_j - f_{j-1}, -2 f_j, 2 (finf - f_j)),
// c0 = beta, c1 = beta (1-beta)(2-beta)/6, c2 = beta (1-beta)(1+beta)/6 and
// finf the line maximum.  With every clamp arm, the integer shift s and the
// position of the line maximum frozen at the forward input, the map is
// linear in f; its transpose is applied here line by line.  The shift's
// fractional part also depends on the acceleration in velocity sweeps:
//   d out_i / d beta = -phi'_{i-s} + phi'_{i-s-1},
//   phi'_j = f_j + c1'(beta) E+_j + c2'(beta) E-_j,
// which gives the cotangent of g through alpha = g tau / dv.  Arms: an E arm
// is limited only when the difference lies strictly beyond its bound; the
// cotangent of finf goes to the first maximum in upwind order.  The
// rounding guard phi <= f of the forward kernels is treated as inactive.
//
// The field part reverses g = -grad phi, phi = G * rho, rho = dv^3 sum_v f:
// the transposed central difference, the same (symmetric) convolution, and
// a broadcast over velocity.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "vp_device.cuh"
#include "vp_internal.cuh"

int vp_sm_count();

namespace {

struct LineGeom {
    int axis;                 // 0..5
    int n;                    // line length
    // position axes: line (o, v): base = cell(o) * nvc + v
    long long cell_stride;
    int od;
    long long m1, m2;
    // velocity axes: line (cell, w): base = cell * nvc + voff(w), stride vstride
    int wdiv, wmul_hi, wmul_lo;   // voff = (w / wdiv) * wmul_hi + (w % wdiv) * wmul_lo
    long long nvc;
    long long stride;             // element stride along the line
    long long nlines_inner;       // v cells (position axes) or lines per cube (velocity)
    int pairs;                    // fix-up after the pair kernels: a z line whose pair
                                  // partner (v ^ 1) was shifted was skipped as well
    int cube3;                    // fix-up after the fused kick adjoint: every line of a
                                  // cube with a shift on any velocity axis
};

template <typename T>
struct AdjArgs {
    const T *fin;                 // sweep input
    T *lam;                       // in: cotangent of the output, out: of the input
    const LineCoef<T> *coef;      // position axes: [maxnv] of this axis; velocity: [np][3]
    int va_stride, va_n;          // position axes: velocity index along the axis
    int periodic;
    double *lam_g;                // velocity axes: cotangent of g (axis slice), or null
    double dalpha_scale;          // tau / dv
};

template <typename T>
__device__ __forceinline__ T dget(const T *tile, int C, int n, int j, int neg, int periodic, int t)
{
    if (periodic) {
        j %= n;
        if (j < 0) j += n;
    } else if (j < 0 || j >= n) {
        return T(0);
    }
    return tile[(neg ? n - 1 - j : j) * C + t];
}

template <typename T>
__device__ __forceinline__ void dadd(T *tile, int C, int n, int j, int neg, int periodic, int t, T v)
{
    if (periodic) {
        j %= n;
        if (j < 0) j += n;
    } else if (j < 0 || j >= n) {
        return;
    }
    tile[(neg ? n - 1 - j : j) * C + t] += v;
}

// one line: F, LO tiles read-only, LI tile accumulates the input cotangent
template <typename T>
__device__ T line_adjoint(const T *F, const T *LO, T *LI, int C, int t, int n,
                          const LineCoef<T> cf, int periodic)
{
    const int neg = cf.code & 1, s = cf.code >> 1;
    const T c0 = cf.c0, c1 = cf.c1, c2 = cf.c2;
    const T beta = c0;
    const T dc1 = (T(2) - T(6) * beta + T(3) * beta * beta) / T(6);
    const T dc2 = (T(1) - T(3) * beta * beta) / T(6);
    T finf = T(0);
    int arg = 0;
    for (int j = 0; j < n; ++j) {
        const T v = dget(F, C, n, j, neg, 0, t);
        if (v > finf) { finf = v; arg = j; }
    }
    for (int j = 0; j < n; ++j) LI[j * C + t] = T(0);
    T lfinf = T(0), dbeta = T(0);
    for (int j = 0; j < n; ++j) {
        // f_j enters out_{j+s} directly, -phi_j enters out_{j+s}, +phi_j out_{j+s+1}
        const T l1 = (periodic || j + s < n) ? dget(LO, C, n, j + s, neg, periodic, t) : T(0);
        const T l2 = (periodic || j + s + 1 < n) ? dget(LO, C, n, j + s + 1, neg, periodic, t) : T(0);
        dadd(LI, C, n, j, neg, periodic, t, l1);
        const T mu = l2 - l1;
        if (mu == T(0)) continue;
        const T fm = dget(F, C, n, j - 1, neg, periodic, t);
        const T f0 = dget(F, C, n, j, neg, periodic, t);
        const T fp = dget(F, C, n, j + 1, neg, periodic, t);
        T l0 = c0 * mu, lm = T(0), lp = T(0);
        T ep, em;
        // E+ arm
        const T dp = fp - f0;
        if (dp > T(0) && T(2) * f0 < dp) {
            ep = T(2) * f0;
            l0 += T(2) * c1 * mu;
        } else if (dp < T(0) && -T(2) * (finf - f0) > dp) {
            ep = -T(2) * (finf - f0);
            l0 += T(2) * c1 * mu;
            lfinf -= T(2) * c1 * mu;
        } else {
            ep = dp;
            lp += c1 * mu;
            l0 -= c1 * mu;
        }
        // E- arm
        const T dm = f0 - fm;
        if (dm > T(0) && T(2) * (finf - f0) < dm) {
            em = T(2) * (finf - f0);
            lfinf += T(2) * c2 * mu;
            l0 -= T(2) * c2 * mu;
        } else if (dm < T(0) && -T(2) * f0 > dm) {
            em = -T(2) * f0;
            l0 -= T(2) * c2 * mu;
        } else {
            em = dm;
            l0 += c2 * mu;
            lm -= c2 * mu;
        }
        dadd(LI, C, n, j, neg, periodic, t, l0);
        if (lp != T(0)) dadd(LI, C, n, j + 1, neg, periodic, t, lp);
        if (lm != T(0)) dadd(LI, C, n, j - 1, neg, periodic, t, lm);
        dbeta += mu * (f0 + dc1 * ep + dc2 * em);
    }
    dadd(LI, C, n, arg, neg, 0, t, lfinf);
    return neg ? -dbeta : dbeta;
}

// generic line-adjoint kernel: blockIdx.y selects the outer index (position
// axes) or the spatial cell (velocity axes); threads take consecutive lines
// Blocks are virtual: block vb = (bx, by) with bx = vb % vgx, by = vb / vgx,
// vb = blockIdx.x + k gridDim.x, so that the fix-up pass after the register
// kernels (only_shifted) can run on a small grid.
template <typename T>
__device__ void sweep_adjoint_block(const AdjArgs<T> &A, const LineGeom &g, const int *only_shifted,
                                    long long bx, long long by, T *F, T *LO, T *LI, double *red);

template <typename T>
__global__ void __launch_bounds__(128) k_sweep_adjoint(AdjArgs<T> A, LineGeom g,
                                                      const int *only_shifted, long long vgx,
                                                      long long vtotal)
{
    // after the register kernel: nothing to do unless it skipped a line
    if (only_shifted && *only_shifted == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = blockDim.x;
    T *F = reinterpret_cast<T *>(smem_raw);
    T *LO = F + g.n * C;
    T *LI = LO + g.n * C;
    __shared__ double red[32];
    for (long long vb = blockIdx.x; vb < vtotal; vb += gridDim.x) {
        sweep_adjoint_block<T>(A, g, only_shifted, vb % vgx, vb / vgx, F, LO, LI, red);
        __syncthreads();
    }
}

template <typename T>
__device__ void sweep_adjoint_block(const AdjArgs<T> &A, const LineGeom &g, const int *only_shifted,
                                    long long bx, long long by, T *F, T *LO, T *LI, double *red)
{
    const int C = blockDim.x;
    const int n = g.n;
    const int t = threadIdx.x;
    const long long w = bx * C + t;
    bool active = w < g.nlines_inner;
    long long base;
    LineCoef<T> cf;
    if (g.axis < 3) {
        const long long o = by;
        const long long cell0 = (o / g.od) * g.m1 + (o % g.od) * g.m2;
        base = cell0 * g.nvc + w;
        if (active) cf = A.coef[(int)((w / A.va_stride) % A.va_n)];
    } else {
        const long long cell = by;
        const long long voff = (w / g.wdiv) * g.wmul_hi + (w % g.wdiv) * g.wmul_lo;
        base = cell * g.nvc + voff;
        cf = A.coef[cell * 3 + (g.axis - 3)];
    }
    if (only_shifted && active) {
        bool shifted = (cf.code >> 1) != 0;
        if (!shifted && g.cube3 && g.axis >= 3) {
            const LineCoef<T> *cc = A.coef + by * 3;
            shifted = ((cc[0].code >> 1) | (cc[1].code >> 1) | (cc[2].code >> 1)) != 0;
        }
        if (!shifted && g.pairs && g.axis == 2) {
            const long long wp = w ^ 1;
            if (wp < g.nlines_inner)
                shifted = (A.coef[(int)((wp / A.va_stride) % A.va_n)].code >> 1) != 0;
        }
        if (!shifted) active = false;
    }
    for (int j = 0; j < n; ++j) {
        F[j * C + t] = active ? A.fin[base + j * g.stride] : T(0);
        LO[j * C + t] = active ? A.lam[base + j * g.stride] : T(0);
    }
    double da = 0.0;
    if (active) {
        da = (double)line_adjoint<T>(F, LO, LI, C, t, n, cf, A.periodic);
        for (int j = 0; j < n; ++j) A.lam[base + j * g.stride] = LI[j * C + t];
    }
    if (A.lam_g) {
        da = block_sum(da, red);
        if (t == 0 && da != 0.0) atomicAdd(A.lam_g + by, da * A.dalpha_scale);
    }
}

// lam_phi (FFT grid) = transpose of the central-difference force applied to
// lam_g (box): lam_phi[p] = sum_a c_a[p - e_a] - c_a[p + e_a],
// c_a = -lam_g_a / (2 dx_a), zero outside the box
__global__ void k_force_adjoint(const double *__restrict__ lam_g, double *__restrict__ lam_phi,
                                int n0, int n1, int n2, int f0, int f1, int f2, double h0,
                                double h1, double h2)
{
    const long long nf = (long long)f0 * f1 * f2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nf) return;
    const long long np = (long long)n0 * n1 * n2;
    const int k = (int)(t % f2), j = (int)((t / f2) % f1), i = (int)(t / ((long long)f1 * f2));
    auto c = [&](int a, int ii, int jj, int kk) -> double {
        ii = (ii + f0) % f0;
        jj = (jj + f1) % f1;
        kk = (kk + f2) % f2;
        if (ii >= n0 || jj >= n1 || kk >= n2) return 0.0;
        const double h = a == 0 ? h0 : (a == 1 ? h1 : h2);
        return -lam_g[a * np + ((long long)ii * n1 + jj) * n2 + kk] / (2.0 * h);
    };
    double v = c(0, i - 1, j, k) - c(0, i + 1, j, k);
    v += c(1, i, j - 1, k) - c(1, i, j + 1, k);
    v += c(2, i, j, k - 1) - c(2, i, j, k + 1);
    lam_phi[t] = v;
}

__global__ void k_real_to_complex(const double *__restrict__ in, double2 *__restrict__ out,
                                  long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = make_double2(in[t], 0.0);
}

// bc[cell] = dvol_v * lam_rho[cell], lam_rho read from the box part of the
// real part of cbuf
__global__ void k_bc_box(const double2 *__restrict__ cbuf, double *__restrict__ bc, int n1, int n2,
                         int f1, int f2, double dvol_v, long long np)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const int k = (int)(t % n2), j = (int)((t / n2) % n1), i = (int)(t / ((long long)n1 * n2));
    bc[t] = cbuf[((long long)i * f1 + j) * f2 + k].x * dvol_v;
}

// lam_f[cell, v] += bc[cell]
template <typename T>
__global__ void __launch_bounds__(256) k_broadcast_box(T *__restrict__ lam_f,
                                                      const double *__restrict__ bc, long long nvc,
                                                      long long np)
{
    for (long long cell = blockIdx.x; cell < np; cell += gridDim.x) {
        T *q = lam_f + cell * nvc;
        if constexpr (sizeof(T) == 4) {
            // FP32 cotangent: the cell's value rounded once to FP32 and added
            // in FP32 (an FP64 add per element costs GB300 1/64 of the rate)
            const float v = (float)bc[cell];
            if ((nvc & 3) == 0) {
                float4 *q4 = reinterpret_cast<float4 *>(q);
                for (long long e = threadIdx.x; e < nvc / 4; e += blockDim.x) {
                    float4 a = q4[e];
                    a.x += v; a.y += v; a.z += v; a.w += v;
                    q4[e] = a;
                }
            } else {
                for (long long e = threadIdx.x; e < nvc; e += blockDim.x) q[e] += v;
            }
        } else {
            const double v = bc[cell];
            for (long long e = threadIdx.x; e < nvc; e += blockDim.x) q[e] = q[e] + v;
        }
    }
}

template <typename T>
cudaError_t launch_broadcast(vp_ctx *c, const double *bc, T *lam)
{
    long long grid = 8LL * vp_sm_count();
    if (grid > c->np) grid = c->np;
    k_broadcast_box<T><<<(unsigned)grid, 256, 0, c->stream>>>(lam, bc, c->nvc, c->np);
    return cudaGetLastError();
}

// lam_f = scale * w[cell] broadcast over velocity, w = phi (kind 0) or
// rho - target (kind 1)
template <typename T>
__global__ void __launch_bounds__(256) k_functional_grad(T *__restrict__ lam_f,
                                                        const double *__restrict__ phi,
                                                        const double *__restrict__ rho,
                                                        const double *__restrict__ target, int kind,
                                                        long long nvc, int n1, int n2, int f1,
                                                        int f2, double scale, long long np)
{
    for (long long cell = blockIdx.x; cell < np; cell += gridDim.x) {
        double w;
        if (kind == 0) {
            const int k = (int)(cell % n2), j = (int)((cell / n2) % n1);
            const int i = (int)(cell / ((long long)n1 * n2));
            w = phi[((long long)i * f1 + j) * f2 + k];
        } else {
            w = rho[cell] - target[cell];
        }
        const T v = (T)(w * scale);
        T *q = lam_f + cell * nvc;
        for (long long e = threadIdx.x; e < nvc; e += blockDim.x) q[e] = v;
    }
}

// sum (rho - target)^2 (compensated), one CTA
__global__ void k_misfit(const double *__restrict__ rho, const double *__restrict__ target,
                         long long np, double *out)
{
    __shared__ Acc<double> red[32];
    Acc<double> a;
    for (long long t = threadIdx.x; t < np; t += blockDim.x) {
        const double r = rho[t] - target[t];
        a.add(r * r);
    }
    a = block_merge(a, red);
    if (threadIdx.x == 0) out[0] = a.value();
}

// ---------------------------------------------------------------------------
// register-line adjoint (line lengths 16/32/48/64, zero whole-cell shift):
// the line of f, the output cotangent and the input cotangent live in
// registers; the arms are evaluated with the same strict comparisons as
// line_adjoint.  A line with a whole-cell shift is left untouched and
// flagged for the generic kernel.
// ---------------------------------------------------------------------------
template <typename T, int N, bool PERIODIC, bool NEG>
__device__ __forceinline__ T adjoint_regs(const T (&f)[N], const T (&lo)[N], T (&li)[N],
                                          const LineCoef<T> &cf)
{
#define M(j) (NEG ? N - 1 - (j) : (j))
    const T c0 = cf.c0, c1 = cf.c1, c2 = cf.c2;
    const T beta = c0;
    const T dc1 = (T(2) - T(6) * beta + T(3) * beta * beta) / T(6);
    const T dc2 = (T(1) - T(3) * beta * beta) / T(6);
    T finf = T(0);
    int arg = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const T v = f[M(j)];
        if (v > finf) { finf = v; arg = j; }
    }
#pragma unroll
    for (int j = 0; j < N; ++j) li[j] = lo[j];
    T lfinf = T(0), dbeta = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const T lnext = (j + 1 < N) ? lo[M(j + 1)] : (PERIODIC ? lo[M(0)] : T(0));
        const T mu = lnext - lo[M(j)];
        const T fm = (j > 0) ? f[M(j - 1)] : (PERIODIC ? f[M(N - 1)] : T(0));
        const T f0 = f[M(j)];
        const T fp = (j + 1 < N) ? f[M(j + 1)] : (PERIODIC ? f[M(0)] : T(0));
        const T two_f0 = T(2) * f0, two_gap = T(2) * (finf - f0);
        const T dp = fp - f0, dm = f0 - fm;
        const bool pu = dp > T(0) && two_f0 < dp;
        const bool pl = !pu && dp < T(0) && -two_gap > dp;
        const bool mup = dm > T(0) && two_gap < dm;
        const bool mlo = !mup && dm < T(0) && -two_f0 > dm;
        const T ep = pu ? two_f0 : (pl ? -two_gap : dp);
        const T em = mup ? two_gap : (mlo ? -two_f0 : dm);
        const T a = c1 * mu, b = c2 * mu;
        T l0 = c0 * mu;
        l0 += (pu || pl) ? T(2) * a : -a;
        l0 += (mup || mlo) ? -T(2) * b : b;
        lfinf += (pl ? -T(2) * a : T(0)) + (mup ? T(2) * b : T(0));
        li[M(j)] += l0;
        if (!(pu || pl)) {
            if (j + 1 < N) li[M(j + 1)] += a;
            else if (PERIODIC) li[M(0)] += a;
        }
        if (!(mup || mlo)) {
            if (j > 0) li[M(j - 1)] -= b;
            else if (PERIODIC) li[M(N - 1)] -= b;
        }
        dbeta += mu * (f0 + dc1 * ep + dc2 * em);
    }
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (j == arg) li[M(j)] += lfinf;
#undef M
    return NEG ? -dbeta : dbeta;
}

template <typename T, int N, bool PERIODIC, bool ROWS>
__global__ void __launch_bounds__(128) k_adjoint_fast(AdjArgs<T> A, LineGeom g, int *skipped)
{
    __shared__ double red[32];
    const int t = threadIdx.x;
    // velocity axes: blockIdx.x is the cube (any number of cubes), blockIdx.y
    // the chunk of its lines
    const bool vel = g.axis >= 3;
    const long long w = (long long)(vel ? blockIdx.y : blockIdx.x) * blockDim.x + t;
    bool active = w < g.nlines_inner;
    long long base = 0;
    LineCoef<T> cf;
    if (g.axis < 3) {
        const int o = blockIdx.y;
        const long long cell0 = (long long)(o / g.od) * g.m1 + (long long)(o % g.od) * g.m2;
        base = cell0 * g.nvc + w;
        if (active) cf = A.coef[(int)((w / A.va_stride) % A.va_n)];
    } else {
        const long long cell = blockIdx.x;
        const long long voff = (w / g.wdiv) * g.wmul_hi + (w % g.wdiv) * g.wmul_lo;
        base = cell * g.nvc + voff;
        cf = A.coef[cell * 3 + (g.axis - 3)];
    }
    if (active && (cf.code >> 1) != 0) {
        atomicExch(skipped, 1);
        active = false;
    }
    double da = 0.0;
    if (active) {
        T f[N], lo[N], li[N];
        if constexpr (ROWS && sizeof(T) == 4) {
#pragma unroll
            for (int j = 0; j < N; j += 4) {
                const float4 a = *reinterpret_cast<const float4 *>(A.fin + base + j);
                const float4 b = *reinterpret_cast<const float4 *>(A.lam + base + j);
                f[j] = a.x; f[j + 1] = a.y; f[j + 2] = a.z; f[j + 3] = a.w;
                lo[j] = b.x; lo[j + 1] = b.y; lo[j + 2] = b.z; lo[j + 3] = b.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) {
                f[j] = A.fin[base + j * g.stride];
                lo[j] = A.lam[base + j * g.stride];
            }
        }
        const T d = (cf.code & 1) ? adjoint_regs<T, N, PERIODIC, true>(f, lo, li, cf)
                                  : adjoint_regs<T, N, PERIODIC, false>(f, lo, li, cf);
        da = (double)d;
        if constexpr (ROWS && sizeof(T) == 4) {
#pragma unroll
            for (int j = 0; j < N; j += 4)
                *reinterpret_cast<float4 *>(A.lam + base + j) =
                    make_float4(li[j], li[j + 1], li[j + 2], li[j + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) A.lam[base + j * g.stride] = li[j];
        }
    }
    if (A.lam_g) {
        da = block_sum(da, red);
        if (t == 0 && da != 0.0) atomicAdd(A.lam_g + blockIdx.x, da * A.dalpha_scale);
    }
}

int vp_adjoint_fast_ok(const vp_ctx *c, int axis)
{
    const int n = axis < 3 ? c->n[axis] : c->nv[axis - 3];
    if (c->isdouble) return n == 16;
    return n == 16 || n == 32 || n == 48 || n == 64;
}

template <typename T, int N>
cudaError_t adjoint_fast_n(vp_ctx *c, const AdjArgs<T> &A, const LineGeom &g, dim3 grid)
// grid: (line chunks, outer index or cube)
{
    const bool rows = g.stride == 1 && sizeof(T) == 4 && (c->nvc % 4) == 0;
    if (g.axis >= 3) grid = dim3(grid.y, grid.x);        // (cube, chunk)
    if (A.periodic) {
        if (rows) k_adjoint_fast<T, N, true, true><<<grid, 128, 0, c->stream>>>(A, g, c->adj_flag);
        else k_adjoint_fast<T, N, true, false><<<grid, 128, 0, c->stream>>>(A, g, c->adj_flag);
    } else {
        if (rows) k_adjoint_fast<T, N, false, true><<<grid, 128, 0, c->stream>>>(A, g, c->adj_flag);
        else k_adjoint_fast<T, N, false, false><<<grid, 128, 0, c->stream>>>(A, g, c->adj_flag);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_fast(vp_ctx *c, const AdjArgs<T> &A, const LineGeom &g, dim3 grid)
{
    cudaError_t e = cudaMemsetAsync(c->adj_flag, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(T) == 8) {
        return adjoint_fast_n<T, 16>(c, A, g, grid);
    } else {
        switch (g.n) {
        case 16: return adjoint_fast_n<T, 16>(c, A, g, grid);
        case 32: return adjoint_fast_n<T, 32>(c, A, g, grid);
        case 48: return adjoint_fast_n<T, 48>(c, A, g, grid);
        default: return adjoint_fast_n<T, 64>(c, A, g, grid);
        }
    }
}

// bc (position x only): add the density broadcast dvol_v lam_rho[cell] to
// lam before the sweep's adjoint
// cube3: only the fix-up pass after the fused kick adjoint
template <typename T>
cudaError_t sweep_adjoint_t(vp_ctx *c, const T *fin, T *lam, int axis, const LineCoef<T> *coef,
                            double *lam_g, double dalpha_scale, const double *bc = nullptr,
                            int cube3 = 0)
{
    LineGeom g;
    AdjArgs<T> A;
    g.axis = axis;
    g.pairs = 0;
    g.cube3 = cube3;
    g.nvc = c->nvc;
    A.fin = fin;
    A.lam = lam;
    A.lam_g = nullptr;
    A.dalpha_scale = 0.0;
    const int C = 128;
    dim3 grid;
    if (axis < 3) {
        g.n = c->n[axis];
        if (axis == 0) { g.cell_stride = (long long)c->n[1] * c->n[2]; g.od = 1; g.m1 = 1; g.m2 = 0; }
        else if (axis == 1) { g.cell_stride = c->n[2]; g.od = c->n[2]; g.m1 = (long long)c->n[1] * c->n[2]; g.m2 = 1; }
        else { g.cell_stride = 1; g.od = 1; g.m1 = c->n[2]; g.m2 = 0; }
        g.stride = g.cell_stride * c->nvc;
        g.nlines_inner = c->nvc;
        A.coef = coef + (size_t)axis * c->maxnv;
        A.va_stride = axis == 0 ? c->nv[1] * c->nv[2] : (axis == 1 ? c->nv[2] : 1);
        A.va_n = c->nv[axis];
        A.periodic = c->periodic_space;
        grid = dim3((unsigned)((c->nvc + C - 1) / C), (unsigned)(c->np / g.n));
    } else {
        const int va = axis - 3;
        const int nx = c->nv[0], ny = c->nv[1], nz = c->nv[2];
        g.n = c->nv[va];
        if (va == 0) { g.stride = (long long)ny * nz; g.wdiv = nz; g.wmul_hi = nz; g.wmul_lo = 1; g.nlines_inner = (long long)ny * nz; }
        else if (va == 1) { g.stride = nz; g.wdiv = nz; g.wmul_hi = ny * nz; g.wmul_lo = 1; g.nlines_inner = (long long)nx * nz; }
        else { g.stride = 1; g.wdiv = 1; g.wmul_hi = nz; g.wmul_lo = 0; g.nlines_inner = (long long)nx * ny; }
        A.coef = coef;
        A.va_stride = 1;
        A.va_n = 1;
        A.periodic = 0;
        A.lam_g = lam_g ? lam_g + (size_t)va * c->np : nullptr;
        A.dalpha_scale = dalpha_scale;
        grid = dim3((unsigned)((g.nlines_inner + C - 1) / C), (unsigned)c->np);
    }
    const size_t smem = 3 * (size_t)g.n * C * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_sweep_adjoint<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const long long vtotal = (long long)grid.x * grid.y;
    if (cube3) {
        long long small = 4LL * vp_sm_count();
        if (small > vtotal) small = vtotal;
        k_sweep_adjoint<T><<<(unsigned)small, C, smem, c->stream>>>(A, g, c->adj_flag, grid.x, vtotal);
        return cudaGetLastError();
    }
    bool fast = false;
    if constexpr (sizeof(T) == 4) {
        if (vp_adjoint_pairs_ok(c, axis)) {
            e = launch_adjoint_pairs(c, fin, lam, axis, coef, lam_g, dalpha_scale, bc);
            if (e != cudaSuccess) return e;
            fast = true;
            g.pairs = 1;
        }
    }
    if (bc && !fast) {
        if ((e = launch_broadcast(c, bc, lam)) != cudaSuccess) return e;
    }
    if (!fast && vp_adjoint_fast_ok(c, axis)) {
        e = launch_adjoint_fast<T>(c, A, g, grid);
        if (e != cudaSuccess) return e;
        fast = true;
    }
    if (fast) {
        // lines the register kernels skipped (whole-cell shifts), if any
        long long small = 4LL * vp_sm_count();
        if (small > vtotal) small = vtotal;
        k_sweep_adjoint<T><<<(unsigned)small, C, smem, c->stream>>>(A, g, c->adj_flag, grid.x, vtotal);
        return cudaGetLastError();
    }
    k_sweep_adjoint<T><<<(unsigned)vtotal, C, smem, c->stream>>>(A, g, nullptr, grid.x, vtotal);
    return cudaGetLastError();
}

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

#define TRY(x)                      \
    do {                            \
        int _r = (x);               \
        if (_r != VP_OK) return _r; \
    } while (0)

// n slots of f's size, allocated where want[i] (slots marked with the same
// alias share one buffer: alias[i] = i, or the index of the slot whose
// buffer it uses); false (nothing kept) if they do not fit
bool alloc_adjoint_states(vp_ctx *c, int n, const bool *want, const int *alias)
{
    const size_t bytes = (size_t)c->ncells * c->esize;
    c->adj_states = (void **)calloc(n, sizeof(void *));
    if (!c->adj_states) return false;
    c->adj_nstates = n;
    for (int i = 0; i < n; ++i) {
        if (!want[i]) continue;
        if (alias[i] != i) {
            c->adj_states[i] = c->adj_states[alias[i]];
            continue;
        }
        if (cudaMalloc(&c->adj_states[i], bytes) != cudaSuccess) {
            cudaGetLastError();
            vp_free_adjoint_states(c);
            return false;
        }
    }
    return true;
}

// Modes: 0 the nine-slot mode if it fits, else three states, else two; 1
// two states; 2 the nine-slot mode; 3 three states.
// The nine-slot mode keeps S1..S8 (S[k]: the input of sweep k of the step;
// S0 = f^n is the caller's): only the slots the step's path reads — with
// the register kick adjoint S2 and S8 are scratch for the fix-up of
// shifted cubes only and share one buffer, and with the fused y+z drift
// adjoint S4 is not kept.
int ensure_adjoint_scratch(vp_ctx *c)
{
    if (c->adj_states) return VP_OK;
    if (!c->adj_f) {
        const size_t cs = c->isdouble ? sizeof(LineCoef<double>) : sizeof(LineCoef<float>);
        if (!c->adj_flag && cudaMalloc((void **)&c->adj_flag, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return VP_ERR_OOM;
        }
        if (cudaMalloc(&c->adj_f, cs * 3 * c->np) != cudaSuccess ||   // K1 table of the replay
            cudaMalloc((void **)&c->adj_g, sizeof(double) * 3 * c->np) != cudaSuccess ||
            cudaMalloc((void **)&c->adj_lg, sizeof(double) * 3 * c->np) != cudaSuccess ||
            cudaMalloc((void **)&c->adj_tmp, sizeof(double) * c->nfft) != cudaSuccess) {
            cudaGetLastError();
            return VP_ERR_OOM;
        }
    }
    if (c->adj_mode == 0 || c->adj_mode == 2) {
        const bool reg = vp_kick_adjoint3_ok(c);
        const bool yz = vp_drift_alpha_bound(c, c->cfg.dt_fixed) < 1.0 && vp_drift_adjoint_yz_ok(c);
        bool want[9];
        int alias[9];
        for (int i = 0; i < 9; ++i) {
            want[i] = i > 0;
            alias[i] = i;
        }
        if (reg) alias[8] = 2;
        if (yz) want[4] = false;
        if (alloc_adjoint_states(c, 9, want, alias)) return VP_OK;
    }
    if (c->adj_mode == 2) return VP_ERR_OOM;
    const bool all[3] = {true, true, true};
    const int id[3] = {0, 1, 2};
    if (c->adj_mode == 0 || c->adj_mode == 3) {
        if (alloc_adjoint_states(c, 3, all, id)) return VP_OK;
        if (c->adj_mode == 3) return VP_ERR_OOM;
    }
    return alloc_adjoint_states(c, 2, all, id) ? VP_OK : VP_ERR_OOM;
}

// scalar on the device used as the replay's tau
__global__ void k_set(double *p, double v) { *p = v; }

}  // namespace

// frees the adjoint's scratch states (each buffer once: slots may share one)
void vp_free_adjoint_states(vp_ctx *c)
{
    if (!c->adj_states) return;
    for (int i = 0; i < c->adj_nstates; ++i) {
        void *p = c->adj_states[i];
        if (!p) continue;
        bool seen = false;
        for (int j = 0; j < i; ++j) seen |= c->adj_states[j] == p;
        if (!seen) cudaFree(p);
    }
    free(c->adj_states);
    c->adj_states = nullptr;
    c->adj_nstates = 0;
}

cudaError_t launch_drift_adjoint(vp_ctx *c, const void *fin, void *lam, int axis, const void *coef,
                                 const double *bc)
{
    if (c->isdouble)
        return sweep_adjoint_t<double>(c, (const double *)fin, (double *)lam, axis,
                                       (const LineCoef<double> *)coef, nullptr, 0.0, bc);
    return sweep_adjoint_t<float>(c, (const float *)fin, (float *)lam, axis,
                                  (const LineCoef<float> *)coef, nullptr, 0.0, bc);
}

cudaError_t launch_kick_adjoint(vp_ctx *c, const void *fin, void *lam, int vaxis, const void *coef,
                                double tau, double *lam_g)
{
    const double scale = tau / c->dv[vaxis];
    if (c->isdouble)
        return sweep_adjoint_t<double>(c, (const double *)fin, (double *)lam, 3 + vaxis,
                                       (const LineCoef<double> *)coef, lam_g, scale);
    return sweep_adjoint_t<float>(c, (const float *)fin, (float *)lam, 3 + vaxis,
                                  (const LineCoef<float> *)coef, lam_g, scale);
}

// the three velocity-sweep adjoints of a half kick: vz (input sc), vy (sb),
// vx (sa), in that order.  sc may be null when the register path serves the
// grid: the vz input is then recomputed, and for the cubes the register
// kernels skip (whole-cell shifts) it is swept into scratch for the fix-up.
static int kick_adjoint3(vp_ctx *c, const void *sa, const void *sb, const void *sc, void *scratch,
                         void *lam, const void *coef, double tau, double *lam_g)
{
    if (vp_kick_adjoint3_ok(c)) {
        VP_CUDA_TRY(launch_kick_adjoint3(c, sa, sb, lam, coef, lam_g, tau));
        if (!sc) {
            VP_CUDA_TRY(launch_kick_fast(c, const_cast<void *>(sb), coef, nullptr, 1, 1, scratch,
                                         nullptr, nullptr, c->adj_flag));
            sc = scratch;
        }
        const void *S[3] = {sa, sb, sc};
        for (int va = 2; va >= 0; --va)
            VP_CUDA_TRY(sweep_adjoint_t<float>(c, (const float *)S[va], (float *)lam, 3 + va,
                                               (const LineCoef<float> *)coef, lam_g,
                                               tau / c->dv[va], nullptr, 1));
        return VP_OK;
    }
    if (!sc) return VP_ERR_STATE;
    const void *S[3] = {sa, sb, sc};
    for (int va = 2; va >= 0; --va)
        VP_CUDA_TRY(launch_kick_adjoint(c, S[va], lam, va, coef, tau, lam_g));
    return VP_OK;
}

// lam_f += R^T P^T F^T lam_g.  With defer, the density cotangent times
// dvol_v is left in c->rho2 (box layout) for the next sweep adjoint to add
// instead of being broadcast here.
cudaError_t launch_field_adjoint(vp_ctx *c, const double *lam_g, void *lam_f, bool defer)
{
    const int T = 256;
    double *lam_phi = c->phi;   // scratch: the stored potential is recomputed by the next solve
    k_force_adjoint<<<nblk(c->nfft, T), T, 0, c->stream>>>(lam_g, lam_phi, c->n[0], c->n[1], c->n[2],
                                                           c->fn[0], c->fn[1], c->fn[2], c->dx[0],
                                                           c->dx[1], c->dx[2]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_real_to_complex<<<nblk(c->nfft, T), T, 0, c->stream>>>(lam_phi, c->cbuf, c->nfft);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int a = 2; a >= 0; --a)
        if ((e = launch_fft(c, c->cbuf, a, 0)) != cudaSuccess) return e;
    if ((e = launch_green_mul(c)) != cudaSuccess) return e;
    for (int a = 0; a < 3; ++a)
        if ((e = launch_fft(c, c->cbuf, a, 1)) != cudaSuccess) return e;
    k_bc_box<<<nblk(c->np, T), T, 0, c->stream>>>(c->cbuf, c->rho2, c->n[1], c->n[2], c->fn[1],
                                                  c->fn[2], c->dvol_v, c->np);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (defer) return cudaSuccess;
    if (c->isdouble) return launch_broadcast<double>(c, c->rho2, (double *)lam_f);
    return launch_broadcast<float>(c, c->rho2, (float *)lam_f);
}

extern "C" {

int vp_sweep_adjoint(vp_ctx *c, int axis, double tau, const void *f_in, void *lambda,
                     double *lambda_g)
{
    if (!c || !f_in || !lambda || axis < 0 || axis > 5 || !isfinite(tau)) return VP_ERR_ARG;
    if (!c->adj_flag && cudaMalloc((void **)&c->adj_flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return VP_ERR_OOM;
    }
    double *tau_ptr = &c->sc->pad[3];
    k_set<<<1, 1, 0, c->stream>>>(tau_ptr, tau);
    VP_CUDA_TRY(cudaGetLastError());
    if (axis < 3) {
        VP_CUDA_TRY(launch_coef_drift(c, tau_ptr, 1.0, c->coef_drift));
        VP_CUDA_TRY(launch_drift_adjoint(c, f_in, lambda, axis, c->coef_drift, nullptr));
    } else {
        VP_CUDA_TRY(launch_coef_kick(c, c->g, tau_ptr, 1.0, c->coef_kick1));
        VP_CUDA_TRY(launch_kick_adjoint(c, f_in, lambda, axis - 3, c->coef_kick1, tau, lambda_g));
    }
    return VP_OK;
}

int vp_field_adjoint(vp_ctx *c, const double *lambda_g, void *lambda_f)
{
    if (!c || !lambda_g || !lambda_f) return VP_ERR_ARG;
    VP_CUDA_TRY(launch_field_adjoint(c, lambda_g, lambda_f, false));
    return VP_OK;
}

int vp_functional(vp_ctx *c, int kind, const double *target, void *lambda_f, double *J_out)
{
    if (!c || !lambda_f || (kind != 0 && kind != 1) || (kind == 1 && !target)) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    const int T = 256;
    VP_CUDA_TRY(launch_density(c, c->f, c->rho2));
    double *sums = c->red + 2 * c->np;
    if (kind == 0) {
        VP_CUDA_TRY(launch_field_solve(c, c->rho2, nullptr));
        VP_CUDA_TRY(launch_dot_rho_phi(c, c->rho2, sums));
    } else {
        k_misfit<<<1, 1024, 0, c->stream>>>(c->rho2, target, c->np, sums);
        VP_CUDA_TRY(cudaGetLastError());
    }
    const double scale = c->dvol_v * c->dvol_x;
    long long grid = 8LL * vp_sm_count();
    if (grid > c->np) grid = c->np;
    if (c->isdouble)
        k_functional_grad<double><<<(unsigned)grid, T, 0, c->stream>>>(
            (double *)lambda_f, c->phi, c->rho2, target, kind, c->nvc, c->n[1], c->n[2], c->fn[1],
            c->fn[2], scale, c->np);
    else
        k_functional_grad<float><<<(unsigned)grid, T, 0, c->stream>>>(
            (float *)lambda_f, c->phi, c->rho2, target, kind, c->nvc, c->n[1], c->n[2], c->fn[1],
            c->fn[2], scale, c->np);
    VP_CUDA_TRY(cudaGetLastError());
    double h;
    VP_CUDA_TRY(cudaMemcpyAsync(&h, sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    VP_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (J_out) *J_out = 0.5 * h * c->dvol_x;
    return VP_OK;
}

int vp_set_adjoint_states(vp_ctx *c, int mode)
{
    if (!c || mode < 0 || mode > 3) return VP_ERR_ARG;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return VP_ERR_CUDA;
    }
    vp_free_adjoint_states(c);
    c->adj_mode = mode;
    return VP_OK;
}

}  // extern "C"

namespace {

// the first nsweeps (2 or 3) velocity sweeps of a half kick with table
// coef from src into dst, in one launch sequence
int replay_kick(vp_ctx *c, const void *src, void *dst, const void *coef, int nsweeps)
{
    void *s = const_cast<void *>(src);
    if (vp_kick_fast_ok(c)) {
        VP_CUDA_TRY(launch_kick_fast(c, s, coef, nullptr, nsweeps, 0, dst));
    } else if (vp_kick_big_ok(c)) {
        VP_CUDA_TRY(launch_kick_big(c, s, coef, nullptr, nsweeps, 0, dst));
    } else {
        VP_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)c->ncells * c->esize, cudaMemcpyDeviceToDevice,
                                    c->stream));
        VP_CUDA_TRY(launch_kick(c, dst, coef, nullptr, nsweeps, 0));
    }
    return VP_OK;
}

// The adjoint step with two scratch states X, Y.  The sweep inputs S1..S8
// are recomputed from S0 = f_start, keeping at most two at a time, so that
// each adjoint sweep finds its input in X or Y (or S0):
//   S0 -> S3 -> S4 -> S5 -> S6 (Y, kept) [g^{n+1}];  S8 from S6 (vx and vy
//   in one pass, X): vz;  S7 from S6 (X): vy;  S6: vx;  field
//   S0 -> S3 -> S4 (Y) -> S5 (X): x;  S4: y         (fused y+z: S3 again)
//   S0 -> S3 (X): z
//   S2 from S0 (vx and vy, X): vz;  S1 from S0 (X): vy;  S0: vx
int adjoint_step_two_states(vp_ctx *c, const void *S0, void *lambda_f, double *lambda_g,
                            const void *k1, const double *tau_ptr, double dt, double amax)
{
    void *X = c->adj_states[0], *Y = c->adj_states[1];
    const double tau = 0.5 * dt;
    const bool yz = amax < 1.0 && vp_drift_adjoint_yz_ok(c);
    // replay to S6; its density gives g^{n+1}
    TRY(replay_kick(c, S0, X, k1, 3));                                            // X = S3
    VP_CUDA_TRY(launch_sweep_into(c, X, Y, 2, c->coef_drift, amax));              // Y = S4
    VP_CUDA_TRY(launch_sweep_into(c, Y, X, 1, c->coef_drift, amax));              // X = S5
    VP_CUDA_TRY(launch_sweep_into(c, X, Y, 0, c->coef_drift, amax));              // Y = S6
    VP_CUDA_TRY(launch_density(c, Y, c->rho2));
    VP_CUDA_TRY(launch_field_solve(c, c->rho2, c->adj_g));
    VP_CUDA_TRY(launch_coef_kick(c, c->adj_g, tau_ptr, 0.5, c->coef_kick2));
    // K2 reversed with S6 kept in Y
    TRY(replay_kick(c, Y, X, c->coef_kick2, 2));                                  // X = S8
    VP_CUDA_TRY(launch_kick_adjoint(c, X, lambda_f, 2, c->coef_kick2, tau, lambda_g));
    VP_CUDA_TRY(launch_sweep_into(c, Y, X, 3, c->coef_kick2, amax));              // X = S7
    VP_CUDA_TRY(launch_kick_adjoint(c, X, lambda_f, 1, c->coef_kick2, tau, lambda_g));
    VP_CUDA_TRY(launch_kick_adjoint(c, Y, lambda_f, 0, c->coef_kick2, tau, lambda_g));
    VP_CUDA_TRY(launch_field_adjoint(c, lambda_g, lambda_f, true));
    // the drifts reversed: replay to S5 keeping S4
    TRY(replay_kick(c, S0, X, k1, 3));                                            // X = S3
    VP_CUDA_TRY(launch_sweep_into(c, X, Y, 2, c->coef_drift, amax));              // Y = S4
    VP_CUDA_TRY(launch_sweep_into(c, Y, X, 1, c->coef_drift, amax));              // X = S5
    VP_CUDA_TRY(launch_drift_adjoint(c, X, lambda_f, 0, c->coef_drift, c->rho2));
    if (!yz) VP_CUDA_TRY(launch_drift_adjoint(c, Y, lambda_f, 1, c->coef_drift, nullptr));
    TRY(replay_kick(c, S0, X, k1, 3));                                            // X = S3
    if (yz) {
        VP_CUDA_TRY(launch_drift_adjoint_yz(c, X, lambda_f, c->coef_drift));
    } else {
        VP_CUDA_TRY(launch_drift_adjoint(c, X, lambda_f, 2, c->coef_drift, nullptr));
    }
    // K1 reversed
    VP_CUDA_TRY(cudaMemsetAsync(lambda_g, 0, sizeof(double) * 3 * c->np, c->stream));
    TRY(replay_kick(c, S0, X, k1, 2));                                            // X = S2
    VP_CUDA_TRY(launch_kick_adjoint(c, X, lambda_f, 2, k1, tau, lambda_g));
    VP_CUDA_TRY(launch_sweep_into(c, S0, X, 3, k1, amax));                        // X = S1
    VP_CUDA_TRY(launch_kick_adjoint(c, X, lambda_f, 1, k1, tau, lambda_g));
    VP_CUDA_TRY(launch_kick_adjoint(c, S0, lambda_f, 0, k1, tau, lambda_g));
    return VP_OK;
}

// The adjoint step with three scratch states X, Y, Z (the replays move 96
// bytes per cell against 120 with two states):
//   S0 -> S3 (X) -> S4 (Y) -> S5 (Z) -> S6 (Y) [g^{n+1}];  S8 from S6 (vx
//   and vy in one pass, X): vz;  S7 from S6 (X): vy;  S6: vx;  field
//   S5: x
//   S0 -> S3 (X) -> S4 (Y): y;  S3: z               (fused y+z: S3 alone)
//   S2 from S0 (vx and vy, X): vz;  S1 from S0 (X): vy;  S0: vx
int adjoint_step_three_states(vp_ctx *c, const void *S0, void *lambda_f, double *lambda_g,
                              const void *k1, const double *tau_ptr, double dt, double amax)
{
    void *X = c->adj_states[0], *Y = c->adj_states[1], *Z = c->adj_states[2];
    const double tau = 0.5 * dt;
    const bool yz = amax < 1.0 && vp_drift_adjoint_yz_ok(c);
    // replay to S6 keeping S5; the density of S6 gives g^{n+1}
    TRY(replay_kick(c, S0, X, k1, 3));                                            // X = S3
    VP_CUDA_TRY(launch_sweep_into(c, X, Y, 2, c->coef_drift, amax));              // Y = S4
    VP_CUDA_TRY(launch_sweep_into(c, Y, Z, 1, c->coef_drift, amax));              // Z = S5
    VP_CUDA_TRY(launch_sweep_into(c, Z, Y, 0, c->coef_drift, amax));              // Y = S6
    VP_CUDA_TRY(launch_density(c, Y, c->rho2));
    VP_CUDA_TRY(launch_field_solve(c, c->rho2, c->adj_g));
    VP_CUDA_TRY(launch_coef_kick(c, c->adj_g, tau_ptr, 0.5, c->coef_kick2));
    // K2 reversed with S6 in Y
    TRY(replay_kick(c, Y, X, c->coef_kick2, 2));                                  // X = S8
    VP_CUDA_TRY(launch_kick_adjoint(c, X, lambda_f, 2, c->coef_kick2, tau, lambda_g));
    VP_CUDA_TRY(launch_sweep_into(c, Y, X, 3, c->coef_kick2, amax));              // X = S7
    VP_CUDA_TRY(launch_kick_adjoint(c, X, lambda_f, 1, c->coef_kick2, tau, lambda_g));
    VP_CUDA_TRY(launch_kick_adjoint(c, Y, lambda_f, 0, c->coef_kick2, tau, lambda_g));
    VP_CUDA_TRY(launch_field_adjoint(c, lambda_g, lambda_f, true));
    // the drifts reversed: S5 is in Z; S3 and S4 replayed again
    VP_CUDA_TRY(launch_drift_adjoint(c, Z, lambda_f, 0, c->coef_drift, c->rho2));
    TRY(replay_kick(c, S0, X, k1, 3));                                            // X = S3
    if (yz) {
        VP_CUDA_TRY(launch_drift_adjoint_yz(c, X, lambda_f, c->coef_drift));
    } else {
        VP_CUDA_TRY(launch_sweep_into(c, X, Y, 2, c->coef_drift, amax));          // Y = S4
        VP_CUDA_TRY(launch_drift_adjoint(c, Y, lambda_f, 1, c->coef_drift, nullptr));
        VP_CUDA_TRY(launch_drift_adjoint(c, X, lambda_f, 2, c->coef_drift, nullptr));
    }
    // K1 reversed
    VP_CUDA_TRY(cudaMemsetAsync(lambda_g, 0, sizeof(double) * 3 * c->np, c->stream));
    TRY(replay_kick(c, S0, X, k1, 2));                                            // X = S2
    VP_CUDA_TRY(launch_kick_adjoint(c, X, lambda_f, 2, k1, tau, lambda_g));
    VP_CUDA_TRY(launch_sweep_into(c, S0, X, 3, k1, amax));                        // X = S1
    VP_CUDA_TRY(launch_kick_adjoint(c, X, lambda_f, 1, k1, tau, lambda_g));
    VP_CUDA_TRY(launch_kick_adjoint(c, S0, lambda_f, 0, k1, tau, lambda_g));
    return VP_OK;
}

}  // namespace

extern "C" {

int vp_adjoint_step(vp_ctx *c, const void *f_start, const double *g_start, void *lambda_f,
                    double *lambda_g)
{
    if (!c || !f_start || !g_start || !lambda_f || !lambda_g) return VP_ERR_ARG;
    if (!c->f) return VP_ERR_STATE;
    if (!(c->cfg.dt_fixed > 0.0)) return VP_ERR_STATE;
    TRY(ensure_adjoint_scratch(c));
    const double dt = c->cfg.dt_fixed;
    void **S = c->adj_states;
    double *tau_ptr = &c->sc->pad[2];
    k_set<<<1, 1, 0, c->stream>>>(tau_ptr, dt);
    VP_CUDA_TRY(cudaGetLastError());
    // the replay's outflow is not the simulation's: keep the counter aside
    VP_CUDA_TRY(cudaMemcpyAsync(&c->sc->pad[1], &c->sc->lost, sizeof(double),
                                cudaMemcpyDeviceToDevice, c->stream));
    // tables of the replay: K1 from g^n, drift, K2 from the recomputed g^{n+1}
    void *k1 = c->adj_f;
    VP_CUDA_TRY(launch_coef_kick(c, g_start, tau_ptr, 0.5, k1));
    VP_CUDA_TRY(launch_coef_drift(c, tau_ptr, 1.0, c->coef_drift));
    const double amax = vp_drift_alpha_bound(c, dt);
    const void *S0 = f_start;     // S[k]: input of sweep k of the step (S[0] = f^n)
    if (c->adj_nstates == 2 || c->adj_nstates == 3) {
        const int r = c->adj_nstates == 2
                          ? adjoint_step_two_states(c, S0, lambda_f, lambda_g, k1, tau_ptr, dt, amax)
                          : adjoint_step_three_states(c, S0, lambda_f, lambda_g, k1, tau_ptr, dt, amax);
        VP_CUDA_TRY(cudaMemcpyAsync(&c->sc->lost, &c->sc->pad[1], sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->stream));
        return r;
    }
    const bool reg = vp_kick_adjoint3_ok(c);
    // --- forward replay
    if (reg) {
        // K1 in one pass keeping the vx output (the vz input is recomputed)
        VP_CUDA_TRY(launch_kick_fast(c, const_cast<void *>(S0), k1, nullptr, 3, 0, S[3], S[1], nullptr));
    } else if (vp_kick_fast_ok(c)) {
        VP_CUDA_TRY(launch_kick_fast(c, const_cast<void *>(S0), k1, nullptr, 3, 0, S[3], S[1], S[2]));
    } else {
        for (int k = 0; k < 3; ++k)
            VP_CUDA_TRY(launch_sweep_into(c, k ? S[k] : S0, S[k + 1], 3 + k, k1, amax));
    }
    // the fused y+z drift adjoint recomputes the y input S4 from S3: the
    // replay then keeps S5 only
    const bool yz = amax < 1.0 && vp_drift_adjoint_yz_ok(c);
    if (yz) {
        VP_CUDA_TRY(launch_drift_yz(c, S[3], c->coef_drift, S[5]));
    } else {
        VP_CUDA_TRY(launch_sweep_into(c, S[3], S[4], 2, c->coef_drift, amax));
        VP_CUDA_TRY(launch_sweep_into(c, S[4], S[5], 1, c->coef_drift, amax));
    }
    if (c->rho_part && vp_rho_fuse_ok(c) && amax < 1.0) {
        VP_CUDA_TRY(launch_drift_fast(c, S[5], 0, c->coef_drift, c->rho_part, S[6]));
        VP_CUDA_TRY(launch_rho_finish(c, c->rho_part, c->rho_nparts, c->rho2));
    } else {
        VP_CUDA_TRY(launch_sweep_into(c, S[5], S[6], 0, c->coef_drift, amax));
        VP_CUDA_TRY(launch_density(c, S[6], c->rho2));
    }
    VP_CUDA_TRY(launch_field_solve(c, c->rho2, c->adj_g));
    VP_CUDA_TRY(launch_coef_kick(c, c->adj_g, tau_ptr, 0.5, c->coef_kick2));
    if (reg) {
        VP_CUDA_TRY(launch_kick_fast(c, S[6], c->coef_kick2, nullptr, 1, 0, S[7]));
    } else if (vp_kick_fast_ok(c)) {
        VP_CUDA_TRY(launch_kick_fast(c, S[6], c->coef_kick2, nullptr, 2, 0, S[8], S[7], nullptr));
    } else {
        VP_CUDA_TRY(launch_sweep_into(c, S[6], S[7], 3, c->coef_kick2, amax));
        VP_CUDA_TRY(launch_sweep_into(c, S[7], S[8], 4, c->coef_kick2, amax));
    }
    // --- reverse
    // K2 (vz, vy, vx); its g-cotangent is added to lambda_g^{n+1}
    TRY(kick_adjoint3(c, S[6], S[7], reg ? nullptr : S[8], S[8], lambda_f, c->coef_kick2, 0.5 * dt,
                      lambda_g));
    // g^{n+1} = field(f_b); its density broadcast is added by the x-drift
    // adjoint as it loads lambda_f
    VP_CUDA_TRY(launch_field_adjoint(c, lambda_g, lambda_f, true));
    // drift x, y, z reversed
    VP_CUDA_TRY(launch_drift_adjoint(c, S[5], lambda_f, 0, c->coef_drift, c->rho2));
    if (yz) {
        VP_CUDA_TRY(launch_drift_adjoint_yz(c, S[3], lambda_f, c->coef_drift));
    } else {
        VP_CUDA_TRY(launch_drift_adjoint(c, S[4], lambda_f, 1, c->coef_drift, nullptr));
        VP_CUDA_TRY(launch_drift_adjoint(c, S[3], lambda_f, 2, c->coef_drift, nullptr));
    }
    // K1 reversed; its g-cotangent is that of g^n
    VP_CUDA_TRY(cudaMemsetAsync(lambda_g, 0, sizeof(double) * 3 * c->np, c->stream));
    TRY(kick_adjoint3(c, S0, S[1], reg ? nullptr : S[2], S[2], lambda_f, k1, 0.5 * dt, lambda_g));
    VP_CUDA_TRY(cudaMemcpyAsync(&c->sc->lost, &c->sc->pad[1], sizeof(double),
                                cudaMemcpyDeviceToDevice, c->stream));
    return VP_OK;
}

}  // extern "C"
