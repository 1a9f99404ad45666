// vp_adjoint_fast.cu -- FP32 register-line adjoint sweeps for line lengths
// 16, 32 and 48 (zero whole-cell shift): the transpose of the forward kernels
// of vp_sweep_fast.cu with their own limiter arms.
//
// Forward (vp_line.cuh), in the upwind frame of a line with F = 2 f_inf,
// h_j = -f_j / F and r3 = 3 / F:
//   u1_j = r3 f_j + h_{j+1},  u2_j = r3 f_j + h_{j-1},
//   s1 = sat(u1), s2 = sat(u2),
//   E+ = 2 f_j - F s1,  E- = F s2 - 2 f_j,
//   phi_j = c0 f_j + c1 E+ + c2 E-,   out_j = f_j - phi_j + phi_{j-1}.
// The E+ arm is interior iff sat(u1) == u1 (0 <= u1 <= 1, the arm of
// clamp(f_{j+1} - f_j, -2 (f_inf - f_j), 2 f_j) that returns the difference
// itself); the same for E- with u2.  With the arms frozen, and with
// mu_j = l_{j+1} - l_j, a = c1 mu, b = c2 mu, I1 = [E+ interior],
// I2 = [E- interior]:
//   dl_j     += (c0 + 2 c1 - 2 c2) mu - 3 a I1 + 3 b I2,
//   dl_{j+1} += a I1,     dl_{j-1} -= b I2,
//   l_F      += a (u1 I1 - s1) + b (s2 - u2 I2)    (dE+/dF, dE-/dF),
// where u I - s is minus the indicator of the arm saturated at 1 (so l_F is
// accumulated per line as c2 sum mu g2 - c1 sum mu g1, g = s - I u),
// and l_F reaches the line maximum (2 l_F on f_inf) at its first position
// in upwind order.  The velocity sweeps also return
//   d/dbeta = sum_j mu_j (f_j + c1'(beta) E+ + c2'(beta) E-).
// The limiter values are the forward kernels' own (same F, h, r3 and
// saturating FMAs), so the arms are those the forward pass took.
//
// Every kernel runs one upwind code path: a line with u < 0 is read and
// written mirrored (from its far end with a negative stride, or through a
// tile held in upwind order).
//
// Kernels:
//  * k_adjoint_pairs: two lines per thread (adjacent vz for the vx and vy
//    sweeps, adjacent velocity cells for the drifts), packed f32x2; the
//    state line read from global memory into registers, the cotangent line
//    copied by cp.async into the thread's shared-memory slots and streamed
//    from there (a warp reads two 128-byte rows per load).  The x-drift
//    adjoint can add the broadcast of the density cotangent on load.
//  * k_adjoint_rows: the vz sweep; persistent warps each stage 32 rows of
//    the state and of the cotangent in shared memory by 16-byte asynchronous
//    copies (the next 32 rows prefetched into L2 meanwhile), sweep one row
//    per lane, and write the rows back with coalesced 16-byte stores.
//  * k_kick_adjoint_zy: the vz and then the vy adjoint of a half kick on the
//    same staged rows (a warp holds whole vx planes), followed by the vx
//    adjoint as line pairs: the cotangent crosses HBM twice for three sweeps.
//  * k_drift_adjoint_yz: the y and then the z drift adjoint in one pass,
//    the y input recomputed from the z input in a shared tile.
#include <cuda_runtime.h>

#include "vp_device.cuh"
#include "vp_internal.cuh"
#include "vp_fast_line.cuh"
#include "vp_line.cuh"

using namespace vpline;

int vp_sm_count();

namespace {

// per-line weights of the adjoint: K0 = c0 + 2 (c1 - c2), the cotangent
// weights 3 c1, -3 c2, -c1, c2 of the frozen-arm terms, and with c' = dc/dbeta
// the beta derivative of phi_j, f_j + c1' E+ + c2' E-
//   = kf f_j + Fd1 s1 + Fd2 s2,  kf = 1 + 2 (c1' - c2'), Fd1 = -F c1', Fd2 = F c2'
template <typename V>
struct AdjW {
    V nK0, c3a, c3b, nc1, c2, kf, Fd1, Fd2;    // nK0 = -K0
    V ninvF, r3;
};

// an arm with saturation s of its argument u: interior iff s == u.  Returns
// nm = -mu [interior] and g = [saturated at 1] (s when not interior, which
// is 0 when saturated at 0), both selected by the one comparison
__device__ __forceinline__ void arm1(float s, float u, float nmu, float &nm, float &g)
{
    const bool in = s == u;
    nm = in ? nmu : 0.f;
    g = in ? 0.f : s;
}

template <typename V>
struct AOps;
template <>
struct AOps<float2> {
    __device__ __forceinline__ static void arm(float2 s, float2 u, float2 nmu, float2 &nm, float2 &g)
    {
        arm1(s.x, u.x, nmu.x, nm.x, g.x);
        arm1(s.y, u.y, nmu.y, nm.y, g.y);
    }
    __device__ __forceinline__ static float2 fsat(float2 a, float2 b, float2 c)
    {
        return make_float2(fmasat(a.x, b.x, c.x), fmasat(a.y, b.y, c.y));
    }
};
template <>
struct AOps<float> {
    __device__ __forceinline__ static void arm(float s, float u, float nmu, float &nm, float &g)
    {
        arm1(s, u, nmu, nm, g);
    }
    __device__ __forceinline__ static float fsat(float a, float b, float c) { return fmasat(a, b, c); }
};

__device__ __forceinline__ void adj_weights1(const LineCoef<float> &cf, float finf, float &nK0,
                                             float &c3a, float &c3b, float &nc1, float &c2,
                                             float &kf, float &Fd1, float &Fd2, float &ninvF)
{
    float A1, A2;
    weights1<float>(cf.c0, cf.c1, cf.c2, cf.code & 1, finf, nK0, A1, A2, ninvF);
    nK0 = -nK0;
    const float beta = cf.c0;
    c3a = 3.f * cf.c1;
    c3b = -3.f * cf.c2;
    nc1 = -cf.c1;
    c2 = cf.c2;
    const float dc1 = (2.f - 6.f * beta + 3.f * beta * beta) * (1.f / 6.f);
    const float dc2 = (1.f - 3.f * beta * beta) * (1.f / 6.f);
    const float F = finf + finf;
    kf = 1.f + 2.f * (dc1 - dc2);
    Fd1 = -F * dc1;
    Fd2 = F * dc2;
}

__device__ __forceinline__ AdjW<float2> adj_weights(const LineCoef<float> &ca,
                                                    const LineCoef<float> &cb, float2 finf)
{
    AdjW<float2> w;
    adj_weights1(ca, finf.x, w.nK0.x, w.c3a.x, w.c3b.x, w.nc1.x, w.c2.x, w.kf.x, w.Fd1.x, w.Fd2.x,
                 w.ninvF.x);
    adj_weights1(cb, finf.y, w.nK0.y, w.c3a.y, w.c3b.y, w.nc1.y, w.c2.y, w.kf.y, w.Fd1.y, w.Fd2.y,
                 w.ninvF.y);
    w.r3 = __fmul2_rn(w.ninvF, make_float2(-3.f, -3.f));
    return w;
}

__device__ __forceinline__ AdjW<float> adj_weights(const LineCoef<float> &cf, float finf)
{
    AdjW<float> w;
    adj_weights1(cf, finf, w.nK0, w.c3a, w.c3b, w.nc1, w.c2, w.kf, w.Fd1, w.Fd2, w.ninvF);
    w.r3 = w.ninvF * -3.f;
    return w;
}

// One cell of the line adjoint (upwind position j).  In: the cell f0, the
// scaled neighbours hprev, hnext, the output cotangents lo = l_j, ln =
// l_{j+1}, the pending input cotangent pend of cell j - 1 and nm1p =
// -m1_{j-1}.  With mu = ln - lo and nm = -mu [arm interior]:
//   l^in_{j-1} = pend - c2 m2_j                         (returned in done)
//   pend'      = lo + K0 mu - 3 c1 m1_j + 3 c2 m2_j + c1 m1_{j-1}
// and the line sums of mu g1, mu g2 with g = [arm saturated at 1] (each term
// exact: no cancellation), so that l_F = c2 sum mu g2 - c1 sum mu g1.  DB:
// the sums of mu s1, mu s2 and mu f as well.  The sums are kept negated (they
// accumulate -mu, which the arms' selection gives for free); finish() turns
// them back, bitwise as the positive sums would be (an FMA rounds
// symmetrically).
template <typename V, bool DB>
struct AdjCell {
    V pend, nm1p, G1, G2, S1, S2, SF;      // G, S: negated sums

    __device__ __forceinline__ void init()
    {
        const V z = VOps<V>::zero();
        pend = z; nm1p = z; G1 = z; G2 = z; S1 = z; S2 = z; SF = z;
    }

    template <bool FIRST>
    __device__ __forceinline__ V step(V f0, V hprev, V hnext, V lo, V ln, const AdjW<V> &w, V &nm2)
    {
        typedef VOps<V> O;
        typedef AOps<V> A;
        const V nmu = O::sub(lo, ln);
        const V u1 = O::fma(f0, w.r3, hnext);
        const V u2 = O::fma(f0, w.r3, hprev);
        const V s1 = A::fsat(f0, w.r3, hnext);
        const V s2 = A::fsat(f0, w.r3, hprev);
        V nm1, g1, g2;
        A::arm(s1, u1, nmu, nm1, g1);
        A::arm(s2, u2, nmu, nm2, g2);
        V x = O::fma(w.nK0, nmu, lo);
        x = O::fma(w.c3a, nm1, x);
        x = O::fma(w.c3b, nm2, x);
        if (!FIRST) x = O::fma(w.nc1, nm1p, x);
        const V done = O::fma(w.c2, nm2, pend);
        pend = x;
        nm1p = nm1;
        G1 = O::fma(nmu, g1, G1);
        G2 = O::fma(nmu, g2, G2);
        if (DB) {
            S1 = O::fma(nmu, s1, S1);
            S2 = O::fma(nmu, s2, S2);
            SF = O::fma(nmu, f0, SF);
        }
        return done;
    }

    __device__ __forceinline__ void finish(const AdjW<V> &w, V &lF, V &db) const
    {
        typedef VOps<V> O;
        const V m1 = O::splat(typename O::S(-1));
        lF = O::mul(O::fma(w.c2, G2, O::mul(w.nc1, G1)), m1);
        db = DB ? O::mul(O::fma(w.Fd2, S2, O::fma(w.Fd1, S1, O::mul(w.kf, SF))), m1) : O::zero();
    }
};

// Cotangent of the zero-shift update of one line in upwind order (lines with
// u < 0 are passed mirrored), through accessors of compile-time position j:
// fget(j) the state, lget(j) the output cotangent, lput(j, v) the input
// cotangent (without the f_inf term: l_F is returned for the caller to
// place).  Every state and cotangent element is read once, in increasing j,
// before position j - 1 is written (at step j), so lput may write over the
// storage of fget or lget; with PERIODIC, positions 0 and N - 1 are written
// last.
template <typename V, int N, bool PERIODIC, bool DB, class FG, class LG, class LP>
__device__ __forceinline__ void adjoint_line_acc(FG fget, LG lget, LP lput, const AdjW<V> &w,
                                                 V &lF, V &db)
{
    typedef VOps<V> O;
    const V z = O::zero();
    const V f0 = fget(0), l0 = lget(0);
    const V h0 = O::mul(f0, w.ninvF);
    V hprev = PERIODIC ? O::mul(fget(N - 1), w.ninvF) : z;
    V fcur = f0, hcur = h0, lo = l0, nm2 = z, nm2first = z, first = z;
    AdjCell<V, DB> c;
    c.init();
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const V fnext = (j + 1 < N) ? fget(j + 1 < N ? j + 1 : 0) : z;
        const V hnext = (j + 1 < N) ? O::mul(fnext, w.ninvF) : (PERIODIC ? h0 : z);
        const V ln = (j + 1 < N) ? lget(j + 1 < N ? j + 1 : 0) : (PERIODIC ? l0 : z);
        if (j == 0) {
            c.template step<true>(fcur, hprev, hnext, lo, ln, w, nm2);
            nm2first = nm2;
        } else {
            const V d = c.template step<false>(fcur, hprev, hnext, lo, ln, w, nm2);
            if (PERIODIC && j == 1) first = d;
            else lput(j - 1, d);
        }
        hprev = hcur;
        hcur = hnext;
        lo = ln;
        fcur = fnext;
    }
    if (PERIODIC) {
        lput(N - 1, O::fma(w.c2, nm2first, c.pend));
        lput(0, O::fma(w.nc1, c.nm1p, first));
    } else {
        lput(N - 1, c.pend);
    }
    c.finish(w, lF, db);
}

// the line in registers: l is overwritten with the input cotangent
template <typename V, int N, bool PERIODIC, bool DB>
__device__ __forceinline__ void adjoint_line(const V (&f)[N], V (&l)[N], const AdjW<V> &w, V &lF,
                                             V &db)
{
    adjoint_line_acc<V, N, PERIODIC, DB>([&](int j) { return f[j]; }, [&](int j) { return l[j]; },
                                         [&](int j, V v) { l[j] = v; }, w, lF, db);
}

// the state in registers, the cotangent in memory (lsrc, stride ls elements
// of V; mirrored lines pass the last element and a negative stride) and the
// input cotangent written to memory (ldst, stride ld; may equal lsrc)
template <typename V, int N, bool PERIODIC, bool DB>
__device__ __forceinline__ void adjoint_line_mem(const V (&f)[N], const V *lsrc, int ls, V *ldst,
                                                 int ld, const AdjW<V> &w, V &lF, V &db)
{
    adjoint_line_acc<V, N, PERIODIC, DB>([&](int j) { return f[j]; },
                                         [&](int j) { return lsrc[j * ls]; },
                                         [&](int j, V v) { ldst[j * ld] = v; }, w, lF, db);
}

// first array position of the maximum m of the line v (lines in upwind order)
template <int N>
__device__ __forceinline__ int first_max(const float (&v)[N], float m)
{
    int a = 0;
#pragma unroll
    for (int j = N - 1; j >= 0; --j) a = v[j] == m ? j : a;
    return a;
}

template <int N>
__device__ __forceinline__ int2 first_max2(const float2 (&x)[N], float2 m)
{
    int ax = 0, ay = 0;
#pragma unroll
    for (int j = N - 1; j >= 0; --j) {
        ax = x[j].x == m.x ? j : ax;
        ay = x[j].y == m.y ? j : ay;
    }
    return make_int2(ax, ay);
}

// one scalar line in upwind order: returns the beta derivative (in the
// frame of the velocity axis), the upwind position of the line maximum and
// its cotangent 2 l_F
template <int N, bool PERIODIC, bool DB>
__device__ __forceinline__ float adjoint_scalar(const float (&f)[N], float (&l)[N],
                                                const LineCoef<float> &cf, int &arg, float &lfinf)
{
    const float finf = line_max(f);
    arg = first_max<N>(f, finf);
    const AdjW<float> w = adj_weights(cf, finf);
    float lF, db;
    adjoint_line<float, N, PERIODIC, DB>(f, l, w, lF, db);
    lfinf = 2.f * lF;
    return (cf.code & 1) ? -db : db;
}

// a pair of lines travelling in opposite directions: two scalar adjoints,
// out of line (the arrays are copies in local memory, each put in upwind
// order; rare).  f, l in array order; arg returns array positions.
template <int N, bool PERIODIC, bool DB>
__device__ __noinline__ float adjoint_pair_mixed(const float2 *f, float2 *l, LineCoef<float> ca,
                                                 LineCoef<float> cb, int *arg, float *lfinf)
{
    float fx[N], fy[N], lx[N], ly[N];
    const bool nx = ca.code & 1, ny = cb.code & 1;
    for (int j = 0; j < N; ++j) {
        const int jx = nx ? N - 1 - j : j, jy = ny ? N - 1 - j : j;
        fx[j] = f[jx].x; fy[j] = f[jy].y;
        lx[j] = l[jx].x; ly[j] = l[jy].y;
    }
    const float dx = adjoint_scalar<N, PERIODIC, DB>(fx, lx, ca, arg[0], lfinf[0]);
    const float dy = adjoint_scalar<N, PERIODIC, DB>(fy, ly, cb, arg[1], lfinf[1]);
    for (int j = 0; j < N; ++j) {
        const int jx = nx ? N - 1 - j : j, jy = ny ? N - 1 - j : j;
        l[jx].x = lx[j];
        l[jy].y = ly[j];
    }
    if (nx) arg[0] = N - 1 - arg[0];
    if (ny) arg[1] = N - 1 - arg[1];
    return dx + dy;
}

// asynchronous 8-byte copy global -> shared (no register staging) and the
// wait for all of the thread's copies
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

struct PairGeom {
    int axis;                  // 0..5
    long long nvc;
    // drift axes: outer index o -> base cell (o / od) m1 + (o % od) m2
    long long cell_stride;
    int od;
    long long m1, m2;
    int va_stride, va_n;       // velocity index along the axis: (v / va_stride) % va_n
    int zremap, nvz;           // z drift: pairs per half vz row of the warp-uniform map (0: off)
    int mixed;                 // z drift: some pair (v, v + 1) has v_z of both signs
    long long units;           // line pairs per outer index (drift) or per cube (kick)
    long long per_part;        // units per CTA (drift)
    // kick axes: pair p -> voff = (p / pd) pm_hi + 2 (p % pd), element stride vstride
    int pd;
    long long pm_hi, vstride;
    int cube3;                 // kick axes: skip a cube with a shift on any velocity axis
};

// DB: the velocity sweeps' beta derivative; BC: add dvol_v lam_rho[cell] to
// the cotangent on load (the density broadcast of the field adjoint)
// MIXED: the two lines of a pair may travel in opposite directions (z drift,
// where they differ in v_z); then they are done as two scalar lines.
// The state pair line is held in registers; the cotangent pair line is
// copied asynchronously into the thread's own shared-memory slots (element j
// of thread t at j * 128 + t: conflict-free) and streamed from there, which
// keeps the kernel at 128 registers (16 warps per SM).
template <int N, bool PERIODIC, bool DB, bool BC, bool MIXED>
__global__ void __launch_bounds__(128, N <= 32 ? 4 : 3) k_adjoint_pairs(const float *__restrict__ fin,
                                                      float *__restrict__ lam,
                                                      const LineCoef<float> *__restrict__ coef,
                                                      PairGeom g, const double *__restrict__ bc,
                                                      double *__restrict__ lam_g, double scale,
                                                      int *skipped)
{
    __shared__ double red[32];
    __shared__ float sbc[BC ? N : 1];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = threadIdx.x;
    float2 *sl = reinterpret_cast<float2 *>(smem_raw) + t;     // slot j: sl[j * 128]
    long long base, u0, u1, stride, cell0 = 0, cube = 0;
    if (g.axis < 3) {
        const int o = blockIdx.y;
        cell0 = (long long)(o / g.od) * g.m1 + (long long)(o % g.od) * g.m2;
        base = cell0 * g.nvc;
        stride = g.cell_stride * g.nvc;
        u0 = (long long)blockIdx.x * g.per_part;
        u1 = u0 + g.per_part;
        if (u1 > g.units) u1 = g.units;
        if constexpr (BC) {
            if (t < N) sbc[t] = (float)bc[cell0 + t * g.cell_stride];
            __syncthreads();
        }
    } else {
        // velocity axes: the cube on the grid's x dimension (any number of
        // cubes), the chunk of its line pairs on y
        cube = blockIdx.x;
        base = cube * g.nvc;
        stride = g.vstride;
        u0 = (long long)blockIdx.y * blockDim.x;
        u1 = u0 + blockDim.x;
        if (u1 > g.units) u1 = g.units;
    }
    float da = 0.f;
    for (long long u = u0 + t; u < u1; u += blockDim.x) {
        long long off;
        LineCoef<float> ca, cb;
        if (g.axis < 3) {
            long long v = 2 * u;
            if (g.zremap > 0) {
                // a warp takes the same half (the same sign of v_z) of 32 / H
                // consecutive vz rows, H pairs each
                const int H = g.zremap, RW = 32 / H;
                const long long q = u % H, r1 = u / H, ri = r1 % RW, r2 = r1 / RW;
                v = ((r2 >> 1) * RW + ri) * g.nvz + ((r2 & 1) * H + q) * 2;
            }
            off = base + v;
            ca = coef[(int)((v / g.va_stride) % g.va_n)];
            cb = coef[(int)(((v + 1) / g.va_stride) % g.va_n)];
        } else {
            off = base + (u / g.pd) * g.pm_hi + 2 * (u % g.pd);
            ca = coef[cube * 3 + (g.axis - 3)];
            cb = ca;
            if (g.cube3) {
                const LineCoef<float> *cc = coef + cube * 3;
                cb.code |= (cc[0].code | cc[1].code | cc[2].code) & ~1;
            }
        }
        if ((ca.code >> 1) != 0 || (cb.code >> 1) != 0) {
            atomicExch(skipped, 1);
            if constexpr (BC) {
                // the fix-up pass sweeps this pair: it gets its density
                // broadcast here, as the pairs swept below do on load
#pragma unroll 4
                for (int j = 0; j < N; ++j) {
                    float2 *p = reinterpret_cast<float2 *>(lam + off + j * stride);
                    float2 v = *p;
                    v.x += sbc[j];
                    v.y += sbc[j];
                    *p = v;
                }
            }
            continue;
        }
        // lines of one direction are read in upwind order (u < 0: from the
        // far end with a negative stride); a mixed pair in array order
        const bool same = !MIXED || (ca.code & 1) == (cb.code & 1);
        const bool neg = same && (ca.code & 1);
        const long long st = neg ? -stride : stride;
        const long long o0 = neg ? off + (N - 1) * stride : off;
#pragma unroll
        for (int j = 0; j < N; ++j) cp_async8(sl + j * 128, lam + o0 + j * st);
        float2 f[N];
#pragma unroll
        for (int j = 0; j < N; ++j) f[j] = *reinterpret_cast<const float2 *>(fin + o0 + j * st);
        cp_async_wait_all();
        const float *sb = sbc + (neg ? N - 1 : 0);
        const int ss = neg ? -1 : 1;
        auto lget = [&](int j) {
            float2 v = sl[j * 128];
            if constexpr (BC) {
                const float b = sb[j * ss];
                v.x += b;
                v.y += b;
            }
            return v;
        };
        auto lput = [&](int j, float2 v) { *reinterpret_cast<float2 *>(lam + o0 + j * st) = v; };
        int ax, ay;
        float lfx, lfy;
        if (same) {
            const float2 finf = line_max(f);
            const int2 a2 = first_max2<N>(f, finf);
            const AdjW<float2> w = adj_weights(ca, cb, finf);
            float2 lF, db;
            adjoint_line_acc<float2, N, PERIODIC, DB>([&](int j) { return f[j]; }, lget, lput, w,
                                                      lF, db);
            ax = a2.x;
            ay = a2.y;
            lfx = 2.f * lF.x;
            lfy = 2.f * lF.y;
            if (DB) da += neg ? -(db.x + db.y) : db.x + db.y;
        } else if constexpr (MIXED) {
            float2 fm[N], lm[N];
#pragma unroll
            for (int j = 0; j < N; ++j) { fm[j] = f[j]; lm[j] = lget(j); }
            int am[2];
            float lfm[2];
            const float d = adjoint_pair_mixed<N, PERIODIC, DB>(fm, lm, ca, cb, am, lfm);
            if (DB) da += d;
            ax = am[0]; ay = am[1];
            lfx = lfm[0]; lfy = lfm[1];
#pragma unroll
            for (int j = 0; j < N; ++j) lput(j, lm[j]);
        }
        lam[o0 + ax * st] += lfx;
        lam[o0 + ay * st + 1] += lfy;
    }
    if (DB) {
        const double s = block_sum((double)da, red);
        if (t == 0 && s != 0.0) atomicAdd(lam_g + cube, s * scale);
    }
}

// 32 contiguous rows of N floats (global) to a tile of pitch P and back,
// each row reversed when rev (warp-uniform): a row of a line with u < 0 is
// held in upwind order
template <int N, int P>
__device__ __forceinline__ void rows_in(float *tile, const float *g, bool rev, int lane)
{
    constexpr int Q = N / 4;
    if (!rev) {
#pragma unroll 4
        for (int e = lane; e < 32 * Q; e += 32) {
            const int r = e / Q, c = 4 * (e % Q);
            *reinterpret_cast<float4 *>(tile + r * P + c) = *reinterpret_cast<const float4 *>(g + r * N + c);
        }
    } else {
#pragma unroll 4
        for (int e = lane; e < 32 * Q; e += 32) {
            const int r = e / Q, c = 4 * (e % Q);
            const float4 v = *reinterpret_cast<const float4 *>(g + r * N + c);
            *reinterpret_cast<float4 *>(tile + r * P + (N - 4 - c)) = make_float4(v.w, v.z, v.y, v.x);
        }
    }
}

template <int N, int P>
__device__ __forceinline__ void rows_out(float *g, const float *tile, bool rev, int lane)
{
    constexpr int Q = N / 4;
    if (!rev) {
#pragma unroll 4
        for (int e = lane; e < 32 * Q; e += 32) {
            const int r = e / Q, c = 4 * (e % Q);
            *reinterpret_cast<float4 *>(g + r * N + c) = *reinterpret_cast<const float4 *>(tile + r * P + c);
        }
    } else {
#pragma unroll 4
        for (int e = lane; e < 32 * Q; e += 32) {
            const int r = e / Q, c = 4 * (e % Q);
            const float4 v = *reinterpret_cast<const float4 *>(tile + r * P + (N - 4 - c));
            *reinterpret_cast<float4 *>(g + r * N + c) = make_float4(v.w, v.z, v.y, v.x);
        }
    }
}

// one row of the tile (pitch P) to registers and back
template <int N>
__device__ __forceinline__ void row_load(float (&x)[N], const float *row)
{
#pragma unroll
    for (int c = 0; c < N; c += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(row + c);
        x[c] = a.x; x[c + 1] = a.y; x[c + 2] = a.z; x[c + 3] = a.w;
    }
}

template <int N>
__device__ __forceinline__ void row_store(float *row, const float (&x)[N])
{
#pragma unroll
    for (int c = 0; c < N; c += 4)
        *reinterpret_cast<float4 *>(row + c) = make_float4(x[c], x[c + 1], x[c + 2], x[c + 3]);
}

// asynchronous 16-byte copy global -> shared, and an asynchronous prefetch
// of [p, p + bytes) into L2 (16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// 32 contiguous rows of N floats (global) into a tile of pitch P, in array
// order, by 16-byte asynchronous copies (the caller waits)
template <int N, int P>
__device__ __forceinline__ void rows_in_async(float *tile, const float *g, int lane)
{
    constexpr int Q = N / 4;
#pragma unroll
    for (int e = lane; e < 32 * Q; e += 32) {
        const int r = e / Q, c = 4 * (e % Q);
        cp_async16(tile + r * P + c, g + r * N + c);
    }
}

// one tile row to registers in upwind order (rev: the row mirrored) and back
template <int N>
__device__ __forceinline__ void row_load_dir(float (&x)[N], const float *row, bool rev)
{
    if (!rev) {
        row_load<N>(x, row);
        return;
    }
#pragma unroll
    for (int c = 0; c < N; c += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(row + N - 4 - c);
        x[c] = a.w; x[c + 1] = a.z; x[c + 2] = a.y; x[c + 3] = a.x;
    }
}

template <int N>
__device__ __forceinline__ void row_store_dir(float *row, const float (&x)[N], bool rev)
{
    if (!rev) {
        row_store<N>(row, x);
        return;
    }
#pragma unroll
    for (int c = 0; c < N; c += 4)
        *reinterpret_cast<float4 *>(row + N - 4 - c) = make_float4(x[c + 3], x[c + 2], x[c + 1], x[c]);
}

// vz sweep of FP32 cubes of edge N (16, 32 or 48): persistent warps taking
// units of 32 rows in turn, each staged in shared memory by 16-byte
// asynchronous copies (array order; a row with u_z < 0 is read mirrored)
// while the next unit's rows are prefetched into L2
template <int N>
__global__ void __launch_bounds__(128) k_adjoint_rows(const float *__restrict__ fin,
                                                     float *__restrict__ lam,
                                                     const LineCoef<float> *__restrict__ coef,
                                                     long long np, double *__restrict__ lam_g,
                                                     double scale, int *skipped)
{
    constexpr int P = N + 4, UPC = N * N / 32;   // pitch, units per cube
    constexpr unsigned UB = 32 * N * sizeof(float);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *tf = reinterpret_cast<float *>(smem_raw) + warp * 2 * 32 * P;
    float *tl = tf + 32 * P;
    const long long nunits = np * UPC;
    const long long ustride = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long unit = (long long)blockIdx.x * (blockDim.x >> 5) + warp; unit < nunits;
         unit += ustride) {
        const long long cell = unit / UPC;
        const LineCoef<float> cf = coef[cell * 3 + 2];
        const long long next = unit + ustride;
        if (lane == 0 && next < nunits) {
            prefetch_l2(fin + next * 32 * N, UB);
            prefetch_l2(lam + next * 32 * N, UB);
        }
        if ((cf.code >> 1) != 0) {
            if (lane == 0) atomicExch(skipped, 1);
            continue;
        }
        const bool neg = cf.code & 1;
        const long long off = unit * 32 * N;          // 32 contiguous rows
        __syncwarp();       // the previous unit's tiles are read out
        rows_in_async<N, P>(tf, fin + off, lane);
        rows_in_async<N, P>(tl, lam + off, lane);
        cp_async_wait_all();
        __syncwarp();
        float f[N], l[N];
        row_load_dir<N>(f, tf + lane * P, neg);
        row_load_dir<N>(l, tl + lane * P, neg);
        int arg;
        float lfinf;
        const float db = adjoint_scalar<N, false, true>(f, l, cf, arg, lfinf);
        row_store_dir<N>(tl + lane * P, l, neg);
        tl[lane * P + (neg ? N - 1 - arg : arg)] += lfinf;
        __syncwarp();
        rows_out<N, P>(lam + off, tl, false, lane);
        if (lam_g) {
            float sum = db;
            for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
            if (lane == 0 && sum != 0.f) atomicAdd(lam_g + cell, (double)sum * scale);
        }
    }
}

// The vz and vy adjoints of a half kick in one pass: each warp takes 32
// rows of one cube (one vx plane for N = 32, two for N = 16) and stages the
// cotangent and the vy input of those rows in shared memory with coalesced
// 16-byte loads.  It recomputes the vz input (the forward vy sweep, one
// column per lane, bitwise as the forward kernels), does the vz adjoint one
// row per lane and the vy adjoint one column per lane, and writes the rows
// back.  A cube with a whole-cell shift on any velocity axis is skipped:
// all three of its sweeps go to the fix-up pass.  (A packed variant with two
// rows or columns per lane needs 255 registers, leaves 8 warps per SM and
// ran slower.)
template <int N>
struct KickZY {
    static constexpr int P = N + 4, UPC = N * N / 32, WPC = 4;   // warps per CTA
    static constexpr size_t SMEM = (size_t)WPC * 3 * 32 * P * sizeof(float);
};

template <int N>
__global__ void __launch_bounds__(128) k_kick_adjoint_zy(const float *__restrict__ sb,
                                                        float *__restrict__ lam,
                                                        const LineCoef<float> *__restrict__ coef,
                                                        long long np, double *__restrict__ lam_g,
                                                        double scale_y, double scale_z,
                                                        int *skipped)
{
    constexpr int P = KickZY<N>::P, UPC = KickZY<N>::UPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *tl = reinterpret_cast<float *>(smem_raw) + warp * 3 * 32 * P;
    float *tb = tl + 32 * P;       // vy input rows
    float *tc = tb + 32 * P;       // vz input rows (recomputed)
    const long long unit = (long long)blockIdx.x * KickZY<N>::WPC + warp;
    if (unit >= np * UPC) return;
    const long long cell = unit / UPC;
    const LineCoef<float> cx = coef[cell * 3], cy = coef[cell * 3 + 1], cz = coef[cell * 3 + 2];
    if (((cx.code | cy.code | cz.code) >> 1) != 0) {
        if (lane == 0) atomicExch(skipped, 1);
        return;
    }
    const long long off = unit * 32 * N;
    const bool negy = cy.code & 1, negz = cz.code & 1;
    // the cotangent rows in upwind order along vz; the vy input as it is
    rows_in<N, P>(tl, lam + off, negz, lane);
    rows_in<N, P>(tb, sb + off, false, lane);
    __syncwarp();
    const int pl = lane / N, k = lane % N;          // this lane's vy column
    const int kt = negz ? N - 1 - k : k;            // its position in the upwind rows
    {
        float x[N];
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = tb[(pl * N + j) * P + k];
        const LineW<float> w = weights_one<float>(cy, line_max(x));
        update_line<float, N, false>(x, w, negy);
#pragma unroll
        for (int j = 0; j < N; ++j) tc[(pl * N + j) * P + kt] = x[j];
    }
    __syncwarp();
    float dz, dy;
    {
        float f[N], l[N];
        row_load<N>(f, tc + lane * P);
        row_load<N>(l, tl + lane * P);
        int arg;
        float lfinf;
        dz = adjoint_scalar<N, false, true>(f, l, cz, arg, lfinf);
        row_store<N>(tl + lane * P, l);
        tl[lane * P + arg] += lfinf;
    }
    __syncwarp();
    {
        // the vy column in upwind order (u < 0: from the last row up)
        const int r0 = negy ? N - 1 : 0, rs = negy ? -P : P;
        const float *B = tb + (pl * N + r0) * P + k;
        float f[N];
#pragma unroll
        for (int j = 0; j < N; ++j) f[j] = B[j * rs];
        const float finf = line_max(f);
        const int arg = first_max<N>(f, finf);
        const AdjW<float> w = adj_weights(cy, finf);
        float *L = tl + (pl * N + r0) * P + kt;
        float lF, db;
        adjoint_line_mem<float, N, false, true>(f, L, rs, L, rs, w, lF, db);
        L[arg * rs] += 2.f * lF;
        dy = negy ? -db : db;
    }
    __syncwarp();
    rows_out<N, P>(lam + off, tl, negz, lane);
    if (!lam_g) return;
    for (int d = 16; d > 0; d >>= 1) {
        dz += __shfl_xor_sync(0xffffffffu, dz, d);
        dy += __shfl_xor_sync(0xffffffffu, dy, d);
    }
    if (lane == 0) {
        if (dz != 0.f) atomicAdd(lam_g + 2 * np + cell, (double)dz * scale_z);
        if (dy != 0.f) atomicAdd(lam_g + np + cell, (double)dy * scale_y);
    }
}

// The y and then the z drift adjoint in one pass (FP32, N_y = N_z = N, 16
// (N = 32) or 32 (N = 16) velocity cells per CTA, zero-shift drifts), the
// transpose of k_drift_yz.  The y input is not stored: the CTA recomputes it
// from the z input s3 (the z sweep of its lines, bitwise as the forward pass)
// into a shared tile [y][z][VC].  The y adjoint (lines of two adjacent
// velocity cells) holds its cotangent line, read from global memory, in
// registers and streams the state from the tile, writing the result over it
// (each thread reads and writes only its own line); the z adjoint holds the
// z input, read again from global memory (the CTA's 64 KB of s3 are still in
// L2), in registers and streams its cotangent from the tile, writing the
// result to global memory.  One line array per thread keeps two CTAs per SM.
// The cotangent crosses HBM once for the two sweeps.  Pairs of z lines with
// directions of both signs go through the scalar path.
template <int N>
struct AdjYZ {
    static constexpr int VC = 512 / N, NT = N * VC / 2;
    static constexpr int YP = N * VC + (VC == 16 ? 16 : 0);
    static constexpr size_t SMEM = (size_t)N * YP * sizeof(float);
};

// maximum (at least 0) and its first position of a line read through fget
template <int N, class FG>
__device__ __forceinline__ float2 scan_max2(FG fget, int2 &arg)
{
    float2 m = make_float2(0.f, 0.f);
    int ax = 0, ay = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const float2 v = fget(j);
        ax = v.x > m.x ? j : ax;
        ay = v.y > m.y ? j : ay;
        m.x = fmaxf(m.x, v.x);
        m.y = fmaxf(m.y, v.y);
    }
    arg = make_int2(ax, ay);
    return m;
}

template <int N, bool PERIODIC>
__global__ void __launch_bounds__(AdjYZ<N>::NT, 2) k_drift_adjoint_yz(
    const float *__restrict__ s3, float *__restrict__ lam, const LineCoef<float> *__restrict__ cz,
    const LineCoef<float> *__restrict__ cy, long long nvc, int nvy, int nvz)
{
    constexpr int VC = AdjYZ<N>::VC, YP = AdjYZ<N>::YP, H = VC / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw);
    const int t = threadIdx.x, vp = t % H, r = t / H;    // r: y in the z sweeps, z in the y adjoint
    const long long v0 = (long long)blockIdx.x * VC;
    const long long x0 = (long long)blockIdx.y * N * N;
    const long long v = v0 + 2 * vp;
    const LineCoef<float> ca = cz[(int)(v % nvz)], cb = cz[(int)((v + 1) % nvz)];
    const long long zoff = (x0 + (long long)r * N) * nvc + v;   // z line (y = r, v pair)
    {
        // the y input: the forward z sweep of the line (y = r, v pair)
        float2 x[N];
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = *reinterpret_cast<const float2 *>(s3 + zoff + j * nvc);
        drift_pair<N, PERIODIC>(x, ca, cb);
        float *q = tile + r * YP + 2 * vp;
#pragma unroll
        for (int j = 0; j < N; ++j) *reinterpret_cast<float2 *>(q + j * VC) = x[j];
    }
    __syncthreads();
    {
        // y adjoint: line (z = r, v pair), cells y = 0..N-1 in upwind order
        const LineCoef<float> c = cy[(int)((v0 / nvz) % nvy)];
        const bool neg = c.code & 1;
        const long long st = neg ? -(long long)N * nvc : (long long)N * nvc;
        const long long o0 = (x0 + r) * nvc + v + (neg ? (N - 1) * (long long)N * nvc : 0);
        const int ys = neg ? -YP : YP;
        float2 *q = reinterpret_cast<float2 *>(tile + r * VC + 2 * vp + (neg ? (N - 1) * YP : 0));
        const int qs = ys / 2;
        float2 l[N];
#pragma unroll
        for (int j = 0; j < N; ++j) l[j] = *reinterpret_cast<const float2 *>(lam + o0 + j * st);
        int2 am;
        const float2 finf = scan_max2<N>([&](int j) { return q[j * qs]; }, am);
        const AdjW<float2> w = adj_weights(c, c, finf);
        float2 lF, db;
        adjoint_line_acc<float2, N, PERIODIC, false>(
            [&](int j) { return q[j * qs]; }, [&](int j) { return l[j]; },
            [&](int j, float2 u) { q[j * qs] = u; }, w, lF, db);
        float *qf = reinterpret_cast<float *>(q);
        qf[am.x * ys] += 2.f * lF.x;
        qf[am.y * ys + 1] += 2.f * lF.y;
    }
    __syncthreads();
    {
        // z adjoint: line (y = r, v pair), cells z = 0..N-1
        const bool same = (ca.code & 1) == (cb.code & 1);
        const bool neg = same && (ca.code & 1);
        const long long st = neg ? -(long long)nvc : (long long)nvc;
        const long long o0 = zoff + (neg ? (N - 1) * (long long)nvc : 0);
        const int ts = neg ? -VC / 2 : VC / 2;
        const float2 *q = reinterpret_cast<const float2 *>(tile + r * YP + 2 * vp + (neg ? (N - 1) * VC : 0));
        float2 f[N];
#pragma unroll
        for (int j = 0; j < N; ++j) f[j] = *reinterpret_cast<const float2 *>(s3 + o0 + j * st);
        float2 *out = reinterpret_cast<float2 *>(lam + o0);
        int ax, ay;
        float lfx, lfy;
        if (same) {
            const float2 finf = line_max(f);
            const int2 am = first_max2<N>(f, finf);
            const AdjW<float2> w = adj_weights(ca, cb, finf);
            float2 lF, db;
            adjoint_line_acc<float2, N, PERIODIC, false>(
                [&](int j) { return f[j]; }, [&](int j) { return q[j * ts]; },
                [&](int j, float2 u) { out[j * st / 2] = u; }, w, lF, db);
            ax = am.x; ay = am.y;
            lfx = 2.f * lF.x; lfy = 2.f * lF.y;
        } else {
            float2 fm[N], lm[N];
#pragma unroll
            for (int j = 0; j < N; ++j) { fm[j] = f[j]; lm[j] = q[j * ts]; }
            int am[2];
            float lfm[2];
            adjoint_pair_mixed<N, PERIODIC, false>(fm, lm, ca, cb, am, lfm);
            ax = am[0]; ay = am[1];
            lfx = lfm[0]; lfy = lfm[1];
#pragma unroll
            for (int j = 0; j < N; ++j) out[j * st / 2] = lm[j];
        }
        lam[o0 + ax * st] += lfx;
        lam[o0 + ay * st + 1] += lfy;
    }
}

// persistent warps: as many CTAs of 128 threads as fit on the SMs at once
// (the kernel's register and shared-memory limits), or fewer where there
// are fewer units of four warps
template <class K>
unsigned persistent_grid(K kernel, size_t smem, long long units)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const long long g = (units + 3) / 4, cap = (long long)per_sm * vp_sm_count();
    return (unsigned)(g < cap ? g : cap);
}

// dynamic shared memory above the default 48 KB (static included) must be
// allowed per kernel before its launch
template <class K>
cudaError_t allow_smem(K kernel, size_t dyn)
{
    if (dyn + 1024 <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

template <int N, bool PERIODIC, bool DB, bool BC, bool MIXED>
cudaError_t pairs_launch(vp_ctx *c, const float *fin, float *lam, const LineCoef<float> *coef,
                         const PairGeom &g, dim3 grid, const double *bc, double *lam_g, double scale)
{
    constexpr size_t smem = (size_t)N * 128 * sizeof(float2);     // cotangent slots
    auto *k = k_adjoint_pairs<N, PERIODIC, DB, BC, MIXED>;
    const cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 128, smem, c->stream>>>(fin, lam, coef, g, bc, lam_g, scale, c->adj_flag);
    return cudaGetLastError();
}

template <int N, bool PERIODIC>
cudaError_t pairs_n(vp_ctx *c, const float *fin, float *lam, const LineCoef<float> *coef,
                    const PairGeom &g, dim3 grid, const double *bc, double *lam_g, double scale)
{
    if (g.axis >= 3 && lam_g)
        return pairs_launch<N, PERIODIC, true, false, false>(c, fin, lam, coef, g, grid, bc, lam_g, scale);
    if (bc)
        return pairs_launch<N, PERIODIC, false, true, false>(c, fin, lam, coef, g, grid, bc, lam_g, scale);
    if (g.axis == 2 && g.mixed)
        return pairs_launch<N, PERIODIC, false, false, true>(c, fin, lam, coef, g, grid, bc, lam_g, scale);
    return pairs_launch<N, PERIODIC, false, false, false>(c, fin, lam, coef, g, grid, bc, lam_g, scale);
}

template <int N>
cudaError_t rows_n(vp_ctx *c, const float *fin, float *lam, const LineCoef<float> *coef,
                   double *lam_g, double scale)
{
    constexpr int P = N + 4;
    const size_t smem = 4 * 2 * 32 * P * sizeof(float);
    const cudaError_t e = allow_smem(k_adjoint_rows<N>, smem);
    if (e != cudaSuccess) return e;
    const long long units = c->np * (N * N / 32);
    k_adjoint_rows<N><<<persistent_grid(k_adjoint_rows<N>, smem, units), 128, smem, c->stream>>>(fin, lam, coef, c->np,
                                                                            lam_g, scale, c->adj_flag);
    return cudaGetLastError();
}

}  // namespace

int vp_kick_adjoint3_ok(const vp_ctx *c)
{
    const int n = c->nv[0];
    return !c->isdouble && c->adj_flag && n == c->nv[1] && n == c->nv[2] && (n == 16 || n == 32) &&
           c->np <= 65535;
}

// the three velocity-sweep adjoints of a half kick: sa, sb the inputs of
// the vx and vy sweeps (the vz input is recomputed); lam_g (3 np)
// accumulates the g cotangent with d alpha / d g = tau / dv per axis.  vz and
// vy in one pass, then vx.  Skipped cubes set c->adj_flag.
cudaError_t launch_kick_adjoint3(vp_ctx *c, const void *sa, const void *sb, void *lam,
                                 const void *coef, double *lam_g, double tau)
{
    cudaError_t e = cudaMemsetAsync(c->adj_flag, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    const int n = c->nv[0];
    const LineCoef<float> *cf = (const LineCoef<float> *)coef;
    if (n == 32) {
        typedef KickZY<32> K;
        const unsigned grid = (unsigned)((c->np * K::UPC + K::WPC - 1) / K::WPC);
        if ((e = cudaFuncSetAttribute(k_kick_adjoint_zy<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)K::SMEM)) != cudaSuccess)
            return e;
        k_kick_adjoint_zy<32><<<grid, 32 * K::WPC, K::SMEM, c->stream>>>(
            (const float *)sb, (float *)lam, cf, c->np, lam_g, tau / c->dv[1], tau / c->dv[2],
            c->adj_flag);
    } else {
        typedef KickZY<16> K;
        const unsigned grid = (unsigned)((c->np * K::UPC + K::WPC - 1) / K::WPC);
        k_kick_adjoint_zy<16><<<grid, 32 * K::WPC, K::SMEM, c->stream>>>(
            (const float *)sb, (float *)lam, cf, c->np, lam_g, tau / c->dv[1], tau / c->dv[2],
            c->adj_flag);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_adjoint_pairs(c, sa, lam, 3, coef, lam_g, tau / c->dv[0], nullptr, 1);
}

// the y then z drift adjoints in one pass (zero-shift drifts: the caller
// checks the shift bound); s4, s3 the inputs of the y and z drifts
int vp_drift_adjoint_yz_ok(const vp_ctx *c) { return vp_drift_yz_ok(c); }

// the y then z drift adjoints in one pass (zero-shift drifts: the caller
// checks the shift bound); s3 the input of the z drift (the input of the y
// drift is recomputed from it)
cudaError_t launch_drift_adjoint_yz(vp_ctx *c, const void *s3, void *lam, const void *coef)
{
    const LineCoef<float> *cf = (const LineCoef<float> *)coef;
    const LineCoef<float> *cz = cf + (size_t)2 * c->maxnv, *cy = cf + (size_t)c->maxnv;
    const float *b = (const float *)s3;
    float *l = (float *)lam;
    cudaError_t e;
    if (c->n[1] == 32) {
        typedef AdjYZ<32> K;
        const dim3 grid((unsigned)(c->nvc / K::VC), (unsigned)c->n[0]);
        auto k = c->periodic_space ? k_drift_adjoint_yz<32, true> : k_drift_adjoint_yz<32, false>;
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM)) !=
            cudaSuccess)
            return e;
        k<<<grid, K::NT, K::SMEM, c->stream>>>(b, l, cz, cy, c->nvc, c->nv[1], c->nv[2]);
    } else {
        typedef AdjYZ<16> K;
        const dim3 grid((unsigned)(c->nvc / K::VC), (unsigned)c->n[0]);
        auto k = c->periodic_space ? k_drift_adjoint_yz<16, true> : k_drift_adjoint_yz<16, false>;
        k<<<grid, K::NT, K::SMEM, c->stream>>>(b, l, cz, cy, c->nvc, c->nv[1], c->nv[2]);
    }
    return cudaGetLastError();
}

int vp_adjoint_pairs_ok(const vp_ctx *c, int axis)
{
    if (c->isdouble || !c->adj_flag) return 0;
    if (axis < 3) {
        const int n = c->n[axis];
        // the two lines of a pair (v, v + 1) share their velocity along x or
        // y (an even count of inner velocity cells); along z they may differ
        const long long inner = axis == 0 ? (long long)c->nv[1] * c->nv[2] : (axis == 1 ? c->nv[2] : 2);
        return (n == 16 || n == 32 || n == 48) && c->nvc % 2 == 0 && inner % 2 == 0 &&
               c->np / n <= 65535;
    }
    const int n = c->nv[0];
    return n == c->nv[1] && n == c->nv[2] && (n == 16 || n == 32 || n == 48) && c->np <= 0x7fffffffLL;
}

cudaError_t launch_adjoint_pairs(vp_ctx *c, const void *fin_, void *lam_, int axis,
                                 const void *coef_, double *lam_g, double scale, const double *bc,
                                 int cube3)
{
    const float *fin = (const float *)fin_;
    float *lam = (float *)lam_;
    const LineCoef<float> *coef = (const LineCoef<float> *)coef_;
    if (!cube3) {
        cudaError_t e = cudaMemsetAsync(c->adj_flag, 0, sizeof(int), c->stream);
        if (e != cudaSuccess) return e;
    }
    PairGeom g{};
    g.cube3 = cube3;
    g.axis = axis;
    g.nvc = c->nvc;
    if (axis < 3) {
        const int n = c->n[axis];
        if (axis == 0) { g.cell_stride = (long long)c->n[1] * c->n[2]; g.od = 1; g.m1 = 1; g.m2 = 0; }
        else if (axis == 1) { g.cell_stride = c->n[2]; g.od = c->n[2]; g.m1 = (long long)c->n[1] * c->n[2]; g.m2 = 1; }
        else { g.cell_stride = 1; g.od = 1; g.m1 = c->n[2]; g.m2 = 0; }
        g.va_stride = axis == 0 ? c->nv[1] * c->nv[2] : (axis == 1 ? c->nv[2] : 1);
        g.va_n = c->nv[axis];
        g.units = c->nvc / 2;
        g.nvz = c->nv[2];
        if (axis == 2) {
            // the directions of the two lines of a pair (2m, 2m + 1) differ only
            // where the cell centres straddle v_z = 0 (tau has one sign)
            const double vl = c->cfg.vlo[2], dvz = c->dv[2];
            auto sgn = [](double v) { return v < 0.0 ? -1 : (v > 0.0 ? 1 : 0); };
            for (int k = 0; k + 1 < c->nv[2]; k += 2)
                if (sgn(vl + (k + 0.5) * dvz) != sgn(vl + (k + 1.5) * dvz)) g.mixed = 1;
        }
        if (axis == 2 && c->nv[2] % 4 == 0) {
            const int H = c->nv[2] / 4;
            if (32 % H == 0 && ((long long)c->nv[0] * c->nv[1]) % (2 * (32 / H)) == 0) g.zremap = H;
        }
        const long long outer = c->np / n;
        // one line pair per thread: a thread holds two lines of f and of the
        // cotangent, so latency is hidden by many resident CTAs
        g.per_part = 128;
        const long long nparts = (g.units + 127) / 128;
        const dim3 grid((unsigned)nparts, (unsigned)outer);
        const LineCoef<float> *cf = coef + (size_t)axis * c->maxnv;
        if (c->periodic_space) {
            if (n == 48) return pairs_n<48, true>(c, fin, lam, cf, g, grid, bc, nullptr, 0.0);
            return n == 32 ? pairs_n<32, true>(c, fin, lam, cf, g, grid, bc, nullptr, 0.0)
                           : pairs_n<16, true>(c, fin, lam, cf, g, grid, bc, nullptr, 0.0);
        }
        if (n == 48) return pairs_n<48, false>(c, fin, lam, cf, g, grid, bc, nullptr, 0.0);
        return n == 32 ? pairs_n<32, false>(c, fin, lam, cf, g, grid, bc, nullptr, 0.0)
                       : pairs_n<16, false>(c, fin, lam, cf, g, grid, bc, nullptr, 0.0);
    }
    const int va = axis - 3, n = c->nv[0];
    double *lg = lam_g ? lam_g + (size_t)va * c->np : nullptr;
    if (va == 2) {
        if (n == 48) return rows_n<48>(c, fin, lam, coef, lg, scale);
        return n == 32 ? rows_n<32>(c, fin, lam, coef, lg, scale)
                       : rows_n<16>(c, fin, lam, coef, lg, scale);
    }
    g.pd = n / 2;
    g.pm_hi = va == 0 ? n : (long long)n * n;
    g.vstride = va == 0 ? (long long)n * n : n;
    g.units = (long long)n * n / 2;
    const dim3 grid((unsigned)c->np, (unsigned)((g.units + 127) / 128));
    if (n == 48) return pairs_n<48, false>(c, fin, lam, coef, g, grid, nullptr, lg, scale);
    return n == 32 ? pairs_n<32, false>(c, fin, lam, coef, g, grid, nullptr, lg, scale)
                   : pairs_n<16, false>(c, fin, lam, coef, g, grid, nullptr, lg, scale);
}
