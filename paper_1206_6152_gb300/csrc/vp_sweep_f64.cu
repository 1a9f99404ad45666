// vp_sweep_f64.cu -- velocity sweeps of FP64 velocity cubes of edge 16 or 32
// (Sec. 2.1, the kick T_vx T_vy T_vz of Eq. integration) with lines in
// registers.
//
// GB300 executes FP64 arithmetic at a small fraction of its FP32 rate, so
// an FP64 sweep is bound by its FP64 instructions, not by HBM (16 bytes per
// cell).  Each thread takes one whole line: it reads the line straight from
// global memory into registers (a warp reads 256 contiguous bytes per load
// along vx and vy; along vz each thread reads its own contiguous row), sweeps
// it in the saturating form of the register-line kernels (about 14 FP64
// instructions per cell, against about 21 for the shared-memory line routine
// in the clamp form), and writes it back.  A FP64 cube of 32^3 (256 KB) does
// not fit in shared memory; one launch per sweep costs 16 bytes per cell of
// HBM traffic, far below the arithmetic time.  Lines of a cube with a
// whole-cell shift (|alpha| >= 1) go through the generic in-place routine.
#include <cuda_runtime.h>

#include "vp_device.cuh"
#include "vp_fast_line.cuh"
#include "vp_internal.cuh"
#include "vp_line.cuh"

using namespace vpline;

int vp_sm_count();

namespace {

// sweep along velocity axis va of every cube, one line per thread, from src
// into dst (dst == src in place: each thread reads its whole line before
// writing it, and lines are disjoint)
template <int N>
__global__ void __launch_bounds__(128) k_kick_lines_f64(const double *src, double *dst,
                                                       const LineCoef<double> *__restrict__ coef,
                                                       int va, long long np, double *lost_out)
{
    __shared__ Acc<double> red[32];
    constexpr int NN = N * N;
    const long long nlines = np * NN;
    double lost = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nlines;
         q += (long long)gridDim.x * blockDim.x) {
        const long long cell = q / NN;
        const int u = (int)(q % NN);
        // line u of the cube: va 0 at (vy, vz) = (u / N, u % N), va 1 at (vx,
        // vz), va 2 at (vx, vy); elements base + j * st
        int base, st;
        if (va == 0) { base = u; st = NN; }
        else if (va == 1) { base = (u / N) * NN + u % N; st = N; }
        else { base = u * N; st = 1; }
        const long long off = cell * (long long)(N * NN) + base;
        const LineCoef<double> cf = coef[cell * 3 + va];
        double x[N];
#pragma unroll
        for (int j = 0; j < N; ++j) x[j] = src[off + j * st];
        if ((cf.code >> 1) == 0) {
            lost += update_line_f64<N, false>(x, cf.c0, cf.c1, cf.c2, cf.code & 1);
#pragma unroll
            for (int j = 0; j < N; ++j) dst[off + j * st] = x[j];
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) dst[off + j * st] = x[j];
            lost += kick_line_shifted(dst + off, st, N, cf);
        }
    }
    Acc<double> a;
    a.add(lost);
    a = block_merge(a, red);
    if (threadIdx.x == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

template <int N>
cudaError_t kick_f64_n(vp_ctx *c, const double *src, double *dst, const LineCoef<double> *coef,
                       int va)
{
    const long long nlines = c->np * N * N;
    long long grid = (nlines + 127) / 128;
    const long long cap = 8LL * vp_sm_count();
    if (grid > cap) grid = cap;
    k_kick_lines_f64<N><<<(unsigned)grid, 128, 0, c->stream>>>(src, dst, coef, va, c->np,
                                                              &c->sc->lost);
    return cudaGetLastError();
}

}  // namespace

int vp_kick_f64_ok(const vp_ctx *c)
{
    const int n = c->nv[0];
    return c->isdouble && n == c->nv[1] && n == c->nv[2] && (n == 16 || n == 32);
}

cudaError_t launch_kick_f64(vp_ctx *c, void *f, const void *ca, const void *cb, int nsweeps,
                            int first_axis, void *fo)
{
    double *src = (double *)f;
    double *dst = fo ? (double *)fo : src;
    for (int sw = 0; sw < nsweeps; ++sw) {
        const int va = (first_axis + sw) % 3;
        const LineCoef<double> *cf = (const LineCoef<double> *)(sw < 3 ? ca : cb);
        const double *s = sw ? dst : src;       // the first sweep reads f, the rest dst
        const cudaError_t e = c->nv[0] == 32 ? kick_f64_n<32>(c, s, dst, cf, va)
                                             : kick_f64_n<16>(c, s, dst, cf, va);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
