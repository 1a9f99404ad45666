// vp_sweep.cu -- PFC advection sweeps of the 6D distribution function
// (Sec. 2.1 of Yoshikawa, Yoshida & Umemura 2013) on sm_103a.
//
// Layout: f[x][y][z][vx][vy][vz], vz fastest.  Every velocity cube (the
// N^v_x N^v_y N^v_z cells of one spatial cell) is contiguous.
//
//  * kick kernel (T_vx, T_vy, T_vz): one CTA holds one velocity cube in
//    shared memory (rows padded to an odd length so that every sweep
//    direction is bank-conflict free), runs 3 or 6 sweeps on it in place and
//    writes it back.  The acceleration is uniform over the cube, so the shift
//    of all lines of one sweep is uniform.
//  * drift kernel (T_x, T_y, T_z): one CTA stages an N_l x C tile (N_l cells
//    along the swept spatial axis times C contiguous velocity cells) in shared
//    memory with coalesced row loads; each thread owns one line (one velocity
//    cell) and writes its updated line straight back to global memory.
//
// Per line the update is f'_i = (f_{i-s} - phi_{i-s}) + phi_{i-s-1}: the
// conservative form f + Phi^- - Phi^+ of Sec. 2.1 with the whole cells of a
// shift of s cells cancelled.  Lines with u < 0 are processed in the mirrored
// index order.
#include <cuda_runtime.h>

#include "vp_device.cuh"
#include "vp_internal.cuh"

namespace {

// position in memory of upwind-frame index j of a line of n cells
__device__ __forceinline__ int upos(int j, int n, int neg) { return neg ? n - 1 - j : j; }

// ---------------------------------------------------------------------------
// one velocity line in shared memory, in place, outflow boundaries
// (matter leaving [V^-, V^+] vanishes; ghost cells are 0).  Returns the
// amount of f that left the line.
// ---------------------------------------------------------------------------
template <typename T>
__device__ T kick_line(T *L, int st, int n, const LineCoef<T> cf)
{
    const int s = cf.code >> 1, neg = cf.code & 1;
    const T c0 = cf.c0, c1 = cf.c1, c2 = cf.c2;
    T finf = T(0);
    for (int j = 0; j < n; ++j) finf = vmax(finf, L[j * st]);
    if (s == 0) {
        T fm = T(0), f0 = L[upos(0, n, neg) * st], phim = T(0);
        for (int i = 0; i < n; ++i) {
            const T fp = (i + 1 < n) ? L[upos(i + 1, n, neg) * st] : T(0);
            const T ph = pfc_flux(fm, f0, fp, finf, c0, c1, c2);
            L[upos(i, n, neg) * st] = (f0 - ph) + phim;
            phim = ph;
            fm = f0;
            f0 = fp;
        }
        return phim;
    }
    // shift of s >= 1 whole cells: walk downward so that only cells below
    // the one being written are read afterwards
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

// ---------------------------------------------------------------------------
// one kick sweep along velocity axis va for cubes too large for shared
// memory: each CTA stages C lines of one cube in a tile [n][C + 1] (line t
// in column t), lines along vx or vy with one coalesced load per cell
// index, rows (vz) with a cooperative load of the contiguous rows
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_kick_axis(T *__restrict__ f,
                                                  const LineCoef<T> *__restrict__ coef, int va,
                                                  int nx, int ny, int nz, long long np,
                                                  double *lost_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    __shared__ Acc<double> red[32];
    const int C = blockDim.x, CP = C + 1, t = threadIdx.x;
    const int n = va == 0 ? nx : (va == 1 ? ny : nz);
    const int lines = nx * ny * nz / n;
    const long long cell = blockIdx.x;
    T *g = f + cell * (long long)nx * ny * nz;
    const int l0 = blockIdx.y * C;
    const int cnt = lines - l0 < C ? lines - l0 : C;
    const int l = l0 + t;
    const bool active = t < cnt;
    long long off = 0, stride = 1;
    if (va == 0) { off = l; stride = (long long)ny * nz; }            // l = j nz + k
    else if (va == 1) { off = (long long)(l / nz) * ny * nz + l % nz; stride = nz; }
    if (va < 2) {
        if (active)
            for (int j = 0; j < n; ++j) tile[j * CP + t] = g[off + j * stride];
    } else {
        for (int e = t; e < cnt * nz; e += C) tile[(e % nz) * CP + e / nz] = g[(long long)l0 * nz + e];
        __syncthreads();
    }
    T lost = T(0);
    if (active) lost = kick_line(tile + t, CP, n, coef[cell * 3 + va]);
    if (va < 2) {
        if (active)
            for (int j = 0; j < n; ++j) g[off + j * stride] = tile[j * CP + t];
    } else {
        __syncthreads();
        for (int e = t; e < cnt * nz; e += C) g[(long long)l0 * nz + e] = tile[(e % nz) * CP + e / nz];
    }
    Acc<double> a;
    a.add((double)lost);
    a = block_merge(a, red);
    if (t == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

// ---------------------------------------------------------------------------
// consecutive kick sweeps along vy and vz (in the order given) for cubes too
// large for shared memory: both are local to one vx plane, so one CTA stages
// one plane [ny][nz + 1] (odd pitch: rows and columns conflict-free), runs
// the sweeps (one line per thread) and writes the plane back
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_kick_plane(T *__restrict__ f,
                                                   const LineCoef<T> *__restrict__ c0, int a0,
                                                   const LineCoef<T> *__restrict__ c1, int a1,
                                                   int nsw, int nx, int ny, int nz,
                                                   double *lost_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    __shared__ Acc<double> red[32];
    const int P = nz + 1, t = threadIdx.x;
    const long long cell = blockIdx.x;
    T *g = f + (cell * nx + blockIdx.y) * (long long)ny * nz;
    for (int e = t; e < ny * nz; e += blockDim.x) tile[(e / nz) * P + e % nz] = g[e];
    __syncthreads();
    T lost = T(0);
    for (int sw = 0; sw < nsw; ++sw) {
        const int va = sw ? a1 : a0;
        const LineCoef<T> cf = (sw ? c1 : c0)[cell * 3 + va];
        if (va == 1) {
            for (int k = t; k < nz; k += blockDim.x) lost += kick_line(tile + k, P, ny, cf);
        } else {
            for (int j = t; j < ny; j += blockDim.x) lost += kick_line(tile + j * P, 1, nz, cf);
        }
        __syncthreads();
    }
    for (int e = t; e < ny * nz; e += blockDim.x) g[e] = tile[(e / nz) * P + e % nz];
    Acc<double> a;
    a.add((double)lost);
    a = block_merge(a, red);
    if (t == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

// ---------------------------------------------------------------------------
// kick: NX, NY, NZ compile-time cube edges (0 = runtime)
// ---------------------------------------------------------------------------
template <typename T, int NX, int NY, int NZ>
__global__ void __launch_bounds__(1024) k_kick(T *__restrict__ f, const LineCoef<T> *__restrict__ ca,
                                               const LineCoef<T> *__restrict__ cb, int nsweeps,
                                               int first_axis, int rnx, int rny, int rnz,
                                               long long np, double *lost_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *cube = reinterpret_cast<T *>(smem_raw);
    __shared__ Acc<double> red[32];
    const int nx = NX ? NX : rnx, ny = NY ? NY : rny, nz = NZ ? NZ : rnz;
    const int P = nz | 1;                      // odd row pitch
    const int ncube = nx * ny * nz;
    T lost = T(0);
    for (long long cell = blockIdx.x; cell < np; cell += gridDim.x) {
        T *g = f + cell * (long long)ncube;
        for (int e = threadIdx.x; e < ncube; e += blockDim.x) {
            const int r = e / nz, k = e - r * nz;
            cube[r * P + k] = g[e];
        }
        __syncthreads();
        for (int sw = 0; sw < nsweeps; ++sw) {
            const int va = (first_axis + sw) % 3;
            const LineCoef<T> cf = (sw < 3 ? ca : cb)[cell * 3 + va];
            if (va == 0) {                         // lines along vx
                for (int l = threadIdx.x; l < ny * nz; l += blockDim.x) {
                    const int j = l / nz, k = l - j * nz;
                    lost += kick_line(cube + j * P + k, ny * P, nx, cf);
                }
            } else if (va == 1) {                  // lines along vy
                for (int l = threadIdx.x; l < nx * nz; l += blockDim.x) {
                    const int i = l / nz, k = l - i * nz;
                    lost += kick_line(cube + i * ny * P + k, P, ny, cf);
                }
            } else {                               // lines along vz
                for (int l = threadIdx.x; l < nx * ny; l += blockDim.x)
                    lost += kick_line(cube + l * P, 1, nz, cf);
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < ncube; e += blockDim.x) {
            const int r = e / nz, k = e - r * nz;
            g[e] = cube[r * P + k];
        }
        __syncthreads();
    }
    Acc<double> a;
    a.add((double)lost);
    a = block_merge(a, red);
    if (threadIdx.x == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

// ---------------------------------------------------------------------------
// drift: one line per thread from a read-only shared tile; output to global
// ---------------------------------------------------------------------------
template <typename T, bool PERIODIC>
__device__ T drift_line(const T *L, int st, int n, const LineCoef<T> cf, T *out,
                        long long ostride)
{
    const int neg = cf.code & 1;
    const int s = cf.code >> 1;
    const T c0 = cf.c0, c1 = cf.c1, c2 = cf.c2;
    T finf = T(0);
    for (int j = 0; j < n; ++j) finf = vmax(finf, L[j * st]);
    if (PERIODIC) {
        const int sm = s % n;
        T fm = L[upos(n - 1, n, neg) * st], f0 = L[upos(0, n, neg) * st];
        T phim = pfc_flux(L[upos((2 * n - 2) % n, n, neg) * st], fm, f0, finf, c0, c1, c2);
        int i = sm;
        for (int j = 0; j < n; ++j) {
            const int jn = (j + 1 == n) ? 0 : j + 1;
            const T fp = L[upos(jn, n, neg) * st];
            const T ph = pfc_flux(fm, f0, fp, finf, c0, c1, c2);
            out[upos(i, n, neg) * ostride] = (f0 - ph) + phim;
            phim = ph;
            fm = f0;
            f0 = fp;
            i = (i + 1 == n) ? 0 : i + 1;
        }
        return T(0);
    } else {
        T lost = T(0);
        for (int j = (n - s > 0 ? n - s : 0); j < n; ++j) lost += L[upos(j, n, neg) * st];
        for (int i = 0; i < s && i < n; ++i) out[upos(i, n, neg) * ostride] = T(0);
        T fm = T(0), f0 = L[upos(0, n, neg) * st], phim = T(0);
        for (int j = 0; j < n; ++j) {
            const T fp = (j + 1 < n) ? L[upos(j + 1, n, neg) * st] : T(0);
            const T ph = pfc_flux(fm, f0, fp, finf, c0, c1, c2);
            const int i = j + s;
            if (i < n) out[upos(i, n, neg) * ostride] = (f0 - ph) + phim;
            if (j == n - 1 - s) lost += ph;
            phim = ph;
            fm = f0;
            f0 = fp;
        }
        return lost;
    }
}

template <typename T, bool PERIODIC>
__global__ void __launch_bounds__(256) k_drift(T *__restrict__ f, const LineCoef<T> *__restrict__ coef,
                                              int n, long long cell_stride, int od, long long m1,
                                              long long m2, long long nvc, int va_stride,
                                              int va_n, double *lost_out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    __shared__ Acc<double> red[32];
    const int C = blockDim.x;
    const long long v = (long long)blockIdx.x * C + threadIdx.x;
    const int o = blockIdx.y;
    const long long base_cell = (long long)(o / od) * m1 + (long long)(o % od) * m2;
    const bool active = v < nvc;
    T *gline = f + base_cell * nvc + v;
    const long long gstride = cell_stride * nvc;
#pragma unroll 4
    for (int p = 0; p < n; ++p) tile[p * C + threadIdx.x] = active ? gline[p * gstride] : T(0);
    __syncthreads();
    T lost = T(0);
    if (active) {
        const int vi = (int)((v / va_stride) % va_n);
        const LineCoef<T> cf = coef[vi];
        lost = drift_line<T, PERIODIC>(tile + threadIdx.x, C, n, cf, gline, gstride);
    }
    if (!PERIODIC) {
        Acc<double> a;
        a.add((double)lost);
        a = block_merge(a, red);
        if (threadIdx.x == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
    }
}

// ---------------------------------------------------------------------------
// coefficient tables (FP64 shift -> storage-type weights)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_coef_drift(LineCoef<T> *out, int maxnv, int nv0, int nv1, int nv2,
                             const double *vc0, const double *vc1, const double *vc2,
                             double dx0, double dx1, double dx2, const double *tau_ptr,
                             double factor)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = t / maxnv, j = t - a * maxnv;
    if (a >= 3) return;
    const int nva = a == 0 ? nv0 : (a == 1 ? nv1 : nv2);
    if (j >= nva) return;
    const double *vc = a == 0 ? vc0 : (a == 1 ? vc1 : vc2);
    const double dx = a == 0 ? dx0 : (a == 1 ? dx1 : dx2);
    const double tau = (*tau_ptr) * factor;
    out[a * maxnv + j] = make_line_coef<T>(vc[j] * tau / dx);
}

template <typename T>
__global__ void k_coef_kick(LineCoef<T> *out, const double *__restrict__ g, long long np,
                            double dv0, double dv1, double dv2, const double *tau_ptr,
                            double factor)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * np) return;
    const long long cell = t / 3;
    const int a = (int)(t - cell * 3);
    const double dv = a == 0 ? dv0 : (a == 1 ? dv1 : dv2);
    const double tau = (*tau_ptr) * factor;
    out[t] = make_line_coef<T>(g[a * np + cell] * tau / dv);
}

// dt = C min(dt_p, dt_v) (Sec. 2.4), or the fixed dt.  One CTA.
__global__ void k_dt(DevScalars *sc, const double *__restrict__ g, long long np, double idv0,
                     double idv1, double idv2, double dtp, double courant, double dt_fixed)
{
    __shared__ double red[32];
    double m = 0.0;
    for (long long i = threadIdx.x; i < np; i += blockDim.x) {
        m = fmax(m, fabs(g[i]) * idv0);
        m = fmax(m, fabs(g[np + i]) * idv1);
        m = fmax(m, fabs(g[2 * np + i]) * idv2);
    }
    m = block_max(m, red);
    if (threadIdx.x == 0) {
        sc->amax = m;
        if (dt_fixed > 0.0) {
            sc->dt = dt_fixed;
        } else {
            const double dtv = m > 0.0 ? 1.0 / m : INFINITY;
            sc->dt = courant * fmin(dtp, dtv);
        }
    }
}

__global__ void k_advance_time(DevScalars *sc) { sc->t += sc->dt; }

// ---------------------------------------------------------------------------
// rho(x) = dv^3 sum_v f (Sec. 2.2): one CTA per velocity cube, compensated
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_density(const T *__restrict__ f, long long np, int nvc,
                                                double dvol, double *__restrict__ rho)
{
    __shared__ Acc<T> red[32];
    for (long long cell = blockIdx.x; cell < np; cell += gridDim.x) {
        const T *q = f + cell * (long long)nvc;
        Acc<T> a;
        if (sizeof(T) == 4 && (nvc & 3) == 0) {
            // four independent compensated sums (one per float4 lane) for
            // memory-level parallelism, merged at the end
            Acc<T> b, c2, d;
            const float4 *q4 = reinterpret_cast<const float4 *>(q);
            for (int e = threadIdx.x; e < nvc / 4; e += blockDim.x) {
                const float4 v = q4[e];
                a.add((T)v.x);
                b.add((T)v.y);
                c2.add((T)v.z);
                d.add((T)v.w);
            }
            a.merge(b);
            c2.merge(d);
            a.merge(c2);
        } else {
            for (int e = threadIdx.x; e < nvc; e += blockDim.x) a.add(q[e]);
        }
        a = block_merge(a, red);
        if (threadIdx.x == 0) rho[cell] = a.value() * dvol;
        __syncthreads();
    }
}

// per spatial cell: sum f and sum f |v|^2 (FP64, Neumaier) -> partials[2*cell]
template <typename T>
__global__ void __launch_bounds__(256) k_energy_partials(const T *__restrict__ f, long long np,
                                                        int nvx, int nvy, int nvz,
                                                        const double *vcx, const double *vcy,
                                                        const double *vcz, double *partials)
{
    __shared__ Acc<double> red[32];
    const int nvc = nvx * nvy * nvz;
    for (long long cell = blockIdx.x; cell < np; cell += gridDim.x) {
        const T *q = f + cell * (long long)nvc;
        Acc<double> a0, a2;
        for (int e = threadIdx.x; e < nvc; e += blockDim.x) {
            const int i = e / (nvy * nvz);
            const int r = e - i * nvy * nvz;
            const int j = r / nvz, k = r - j * nvz;
            const double v2 = vcx[i] * vcx[i] + vcy[j] * vcy[j] + vcz[k] * vcz[k];
            const double x = (double)q[e];
            a0.add(x);
            a2.add(x * v2);
        }
        a0 = block_merge(a0, red);
        if (threadIdx.x == 0) partials[2 * cell] = a0.value();
        __syncthreads();
        a2 = block_merge(a2, red);
        if (threadIdx.x == 0) partials[2 * cell + 1] = a2.value();
        __syncthreads();
    }
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 152;
    }
    return n;
}

template <typename T, int NX, int NY, int NZ>
cudaError_t launch_kick_t(vp_ctx *c, T *f, const LineCoef<T> *ca, const LineCoef<T> *cb,
                          int nsweeps, int first_axis)
{
    const int nx = c->nv[0], ny = c->nv[1], nz = c->nv[2];
    const int P = nz | 1;
    const size_t smem = (size_t)nx * ny * P * sizeof(T);
    int lines = ny * nz;
    if (nx * nz > lines) lines = nx * nz;
    if (nx * ny > lines) lines = nx * ny;
    int threads = ((lines + 31) / 32) * 32;
    if (threads > 1024) threads = 1024;
    if (threads < 64) threads = 64;
    auto kern = k_kick<T, NX, NY, NZ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)per_sm * sm_count();
    if (grid > c->np) grid = c->np;
    kern<<<(unsigned)grid, threads, smem, c->stream>>>(f, ca, cb, nsweeps, first_axis, nx, ny,
                                                       nz, c->np, &c->sc->lost);
    return cudaGetLastError();
}

// cube in shared memory (odd row pitch) for the whole-cube kernel
size_t kick_cube_bytes(const vp_ctx *c)
{
    return (size_t)c->nv[0] * c->nv[1] * (c->nv[2] | 1) * c->esize;
}

template <typename T>
cudaError_t launch_kick_axes(vp_ctx *c, T *f, const LineCoef<T> *ca, const LineCoef<T> *cb,
                             int nsweeps, int first_axis)
{
    const int C = sizeof(T) == 8 ? 128 : 256;
    cudaError_t e;
    for (int sw = 0; sw < nsweeps;) {
        const int va = (first_axis + sw) % 3;
        const LineCoef<T> *cf = sw < 3 ? ca : cb;
        if (va > 0) {
            // a run of sweeps local to vx planes: this one and, if it is
            // along the other of vy / vz, the next
            int nsw = 1;
            const int vb = (first_axis + sw + 1) % 3;
            if (sw + 1 < nsweeps && vb > 0) nsw = 2;
            const size_t smem = (size_t)c->nv[1] * (c->nv[2] + 1) * sizeof(T);
            if ((e = cudaFuncSetAttribute(k_kick_plane<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem)) != cudaSuccess)
                return e;
            int threads = ((c->nv[1] > c->nv[2] ? c->nv[1] : c->nv[2]) + 31) / 32 * 32;
            if (threads > 256) threads = 256;
            const dim3 grid((unsigned)c->np, (unsigned)c->nv[0]);
            k_kick_plane<T><<<grid, threads, smem, c->stream>>>(
                f, cf, va, (sw + 1 < 3 ? ca : cb), vb, nsw, c->nv[0], c->nv[1], c->nv[2],
                &c->sc->lost);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            sw += nsw;
            continue;
        }
        const int n = c->nv[va];
        const long long lines = c->nvc / n;
        const size_t smem = (size_t)n * (C + 1) * sizeof(T);
        if ((e = cudaFuncSetAttribute(k_kick_axis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        const dim3 grid((unsigned)c->np, (unsigned)((lines + C - 1) / C));
        k_kick_axis<T><<<grid, C, smem, c->stream>>>(f, cf, va, c->nv[0], c->nv[1], c->nv[2],
                                                     c->np, &c->sc->lost);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++sw;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_kick_dispatch(vp_ctx *c, T *f, const LineCoef<T> *ca, const LineCoef<T> *cb,
                                 int nsweeps, int first_axis)
{
    if (kick_cube_bytes(c) > 220 * 1024)
        return launch_kick_axes<T>(c, f, ca, cb, nsweeps, first_axis);
    const int nx = c->nv[0], ny = c->nv[1], nz = c->nv[2];
    if (nx == ny && ny == nz) {
        if (nx == 16) return launch_kick_t<T, 16, 16, 16>(c, f, ca, cb, nsweeps, first_axis);
        if (nx == 32) return launch_kick_t<T, 32, 32, 32>(c, f, ca, cb, nsweeps, first_axis);
    }
    return launch_kick_t<T, 0, 0, 0>(c, f, ca, cb, nsweeps, first_axis);
}

template <typename T>
cudaError_t launch_drift_t(vp_ctx *c, T *f, int axis, const LineCoef<T> *coef)
{
    const int n = c->n[axis];
    long long cell_stride;
    int od;
    long long m1, m2;
    if (axis == 0) {
        cell_stride = (long long)c->n[1] * c->n[2];
        od = 1; m1 = 1; m2 = 0;
    } else if (axis == 1) {
        cell_stride = c->n[2];
        od = c->n[2]; m1 = (long long)c->n[1] * c->n[2]; m2 = 1;
    } else {
        cell_stride = 1;
        od = 1; m1 = c->n[2]; m2 = 0;
    }
    const int va_stride = axis == 0 ? c->nv[1] * c->nv[2] : (axis == 1 ? c->nv[2] : 1);
    const int va_n = c->nv[axis];
    const int C = c->isdouble ? 128 : 256;
    const size_t smem = (size_t)n * C * sizeof(T);
    const long long outer = c->np / n;
    dim3 grid((unsigned)((c->nvc + C - 1) / C), (unsigned)outer);
    const LineCoef<T> *cf = coef + (size_t)axis * c->maxnv;
    if (c->periodic_space) {
        auto kern = k_drift<T, true>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, C, smem, c->stream>>>(f, cf, n, cell_stride, od, m1, m2, c->nvc, va_stride,
                                           va_n, &c->sc->lost);
    } else {
        auto kern = k_drift<T, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, C, smem, c->stream>>>(f, cf, n, cell_stride, od, m1, m2, c->nvc, va_stride,
                                           va_n, &c->sc->lost);
    }
    return cudaGetLastError();
}

}  // namespace

int vp_sm_count() { return sm_count(); }

cudaError_t launch_coef_drift(vp_ctx *c, const double *tau_ptr, double factor, void *out)
{
    const int total = 3 * c->maxnv;
    const int threads = 128, blocks = (total + threads - 1) / threads;
    if (c->isdouble)
        k_coef_drift<double><<<blocks, threads, 0, c->stream>>>(
            (LineCoef<double> *)out, c->maxnv, c->nv[0], c->nv[1], c->nv[2], c->vc[0], c->vc[1],
            c->vc[2], c->dx[0], c->dx[1], c->dx[2], tau_ptr, factor);
    else
        k_coef_drift<float><<<blocks, threads, 0, c->stream>>>(
            (LineCoef<float> *)out, c->maxnv, c->nv[0], c->nv[1], c->nv[2], c->vc[0], c->vc[1],
            c->vc[2], c->dx[0], c->dx[1], c->dx[2], tau_ptr, factor);
    return cudaGetLastError();
}

cudaError_t launch_coef_kick(vp_ctx *c, const double *g, const double *tau_ptr, double factor,
                             void *out)
{
    const long long total = 3 * c->np;
    const int threads = 256;
    const unsigned blocks = (unsigned)((total + threads - 1) / threads);
    if (c->isdouble)
        k_coef_kick<double><<<blocks, threads, 0, c->stream>>>(
            (LineCoef<double> *)out, g, c->np, c->dv[0], c->dv[1], c->dv[2], tau_ptr, factor);
    else
        k_coef_kick<float><<<blocks, threads, 0, c->stream>>>(
            (LineCoef<float> *)out, g, c->np, c->dv[0], c->dv[1], c->dv[2], tau_ptr, factor);
    return cudaGetLastError();
}

cudaError_t launch_dt(vp_ctx *c, const double *g)
{
    double dtp = INFINITY;
    for (int a = 0; a < 3; ++a) {
        const double vmax = fmax(fabs(c->cfg.vlo[a]), fabs(c->cfg.vhi[a]));
        if (vmax > 0) dtp = fmin(dtp, c->dx[a] / vmax);
    }
    k_dt<<<1, 1024, 0, c->stream>>>(c->sc, g, c->np, 1.0 / c->dv[0], 1.0 / c->dv[1],
                                    1.0 / c->dv[2], dtp, c->cfg.courant, c->cfg.dt_fixed);
    return cudaGetLastError();
}

cudaError_t launch_advance_time(vp_ctx *c)
{
    k_advance_time<<<1, 1, 0, c->stream>>>(c->sc);
    return cudaGetLastError();
}

cudaError_t launch_drift(vp_ctx *c, void *f, int axis, const void *coef, double max_alpha,
                         double *rho_part)
{
    const bool fast = vp_drift_fast_ok(c, axis) && max_alpha < 1.0;
    if (rho_part && !(fast && axis == 0 && vp_rho_fuse_ok(c))) return cudaErrorNotSupported;
    if (fast) return launch_drift_fast(c, f, axis, coef, rho_part);
    if (c->isdouble)
        return launch_drift_t<double>(c, (double *)f, axis, (const LineCoef<double> *)coef);
    return launch_drift_t<float>(c, (float *)f, axis, (const LineCoef<float> *)coef);
}

cudaError_t launch_kick(vp_ctx *c, void *f, const void *coef_a, const void *coef_b, int nsweeps,
                        int first_axis)
{
    if (vp_kick_fast_ok(c)) return launch_kick_fast(c, f, coef_a, coef_b, nsweeps, first_axis);
    if (vp_kick_big_ok(c)) return launch_kick_big(c, f, coef_a, coef_b, nsweeps, first_axis);
    if (vp_kick_f64_ok(c)) return launch_kick_f64(c, f, coef_a, coef_b, nsweeps, first_axis, nullptr);
    if (c->isdouble)
        return launch_kick_dispatch<double>(c, (double *)f, (const LineCoef<double> *)coef_a,
                                            (const LineCoef<double> *)coef_b, nsweeps,
                                            first_axis);
    return launch_kick_dispatch<float>(c, (float *)f, (const LineCoef<float> *)coef_a,
                                       (const LineCoef<float> *)coef_b, nsweeps, first_axis);
}

cudaError_t launch_sweep_into(vp_ctx *c, const void *src, void *dst, int axis, const void *coef,
                              double drift_alpha_bound)
{
    if (axis >= 3 && vp_kick_fast_ok(c))
        return launch_kick_fast(c, const_cast<void *>(src), coef, nullptr, 1, axis - 3, dst);
    if (axis >= 3 && vp_kick_big_ok(c))
        return launch_kick_big(c, const_cast<void *>(src), coef, nullptr, 1, axis - 3, dst);
    if (axis >= 3 && vp_kick_f64_ok(c))
        return launch_kick_f64(c, const_cast<void *>(src), coef, nullptr, 1, axis - 3, dst);
    if (axis < 3 && vp_drift_fast_ok(c, axis) && drift_alpha_bound < 1.0)
        return launch_drift_fast(c, const_cast<void *>(src), axis, coef, nullptr, dst);
    cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)c->ncells * c->esize,
                                    cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
    if (axis < 3) return launch_drift(c, dst, axis, coef, drift_alpha_bound, nullptr);
    return launch_kick(c, dst, coef, nullptr, 1, axis - 3);
}

cudaError_t launch_density(vp_ctx *c, const void *f, double *rho)
{
    long long grid = (long long)sm_count() * 8;
    if (grid > c->np) grid = c->np;
    if (c->isdouble)
        k_density<double><<<(unsigned)grid, 256, 0, c->stream>>>((const double *)f, c->np,
                                                                 (int)c->nvc, c->dvol_v, rho);
    else
        k_density<float><<<(unsigned)grid, 256, 0, c->stream>>>((const float *)f, c->np,
                                                                (int)c->nvc, c->dvol_v, rho);
    return cudaGetLastError();
}

cudaError_t launch_energy_partials(vp_ctx *c, const void *f, double *partials)
{
    long long grid = (long long)sm_count() * 8;
    if (grid > c->np) grid = c->np;
    if (c->isdouble)
        k_energy_partials<double><<<(unsigned)grid, 256, 0, c->stream>>>(
            (const double *)f, c->np, c->nv[0], c->nv[1], c->nv[2], c->vc[0], c->vc[1],
            c->vc[2], partials);
    else
        k_energy_partials<float><<<(unsigned)grid, 256, 0, c->stream>>>(
            (const float *)f, c->np, c->nv[0], c->nv[1], c->nv[2], c->vc[0], c->vc[1], c->vc[2],
            partials);
    return cudaGetLastError();
}
