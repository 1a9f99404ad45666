// vp_sweep_fast.cu -- register-line PFC sweep kernels for the grid sizes of
// the measured workloads (line lengths 16, 32, 48, 64), zero-shift sweeps
// (|alpha| < 1, which every Courant-limited step satisfies).
//
//  * k_kick_fast<N>: one velocity cube of N^3 floats per CTA in shared memory
//    (row pitch N + 4 floats: 16-byte aligned rows, conflict-free columns and
//    rows).  vx and vy sweeps: each thread loads two neighbouring lines
//    (adjacent vz) with 8-byte shared loads and updates both with packed
//    f32x2 arithmetic; vz sweep: one contiguous line per thread with 16-byte
//    shared loads.  A cube-sweep whose shift has a whole-cell part falls back
//    to the generic in-place line routine.
//  * k_drift_fast<T, N>: each thread owns two (float) or one (double)
//    position lines, loads them straight from global memory into registers
//    (a warp reads 256 contiguous bytes per load), updates them and stores
//    them back.  Optionally (x sweep) it accumulates the density of the
//    updated f: per-thread double-float sums over the velocity cells it
//    visits (kept in the thread's shared-memory slots), one reduction per
//    CTA into a small partial buffer.
//  * k_drift_yz<N>: the z and the y drift in one pass through a shared tile.
//  * k_kick6<N>: the six sweeps of two consecutive half kicks in one pass.
//  * k_kick_vx_big / k_kick_plane_big: cubes of 48^3, above shared memory.
#include <cuda_runtime.h>

#include "vp_device.cuh"
#include "vp_internal.cuh"
#include "vp_fast_line.cuh"
#include "vp_line.cuh"

using namespace vpline;

int vp_sm_count();

namespace {

// ---------------------------------------------------------------------------
// kick: FP32 velocity cubes of edge N (16 or 32)
//
// Line ownership: for sweeps along vx and vy each thread owns the two lines
// at vz = k, k + 1 of one (vy resp. vx) index; for vz it owns two contiguous
// rows.  The first sweep of a cube reads its lines straight from global
// memory into registers.  A last sweep along vx or vy writes its lines
// straight back (a warp store covers two 128-byte rows); a last sweep along
// vz first writes its rows to shared memory, after which each warp copies
// the 64 rows it owns out with 16-byte stores that cover 512 contiguous
// bytes.  The next cube's loads are issued before the barrier that protects
// the buffer, so they overlap the end of the previous cube, and one bulk L2
// prefetch per cube brings the cube after next into L2.
// ---------------------------------------------------------------------------
template <int N>
struct KickCube {
    static constexpr int P = N + 4;           // row pitch (floats)
    static constexpr int NU = N * N / 2;      // units of two packed lines per sweep
    static constexpr int NT = NU;             // threads: one unit each
    static constexpr int NC = N * N * N;
};

// element (i, j, k) of the cube: global offset and shared offset
template <int N>
__device__ __forceinline__ int goff(int i, int j, int k) { return (i * N + j) * N + k; }
template <int N>
__device__ __forceinline__ int soff(int i, int j, int k) { return (i * N + j) * KickCube<N>::P + k; }

// pair lines along va (0: vx, 1: vy) owned by thread t: returns the element
// offsets of line cell j through base + j * step (k is even)
template <int N, bool GLOBAL>
__device__ __forceinline__ void pair_geom(int va, int t, int &base, int &step)
{
    const int other = t / (N / 2), k = 2 * (t % (N / 2));
    if (va == 0) {
        base = GLOBAL ? goff<N>(0, other, k) : soff<N>(0, other, k);
        step = GLOBAL ? N * N : N * KickCube<N>::P;
    } else {
        base = GLOBAL ? goff<N>(other, 0, k) : soff<N>(other, 0, k);
        step = GLOBAL ? N : KickCube<N>::P;
    }
}

template <int N, bool GLOBAL>
__device__ __forceinline__ void load_pairs(const float *src, int va, int t, float2 (&x)[N])
{
    int base, step;
    pair_geom<N, GLOBAL>(va, t, base, step);
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = *reinterpret_cast<const float2 *>(src + base + j * step);
}

template <int N, bool GLOBAL>
__device__ __forceinline__ void store_pairs(float *dst, int va, int t, const float2 (&x)[N])
{
    int base, step;
    pair_geom<N, GLOBAL>(va, t, base, step);
#pragma unroll
    for (int j = 0; j < N; ++j) *reinterpret_cast<float2 *>(dst + base + j * step) = x[j];
}

// rows (vz lines) (i, j) = (2q, j) and (2q + 1, j) with q = t / N, j = t % N,
// packed as one float2 line x[k] = (row a cell k, row b cell k).  A warp
// owns the same vx planes here as in the vy sweep (plane t / (N/2)), so a
// vy -> vz (or vz -> vy) transition only needs a warp barrier.
template <int N>
__device__ __forceinline__ void row_pair(int t, int &ra, int &rb)
{
    const int q = t / N, j = t % N;
    ra = (2 * q) * N + j;
    rb = (2 * q + 1) * N + j;
}

template <int N, bool GLOBAL>
__device__ __forceinline__ void load_rows(const float *src, int t, float2 (&x)[N])
{
    int r0, r1;
    row_pair<N>(t, r0, r1);
    const float *ra = src + (GLOBAL ? r0 * N : r0 * KickCube<N>::P);
    const float *rb = src + (GLOBAL ? r1 * N : r1 * KickCube<N>::P);
#pragma unroll
    for (int j = 0; j < N; j += 4) {
        const float4 qa = *reinterpret_cast<const float4 *>(ra + j);
        const float4 qb = *reinterpret_cast<const float4 *>(rb + j);
        x[j] = make_float2(qa.x, qb.x);
        x[j + 1] = make_float2(qa.y, qb.y);
        x[j + 2] = make_float2(qa.z, qb.z);
        x[j + 3] = make_float2(qa.w, qb.w);
    }
}

template <int N, bool GLOBAL>
__device__ __forceinline__ void store_rows(float *dst, int t, const float2 (&x)[N])
{
    int r0, r1;
    row_pair<N>(t, r0, r1);
    float *ra = dst + (GLOBAL ? r0 * N : r0 * KickCube<N>::P);
    float *rb = dst + (GLOBAL ? r1 * N : r1 * KickCube<N>::P);
#pragma unroll
    for (int j = 0; j < N; j += 4) {
        *reinterpret_cast<float4 *>(ra + j) = make_float4(x[j].x, x[j + 1].x, x[j + 2].x, x[j + 3].x);
        *reinterpret_cast<float4 *>(rb + j) = make_float4(x[j].y, x[j + 1].y, x[j + 2].y, x[j + 3].y);
    }
}

// rows [64 w, 64 w + 64) of the cube belong to warp w in the vz sweep (for
// N = 16 and N = 32): copy them from shared to global memory, coalesced
template <int N>
__device__ __forceinline__ void copy_out_rows(float *go, const float *cube, int warp, int lane)
{
    constexpr int Q = N / 4;                    // 16-byte chunks per row
#pragma unroll 4
    for (int e = lane; e < 64 * Q; e += 32) {
        const int r = 64 * warp + e / Q, c = 4 * (e % Q);
        *reinterpret_cast<float4 *>(go + r * N + c) =
            *reinterpret_cast<const float4 *>(cube + r * KickCube<N>::P + c);
    }
}

// asynchronous prefetch of [p, p + bytes) into L2 (16-byte aligned, bytes a
// multiple of 16)
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// whole cube through shared memory (a sweep moves by whole cells)
template <int N>
__device__ __noinline__ float kick_cube_shifted(const float *g, float *go, float *cube,
                                                const LineCoef<float> *cf, int nsweeps,
                                                int first_axis, float *inter0 = nullptr,
                                                float *inter1 = nullptr)
{
    constexpr int P = KickCube<N>::P;
    constexpr int NT = KickCube<N>::NT;
    constexpr int NC = KickCube<N>::NC;
    const int t = threadIdx.x;
    float lost = 0.f;
    for (int e = t; e < NC / 4; e += NT) {
        const int r = (4 * e) / N, k = (4 * e) % N;
        *reinterpret_cast<float4 *>(cube + r * P + k) = reinterpret_cast<const float4 *>(g)[e];
    }
    __syncthreads();
    for (int sw = 0; sw < nsweeps; ++sw) {
        const int va = (first_axis + sw) % 3;
        const LineCoef<float> c = cf[sw];
        for (int l = t; l < N * N; l += NT) {
            float *base;
            int st;
            if (va == 0) { base = cube + (l / N) * P + (l % N); st = N * P; }
            else if (va == 1) { base = cube + (l / N) * N * P + (l % N); st = P; }
            else { base = cube + l * P; st = 1; }
            lost += kick_line_shifted(base, st, N, c);
        }
        __syncthreads();
        float *ist = sw == 0 ? inter0 : (sw == 1 ? inter1 : nullptr);
        if (ist && sw < nsweeps - 1) {
            for (int e = t; e < NC / 4; e += NT) {
                const int r = (4 * e) / N, k = (4 * e) % N;
                reinterpret_cast<float4 *>(ist)[e] = *reinterpret_cast<const float4 *>(cube + r * P + k);
            }
            __syncthreads();
        }
    }
    for (int e = t; e < NC / 4; e += NT) {
        const int r = (4 * e) / N, k = (4 * e) % N;
        reinterpret_cast<float4 *>(go)[e] = *reinterpret_cast<const float4 *>(cube + r * P + k);
    }
    return lost;
}

template <int N>
__global__ void __launch_bounds__(KickCube<N>::NT) k_kick_fast(float *__restrict__ f,
                                                             const LineCoef<float> *__restrict__ ca,
                                                             const LineCoef<float> *__restrict__ cb,
                                                             int nsweeps, int first_axis, long long np,
                                                             double *lost_out, float *__restrict__ fo,
                                                             float *__restrict__ inter0,
                                                             float *__restrict__ inter1,
                                                             const int *gate)
{
    if (gate && *gate == 0) return;
    constexpr int NC = KickCube<N>::NC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *cube = reinterpret_cast<float *>(smem_raw);
    __shared__ Acc<double> red[32];
    __shared__ LineCoef<float> scf[2][6];
    const int t = threadIdx.x;
    float lost = 0.f;
    int par = 0;
    for (long long cell = blockIdx.x; cell < np; cell += gridDim.x, par ^= 1) {
        float *g = f + cell * (long long)NC;
        float *go = fo + cell * (long long)NC;          // output cube (== g in place)
        if (gate && ((ca[cell * 3].code | ca[cell * 3 + 1].code | ca[cell * 3 + 2].code) >> 1) == 0)
            continue;
        if (t < nsweeps) scf[par][t] = (t < 3 ? ca : cb)[cell * 3 + (first_axis + t) % 3];
        // first sweep: lines straight from global memory, issued before the
        // barrier that publishes the coefficients and retires the previous
        // cube's readers of the buffer
        float2 x[N];
        if (first_axis < 2) load_pairs<N, true>(g, first_axis, t, x);
        else load_rows<N, true>(g, t, x);
        __syncthreads();
        bool shifted = false;
        for (int sw = 0; sw < nsweeps; ++sw) shifted |= (scf[par][sw].code >> 1) != 0;
        if (shifted) {
            lost += kick_cube_shifted<N>(g, go, cube, scf[par], nsweeps, first_axis,
                                         inter0 ? inter0 + cell * (long long)NC : nullptr,
                                         inter1 ? inter1 + cell * (long long)NC : nullptr);
            continue;
        }
        for (int sw = 0; sw < nsweeps; ++sw) {
            const int va = (first_axis + sw) % 3;
            const bool last = sw == nsweeps - 1;
            const LineCoef<float> cf = scf[par][sw];
            if (sw) {
                if (va < 2) load_pairs<N, false>(cube, va, t, x);
                else load_rows<N, false>(cube, t, x);
            }
            lost += sweep_pairs<N>(x, cf);
            if (va < 2) {
                if (last) store_pairs<N, true>(go, va, t, x);
                else store_pairs<N, false>(cube, va, t, x);
            } else {
                store_rows<N, false>(cube, t, x);
                if (last) {
                    __syncwarp();
                    copy_out_rows<N>(go, cube, t >> 5, t & 31);
                }
            }
            // intermediate states for the adjoint's replay
            float *ist = sw == 0 ? inter0 : (sw == 1 ? inter1 : nullptr);
            if (!last && ist) {
                float *gi = ist + cell * (long long)NC;
                if (va < 2) store_pairs<N, true>(gi, va, t, x);
                else store_rows<N, true>(gi, t, x);
            }
            if (!last) {
                const int vb = (first_axis + sw + 1) % 3;
                if (va + vb == 3) __syncwarp();     // vy <-> vz: planes stay with the warp
                else __syncthreads();
            }
        }
    }
    Acc<double> a;
    a.add((double)lost);
    a = block_merge(a, red);
    if (t == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

// The fused kick pass K2^n K1^{n+1}: six sweeps vx vy vz vx vy vz of every
// cube (coefficient tables ca for the first three, cb for the last three),
// in place or into fo.
template <int N>
__global__ void __launch_bounds__(KickCube<N>::NT) k_kick6(float *__restrict__ f,
                                                         const LineCoef<float> *__restrict__ ca,
                                                         const LineCoef<float> *__restrict__ cb,
                                                         long long np, double *lost_out,
                                                         float *__restrict__ fo)
{
    constexpr int NC = KickCube<N>::NC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *cube = reinterpret_cast<float *>(smem_raw);
    __shared__ Acc<double> red[32];
    __shared__ LineCoef<float> scf[2][6];
    const int t = threadIdx.x;
    float lost = 0.f;
    int par = 0;
    for (long long cell = blockIdx.x; cell < np; cell += gridDim.x, par ^= 1) {
        float *g = f + cell * (long long)NC;
        float *go = fo + cell * (long long)NC;
        if (t < 4) {
            const long long nx = cell + gridDim.x;
            if (nx < np) prefetch_l2(f + nx * NC + t * (NC / 4), NC);
        }
        if (t < 6) scf[par][t] = (t < 3 ? ca : cb)[cell * 3 + t % 3];
        float2 x[N];
        load_pairs<N, true>(g, 0, t, x);
        __syncthreads();
        bool shifted = false;
#pragma unroll
        for (int sw = 0; sw < 6; ++sw) shifted |= (scf[par][sw].code >> 1) != 0;
        if (shifted) {
            lost += kick_cube_shifted<N>(g, go, cube, scf[par], 6, 0);
            continue;
        }
        lost += sweep_pairs<N>(x, scf[par][0]);
        store_pairs<N, false>(cube, 0, t, x);
        __syncthreads();
        load_pairs<N, false>(cube, 1, t, x);
        lost += sweep_pairs<N>(x, scf[par][1]);
        store_pairs<N, false>(cube, 1, t, x);
        __syncwarp();
        load_rows<N, false>(cube, t, x);
        lost += sweep_pairs<N>(x, scf[par][2]);
        store_rows<N, false>(cube, t, x);
        __syncthreads();
        load_pairs<N, false>(cube, 0, t, x);
        lost += sweep_pairs<N>(x, scf[par][3]);
        store_pairs<N, false>(cube, 0, t, x);
        __syncthreads();
        load_pairs<N, false>(cube, 1, t, x);
        lost += sweep_pairs<N>(x, scf[par][4]);
        store_pairs<N, false>(cube, 1, t, x);
        __syncwarp();
        load_rows<N, false>(cube, t, x);
        lost += sweep_pairs<N>(x, scf[par][5]);
        store_rows<N, false>(cube, t, x);
        __syncwarp();
        copy_out_rows<N>(go, cube, t >> 5, t & 31);
    }
    Acc<double> a;
    a.add((double)lost);
    a = block_merge(a, red);
    if (t == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

// ---------------------------------------------------------------------------
// kick sweeps for FP32 cubes too large for shared memory (edge N = 48):
//  * k_kick_vx_big: lines along vx, two per thread (adjacent vz, packed),
//    straight from global memory (a warp reads two 192-byte row pieces);
//  * k_kick_plane_big: one or two consecutive sweeps along vy / vz, which
//    are local to a vx plane: each CTA stages four planes [N][N + 1] (odd
//    pitch: rows and columns conflict-free) and sweeps one line per thread
//    in registers.
// A line with a whole-cell shift takes the generic in-place routine.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128) k_kick_vx_big(const float *__restrict__ f,
                                                    const LineCoef<float> *__restrict__ coef,
                                                    long long np, double *lost_out,
                                                    float *__restrict__ fo)
{
    __shared__ Acc<double> red[32];
    constexpr int H = N / 2;
    const int t = threadIdx.x;
    const long long cell = blockIdx.x;
    const int u = blockIdx.y * blockDim.x + t;            // pair index (j, k)
    float lost = 0.f;
    if (u < N * H) {
        const LineCoef<float> cf = coef[cell * 3];
        const long long off = cell * (long long)N * N * N + (u / H) * N + 2 * (u % H);
        const float *g = f + off;
        float *go = fo + off;
        float2 x[N];
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = *reinterpret_cast<const float2 *>(g + i * N * N);
        if ((cf.code >> 1) == 0) {
            lost += sweep_pairs<N>(x, cf);
#pragma unroll
            for (int i = 0; i < N; ++i) *reinterpret_cast<float2 *>(go + i * N * N) = x[i];
        } else {
#pragma unroll
            for (int i = 0; i < N; ++i) *reinterpret_cast<float2 *>(go + i * N * N) = x[i];
            lost += kick_line_shifted(go, N * N, N, cf);
            lost += kick_line_shifted(go + 1, N * N, N, cf);
        }
    }
    Acc<double> a;
    a.add((double)lost);
    a = block_merge(a, red);
    if (t == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

template <int N>
struct PlaneBig {
    static constexpr int P = N + 1, PPC = 4, NT = PPC * N;   // planes per group, threads
    static constexpr int G = N / PPC;                         // groups per cube
    static constexpr int TILE = PPC * N * P;                  // floats per buffer
    static constexpr size_t SMEM = (size_t)2 * TILE * sizeof(float);
};

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}

// Persistent: each CTA takes groups of PPC consecutive vx planes in turn
// (group g: cube g / G, planes (g % G) PPC ...) with two tile buffers; the
// next group is copied asynchronously (cp.async, 4 bytes a thread per
// element: the odd pitch keeps rows and columns conflict-free) while the
// current one is swept.  Groups are disjoint, so in-place use (fo == f) is
// safe.
template <int N>
__global__ void __launch_bounds__(PlaneBig<N>::NT, 3) k_kick_plane_big(
    const float *__restrict__ f, const LineCoef<float> *__restrict__ c0, int a0,
    const LineCoef<float> *__restrict__ c1, int a1, int nsw, long long ngroups, double *lost_out,
    float *__restrict__ fo)
{
    constexpr int P = PlaneBig<N>::P, PPC = PlaneBig<N>::PPC, NT = PlaneBig<N>::NT;
    constexpr int G = PlaneBig<N>::G, TILE = PlaneBig<N>::TILE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tiles = reinterpret_cast<float *>(smem_raw);
    __shared__ Acc<double> red[32];
    const int t = threadIdx.x, pl = t / N, m = t % N;
    // thread t moves column t % N of rows t / N, t / N + NT / N, ... (the
    // PPC planes of a group are PPC * N contiguous rows)
    constexpr int RS = NT / N, NR = PPC * N / RS;         // rows per step, rows per thread
    auto issue = [&](long long g, float *buf) {
        const float *src = f + ((g / G) * N + (g % G) * PPC) * (long long)N * N + (t / N) * N + m;
        float *dst = buf + (t / N) * P + m;
#pragma unroll 8
        for (int i = 0; i < NR; ++i) cp_async4(dst + i * RS * P, src + i * RS * N);
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float lost = 0.f;
    long long g = blockIdx.x;
    if (g < ngroups) issue(g, tiles);
    for (int b = 0; g < ngroups; g += gridDim.x, b ^= 1) {
        float *cur = tiles + b * TILE, *nxt = tiles + (b ^ 1) * TILE;
        const long long gn = g + gridDim.x;
        if (gn < ngroups) {
            issue(gn, nxt);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const long long cell = g / G;
        float *pt = cur + pl * N * P;
        for (int sw = 0; sw < nsw; ++sw) {
            const int va = sw ? a1 : a0;
            const LineCoef<float> cf = (sw ? c1 : c0)[cell * 3 + va];
            float *L = va == 1 ? pt + m : pt + m * P;      // column m (vy) or row m (vz)
            const int st = va == 1 ? P : 1;
            if ((cf.code >> 1) == 0) {
                float x[N];
#pragma unroll
                for (int j = 0; j < N; ++j) x[j] = L[j * st];
                const LineW<float> w = weights_one<float>(cf, line_max(x));
                lost += update_line<float, N, false>(x, w, cf.code & 1);
#pragma unroll
                for (int j = 0; j < N; ++j) L[j * st] = x[j];
            } else {
                lost += kick_line_shifted(L, st, N, cf);
            }
            __syncthreads();
        }
        {
            const float *tp = cur + (t / N) * P + m;
            float *gp = fo + (cell * N + (g % G) * PPC) * (long long)N * N + (t / N) * N + m;
#pragma unroll 8
            for (int i = 0; i < NR; ++i) gp[i * RS * N] = tp[i * RS * P];
        }
        __syncthreads();        // the buffer is refilled two groups later
    }
    Acc<double> a;
    a.add((double)lost);
    a = block_merge(a, red);
    if (t == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

// ---------------------------------------------------------------------------
// drift: lines along a spatial axis, held in registers
// ---------------------------------------------------------------------------
struct DriftGeom {
    long long cell_stride;     // spatial-cell stride of the swept axis
    int od;                    // outer index -> base cell: (o / od) * m1 + (o % od) * m2
    long long m1, m2;
    long long nvc;             // velocity cells per spatial cell
    int va_stride, va_n;       // velocity index along the swept axis: (v / va_stride) % va_n
    long long nunits;          // lines units (pairs for float, cells for double) per outer
    long long per_part;        // units per CTA
    int zremap;                // > 0: warp-uniform direction remap of the z sweep, H pairs
    int nvz;                   // N^v_z
    long long np;
};

template <typename T>
struct DriftVec;
template <>
struct DriftVec<float> { typedef float2 V; static constexpr int W = 2; };
template <>
struct DriftVec<double> { typedef double V; static constexpr int W = 1; };

// logical unit index -> first velocity cell of the unit
__device__ __forceinline__ long long unit_to_v(long long L, const DriftGeom &g, int W)
{
    if (W == 2 && g.zremap > 0) {
        const int H = g.zremap;           // pairs per half row
        const int RW = 32 / H;            // rows per warp
        const long long q = L % H;
        long long r1 = L / H;
        const long long ri = r1 % RW;
        r1 /= RW;
        const long long h = r1 & 1;
        const long long rg = r1 >> 1;
        const long long row = rg * RW + ri;
        return row * g.nvz + (h * H + q) * 2;
    }
    return L * W;
}

// RHO: the per-thread compensated density sums of the N cells of the line
// live in shared memory (slot j of thread t at j * 128 + t: conflict-free),
// which keeps the kernel at 128 registers (16 warps per SM)
template <typename T, int N, bool PERIODIC, bool RHO>
__global__ void __launch_bounds__(128, N <= 32 ? 4 : 1) k_drift_fast(const T *__restrict__ f,
                                                               const LineCoef<T> *__restrict__ coef,
                                                               DriftGeom g, double *__restrict__ rho_part,
                                                               double *lost_out, T *__restrict__ fo)
{
    typedef typename DriftVec<T>::V V;
    constexpr int W = DriftVec<T>::W;
    __shared__ Acc<double> red[32];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Acc<T> *sacc = reinterpret_cast<Acc<T> *>(smem_raw) + threadIdx.x;   // slot j: sacc[j * 128]
    const int o = blockIdx.y;
    const long long base_cell = (long long)(o / g.od) * g.m1 + (long long)(o % g.od) * g.m2;
    const long long gstride = g.cell_stride * g.nvc;
    const T *fb = f + base_cell * g.nvc;
    T *ob = fo + base_cell * g.nvc;
    const long long u0 = (long long)blockIdx.x * g.per_part;
    long long u1 = u0 + g.per_part;
    if (u1 > g.nunits) u1 = g.nunits;
    if constexpr (RHO) {
#pragma unroll
        for (int j = 0; j < N; ++j) sacc[j * 128] = Acc<T>();
    }
    T lost = T(0);
    for (long long L = u0 + threadIdx.x; L < u1; L += blockDim.x) {
        const long long v = unit_to_v(L, g, W);
        V x[N];
        // the line's addresses are stepped through an opaque register: the
        // compiler would otherwise keep all 2 N of them live across the update
        const T *p = fb + v;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            x[j] = *reinterpret_cast<const V *>(p);
            p += gstride;
            asm volatile("" : "+l"(p));
        }
        if constexpr (W == 2) {
            const int via = (int)((v / g.va_stride) % g.va_n);
            const int vib = (int)(((v + 1) / g.va_stride) % g.va_n);
            const LineCoef<float> ca = coef[via];
            const LineCoef<float> cb = coef[vib];
            if ((ca.code & 1) == (cb.code & 1)) {
                const LineW<float2> w = weights_pair2(ca, cb, line_max(x));
                const float2 out = update_line<float2, N, PERIODIC>(x, w, ca.code & 1);
                lost += out.x + out.y;
            } else {
                // the pair straddles the sign change of the velocity: two
                // scalar lines
                float y0[N], y1[N];
#pragma unroll
                for (int j = 0; j < N; ++j) { y0[j] = x[j].x; y1[j] = x[j].y; }
                const LineW<float> w0 = weights_one<float>(ca, line_max(y0));
                const LineW<float> w1 = weights_one<float>(cb, line_max(y1));
                lost += update_line<float, N, PERIODIC>(y0, w0, ca.code & 1);
                lost += update_line<float, N, PERIODIC>(y1, w1, cb.code & 1);
#pragma unroll
                for (int j = 0; j < N; ++j) x[j] = make_float2(y0[j], y1[j]);
            }
        } else {
            const int via = (int)((v / g.va_stride) % g.va_n);
            const LineCoef<T> ca = coef[via];
            lost += update_line_f64<N, PERIODIC>(x, ca.c0, ca.c1, ca.c2, ca.code & 1);
        }
        T *q = ob + v;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            *reinterpret_cast<V *>(q) = x[j];
            q += gstride;
            asm volatile("" : "+l"(q));
        }
        if constexpr (RHO) {
#pragma unroll
            for (int j = 0; j < N; ++j) {
                Acc<T> a = sacc[j * 128];
                if constexpr (W == 2) { a.add(x[j].x); a.add(x[j].y); }
                else a.add(x[j]);
                sacc[j * 128] = a;
            }
        }
    }
    if constexpr (RHO) {
        // per-x reduction over the CTA, written as one partial per (part, cell)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            Acc<T> a = block_merge(sacc[j * 128], reinterpret_cast<Acc<T> *>(red));
            if (threadIdx.x == 0)
                rho_part[(long long)blockIdx.x * g.np + base_cell + j * g.cell_stride] = a.value();
            __syncthreads();
        }
    }
    if (!PERIODIC) {
        Acc<double> a;
        a.add((double)lost);
        a = block_merge(a, red);
        if (threadIdx.x == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
    }
}

// ---------------------------------------------------------------------------
// fused z and y drift (FP32, N_y = N_z = N): a block is (x, chunk of VC
// velocity cells); persistent CTAs take blocks in turn.  A block [y][z][VC]
// is copied into a shared tile with 16-byte cp.async copies; the z sweep
// takes its lines (pairs of adjacent velocity cells) from the tile and
// writes them back in place; the y sweep reads its lines from the tile into
// registers, the copies of the CTA's next block start, and the y lines are
// swept and written straight to global memory.  f crosses HBM once for both
// sweeps.  The chunk lies inside one vz
// row, so every y line of the CTA has the same v_y; the z lines of a pair
// differ in v_z (two coefficients, two scalar lines where the pair
// straddles the sign change of v_z).
// ---------------------------------------------------------------------------
template <int N>
struct DriftYZ {
    static constexpr int VC = 512 / N;                 // velocity cells per CTA
    static constexpr int NT = N * VC / 2;              // threads: one line pair each
    // tile pitch of one y: the r groups of a warp's z-sweep accesses (VC/2
    // lanes each) start on different banks
    static constexpr int YP = N * VC + (VC == 16 ? 16 : 0);
};

template <int N, bool PERIODIC>
__global__ void __launch_bounds__(DriftYZ<N>::NT, 2) k_drift_yz(const float *__restrict__ f,
                                                              const LineCoef<float> *__restrict__ cz,
                                                              const LineCoef<float> *__restrict__ cy,
                                                              long long nvc, int nvy, int nvz,
                                                              long long nblocks, double *lost_out,
                                                              float *__restrict__ fo)
{
    constexpr int VC = DriftYZ<N>::VC, YP = DriftYZ<N>::YP, H = VC / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw);
    __shared__ Acc<double> red[32];
    const int t = threadIdx.x, vp = t % H, r = t / H;    // r: y in the z sweep, z in the y sweep
    const long long nvb = nvc / VC;                      // velocity blocks per x plane
    float lost = 0.f;
    // block b = (x plane b / nvb, velocity cells [VC (b % nvb), + VC)) into
    // the tile [y][z][VC] with asynchronous 16-byte copies (no register
    // staging, few load instructions)
    auto stage = [&](long long b) {
        constexpr int Q = VC / 4, PIECES = N * N * Q;
        const float *src = f + (b / nvb) * N * N * nvc + (b % nvb) * VC;
#pragma unroll 4
        for (int e = t; e < PIECES; e += DriftYZ<N>::NT) {
            const int q = e % Q, yz = e / Q, y = yz / N, z = yz % N;
            const unsigned sa = (unsigned)__cvta_generic_to_shared(tile + y * YP + z * VC + 4 * q);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa),
                         "l"(src + (long long)yz * nvc + 4 * q)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if ((long long)blockIdx.x < nblocks) stage(blockIdx.x);
    for (long long b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const long long v0 = (b % nvb) * VC;
        const long long x0 = (b / nvb) * N * N;          // first spatial cell of the x plane
        const long long v = v0 + 2 * vp;
        float2 x[N];
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        {
            // z sweep of the line (y = r, v pair), in place in the tile
            float *q = tile + r * YP + 2 * vp;
#pragma unroll
            for (int j = 0; j < N; ++j) x[j] = *reinterpret_cast<const float2 *>(q + j * VC);
            const LineCoef<float> ca = cz[(int)(v % nvz)], cb = cz[(int)((v + 1) % nvz)];
            lost += drift_pair<N, PERIODIC>(x, ca, cb);
#pragma unroll
            for (int j = 0; j < N; ++j) *reinterpret_cast<float2 *>(q + j * VC) = x[j];
        }
        __syncthreads();
        {
            const float *q = tile + r * VC + 2 * vp;
#pragma unroll
            for (int j = 0; j < N; ++j) x[j] = *reinterpret_cast<const float2 *>(q + j * YP);
        }
        // every line of the y sweep is in registers: the next block's copies
        // into the tile run under this block's y sweep and stores
        __syncthreads();
        if (b + gridDim.x < nblocks) stage(b + gridDim.x);
        {
            const LineCoef<float> c = cy[(int)((v0 / nvz) % nvy)];
            lost += drift_pair<N, PERIODIC>(x, c, c);
            float *p = fo + (x0 + r) * nvc + v;
            const long long ys = (long long)N * nvc;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                *reinterpret_cast<float2 *>(p) = x[j];
                p += ys;
                asm volatile("" : "+l"(p));
            }
        }
    }
    if (!PERIODIC) {
        Acc<double> a;
        a.add((double)lost);
        a = block_merge(a, red);
        if (t == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
    }
}

template <int N>
cudaError_t drift_yz_n(vp_ctx *c, const float *f, const LineCoef<float> *coef, float *fo)
{
    constexpr int NT = DriftYZ<N>::NT;
    const size_t smem = (size_t)N * DriftYZ<N>::YP * sizeof(float);
    const long long nblocks = (c->nvc / DriftYZ<N>::VC) * (long long)c->n[0];
    const LineCoef<float> *cz = coef + (size_t)2 * c->maxnv, *cy = coef + (size_t)c->maxnv;
    auto kern = c->periodic_space ? k_drift_yz<N, true> : k_drift_yz<N, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // persistent: the CTAs that fit on the GPU at once, each taking blocks
    // in turn
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)per_sm * vp_sm_count();
    if (grid > nblocks) grid = nblocks;
    kern<<<(unsigned)grid, NT, smem, c->stream>>>(f, cz, cy, c->nvc, c->nv[1], c->nv[2], nblocks,
                                                  &c->sc->lost, fo);
    return cudaGetLastError();
}

// rho = dvol * sum_parts partial (Neumaier)
__global__ void k_rho_finish(const double *__restrict__ part, int nparts, long long np, double dvol,
                             double *__restrict__ rho)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    Acc<double> a;
    for (int p = 0; p < nparts; ++p) a.add(part[(long long)p * np + t]);
    rho[t] = a.value() * dvol;
}

template <typename K>
cudaError_t kick_grid(vp_ctx *c, K kern, int threads, size_t smem, long long &grid)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid = (long long)per_sm * vp_sm_count();
    if (grid > c->np) grid = c->np;
    return cudaSuccess;
}

template <int N>
cudaError_t kick_fast_n(vp_ctx *c, float *f, const LineCoef<float> *ca, const LineCoef<float> *cb,
                        int nsweeps, int first_axis, float *fo, float *inter0, float *inter1,
                        const int *gate)
{
    constexpr int P = KickCube<N>::P;
    const size_t smem = (size_t)N * N * P * sizeof(float);
    const int threads = KickCube<N>::NT;
    long long grid = 0;
    cudaError_t e;
    if (nsweeps == 6 && first_axis == 0 && !inter0 && !inter1 && !gate) {
        e = kick_grid(c, k_kick6<N>, threads, smem, grid);
        if (e != cudaSuccess) return e;
        k_kick6<N><<<(unsigned)grid, threads, smem, c->stream>>>(f, ca, cb, c->np, &c->sc->lost,
                                                                  fo ? fo : f);
        return cudaGetLastError();
    }
    e = kick_grid(c, k_kick_fast<N>, threads, smem, grid);
    if (e != cudaSuccess) return e;
    k_kick_fast<N><<<(unsigned)grid, threads, smem, c->stream>>>(
        f, ca, cb, nsweeps, first_axis, c->np, &c->sc->lost, fo ? fo : f, inter0, inter1, gate);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t drift_fast_n(vp_ctx *c, T *f, int axis, const LineCoef<T> *coef, double *rho_part,
                         int nparts, T *fo)
{
    DriftGeom g;
    if (axis == 0) {
        g.cell_stride = (long long)c->n[1] * c->n[2];
        g.od = 1; g.m1 = 1; g.m2 = 0;
    } else if (axis == 1) {
        g.cell_stride = c->n[2];
        g.od = c->n[2]; g.m1 = (long long)c->n[1] * c->n[2]; g.m2 = 1;
    } else {
        g.cell_stride = 1;
        g.od = 1; g.m1 = c->n[2]; g.m2 = 0;
    }
    constexpr int W = DriftVec<T>::W;
    g.nvc = c->nvc;
    g.va_stride = axis == 0 ? c->nv[1] * c->nv[2] : (axis == 1 ? c->nv[2] : 1);
    g.va_n = c->nv[axis];
    g.nunits = c->nvc / W;
    g.nvz = c->nv[2];
    g.np = c->np;
    g.zremap = 0;
    if (W == 2 && axis == 2 && c->nv[2] % 4 == 0) {
        const int H = c->nv[2] / 4;
        if (32 % H == 0 && ((long long)c->nv[0] * c->nv[1]) % (2 * (32 / H)) == 0) g.zremap = H;
    }
    const long long outer = c->np / N;
    if (nparts <= 0) {
        long long target = 4LL * 4 * vp_sm_count();
        nparts = (int)((target + outer - 1) / outer);
        if (nparts < 1) nparts = 1;
        const long long maxparts = (g.nunits + 127) / 128;
        if (nparts > maxparts) nparts = (int)maxparts;
    }
    g.per_part = (g.nunits + nparts - 1) / nparts;
    dim3 grid((unsigned)nparts, (unsigned)outer);
    const bool rho = rho_part != nullptr;
    constexpr bool RHO_OK = (sizeof(T) == 4 && N <= 64) || N <= 16;
    if (rho && !RHO_OK) return cudaErrorNotSupported;
    constexpr size_t racc = (size_t)N * 128 * sizeof(Acc<T>);   // density sums (RHO)
    if constexpr (RHO_OK) {
        if (rho) {
            cudaError_t e = cudaFuncSetAttribute(c->periodic_space ? k_drift_fast<T, N, true, true>
                                                                   : k_drift_fast<T, N, false, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)racc);
            if (e != cudaSuccess) return e;
        }
    }
    if (c->periodic_space) {
        if constexpr (RHO_OK)
            if (rho) {
                k_drift_fast<T, N, true, true><<<grid, 128, racc, c->stream>>>(f, coef, g, rho_part, &c->sc->lost, fo ? fo : f);
                return cudaGetLastError();
            }
        k_drift_fast<T, N, true, false><<<grid, 128, 0, c->stream>>>(f, coef, g, rho_part, &c->sc->lost, fo ? fo : f);
    } else {
        if constexpr (RHO_OK)
            if (rho) {
                k_drift_fast<T, N, false, true><<<grid, 128, racc, c->stream>>>(f, coef, g, rho_part, &c->sc->lost, fo ? fo : f);
                return cudaGetLastError();
            }
        k_drift_fast<T, N, false, false><<<grid, 128, 0, c->stream>>>(f, coef, g, rho_part, &c->sc->lost, fo ? fo : f);
    }
    return cudaGetLastError();
}

}  // namespace

// number of density partials the fused x drift writes per spatial cell
int vp_rho_parts(vp_ctx *c)
{
    const long long outer = c->np / c->n[0];
    long long target = 4LL * 4 * vp_sm_count();
    int nparts = (int)((target + outer - 1) / outer);
    if (nparts < 1) nparts = 1;
    const long long nunits = c->nvc / (c->isdouble ? 1 : 2);
    const long long maxparts = (nunits + 127) / 128;
    if (nparts > maxparts) nparts = (int)maxparts;
    return nparts;
}

// 1 if the register kernels handle this grid
int vp_kick_fast_ok(const vp_ctx *c)
{
    const int n = c->nv[0];
    return !c->isdouble && n == c->nv[1] && n == c->nv[2] && (n == 16 || n == 32);
}

int vp_drift_fast_ok(const vp_ctx *c, int axis)
{
    const int n = c->n[axis];
    if (!(n == 16 || n == 32 || n == 48 || n == 64)) return 0;
    if (!c->isdouble && (c->nvc % 2 != 0)) return 0;
    if (c->isdouble && n > 32) return 0;
    return 1;
}

int vp_rho_fuse_ok(const vp_ctx *c)
{
    return vp_drift_fast_ok(c, 0) && c->n[0] <= (c->isdouble ? 16 : 64);
}

cudaError_t launch_kick_fast(vp_ctx *c, void *f, const void *ca, const void *cb, int nsweeps,
                             int first_axis, void *fo, void *inter0, void *inter1, const int *gate)
{
    if (c->nv[0] == 32)
        return kick_fast_n<32>(c, (float *)f, (const LineCoef<float> *)ca,
                               (const LineCoef<float> *)cb, nsweeps, first_axis, (float *)fo,
                               (float *)inter0, (float *)inter1, gate);
    return kick_fast_n<16>(c, (float *)f, (const LineCoef<float> *)ca, (const LineCoef<float> *)cb,
                           nsweeps, first_axis, (float *)fo, (float *)inter0, (float *)inter1, gate);
}

cudaError_t launch_drift_fast(vp_ctx *c, void *f, int axis, const void *coef, double *rho_part,
                              void *fo)
{
    const int n = c->n[axis];
    const int np = rho_part ? vp_rho_parts(c) : 0;
    if (c->isdouble) {
        const LineCoef<double> *cf = (const LineCoef<double> *)coef + (size_t)axis * c->maxnv;
        if (n == 32) return drift_fast_n<double, 32>(c, (double *)f, axis, cf, rho_part, np, (double *)fo);
        return drift_fast_n<double, 16>(c, (double *)f, axis, cf, rho_part, np, (double *)fo);
    }
    const LineCoef<float> *cf = (const LineCoef<float> *)coef + (size_t)axis * c->maxnv;
    float *o = (float *)fo;
    switch (n) {
    case 16: return drift_fast_n<float, 16>(c, (float *)f, axis, cf, rho_part, np, o);
    case 32: return drift_fast_n<float, 32>(c, (float *)f, axis, cf, rho_part, np, o);
    case 48: return drift_fast_n<float, 48>(c, (float *)f, axis, cf, rho_part, np, o);
    default: return drift_fast_n<float, 64>(c, (float *)f, axis, cf, rho_part, np, o);
    }
}

// 1 if the fused z + y drift handles this grid (FP32, N_y = N_z in {16, 32},
// velocity chunks inside one vz row, zero-shift drift)
int vp_drift_yz_ok(const vp_ctx *c)
{
    if (c->isdouble || c->n[1] != c->n[2]) return 0;
    const int n = c->n[1];
    // (lines of 48: two register-line passes, each near the HBM bound, beat
    // a fused pass of 8-cell chunks)
    if (n != 16 && n != 32) return 0;
    const int vc = 512 / n;
    return c->nv[2] % vc == 0 && c->n[0] <= 65535 && c->nvc / vc <= 0x7fffffffLL;
}

cudaError_t launch_drift_yz(vp_ctx *c, const void *f, const void *coef, void *fo)
{
    if (c->n[1] == 32)
        return drift_yz_n<32>(c, (const float *)f, (const LineCoef<float> *)coef, (float *)fo);
    return drift_yz_n<16>(c, (const float *)f, (const LineCoef<float> *)coef, (float *)fo);
}

// FP32 cubes of edge 48 (too large for shared memory): sweeps one pass per
// vx sweep, one pass per run of consecutive vy / vz sweeps
int vp_kick_big_ok(const vp_ctx *c)
{
    const int n = c->nv[0];
    return !c->isdouble && n == c->nv[1] && n == c->nv[2] && n == 48;
}

cudaError_t launch_kick_big(vp_ctx *c, void *f_, const void *ca_, const void *cb_, int nsweeps,
                            int first_axis, void *fo_)
{
    constexpr int N = 48;
    float *f = (float *)f_;
    float *fo = fo_ ? (float *)fo_ : f;   // the first pass reads f, every pass writes fo
    const LineCoef<float> *ca = (const LineCoef<float> *)ca_, *cb = (const LineCoef<float> *)cb_;
    // whole half kicks and the fused kick: passes of two sweeps on slabs
    cudaError_t e = launch_kick_big3(c, f, ca, cb, nsweeps, first_axis, fo);
    if (e != cudaErrorNotSupported) return e;
    for (int sw = 0; sw < nsweeps;) {
        const int va = (first_axis + sw) % 3;
        const LineCoef<float> *cf = sw < 3 ? ca : cb;
        if (va == 0) {
            const dim3 grid((unsigned)c->np, (unsigned)((N * N / 2 + 127) / 128));
            k_kick_vx_big<N><<<grid, 128, 0, c->stream>>>(sw ? fo : f, cf, c->np, &c->sc->lost, fo);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            ++sw;
            continue;
        }
        int nsw = 1;
        const int vb = (first_axis + sw + 1) % 3;
        if (sw + 1 < nsweeps && vb > 0) nsw = 2;
        typedef PlaneBig<N> PB;
        if ((e = cudaFuncSetAttribute(k_kick_plane_big<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)PB::SMEM)) != cudaSuccess)
            return e;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_kick_plane_big<N>, PB::NT,
                                                               PB::SMEM)) != cudaSuccess)
            return e;
        const long long ngroups = c->np * PB::G;
        long long grid = (long long)vp_sm_count() * (per_sm > 0 ? per_sm : 1);
        if (grid > ngroups) grid = ngroups;
        k_kick_plane_big<N><<<(unsigned)grid, PB::NT, PB::SMEM, c->stream>>>(
            sw ? fo : f, cf, va, sw + 1 < 3 ? ca : cb, vb, nsw, ngroups, &c->sc->lost, fo);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        sw += nsw;
    }
    return cudaSuccess;
}

cudaError_t launch_rho_finish(vp_ctx *c, const double *part, int nparts, double *rho)
{
    k_rho_finish<<<(unsigned)((c->np + 255) / 256), 256, 0, c->stream>>>(part, nparts, c->np,
                                                                        c->dvol_v, rho);
    return cudaGetLastError();
}
