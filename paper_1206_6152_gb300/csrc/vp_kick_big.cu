// vp_kick_big.cu -- the velocity sweeps of FP32 cubes of edge 48 (442 KB per
// cube, twice the shared memory of an SM) in passes of two sweeps each.
//
// Two consecutive sweeps along different velocity axes touch only the lines
// of a slab that is thin along the third axis: vx and vy sweeps stay inside
// a slab of vz planes, vz and vx inside a slab of vy planes, vy and vz inside
// a slab of vx planes.  The fused kick K2^n K1^{n+1} (Sec. 2.1, Eq.
// integration: vx vy vz vx vy vz) therefore runs as three passes over f,
//   A: vx, vy   (K2 table)            on slabs of 8 vz planes
//   B: vz (K2), vx (K1)               on slabs of 8 vy planes
//   C: vy, vz   (K1 table)            on slabs of 8 vx planes
// and a single half kick (vx vy vz) as A followed by C without its first
// sweep.  Each unit (cube, slab) is one CTA's work at a time; persistent
// CTAs take units in turn.  Lines are held in registers two at a time
// (neighbouring lines packed as float2, f32x2 arithmetic); the slab passes
// between the two sweeps through a shared-memory tile.
//
//   A: the vx line pairs are read straight from global memory (a warp reads
//      eight 32-byte row pieces per load), swept and written to the tile with
//      the vy row index XOR-swizzled by the low bits of vx (so that both the
//      vx and the vy line pairs move without bank conflicts), read back as
//      vy line pairs, swept and stored straight to global memory.  The six
//      slabs of a cube go to six CTAs that run at the same time, so every
//      192-byte row is read from DRAM once.  (Slabs of 32-byte row pieces
//      staged by asynchronous copies, cp.async or TMA, read three times
//      their bytes from DRAM, whatever their L2 eviction policy; plain loads
//      read them once.)
//   B: the slab (48 vx planes x 8 rows of 192 bytes) is prefetched into L2
//      one unit ahead and copied into the tile with 16-byte cp.async
//      copies; the vz sweep reads its row pairs from
//      the tile and writes them back; the vx line pairs are read from the
//      tile, the copies of the CTA's next slab start, and the vx lines are
//      swept and stored to global memory.
//   C: the vy line pairs are read from global memory (a warp reads 192
//      contiguous bytes per row), swept and written to the tile; the vz
//      sweep takes row pairs from the tile and writes them back, while the
//      CTA's next slab (73.7 KB, contiguous) is fetched into L2 by a bulk
//      prefetch; the tile is copied out with 16-byte stores that cover
//      contiguous memory.
//
// A unit whose cube has a whole-cell shift in one of the pass's sweeps
// (|alpha| >= 1, outside the Courant limit) is swept line by line in global
// memory by the generic routine.
#include <cuda_runtime.h>

#include "vp_device.cuh"
#include "vp_fast_line.cuh"
#include "vp_internal.cuh"
#include "vp_line.cuh"

using namespace vpline;

int vp_sm_count();

namespace {

template <int N>
struct Big3 {
    static constexpr int H = N / 2;            // line pairs per row
    static constexpr int S = 8;                // planes per slab
    static constexpr int NU = N / S;           // slabs per cube
    static constexpr int NT = S * H;           // threads: one line pair each
    static constexpr int NC = N * N * N;
    // tile of pass A: [vx][vy][8 vz], the vy row index XOR-swizzled with the
    // low two bits of vx (conflict-free both as vx and as vy line pairs)
    static constexpr int A_TILE = N * N * S;
    // tile of passes B and C: [slab plane][row][N], row pitch N + 4 (rows
    // read with 16-byte accesses without conflicts), plane pitch = 16 mod 32
    // banks (line pairs that straddle two planes stay conflict-free)
    static constexpr int RP = N + 4;
    static constexpr int PP = N * RP + 16;
    static constexpr int BC_TILE = S * PP;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

// asynchronous prefetch of [p, p + bytes) into L2 (16-byte aligned, bytes a
// multiple of 16)
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool whole_cell(const LineCoef<float> &c) { return (c.code >> 1) != 0; }

// ---------------------------------------------------------------------------
// pass A: vx then vy on the slab of vz planes [8 s, 8 s + 8) of cube c; in
// place or out of place
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Big3<N>::NT, 2) k_kick_pass_a(
    const float *src, const LineCoef<float> *__restrict__ coef, long long nunits,
    double *lost_out, float *dst)
{
    typedef Big3<N> B;
    constexpr int S = B::S, NU = B::NU, NC = B::NC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw);   // [vx][vy ^ (vx & 3)][8 vz]
    __shared__ Acc<double> red[32];
    const int t = threadIdx.x, p = t % (S / 2), q = t / (S / 2);   // q: vy (sweep 1), vx (sweep 2)
    float lost = 0.f;
    for (long long u = blockIdx.x; u < nunits; u += gridDim.x) {
        const long long c = u / NU;
        const int k0 = (int)(u % NU) * S;
        const LineCoef<float> c1 = coef[c * 3], c2 = coef[c * 3 + 1];
        const float *gs = src + c * NC;
        float *gd = dst + c * NC;
        float2 x[N];
        if (whole_cell(c1) || whole_cell(c2)) {
            // generic: both sweeps in global memory (dst), line by line
#pragma unroll
            for (int i = 0; i < N; ++i)
                x[i] = *reinterpret_cast<const float2 *>(gs + (i * N + q) * N + k0 + 2 * p);
#pragma unroll
            for (int i = 0; i < N; ++i)
                *reinterpret_cast<float2 *>(gd + (i * N + q) * N + k0 + 2 * p) = x[i];
            __syncthreads();
            lost += kick_line_shifted(gd + q * N + k0 + 2 * p, N * N, N, c1);
            lost += kick_line_shifted(gd + q * N + k0 + 2 * p + 1, N * N, N, c1);
            __syncthreads();
            lost += kick_line_shifted(gd + q * N * N + k0 + 2 * p, N, N, c2);
            lost += kick_line_shifted(gd + q * N * N + k0 + 2 * p + 1, N, N, c2);
            __syncthreads();
            continue;
        }
        // sweep 1: vx line pair at (vy = q, vz = k0 + 2p, + 1), from global
        // memory (a warp reads eight 32-byte row pieces per load)
        {
            const float *g = gs + q * N + k0 + 2 * p;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                x[i] = *reinterpret_cast<const float2 *>(g);
                g += N * N;
                asm volatile("" : "+l"(g));
            }
        }
        lost += sweep_pairs<N>(x, c1);
#pragma unroll
        for (int i = 0; i < N; ++i)
            *reinterpret_cast<float2 *>(tile + i * N * S + ((q ^ (i & 3)) * S) + 2 * p) = x[i];
        __syncthreads();
        // sweep 2: vy line pair at (vx = q, vz = k0 + 2p, + 1)
#pragma unroll
        for (int j = 0; j < N; ++j)
            x[j] = *reinterpret_cast<const float2 *>(tile + q * N * S + ((j ^ (q & 3)) * S) + 2 * p);
        lost += sweep_pairs<N>(x, c2);
        {
            float *g = gd + q * N * N + k0 + 2 * p;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                *reinterpret_cast<float2 *>(g) = x[j];
                g += N;
                asm volatile("" : "+l"(g));
            }
        }
        __syncthreads();        // the tile is rewritten by the next unit
    }
    Acc<double> a;
    a.add((double)lost);
    a = block_merge(a, red);
    if (t == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

// ---------------------------------------------------------------------------
// pass B: vz (table ca) then vx (table cb) on the slab of vy planes
// [8 s, 8 s + 8) of cube c; in place (src == dst allowed)
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Big3<N>::NT, 2) k_kick_pass_b(
    const float *__restrict__ src, const LineCoef<float> *__restrict__ ca,
    const LineCoef<float> *__restrict__ cb, long long nunits, double *lost_out, float *dst)
{
    typedef Big3<N> B;
    constexpr int S = B::S, NU = B::NU, NC = B::NC, RP = B::RP, PP = B::PP, NT = B::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw);      // [vy in slab][vx][vz]
    __shared__ Acc<double> red[32];
    const int t = threadIdx.x;
    // rows of the vz sweep: (vx = t % N, slab plane t / N and t / N + S / 2)
    const int ri = t % N, rl = t / N;
    // vx line pair of the second sweep: slab plane t / H, vz = 2 (t % H)
    const int pl = t / B::H, pk = 2 * (t % B::H);
    float lost = 0.f;
    // copy unit u's slab into the tile: per vx plane 8 rows of N floats,
    // contiguous in global memory
    auto stage = [&](long long u) {
        constexpr int Q = N / 4, PER_I = S * Q, CHUNKS = N * PER_I;
        const float *g = src + (u / NU) * NC + (u % NU) * S * N;
#pragma unroll 4
        for (int e = t; e < CHUNKS; e += NT) {
            const int i = e / PER_I, r = e % PER_I, l = r / Q, qq = r % Q;
            cp_async16(tile + l * PP + i * RP + 4 * qq, g + (long long)i * N * N + l * N + 4 * qq);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if ((long long)blockIdx.x < nunits) stage(blockIdx.x);
    for (long long u = blockIdx.x; u < nunits; u += gridDim.x) {
        const long long c = u / NU;
        const int j0 = (int)(u % NU) * S;
        const LineCoef<float> c1 = ca[c * 3 + 2], c2 = cb[c * 3];
        float *gd = dst + c * NC;
        const long long un = u + gridDim.x;
        // the next slab (48 runs of 8 rows, 1.5 KB each) into L2 ahead of
        // its copies, which start only once this slab's vx lines are read
        if (t < N && un < nunits)
            prefetch_l2(src + (un / NU) * NC + (long long)t * N * N + (un % NU) * S * N, S * N * 4);
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        if (whole_cell(c1) || whole_cell(c2)) {
            // generic, in global memory (the tile's copy is not used)
            if (un < nunits) stage(un);
            for (int r = t; r < N * S; r += NT) {
                const int i = r % N, l = r / N;
                lost += kick_line_shifted(gd + (i * N + j0 + l) * N, 1, N, c1);
            }
            __syncthreads();
            for (int r = t; r < N * S; r += NT) {
                const int l = r / N, k = r % N;
                lost += kick_line_shifted(gd + (j0 + l) * N + k, N * N, N, c2);
            }
            __syncthreads();
            continue;
        }
        float2 x[N];
        {
            // sweep 1 (vz): rows (vx = ri, planes rl and rl + S/2), in place
            float *ra = tile + rl * PP + ri * RP, *rb = ra + (S / 2) * PP;
#pragma unroll
            for (int k = 0; k < N; k += 4) {
                const float4 a = *reinterpret_cast<const float4 *>(ra + k);
                const float4 b = *reinterpret_cast<const float4 *>(rb + k);
                x[k] = make_float2(a.x, b.x);
                x[k + 1] = make_float2(a.y, b.y);
                x[k + 2] = make_float2(a.z, b.z);
                x[k + 3] = make_float2(a.w, b.w);
            }
            lost += sweep_pairs<N>(x, c1);
#pragma unroll
            for (int k = 0; k < N; k += 4) {
                *reinterpret_cast<float4 *>(ra + k) = make_float4(x[k].x, x[k + 1].x, x[k + 2].x, x[k + 3].x);
                *reinterpret_cast<float4 *>(rb + k) = make_float4(x[k].y, x[k + 1].y, x[k + 2].y, x[k + 3].y);
            }
        }
        __syncthreads();
        // sweep 2 (vx): line pair (plane pl, vz = pk, pk + 1) from the tile
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = *reinterpret_cast<const float2 *>(tile + pl * PP + i * RP + pk);
        __syncthreads();        // every line is in registers: refill the tile
        if (un < nunits) stage(un);
        lost += sweep_pairs<N>(x, c2);
        {
            float *g = gd + (j0 + pl) * N + pk;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                *reinterpret_cast<float2 *>(g) = x[i];
                g += N * N;
                asm volatile("" : "+l"(g));
            }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    Acc<double> a;
    a.add((double)lost);
    a = block_merge(a, red);
    if (t == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

// ---------------------------------------------------------------------------
// pass C: vy then vz (table coef; the vy sweep skipped when !do1) on the
// slab of vx planes [8 s, 8 s + 8) of cube c; in place (src == dst allowed)
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Big3<N>::NT, 2) k_kick_pass_c(
    const float *src, const LineCoef<float> *__restrict__ coef, int do1, long long nunits,
    double *lost_out, float *dst)
{
    typedef Big3<N> B;
    constexpr int S = B::S, NU = B::NU, NC = B::NC, RP = B::RP, PP = B::PP, NT = B::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *tile = reinterpret_cast<float *>(smem_raw);      // [vx in slab][vy][vz]
    __shared__ Acc<double> red[32];
    const int t = threadIdx.x;
    const int pl = t / B::H, pk = 2 * (t % B::H);           // vy line pair: plane, vz
    const int rj = t % N, rl = t / N;                       // vz rows: vy, planes rl, rl + S/2
    float lost = 0.f;
    for (long long u = blockIdx.x; u < nunits; u += gridDim.x) {
        const long long c = u / NU;
        const int i0 = (int)(u % NU) * S;
        const LineCoef<float> c1 = coef[c * 3 + 1], c2 = coef[c * 3 + 2];
        float *gd = dst + c * NC;
        const long long un = u + gridDim.x;
        if ((do1 && whole_cell(c1)) || whole_cell(c2)) {
            // generic, in global memory
            if (do1)
                for (int r = t; r < N * S; r += NT) {
                    const int l = r / N, k = r % N;
                    lost += kick_line_shifted(gd + (i0 + l) * N * N + k, N, N, c1);
                }
            __syncthreads();
            for (int r = t; r < N * S; r += NT) {
                const int l = r / N, j = r % N;
                lost += kick_line_shifted(gd + ((i0 + l) * N + j) * N, 1, N, c2);
            }
            __syncthreads();
            continue;
        }
        float2 x[N];
        {
            const float *g = src + c * NC + (long long)(i0 + pl) * N * N + pk;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                x[j] = *reinterpret_cast<const float2 *>(g);
                g += N;
                asm volatile("" : "+l"(g));
            }
        }
        if (do1) lost += sweep_pairs<N>(x, c1);
#pragma unroll
        for (int j = 0; j < N; ++j) *reinterpret_cast<float2 *>(tile + pl * PP + j * RP + pk) = x[j];
        __syncthreads();
        // the next slab into L2 while this one's vz rows are swept and the
        // tile is copied out
        if (t < 4 && un < nunits)
            prefetch_l2(src + (un / NU) * NC + (long long)(un % NU) * S * N * N + t * (S * N * N / 4),
                        S * N * N);
        {
            // sweep 2 (vz): rows (vy = rj, planes rl and rl + S/2), in place
            float *ra = tile + rl * PP + rj * RP, *rb = ra + (S / 2) * PP;
#pragma unroll
            for (int k = 0; k < N; k += 4) {
                const float4 a = *reinterpret_cast<const float4 *>(ra + k);
                const float4 b = *reinterpret_cast<const float4 *>(rb + k);
                x[k] = make_float2(a.x, b.x);
                x[k + 1] = make_float2(a.y, b.y);
                x[k + 2] = make_float2(a.z, b.z);
                x[k + 3] = make_float2(a.w, b.w);
            }
            lost += sweep_pairs<N>(x, c2);
#pragma unroll
            for (int k = 0; k < N; k += 4) {
                *reinterpret_cast<float4 *>(ra + k) = make_float4(x[k].x, x[k + 1].x, x[k + 2].x, x[k + 3].x);
                *reinterpret_cast<float4 *>(rb + k) = make_float4(x[k].y, x[k + 1].y, x[k + 2].y, x[k + 3].y);
            }
        }
        __syncthreads();
        {
            constexpr int Q = N / 4, PER_L = N * Q, CHUNKS = S * PER_L;
            float *g = gd + (long long)i0 * N * N;
#pragma unroll 4
            for (int e = t; e < CHUNKS; e += NT) {
                const int l = e / PER_L, r = e % PER_L, j = r / Q, qq = r % Q;
                *reinterpret_cast<float4 *>(g + (long long)l * N * N + j * N + 4 * qq) =
                    *reinterpret_cast<const float4 *>(tile + l * PP + j * RP + 4 * qq);
            }
        }
        __syncthreads();        // the tile is rewritten by the next slab
    }
    Acc<double> a;
    a.add((double)lost);
    a = block_merge(a, red);
    if (t == 0 && a.value() != 0.0) atomicAdd(lost_out, a.value());
}

template <typename K>
cudaError_t persistent_grid(K kern, int threads, size_t smem, long long nunits, unsigned &grid)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long g = (long long)per_sm * vp_sm_count();
    if (g > nunits) g = nunits;
    grid = (unsigned)g;
    return cudaSuccess;
}

}  // namespace

// The fused kick (6 sweeps: A, B, C), one half kick (3 sweeps: A, C
// without its vy sweep) or the vx and vy sweeps of a half kick (2 sweeps:
// A) of FP32 cubes of edge 48, from f into fo (fo == f in place).  Returns
// cudaErrorNotSupported for other sweep runs.
cudaError_t launch_kick_big3(vp_ctx *c, float *f, const LineCoef<float> *ca,
                             const LineCoef<float> *cb, int nsweeps, int first_axis, float *fo)
{
    constexpr int N = 48;
    typedef Big3<N> B;
    if (first_axis != 0 || (nsweeps != 6 && nsweeps != 3 && nsweeps != 2)) return cudaErrorNotSupported;
    const long long nunits = c->np * B::NU;
    cudaError_t e;
    unsigned grid;
    const size_t smem_a = (size_t)B::A_TILE * sizeof(float);
    const size_t smem_bc = (size_t)B::BC_TILE * sizeof(float);
    cudaEvent_t *ev = c->kick_pass_ev;
    if (ev && (e = cudaEventRecord(ev[0], c->stream)) != cudaSuccess) return e;
    if ((e = persistent_grid(k_kick_pass_a<N>, B::NT, smem_a, nunits, grid)) != cudaSuccess) return e;
    k_kick_pass_a<N><<<grid, B::NT, smem_a, c->stream>>>(f, ca, nunits, &c->sc->lost, fo);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], c->stream)) != cudaSuccess) return e;
    if (nsweeps == 2) {             // vx and vy only: pass A
        if (ev && (e = cudaEventRecord(ev[2], c->stream)) != cudaSuccess) return e;
        if (ev && (e = cudaEventRecord(ev[3], c->stream)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    if (nsweeps == 6) {
        if ((e = persistent_grid(k_kick_pass_b<N>, B::NT, smem_bc, nunits, grid)) != cudaSuccess) return e;
        k_kick_pass_b<N><<<grid, B::NT, smem_bc, c->stream>>>(fo, ca, cb, nunits, &c->sc->lost, fo);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[2], c->stream)) != cudaSuccess) return e;
    const LineCoef<float> *cc = nsweeps == 6 ? cb : ca;
    if ((e = persistent_grid(k_kick_pass_c<N>, B::NT, smem_bc, nunits, grid)) != cudaSuccess) return e;
    k_kick_pass_c<N><<<grid, B::NT, smem_bc, c->stream>>>(fo, cc, nsweeps == 6 ? 1 : 0, nunits,
                                                           &c->sc->lost, fo);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[3], c->stream)) != cudaSuccess) return e;
    return cudaSuccess;
}
