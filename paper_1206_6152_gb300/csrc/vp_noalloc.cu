// vp_noalloc.cu -- mass and kinetic-energy sums of a distribution function
// without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// diagnostic: code running inside a CUDA stream capture that must not break
// the capture, host threads of an application whose memory pool is owned by
// another allocator and sized once at start-up, or a plugin embedded in a
// process that forbids new device allocations after initialisation.  For
// them, vp_moments_noalloc() computes sum f and sum f |v|^2 (the two sums
// behind M and K of vp_energy) using a scratch array that lives in the
// library's own static device memory instead of a context.
//
// The scratch is the file-scope array g_moment_scratch below: it holds one
// pair of partial sums per spatial cell, for at most VP_NOALLOC_MAX_CELLS
// spatial cells (4 MiB).  Every GPU that loads this library keeps it until
// the process exits.  Host code may not take the array's address directly
// (its name on the host is only a stand-in for the device symbol), so the
// first call on each device asks the runtime for the device address with
// cudaGetSymbolAddress and caches it for that device, together with the
// unique id of the CUDA context it was looked up in: a call made in another
// context (after a device reset, the runtime creates a new one) looks the
// address up again.  Before any launch the input and output pointers are
// checked to be device memory of the current device (a host pointer would
// fault or read the wrong memory).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <mutex>

#include "vp_device.cuh"
#include "vp_internal.cuh"

#define VP_NOALLOC_MAX_CELLS (1 << 18)
#define VP_NOALLOC_MAX_DEVICES 64

// two partial sums per spatial cell: sum f, sum f |v|^2
static __device__ __align__(256) double g_moment_scratch[2 * VP_NOALLOC_MAX_CELLS];

namespace {

int sm_count_of(int dev)
{
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 152;
    return n;
}

// per spatial cell: compensated sums of f and f |v|^2 with the velocity cell
// centres V^- + (j + 1/2) dv computed in place
template <typename T>
__global__ void __launch_bounds__(256) k_moment_partials(const T *__restrict__ f, long long np,
                                                        int nvx, int nvy, int nvz, double vlx,
                                                        double vly, double vlz, double dvx,
                                                        double dvy, double dvz,
                                                        double *__restrict__ partials)
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
            const double vx = vlx + (i + 0.5) * dvx;
            const double vy = vly + (j + 0.5) * dvy;
            const double vz = vlz + (k + 0.5) * dvz;
            const double x = (double)q[e];
            a0.add(x);
            a2.add(x * (vx * vx + vy * vy + vz * vz));
        }
        a0 = block_merge(a0, red);
        if (threadIdx.x == 0) partials[2 * cell] = a0.value();
        __syncthreads();
        a2 = block_merge(a2, red);
        if (threadIdx.x == 0) partials[2 * cell + 1] = a2.value();
        __syncthreads();
    }
}

// out[j] = sum over cells of partials[2 cell + j], j = 0, 1 (one CTA each)
__global__ void k_moment_finish(const double *__restrict__ partials, long long np,
                                double *__restrict__ out)
{
    __shared__ Acc<double> red[32];
    Acc<double> a;
    for (long long i = threadIdx.x; i < np; i += blockDim.x) a.add(partials[2 * i + blockIdx.x]);
    a = block_merge(a, red);
    if (threadIdx.x == 0) out[blockIdx.x] = a.value();
}

std::mutex g_setup_lock;
double *g_scratch_addr[VP_NOALLOC_MAX_DEVICES];
unsigned long long g_scratch_ctx[VP_NOALLOC_MAX_DEVICES];     // context id of the lookup

// unique id of the current CUDA context (0 if the driver cannot say: the
// address is then looked up on every call)
unsigned long long current_context_id()
{
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
        cudaGetLastError();
        resolved = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// device address of g_moment_scratch in the current context (set up on the
// first call on each device and again whenever the device's context has
// changed; the device must be current)
int scratch_for_current_device(int dev, double **out)
{
    if (dev < 0 || dev >= VP_NOALLOC_MAX_DEVICES) return VP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_setup_lock);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_moment_scratch);
        if (e != cudaSuccess || !p) {
            vp_note_cuda_error(e, "cudaGetSymbolAddress(g_moment_scratch)", __FILE__, __LINE__);
            return VP_ERR_CUDA;
        }
        g_scratch_addr[dev] = (double *)p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return VP_OK;
}

// true if p is device (or managed) memory the current device can address as
// its own
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" int vp_moments_noalloc(const void *f_dev, int dtype, const int n[3], const int nv[3],
                                  const double vlo[3], const double vhi[3], double *sums_dev,
                                  void *cuda_stream)
{
    if (!f_dev || !n || !nv || !vlo || !vhi || !sums_dev) return VP_ERR_ARG;
    if (dtype != 0 && dtype != 1) return VP_ERR_ARG;
    long long np = 1;
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || nv[a] < 1 || !(vhi[a] > vlo[a])) return VP_ERR_CONFIG;
        np *= n[a];
    }
    const long long nvc = (long long)nv[0] * nv[1] * nv[2];
    if (np > VP_NOALLOC_MAX_CELLS || nvc > 0x7fffffffLL) return VP_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return VP_ERR_CUDA;
    }
    if (!on_device(f_dev, dev) || !on_device(sums_dev, dev)) return VP_ERR_ARG;
    double *scratch = nullptr;
    const int r = scratch_for_current_device(dev, &scratch);
    if (r != VP_OK) return r;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    long long grid = (long long)sm_count_of(dev) * 8;
    if (grid > np) grid = np;
    const double dv[3] = {(vhi[0] - vlo[0]) / nv[0], (vhi[1] - vlo[1]) / nv[1],
                          (vhi[2] - vlo[2]) / nv[2]};
    if (dtype == 1)
        k_moment_partials<double><<<(unsigned)grid, 256, 0, s>>>(
            (const double *)f_dev, np, nv[0], nv[1], nv[2], vlo[0], vlo[1], vlo[2], dv[0], dv[1],
            dv[2], scratch);
    else
        k_moment_partials<float><<<(unsigned)grid, 256, 0, s>>>(
            (const float *)f_dev, np, nv[0], nv[1], nv[2], vlo[0], vlo[1], vlo[2], dv[0], dv[1],
            dv[2], scratch);
    VP_CUDA_TRY(cudaGetLastError());
    k_moment_finish<<<2, 1024, 0, s>>>(scratch, np, sums_dev);
    VP_CUDA_TRY(cudaGetLastError());
    return VP_OK;
}
