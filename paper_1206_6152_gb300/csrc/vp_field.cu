// vp_field.cu -- density -> potential -> acceleration (Sec. 2.2 of Yoshikawa,
// Yoshida & Umemura 2013) in FP64 on sm_103a.
//
//  * 3D FFT: batched 1D complex transforms along one axis at a time, each
//    CTA staging a batch of lines in shared memory and running a mixed-radix
//    Stockham transform (radices 2..13) with FP64 twiddle tables built on the
//    host at set-up.
//  * periodic Poisson: phi = IFFT( G(k) FFT(rho) ), G(k) the Green's function
//    of the 7-point discrete Laplacian, -pi G / sum_l sin^2(k_l D_l/2)/D_l^2
//    (equal to -pi G D^2 / sum sin^2(k_l D/2) for equal spacings), G(0) = 0.
//  * isolated Poisson: Hockney's doubling; rho zero-padded to 2N per axis,
//    kernel -G/r on 0..N mirrored to N+1..2N-1, its r = 0 value the mean of
//    -G/r over one cubic cell, -G (3 ln(2 + sqrt 3) - pi/2) / D.
//  * force: g = -(phi_{i+1} - phi_{i-1}) / (2 D) per axis; for the isolated
//    case the neighbours outside the box come from the doubled grid.
#include <cuda_runtime.h>
#include <math.h>

#include "vp_device.cuh"
#include "vp_internal.cuh"

int vp_sm_count();

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

struct FFTParams {
    int n;
    int nrad;
    int rad[24];
    long long so, si, sp;   // strides of outer index, inner index, position
    int ni;                 // number of inner indices
    int B;                  // lines per CTA
    int inverse;
};

template <int R>
__device__ __forceinline__ void butterfly(const double2 *__restrict__ src, double2 *__restrict__ dst,
                                          int n, int Ns, int j, const double2 *__restrict__ tw,
                                          int inverse)
{
    const int k = j % Ns;
    const int nr = n / R;
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        double2 x = src[j + r * nr];
        if (r) {
            const int m = (int)(((long long)r * k * (n / (Ns * R))) % n);
            double2 w = tw[m];
            if (inverse) w.y = -w.y;
            x = cmul(x, w);
        }
        v[r] = x;
    }
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int p = 0; p < R; ++p) {
        double2 acc = v[0];
#pragma unroll
        for (int q = 1; q < R; ++q) {
            const int m = (int)(((long long)q * p % R) * nr);
            double2 w = tw[m];
            if (inverse) w.y = -w.y;
            const double2 t = cmul(v[q], w);
            acc.x += t.x;
            acc.y += t.y;
        }
        dst[base + p * Ns] = acc;
    }
}

__global__ void __launch_bounds__(256) k_fft(double2 *__restrict__ data, FFTParams P,
                                            const double2 *__restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *buf0 = reinterpret_cast<double2 *>(smem_raw);
    double2 *buf1 = buf0 + P.B * P.n;
    const int n = P.n, B = P.B;
    const long long o = blockIdx.y;
    const int i0 = blockIdx.x * B;
    const int nb = min(B, P.ni - i0);
    double2 *gbase = data + o * P.so + (long long)i0 * P.si;
    // load (fastest-varying global index first)
    for (int e = threadIdx.x; e < nb * n; e += blockDim.x) {
        int b, p;
        if (P.sp == 1) { b = e / n; p = e - b * n; }
        else { p = e / nb; b = e - p * nb; }
        buf0[b * n + p] = gbase[b * P.si + p * P.sp];
    }
    __syncthreads();
    double2 *src = buf0, *dst = buf1;
    int Ns = 1;
    for (int st = 0; st < P.nrad; ++st) {
        const int R = P.rad[st];
        const int nbf = n / R;
        for (int t = threadIdx.x; t < nb * nbf; t += blockDim.x) {
            const int b = t / nbf, j = t - b * nbf;
            const double2 *s = src + b * n;
            double2 *d = dst + b * n;
            switch (R) {
            case 2: butterfly<2>(s, d, n, Ns, j, tw, P.inverse); break;
            case 3: butterfly<3>(s, d, n, Ns, j, tw, P.inverse); break;
            case 4: butterfly<4>(s, d, n, Ns, j, tw, P.inverse); break;
            case 5: butterfly<5>(s, d, n, Ns, j, tw, P.inverse); break;
            case 7: butterfly<7>(s, d, n, Ns, j, tw, P.inverse); break;
            case 11: butterfly<11>(s, d, n, Ns, j, tw, P.inverse); break;
            default: butterfly<13>(s, d, n, Ns, j, tw, P.inverse); break;
            }
        }
        __syncthreads();
        double2 *t = src; src = dst; dst = t;
        Ns *= R;
    }
    for (int e = threadIdx.x; e < nb * n; e += blockDim.x) {
        int b, p;
        if (P.sp == 1) { b = e / n; p = e - b * n; }
        else { p = e / nb; b = e - p * nb; }
        gbase[b * P.si + p * P.sp] = src[b * n + p];
    }
}

// rho (box, N^p) -> complex buffer on the FFT grid (zero padding if larger)
__global__ void k_pack(const double *__restrict__ rho, double2 *__restrict__ cbuf, int n0, int n1,
                       int n2, int f0, int f1, int f2)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)f0 * f1 * f2;
    if (t >= total) return;
    const int k = (int)(t % f2);
    const int j = (int)((t / f2) % f1);
    const int i = (int)(t / ((long long)f1 * f2));
    double v = 0.0;
    if (i < n0 && j < n1 && k < n2) v = rho[((long long)i * n1 + j) * n2 + k];
    cbuf[t] = make_double2(v, 0.0);
}

__global__ void k_green_mul(double2 *__restrict__ cbuf, const double *__restrict__ ghat,
                            long long total)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const double gk = ghat[t];
    double2 v = cbuf[t];
    v.x *= gk;
    v.y *= gk;
    cbuf[t] = v;
}

__global__ void k_real_part(const double2 *__restrict__ cbuf, double *__restrict__ phi,
                            long long total)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    phi[t] = cbuf[t].x;
}

// g_a = -(phi(i+1) - phi(i-1)) / (2 dx_a), neighbours wrapped on the FFT grid
__global__ void k_force(const double *__restrict__ phi, double *__restrict__ g, int n0, int n1,
                        int n2, int f0, int f1, int f2, double idx0, double idx1, double idx2)
{
    const long long np = (long long)n0 * n1 * n2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const int k = (int)(t % n2);
    const int j = (int)((t / n2) % n1);
    const int i = (int)(t / ((long long)n1 * n2));
    auto at = [&](int a, int b, int c) -> double {
        return phi[((long long)a * f1 + b) * f2 + c];
    };
    const int ip = i + 1 == f0 ? 0 : i + 1, im = i == 0 ? f0 - 1 : i - 1;
    const int jp = j + 1 == f1 ? 0 : j + 1, jm = j == 0 ? f1 - 1 : j - 1;
    const int kp = k + 1 == f2 ? 0 : k + 1, km = k == 0 ? f2 - 1 : k - 1;
    g[t] = -(at(ip, j, k) - at(im, j, k)) * 0.5 * idx0;
    g[np + t] = -(at(i, jp, k) - at(i, jm, k)) * 0.5 * idx1;
    g[2 * np + t] = -(at(i, j, kp) - at(i, j, km)) * 0.5 * idx2;
}

__global__ void k_copy_box(const double *__restrict__ src, double *__restrict__ dst, int n0,
                           int n1, int n2, int f1, int f2)
{
    const long long np = (long long)n0 * n1 * n2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= np) return;
    const int k = (int)(t % n2);
    const int j = (int)((t / n2) % n1);
    const int i = (int)(t / ((long long)n1 * n2));
    dst[t] = src[((long long)i * f1 + j) * f2 + k];
}

// out[0] += sum rho * phi_box (compensated), one CTA
__global__ void k_dot_rho_phi(const double *__restrict__ rho, const double *__restrict__ phi,
                              int n0, int n1, int n2, int f1, int f2, double *out)
{
    __shared__ Acc<double> red[32];
    const long long np = (long long)n0 * n1 * n2;
    Acc<double> a;
    for (long long t = threadIdx.x; t < np; t += blockDim.x) {
        const int k = (int)(t % n2);
        const int j = (int)((t / n2) % n1);
        const int i = (int)(t / ((long long)n1 * n2));
        a.add(rho[t] * phi[((long long)i * f1 + j) * f2 + k]);
    }
    a = block_merge(a, red);
    if (threadIdx.x == 0) out[0] = a.value();
}

// out[j] = sum_i in[i * stride + j] for j < stride (compensated), one CTA per j
__global__ void k_reduce_strided(const double *__restrict__ in, long long n, int stride,
                                 double *__restrict__ out)
{
    __shared__ Acc<double> red[32];
    Acc<double> a;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) a.add(in[i * stride + blockIdx.x]);
    a = block_merge(a, red);
    if (threadIdx.x == 0) out[blockIdx.x] = a.value();
}

inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// radix plan for one axis: 4s first, then 2, 3, 5, 7, 11, 13
int vp_fft_plan_axis(FFTAxis *a, int n)
{
    a->n = n;
    a->nrad = 0;
    int m = n;
    const int order[] = {4, 2, 3, 5, 7, 11, 13};
    for (int r : order) {
        while (m % r == 0) {
            if (a->nrad >= 24) return VP_ERR_UNSUPPORTED;
            a->rad[a->nrad++] = r;
            m /= r;
        }
    }
    if (m != 1) return VP_ERR_UNSUPPORTED;
    return VP_OK;
}

cudaError_t launch_fft(vp_ctx *c, double2 *data, int axis, int inverse)
{
    FFTParams P;
    const FFTAxis &A = c->ax[axis];
    const long long f0 = c->fn[0], f1 = c->fn[1], f2 = c->fn[2];
    P.n = A.n;
    P.nrad = A.nrad;
    for (int i = 0; i < A.nrad; ++i) P.rad[i] = A.rad[i];
    P.inverse = inverse;
    long long nouter;
    if (axis == 2) { P.so = f1 * f2; P.si = f2; P.sp = 1; P.ni = (int)f1; nouter = f0; }
    else if (axis == 1) { P.so = f1 * f2; P.si = 1; P.sp = f2; P.ni = (int)f2; nouter = f0; }
    else { P.so = f2; P.si = 1; P.sp = f1 * f2; P.ni = (int)f2; nouter = f1; }
    int B = 2048 / P.n;
    if (B < 1) B = 1;
    if (B > P.ni) B = P.ni;
    P.B = B;
    const size_t smem = 2 * (size_t)B * P.n * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_fft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((P.ni + B - 1) / B), (unsigned)nouter);
    k_fft<<<grid, 256, smem, c->stream>>>(data, P, A.tw);
    return cudaGetLastError();
}

cudaError_t launch_field_solve(vp_ctx *c, const double *rho, double *g_out)
{
    const int T = 256;
    k_pack<<<blocks_for(c->nfft, T), T, 0, c->stream>>>(rho, c->cbuf, c->n[0], c->n[1], c->n[2],
                                                        c->fn[0], c->fn[1], c->fn[2]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int a = 2; a >= 0; --a)
        if ((e = launch_fft(c, c->cbuf, a, 0)) != cudaSuccess) return e;
    k_green_mul<<<blocks_for(c->nfft, T), T, 0, c->stream>>>(c->cbuf, c->ghat, c->nfft);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int a = 0; a < 3; ++a)
        if ((e = launch_fft(c, c->cbuf, a, 1)) != cudaSuccess) return e;
    k_real_part<<<blocks_for(c->nfft, T), T, 0, c->stream>>>(c->cbuf, c->phi, c->nfft);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (g_out) {
        k_force<<<blocks_for(c->np, T), T, 0, c->stream>>>(
            c->phi, g_out, c->n[0], c->n[1], c->n[2], c->fn[0], c->fn[1], c->fn[2],
            1.0 / c->dx[0], 1.0 / c->dx[1], 1.0 / c->dx[2]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_green_mul(vp_ctx *c)
{
    k_green_mul<<<blocks_for(c->nfft, 256), 256, 0, c->stream>>>(c->cbuf, c->ghat, c->nfft);
    return cudaGetLastError();
}

cudaError_t launch_copy_phi_box(vp_ctx *c, double *dst)
{
    k_copy_box<<<blocks_for(c->np, 256), 256, 0, c->stream>>>(c->phi, dst, c->n[0], c->n[1],
                                                              c->n[2], c->fn[1], c->fn[2]);
    return cudaGetLastError();
}

cudaError_t launch_dot_rho_phi(vp_ctx *c, const double *rho, double *out)
{
    k_dot_rho_phi<<<1, 1024, 0, c->stream>>>(rho, c->phi, c->n[0], c->n[1], c->n[2], c->fn[1],
                                             c->fn[2], out);
    return cudaGetLastError();
}

// sums of `stride` interleaved sequences of length n
cudaError_t launch_reduce_strided(vp_ctx *c, const double *in, long long n, int stride,
                                  double *out)
{
    k_reduce_strided<<<stride, 1024, 0, c->stream>>>(in, n, stride, out);
    return cudaGetLastError();
}
