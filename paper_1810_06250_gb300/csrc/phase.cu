// Plan-time kernels: the phase matrix in FP64 and the RMSF.
//
// theta_jk = 2 phi_k (lambda_j^2 - lambda_0^2) reaches 1e4-1e5 rad for
// low-frequency bands, so the argument is formed and reduced in FP64:
// r = theta - 2 pi n, n = rint(theta / 2 pi), with 2 pi split into a double
// head and tail (Cody & Waite's two-constant reduction), then sincos(r).
// Sec. 2.3 notes that K, 2 phi and lambda^2 - lambda_0^2 are computed once per
// dataset; the phase matrix is the same once-per-plan product.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "rms_internal.h"

namespace {

// 2 pi = kTwoPiHi + kTwoPiLo to about 1e-32 (double head, double tail).
__device__ constexpr double kTwoPiHi = 6.283185307179586232e+00;
__device__ constexpr double kTwoPiLo = 2.449293598294706414e-16;
__device__ constexpr double kInvTwoPi = 1.591549430918953358e-01;

__device__ __forceinline__ void phase_sincos(double phi, double dl2, double *s, double *c)
{
    double x = 2.0 * phi * dl2;
    double n = rint(x * kInvTwoPi);
    double r = fma(-n, kTwoPiHi, x);
    r = fma(-n, kTwoPiLo, r);
    sincos(r, s, c);
}

// FP32 table [nact][nphi] of w_j (cos, sin)(theta_jk), for the FP32 table path.
__global__ void phase_table_kernel(const double *__restrict__ dl2, const double *__restrict__ w,
                                   const double *__restrict__ phi, int32_t nact, int32_t nphi,
                                   float2 *__restrict__ tab)
{
    int64_t total = (int64_t)nact * nphi;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = (int32_t)(t / nphi), k = (int32_t)(t % nphi);
        double s, c;
        phase_sincos(phi[k], dl2[a], &s, &c);
        tab[t] = make_float2((float)(w[a] * c), (float)(w[a] * s));
    }
}

// Window rotation table [ncentre][ld]: T[n][j] = exp(-2i phi_n dl2_j) with
// phi_n = phi0 + n step (FP64 argument, reduced as above), FP32 complex;
// columns j >= nk (padding) hold 1.
__global__ void rotation_table_kernel(const double *__restrict__ dl2, int32_t nk, int32_t ld, double phi0,
                                      double step, int32_t ncentre, float2 *__restrict__ T)
{
    int64_t total = (int64_t)ncentre * ld;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int32_t n = (int32_t)(t / ld), j = (int32_t)(t % ld);
        if (j >= nk) {
            T[t] = make_float2(1.f, 0.f);
            continue;
        }
        double s, c;
        phase_sincos(phi0 + n * step, dl2[j], &s, &c);
        T[t] = make_float2((float)c, (float)-s);
    }
}

template <typename T>
__device__ __forceinline__ T to_half_type(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_half_type<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to_half_type<__half>(float x) { return __float2half_rn(x); }

template <typename T>
__device__ __forceinline__ float from_half_type(T x);
template <>
__device__ __forceinline__ float from_half_type<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ float from_half_type<__half>(__half x) { return __half2float(x); }

template <typename T>
__device__ __forceinline__ uint16_t bits16(T x) { return *reinterpret_cast<uint16_t *>(&x); }

// Split v into hi + lo of the 16-bit type: hi = rn(v), lo = rn(v - hi).
template <typename T>
__device__ __forceinline__ void split16(double v, uint16_t *hi, uint16_t *lo)
{
    T h = to_half_type<T>((float)v);
    double rest = v - (double)from_half_type<T>(h);
    T l = to_half_type<T>((float)rest);
    *hi = bits16(h);
    *lo = bits16(l);
}

// Tensor-core operand B, K-major [npad][kpad] (row n = 2k + {0: Re F, 1: Im F},
// column = 2a + {0: Q_a, 1: U_a}):
//   B[2k][2a] = c, B[2k][2a+1] = s, B[2k+1][2a] = -s, B[2k+1][2a+1] = c,
// with (c, s) = (w_a / w_max) (cos, sin)(theta_ak).  This is the real block of
// Eqs. qPhi/uPhi: Re F = sum(Q c + U s), Im F = sum(U c - Q s).
template <typename T>
__global__ void phase_bsplit_kernel(const double *__restrict__ dl2, const double *__restrict__ w,
                                    const double *__restrict__ phi, int32_t nact, int32_t nphi,
                                    double inv_wmax, int32_t kpad, uint16_t *__restrict__ bhi,
                                    uint16_t *__restrict__ blo)
{
    int64_t total = (int64_t)nact * nphi;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int32_t k = (int32_t)(t / nact), a = (int32_t)(t % nact);
        double s, c;
        phase_sincos(phi[k], dl2[a], &s, &c);
        double wn = w[a] * inv_wmax;
        uint16_t ch, cl, sh, sl, nsh, nsl;
        split16<T>(wn * c, &ch, &cl);
        split16<T>(wn * s, &sh, &sl);
        split16<T>(-(wn * s), &nsh, &nsl);
        size_t r0 = (size_t)(2 * k) * kpad + 2 * a, r1 = r0 + kpad;
        *reinterpret_cast<uint32_t *>(bhi + r0) = (uint32_t)ch | ((uint32_t)sh << 16);
        *reinterpret_cast<uint32_t *>(blo + r0) = (uint32_t)cl | ((uint32_t)sl << 16);
        *reinterpret_cast<uint32_t *>(bhi + r1) = (uint32_t)nsh | ((uint32_t)ch << 16);
        *reinterpret_cast<uint32_t *>(blo + r1) = (uint32_t)nsl | ((uint32_t)cl << 16);
    }
}

// R(phi_k) = K sum_j w_j exp(-i theta_jk), Eq. Rsum, accumulated in FP64.
__global__ void rmsf_kernel(const double *__restrict__ dl2, const double *__restrict__ w,
                            int32_t nact, double K, const double *__restrict__ phi, int32_t n,
                            double *__restrict__ R64, float *__restrict__ R32)
{
    int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double re = 0.0, im = 0.0, ph = phi[k];
    for (int32_t a = 0; a < nact; ++a) {
        double s, c;
        phase_sincos(ph, dl2[a], &s, &c);
        re = fma(w[a], c, re);
        im = fma(-w[a], s, im);
    }
    re *= K;
    im *= K;
    if (R64) { R64[2 * k] = re; R64[2 * k + 1] = im; }
    if (R32) { R32[2 * k] = (float)re; R32[2 * k + 1] = (float)im; }
}

int grid_for(int64_t total, int threads)
{
    int64_t g = (total + threads - 1) / threads;
    return (int)(g < 65535 * 16 ? (g < 1 ? 1 : g) : 65535 * 16);
}

}  // namespace

cudaError_t launch_phase_table(const rms_plan_s &p, cudaStream_t s)
{
    int64_t total = (int64_t)p.nact * p.nphi;
    phase_table_kernel<<<grid_for(total, 256), 256, 0, s>>>(p.d_dl2, p.d_wact, p.d_phi, p.nact,
                                                            p.nphi, p.d_table);
    return cudaGetLastError();
}

// B over the channel list (dl2, w)[0..nk): the active channels for channel-major
// cubes, or every channel (w = 0 where flagged, giving zero rows) for LOS-major.
cudaError_t launch_phase_bsplit(const rms_plan_s &p, const double *dl2, const double *w, int32_t nk,
                                int32_t kpad, uint16_t *bhi, uint16_t *blo, bool fp16, cudaStream_t s)
{
    size_t bytes = (size_t)p.npad * kpad * sizeof(uint16_t);
    cudaError_t e = cudaMemsetAsync(bhi, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(blo, 0, bytes, s);
    if (e != cudaSuccess) return e;
    int64_t total = (int64_t)nk * p.nphi;
    double inv = 1.0 / p.wmax;
    if (fp16)
        phase_bsplit_kernel<__half><<<grid_for(total, 256), 256, 0, s>>>(dl2, w, p.d_phi, nk, p.nphi, inv, kpad,
                                                                          bhi, blo);
    else
        phase_bsplit_kernel<__nv_bfloat16><<<grid_for(total, 256), 256, 0, s>>>(dl2, w, p.d_phi, nk, p.nphi, inv,
                                                                                 kpad, bhi, blo);
    return cudaGetLastError();
}

cudaError_t launch_rmsf(const rms_plan_s &p, const double *d_phi, int32_t n, double *d_R64,
                        float *d_R32, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    rmsf_kernel<<<(n + 127) / 128, 128, 0, s>>>(p.d_dl2, p.d_wact, p.nact, p.K, d_phi, n, d_R64,
                                                 d_R32);
    return cudaGetLastError();
}

cudaError_t launch_rotation_table(const double *dl2, int32_t nk, int32_t ld, double phi0, double step,
                                  int32_t ncentre, float2 *T, cudaStream_t s)
{
    const int64_t total = (int64_t)ncentre * ld;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
    if (blocks < 1) return cudaSuccess;
    rotation_table_kernel<<<blocks, 256, 0, s>>>(dl2, nk, ld, phi0, step, ncentre, T);
    return cudaGetLastError();
}
