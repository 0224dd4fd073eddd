// RM-CLEAN on the device: Hogbom deconvolution of dirty Faraday spectra with the
// RMSF, the step the paper names after synthesis (Sec. 2.2, Sec. 4).  For each
// LOS, repeat at most max_iter times
//     j = argmax_k |res_k| (lowest index on ties);  stop if |res_j| < threshold
//     c = gain res_j;  comp_j += c;  res_k -= c R(phi_k - phi_j)  for every k
// on a uniform phi grid, then restore clean_k = res_k + sum_{|d|<=W} comp_{k-d} B(d)
// with a real Gaussian beam B of the RMSF's FWHM, truncated at W = ceil(3 FWHM / dphi).
//
// One warp per LOS, residual and components in shared memory, R on the doubled
// grid (2 N - 1 points) shared by the CTA.  The greedy choices must be the ones
// the FP64 definition makes, so the iteration runs in FP64 with every product
// and sum rounded separately (no contraction into FMA): with the same R table
// the device reproduces the definition bit for bit.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "rms_internal.h"

struct rms_clean_s {
    rms_plan_s *plan = nullptr;
    int device = 0;
    int32_t N = 0, W = 0;
    double dphi = 0, fwhm = 0;
    double2 *d_R2 = nullptr;     // [2N - 1]: R at (m - N + 1) dphi
    double *d_beam = nullptr;    // [2W + 1]: B at (d - W) dphi
};

namespace {

constexpr int kCleanMaxN = 2048;

struct CleanParams {
    const float2 *F;
    int64_t nlos;
    int32_t N, W, max_iter, wpb;
    const double2 *R2;
    const double *beam;
    double gain, thr2;
    float2 *clean, *res_out, *comp_out;
    int32_t *niter;
};

__device__ __forceinline__ double2 cmul_rn(double2 a, double2 b)
{
    return make_double2(__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                        __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}

__global__ void __launch_bounds__(256) clean_kernel(const CleanParams P)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    double2 *R2 = reinterpret_cast<double2 *>(smem_raw);
    double *beam = reinterpret_cast<double *>(R2 + (2 * P.N - 1));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double2 *res = reinterpret_cast<double2 *>(beam + (2 * P.W + 1 + 1)) + (size_t)warp * 2 * P.N;
    double2 *comp = res + P.N;
    for (int i = threadIdx.x; i < 2 * P.N - 1; i += blockDim.x) R2[i] = P.R2[i];
    for (int i = threadIdx.x; i < 2 * P.W + 1; i += blockDim.x) beam[i] = P.beam[i];
    __syncthreads();
    const int N = P.N;
    for (int64_t l = (int64_t)blockIdx.x * P.wpb + warp; l < P.nlos; l += (int64_t)gridDim.x * P.wpb) {
        const float2 *f = P.F + l * N;
        for (int k = lane; k < N; k += 32) {
            const float2 v = f[k];
            res[k] = make_double2((double)v.x, (double)v.y);
            comp[k] = make_double2(0.0, 0.0);
        }
        __syncwarp();
        int it = 0;
        for (; it < P.max_iter; ++it) {
            double best = -1.0;
            int bj = INT_MAX;
            for (int k = lane; k < N; k += 32) {
                const double2 r = res[k];
                const double m2 = __dadd_rn(__dmul_rn(r.x, r.x), __dmul_rn(r.y, r.y));
                if (m2 > best) { best = m2; bj = k; }   // ascending k: the first maximum; NaN never
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
            }
            if (!(best >= P.thr2) || bj == INT_MAX) break;
            const double2 rj = res[bj];
            const double2 c = make_double2(__dmul_rn(P.gain, rj.x), __dmul_rn(P.gain, rj.y));
            __syncwarp();
            if (lane == 0) comp[bj] = make_double2(__dadd_rn(comp[bj].x, c.x), __dadd_rn(comp[bj].y, c.y));
            for (int k = lane; k < N; k += 32) {
                const double2 cr = cmul_rn(c, R2[k - bj + N - 1]);
                const double2 r = res[k];
                res[k] = make_double2(__dsub_rn(r.x, cr.x), __dsub_rn(r.y, cr.y));
            }
            __syncwarp();
        }
        if (lane == 0 && P.niter) P.niter[l] = it;
        for (int k = lane; k < N; k += 32) {
            double2 s = res[k];
            if (P.clean) {
                for (int d = -P.W; d <= P.W; ++d) {
                    const int kk = k - d;
                    if (kk < 0 || kk >= N) continue;
                    const double2 cc = comp[kk];
                    s.x = __dadd_rn(s.x, __dmul_rn(cc.x, beam[P.W + d]));
                    s.y = __dadd_rn(s.y, __dmul_rn(cc.y, beam[P.W + d]));
                }
                P.clean[l * N + k] = make_float2((float)s.x, (float)s.y);
            }
            if (P.res_out) P.res_out[l * N + k] = make_float2((float)res[k].x, (float)res[k].y);
            if (P.comp_out) P.comp_out[l * N + k] = make_float2((float)comp[k].x, (float)comp[k].y);
        }
        __syncwarp();
    }
}

size_t clean_smem(int N, int W, int wpb) { return (size_t)(2 * N - 1) * 16 + (size_t)(2 * W + 2) * 8 + (size_t)wpb * 2 * N * 16; }

rms_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return RMS_OK;
    if (e == cudaErrorMemoryAllocation) return RMS_ERR_OOM;
    return RMS_ERR_CUDA;
}

void free_clean(rms_clean_s *c)
{
    if (!c) return;
    cudaFree(c->d_R2);
    cudaFree(c->d_beam);
    delete c;
}

}  // namespace

extern "C" {

rms_status rms_clean_create(rms_clean_t *out, rms_plan_t plan, double fwhm, const double *R2_host)
{
    if (!out) return RMS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plan || !std::isfinite(fwhm)) return RMS_ERR_INVALID_ARG;
    const rms_plan_s &p = *plan;
    if (p.nphi < 2 || p.nphi > kCleanMaxN) return RMS_ERR_INVALID_ARG;
    const double D = (p.phi[p.nphi - 1] - p.phi[0]) / (p.nphi - 1);
    if (!(D > 0)) return RMS_ERR_INVALID_ARG;
    for (int k = 0; k < p.nphi; ++k)
        if (std::fabs(p.phi[k] - (p.phi[0] + k * D)) > 1e-9 * std::max(1.0, std::fabs(p.phi[k])))
            return RMS_ERR_INVALID_ARG;
    if (fwhm <= 0) fwhm = p.fwhm_meas;
    if (!(fwhm > 0) || !std::isfinite(fwhm)) return RMS_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p.device && cudaSetDevice(p.device) != cudaSuccess) return RMS_ERR_CUDA;
    rms_clean_s *c = new (std::nothrow) rms_clean_s();
    if (!c) return RMS_ERR_OOM;
    c->plan = plan;
    c->device = p.device;
    c->N = p.nphi;
    c->dphi = D;
    c->fwhm = fwhm;
    c->W = (int32_t)std::min<double>(p.nphi - 1, std::ceil(3.0 * fwhm / D));
    const int M = 2 * p.nphi - 1;
    std::vector<double> beam(2 * c->W + 1), offs(M);
    for (int d = -c->W; d <= c->W; ++d) beam[d + c->W] = std::exp(-4.0 * std::log(2.0) * (d * D) * (d * D) / (fwhm * fwhm));
    for (int m = 0; m < M; ++m) offs[m] = (m - (p.nphi - 1)) * D;
    double *d_offs = nullptr;
    cudaError_t e = cudaMalloc(&c->d_R2, (size_t)M * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_beam, beam.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_beam, beam.data(), beam.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (R2_host) {
            e = cudaMemcpy(c->d_R2, R2_host, (size_t)M * sizeof(double2), cudaMemcpyHostToDevice);
        } else {
            e = cudaMalloc(&d_offs, (size_t)M * sizeof(double));
            if (e == cudaSuccess) e = cudaMemcpy(d_offs, offs.data(), (size_t)M * sizeof(double), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = launch_rmsf(p, d_offs, M, reinterpret_cast<double *>(c->d_R2), nullptr, 0);
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_offs);
    if (prev >= 0 && prev != p.device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_clean(c);
        return from_cuda(e);
    }
    *out = c;
    return RMS_OK;
}

rms_status rms_clean_destroy(rms_clean_t c)
{
    if (!c) return RMS_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    free_clean(c);
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return RMS_OK;
}

rms_status rms_clean(rms_clean_t c, const float *F, int64_t nlos, float gain, int32_t max_iter, float threshold,
                     float *F_clean, float *residual, float *components, int32_t *niter, void *stream)
{
    if (!c || !F || nlos < 0 || max_iter < 0 || !(gain > 0.f && gain <= 1.f) || !(threshold >= 0.f) ||
        !std::isfinite(threshold))
        return RMS_ERR_INVALID_ARG;
    const uintptr_t mis = reinterpret_cast<uintptr_t>(F) | reinterpret_cast<uintptr_t>(F_clean) |
                          reinterpret_cast<uintptr_t>(residual) | reinterpret_cast<uintptr_t>(components);
    if (mis & 7) return RMS_ERR_INVALID_ARG;
    if (nlos == 0 || (!F_clean && !residual && !components && !niter)) return RMS_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device && cudaSetDevice(c->device) != cudaSuccess) return RMS_ERR_CUDA;
    CleanParams P;
    P.F = reinterpret_cast<const float2 *>(F);
    P.nlos = nlos;
    P.N = c->N;
    P.W = c->W;
    P.max_iter = max_iter;
    P.R2 = c->d_R2;
    P.beam = c->d_beam;
    P.gain = (double)gain;
    P.thr2 = (double)threshold * (double)threshold;
    P.clean = reinterpret_cast<float2 *>(F_clean);
    P.res_out = reinterpret_cast<float2 *>(residual);
    P.comp_out = reinterpret_cast<float2 *>(components);
    P.niter = niter;
    const size_t limit = 200 * 1024;
    int wpb = 8;
    while (wpb > 1 && clean_smem(c->N, c->W, wpb) > limit) --wpb;
    P.wpb = wpb;
    const size_t smem = clean_smem(c->N, c->W, wpb);
    cudaError_t e = cudaFuncSetAttribute(clean_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        const int64_t blocks = std::min<int64_t>((nlos + wpb - 1) / wpb, (int64_t)c->plan->num_sms * 8);
        clean_kernel<<<(unsigned)blocks, 32 * wpb, smem, reinterpret_cast<cudaStream_t>(stream)>>>(P);
        e = cudaGetLastError();
    }
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    return from_cuda(e);
}

}  // extern "C"
