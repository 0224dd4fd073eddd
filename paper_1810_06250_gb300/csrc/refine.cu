// Sub-grid refinement of the Faraday-depth peak.  The synthesis reports the
// grid sample where |F| peaks (Sec. 2.2); between samples the main lobe of the
// RMSF is close to a parabola, so the vertex of the parabola through |F| at the
// peak sample and its two neighbours estimates the peak's depth and height
// off the grid.  With t measured from phi_k, d0 = phi_{k-1} - phi_k and
// d2 = phi_{k+1} - phi_k, the parabola y(t) = y_k + b t + a t^2 through the three
// points has
//     a = ((y_{k-1} - y_k) / d0 - (y_{k+1} - y_k) / d2) / (d0 - d2),
//     b = (y_{k-1} - y_k) / d0 - a d0,
// and for a < 0 its vertex is t* = -b / (2a), y* = y_k + b t* + a t*^2.  This
// holds on any strictly monotonic grid, uniform or not.  Everything runs in
// FP64 from the stored FP32 values; one thread per LOS reads three samples.
#include <math.h>

#include "rms_internal.h"

namespace {

struct RefineParams {
    const float2 *F;
    int64_t nlos;
    int32_t nphi;
    const int32_t *idx;
    const double *phi;
    float *phi_ref, *abs_ref;
};

__device__ __forceinline__ double mag(float2 v)
{
    return sqrt((double)v.x * (double)v.x + (double)v.y * (double)v.y);
}

__global__ void __launch_bounds__(256) refine_kernel(const RefineParams P)
{
    const float qnan = __int_as_float(0x7fc00000);
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < P.nlos;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = P.idx[l];
        float pr = qnan, ar = qnan;
        if (k >= 0 && k < P.nphi) {
            const float2 *row = P.F + l * P.nphi;
            const double x1 = P.phi[k], y1 = mag(row[k]);
            double t = 0.0, y = y1;
            if (k > 0 && k + 1 < P.nphi) {
                const double d0 = P.phi[k - 1] - x1, d2 = P.phi[k + 1] - x1;
                const double y0 = mag(row[k - 1]), y2 = mag(row[k + 1]);
                // neighbours on opposite sides (a monotonic triple), finite samples
                if (d0 * d2 < 0.0) {
                    const double s0 = (y0 - y1) / d0, s2 = (y2 - y1) / d2;
                    const double a = (s0 - s2) / (d0 - d2), b = s0 - a * d0;
                    if (a < 0.0) {
                        t = -b / (2.0 * a);
                        const double lo = fmin(d0, d2), hi = fmax(d0, d2);
                        t = fmin(fmax(t, lo), hi);
                        y = y1 + b * t + a * t * t;
                    }
                }
            }
            pr = (float)(x1 + t);
            ar = (float)y;
        }
        if (P.phi_ref) P.phi_ref[l] = pr;
        if (P.abs_ref) P.abs_ref[l] = ar;
    }
}

rms_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return RMS_OK;
    if (e == cudaErrorMemoryAllocation) return RMS_ERR_OOM;
    return RMS_ERR_CUDA;
}

}  // namespace

extern "C" {

rms_status rms_refine_peaks(rms_plan_t plan, const float *F, int64_t nlos, const int32_t *peak_idx,
                            float *phi_ref, float *abs_ref, void *stream)
{
    if (!plan || !F || !peak_idx || nlos < 0) return RMS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(F) & 7) return RMS_ERR_INVALID_ARG;
    if (nlos == 0 || (!phi_ref && !abs_ref)) return RMS_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != plan->device && cudaSetDevice(plan->device) != cudaSuccess) return RMS_ERR_CUDA;
    RefineParams P;
    P.F = reinterpret_cast<const float2 *>(F);
    P.nlos = nlos;
    P.nphi = plan->nphi;
    P.idx = peak_idx;
    P.phi = plan->d_phi;
    P.phi_ref = phi_ref;
    P.abs_ref = abs_ref;
    const int64_t want = (nlos + 255) / 256, cap = (int64_t)plan->num_sms * 16;
    refine_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(P);
    const cudaError_t e = cudaGetLastError();
    if (prev >= 0 && prev != plan->device) cudaSetDevice(prev);
    return from_cuda(e);
}

}  // extern "C"
