// Window synthesis and the learned peak map (not in the paper).
//
// Window: for a plan with a uniform grid phi_k = phi_0 + k D, the fine grid is
// phi_n = phi_0 + n D / 2.  Synthesis on the window n - W/2 .. n + W/2 - 1 uses
// the exact identity (Eq. Fsum)
//     F(phi_n + m D/2) = K sum_j w_j (P_j T[n][j]) exp(-2i (m D/2) (lambda_j^2 - lambda_0^2)),
//     T[n][j] = exp(-2i phi_n (lambda_j^2 - lambda_0^2)),
// so every LOS shares one phase matrix (a plan whose phi grid is the W offsets
// m D/2) once its data has been multiplied by its own row of T.  T is built in
// FP64 and stored in FP32; the multiplication happens in shared memory inside
// the contraction kernel (its rotating variant), so the split operand is read
// from HBM once.
//
// Learned peak map: one split of the cube feeds (1) the network (hi parts of
// the operand image, scaled by 1/RMS per row), (2) the window contraction
// around 2 * proposed bin, (3) for the LOS that fall back (confidence below tau
// or NaN, window maximum on the window edge or absent) a compacted copy of
// their operand rows and the full-grid contraction on those rows only.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "rms_internal.h"

struct rms_window_s {
    rms_plan_s *plan = nullptr;   // the full-grid plan
    rms_plan_s *sub = nullptr;    // same channels, phi = the window offsets
    int device = 0;
    int32_t width = 0, ncentre = 0, cmin = 0, cmax = 0;
    double phi0 = 0, step = 0;    // fine grid phi_0 + n step, step = D / 2
    float2 *d_Tc = nullptr;       // [ncentre][ldc], active-channel order (channel-major images)
    float2 *d_Tr = nullptr;       // [ncentre][ldr], all channels (LOS-major images)
    int32_t ldc = 0, ldr = 0;
};

namespace {

rms_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return RMS_OK;
    if (e == cudaErrorMemoryAllocation) return RMS_ERR_OOM;
    return RMS_ERR_CUDA;
}

struct Guard {
    int prev = -1;
    bool ok = true;
    explicit Guard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~Guard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

void free_window(rms_window_s *w)
{
    if (!w) return;
    cudaFree(w->d_Tc);
    cudaFree(w->d_Tr);
    if (w->sub) rms_plan_destroy(w->sub);
    delete w;
}

rms_status check_cube(const float *Q, const float *U, int64_t nlos, int32_t layout)
{
    if (!Q || !U || nlos < 0) return RMS_ERR_INVALID_ARG;
    if (layout != RMS_CHAN_MAJOR && layout != RMS_LOS_MAJOR) return RMS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(Q) & 3) || (reinterpret_cast<uintptr_t>(U) & 3)) return RMS_ERR_INVALID_ARG;
    if (nlos > ((int64_t)1 << 31) - 128) return RMS_ERR_INVALID_ARG;
    return RMS_OK;
}

__global__ void centre_kernel(const int32_t *bin, int64_t n, int32_t cmin, int32_t cmax, int32_t *centre)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) centre[i] = max(cmin, min(cmax, 2 * bin[i]));
}

// phi of each window maximum: phi_0 + (centre - W/2 + widx) step
__global__ void window_phi_kernel(const int32_t *centre, const int32_t *widx, int64_t n, int32_t half, int32_t cmin,
                                  int32_t cmax, double phi0, double step, float *wphi)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = widx[i];
    const int c = max(cmin, min(cmax, centre[i]));
    wphi[i] = k < 0 ? __int_as_float(0x7fc00000) : (float)(phi0 + (double)(c - half + k) * step);
}

struct MergeParams {
    const int32_t *centre, *widx;
    const float *conf, *wabs;
    int64_t n;
    int32_t width, half;
    float tau;
    double phi0, step;
    float *phi_peak, *peak_abs;
    int32_t *fallback;
    int64_t *rows, *count;
};

// Window result or fallback, per LOS; fallbacks are appended to a compacted
// list (one atomic per warp).
__global__ void merge_kernel(const MergeParams P)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool fb = false;
    if (i < P.n) {
        const int k = P.widx[i];
        const float cf = P.conf[i];
        fb = !(cf >= P.tau) || k <= 0 || k >= P.width - 1;
        if (P.fallback) P.fallback[i] = fb ? 1 : 0;
        if (!fb) {
            if (P.phi_peak) P.phi_peak[i] = (float)(P.phi0 + (double)(P.centre[i] - P.half + k) * P.step);
            if (P.peak_abs) P.peak_abs[i] = P.wabs[i];
        }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, fb);
    if (mask == 0) return;
    int64_t base = 0;
    if (lane == 0) base = (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(P.count), (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (fb) P.rows[base + __popc(mask & ((1u << lane) - 1u))] = i;
}

}  // namespace

extern "C" {

rms_status rms_window_create(rms_window_t *out, rms_plan_t plan, int32_t width)
{
    if (!out) return RMS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plan || width < 8 || width > 128 || width % 8) return RMS_ERR_INVALID_ARG;
    if (plan->precision != RMS_BF16 && plan->precision != RMS_BF16X3) return RMS_ERR_UNSUPPORTED;
    const rms_plan_s &p = *plan;
    if (p.nphi < 2) return RMS_ERR_INVALID_ARG;
    const double D = (p.phi[p.nphi - 1] - p.phi[0]) / (p.nphi - 1);
    if (!(D > 0)) return RMS_ERR_INVALID_ARG;
    for (int k = 0; k < p.nphi; ++k)
        if (std::fabs(p.phi[k] - (p.phi[0] + k * D)) > 1e-9 * std::max(1.0, std::fabs(p.phi[k])))
            return RMS_ERR_INVALID_ARG;
    if (2 * (p.nphi - 1) + 1 < width) return RMS_ERR_INVALID_ARG;
    Guard guard(p.device);
    if (!guard.ok) return RMS_ERR_CUDA;
    rms_window_s *w = new (std::nothrow) rms_window_s();
    if (!w) return RMS_ERR_OOM;
    w->plan = plan;
    w->device = p.device;
    w->width = width;
    w->step = D / 2;
    w->phi0 = p.phi[0];
    w->ncentre = 2 * (p.nphi - 1) + 1;
    w->cmin = width / 2;
    w->cmax = w->ncentre - 1 - (width / 2 - 1);
    std::vector<double> offs(width);
    for (int m = 0; m < width; ++m) offs[m] = (m - width / 2) * w->step;
    rms_status st = plan_create_internal(&w->sub, p.lambda2.data(), p.nchan, RMS_AXIS_LAMBDA2, p.weights.data(),
                                         offs.data(), width, p.precision, p.device, 128);
    if (st != RMS_OK) {
        free_window(w);
        return st;
    }
    w->ldc = p.kblocks * kChanPerKBlock;
    w->ldr = p.kblocks_raw * kChanPerKBlock;
    std::vector<double> dl2c(p.nact), dl2r(p.nchan);
    for (int a = 0; a < p.nact; ++a) dl2c[a] = p.lambda2[p.active[a]] - p.lambda0sq;
    for (int c = 0; c < p.nchan; ++c) dl2r[c] = p.lambda2[c] - p.lambda0sq;
    double *d_tmp = nullptr;
    cudaError_t e = cudaMalloc(&d_tmp, (size_t)(p.nact + p.nchan) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(d_tmp, dl2c.data(), p.nact * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_tmp + p.nact, dl2r.data(), p.nchan * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&w->d_Tc, (size_t)w->ncentre * w->ldc * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&w->d_Tr, (size_t)w->ncentre * w->ldr * sizeof(float2));
    if (e == cudaSuccess) e = launch_rotation_table(d_tmp, p.nact, w->ldc, w->phi0, w->step, w->ncentre, w->d_Tc, 0);
    if (e == cudaSuccess)
        e = launch_rotation_table(d_tmp + p.nact, p.nchan, w->ldr, w->phi0, w->step, w->ncentre, w->d_Tr, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_tmp);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_window(w);
        return from_cuda(e);
    }
    *out = w;
    return RMS_OK;
}

rms_status rms_window_destroy(rms_window_t w)
{
    if (!w) return RMS_OK;
    Guard guard(w->device);   // the parent plan may already be gone: only the window's own state is used
    cudaDeviceSynchronize();
    free_window(w);
    return RMS_OK;
}

rms_status rms_window_centres(rms_window_t w, const int32_t *bin, int64_t nlos, int32_t *centre, void *stream)
{
    if (!w || !bin || !centre || nlos < 0 || nlos > ((int64_t)1 << 31) - 128) return RMS_ERR_INVALID_ARG;
    if (nlos == 0) return RMS_OK;
    Guard guard(w->device);
    if (!guard.ok) return RMS_ERR_CUDA;
    centre_kernel<<<(unsigned)((nlos + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        bin, nlos, w->cmin, w->cmax, centre);
    return from_cuda(cudaGetLastError());
}

rms_status rms_synth_window(rms_window_t w, const float *Q, const float *U, int64_t nlos, int32_t layout,
                            const int32_t *centre, float *F_out, int32_t *widx, float *wabs, float *wphi,
                            void *stream)
{
    if (!w || !centre) return RMS_ERR_INVALID_ARG;
    rms_status st = check_cube(Q, U, nlos, layout);
    if (st != RMS_OK) return st;
    if (F_out && (reinterpret_cast<uintptr_t>(F_out) & 7)) return RMS_ERR_INVALID_ARG;
    const rms_plan_s &p = *w->plan;
    if (*p.h_err || *w->sub->h_err) return RMS_ERR_TIMEOUT;
    if (nlos == 0 || (!F_out && !widx && !wabs && !wphi)) return RMS_OK;
    Guard guard(p.device);
    if (!guard.ok) return RMS_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ib = split_operand_bytes(p, nlos, layout), xb = (size_t)nlos * 4;
    uint8_t *scr = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scr), up(ib) + (widx ? 0 : up(xb)), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
    }
    int32_t *k = widx ? widx : reinterpret_cast<int32_t *>(scr + up(ib));
    SplitOpts so;
    so.Q = Q;
    so.U = U;
    so.nlos_src = nlos;
    so.layout = layout;
    so.nout = nlos;
    so.A = scr;
    e = launch_split(p, so, s);
    if (e == cudaSuccess) {
        GemmOpts go;
        go.A = scr;
        go.nlos = nlos;
        go.layout = layout;
        go.F = F_out;
        go.pidx = k;
        go.pabs = wabs;
        go.centre = centre;
        go.T = layout == RMS_CHAN_MAJOR ? w->d_Tc : w->d_Tr;
        go.ldT = layout == RMS_CHAN_MAJOR ? w->ldc : w->ldr;
        go.cmin = w->cmin;
        go.cmax = w->cmax;
        e = launch_gemm(*w->sub, go, s);
    }
    if (e == cudaSuccess && wphi) {
        window_phi_kernel<<<(unsigned)((nlos + 255) / 256), 256, 0, s>>>(centre, k, nlos, w->width / 2, w->cmin,
                                                                         w->cmax, w->phi0, w->step, wphi);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaFreeAsync(scr, s);
    if (e == cudaSuccess) e = e2;
    return from_cuda(e);
}

rms_status rms_peakmap_learned(rms_window_t w, rms_net_t net, const float *Q, const float *U, int64_t nlos,
                               int32_t layout, float tau, float *phi_peak, float *peak_abs, int32_t *fallback,
                               int64_t *nfallback, void *stream)
{
    if (!w || !net || net->plan != w->plan || std::isnan(tau)) return RMS_ERR_INVALID_ARG;
    rms_status st = check_cube(Q, U, nlos, layout);
    if (st != RMS_OK) return st;
    const rms_plan_s &p = *w->plan;
    if (*p.h_err || *w->sub->h_err) return RMS_ERR_TIMEOUT;
    Guard guard(p.device);
    if (!guard.ok) return RMS_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (nlos == 0) return nfallback ? from_cuda(cudaMemsetAsync(nfallback, 0, sizeof(int64_t), s)) : RMS_OK;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t ib = up(split_operand_bytes(p, nlos, layout));
    const size_t n4 = up((size_t)nlos * 4), n8 = up((size_t)nlos * 8);
    const size_t hb = up((size_t)nlos * net->hidden * 2);
    // image | fallback image | h | rscale | bin | conf | centre | widx | wabs | rows | count | peak keys
    const size_t total = 2 * ib + hb + 7 * n4 + 2 * n8 + 256;
    uint8_t *scr = nullptr;
    cudaError_t e = cudaStreamWaitEvent(s, net->last, 0);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&scr), total, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
    }
    uint8_t *img = scr, *img_fb = scr + ib;
    uint8_t *q = scr + 2 * ib;
    uint16_t *h = reinterpret_cast<uint16_t *>(q);
    q += hb;
    float *rs = reinterpret_cast<float *>(q);
    int32_t *bin = reinterpret_cast<int32_t *>(q + n4);
    float *conf = reinterpret_cast<float *>(q + 2 * n4);
    int32_t *centre = reinterpret_cast<int32_t *>(q + 3 * n4);
    int32_t *widx = reinterpret_cast<int32_t *>(q + 4 * n4);
    float *wabs = reinterpret_cast<float *>(q + 5 * n4);
    int64_t *rows = reinterpret_cast<int64_t *>(q + 7 * n4);
    int64_t *count = reinterpret_cast<int64_t *>(q + 7 * n4 + n8);
    // the fallback contraction's peak keys (its job schedule and CTA pairs)
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(q + 7 * n4 + n8 + 256);
    const unsigned g256 = (unsigned)((nlos + 255) / 256);

    SplitOpts so;
    so.Q = Q;
    so.U = U;
    so.nlos_src = nlos;
    so.layout = layout;
    so.nout = nlos;
    so.A = img;
    so.rscale = rs;
    e = launch_split(p, so, s);
    if (e == cudaSuccess)
        e = net_forward_image(*net, img, layout, rs, nlos, h, nullptr, bin, conf, w->width / 4 - 2, s);
    if (e == cudaSuccess) {
        centre_kernel<<<g256, 256, 0, s>>>(bin, nlos, w->cmin, w->cmax, centre);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        GemmOpts go;
        go.A = img;
        go.nlos = nlos;
        go.layout = layout;
        go.pidx = widx;
        go.pabs = wabs;
        go.centre = centre;
        go.T = layout == RMS_CHAN_MAJOR ? w->d_Tc : w->d_Tr;
        go.ldT = layout == RMS_CHAN_MAJOR ? w->ldc : w->ldr;
        go.cmin = w->cmin;
        go.cmax = w->cmax;
        e = launch_gemm(*w->sub, go, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int64_t), s);
    if (e == cudaSuccess) {
        MergeParams M;
        M.centre = centre;
        M.widx = widx;
        M.conf = conf;
        M.wabs = wabs;
        M.n = nlos;
        M.width = w->width;
        M.half = w->width / 2;
        M.tau = tau;
        M.phi0 = w->phi0;
        M.step = w->step;
        M.phi_peak = phi_peak;
        M.peak_abs = peak_abs;
        M.fallback = fallback;
        M.rows = rows;
        M.count = count;
        merge_kernel<<<g256, 256, 0, s>>>(M);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_image_gather(p, layout, img, rows, count, nlos, img_fb, s);
    if (e == cudaSuccess) {
        GemmOpts go;
        go.A = img_fb;
        go.nlos = nlos;
        go.count = count;
        go.rows = rows;
        go.layout = layout;
        go.pabs = peak_abs;
        go.pphi = phi_peak;
        go.keys = keys;
        e = launch_gemm(p, go, s);
    }
    if (e == cudaSuccess && nfallback) e = cudaMemcpyAsync(nfallback, count, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    cudaError_t e2 = cudaFreeAsync(scr, s);
    if (e == cudaSuccess) e = e2;
    e2 = cudaEventRecord(net->last, s);
    if (e == cudaSuccess) e = e2;
    return from_cuda(e);
}

}  // extern "C"
