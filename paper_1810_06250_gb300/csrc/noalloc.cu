// rms_synth_noalloc: RM synthesis on FP16X3 plans without any device allocation.
//
// rms_synth on an FP16X3 plan takes a per-line-of-sight exponent scratch (one
// byte per LOS) from the stream-ordered memory pool for every call.  Callers
// whose device memory is reserved up front and who must not allocate while
// data streams in cannot accept that; this entry point keeps the scratch in a
// fixed array that is part of the loaded library instead.
#include <mutex>

#include "rms_internal.h"

namespace {

// One byte per line of sight; every GPU that loads the library holds it until exit.
static __device__ __align__(256) int8_t g_noalloc_rexp[RMS_NOALLOC_MAX_LOS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int8_t *g_rexp_ptr[kMaxDevices] = {};

// Device address of g_noalloc_rexp on the current device (looked up once per device).
// The lookup loads this file's module on the device, and with it the array.
cudaError_t rexp_address(int device, int8_t **out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_rexp_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_rexp);
        if (e != cudaSuccess) return e;
        g_rexp_ptr[device] = static_cast<int8_t *>(p);
    }
    *out = g_rexp_ptr[device];
    return cudaSuccess;
}

}  // namespace

// Called by rms_plan_create for FP16X3 plans, with the plan's device current:
// everything rms_synth_noalloc needs on a device is loaded here, where allocating
// is allowed -- the array (through its address lookup) and the code of the two
// kernels it launches -- so that with lazy module loading no later call makes the
// driver allocate module memory.
cudaError_t noalloc_prepare(int device)
{
    int8_t *p = nullptr;
    cudaError_t e = rexp_address(device, &p);
    if (e == cudaSuccess) e = umma_prepare();
    return e;
}

extern "C" rms_status rms_synth_noalloc(rms_plan_t p, const float *Q, const float *U, int64_t nlos, int32_t layout,
                                        float *F_out, int32_t *peak_idx, float *peak_abs, float *phi_peak,
                                        void *stream)
{
    const rms_status st = check_synth_args(p, Q, U, nlos, layout, F_out);   // the checks of rms_synth
    if (st != RMS_OK) return st;
    if (nlos > RMS_NOALLOC_MAX_LOS) return RMS_ERR_INVALID_ARG;   // beyond the fixed scratch
    if (p->precision != RMS_FP16X3) return RMS_ERR_UNSUPPORTED;
    if (*p->h_err) return RMS_ERR_TIMEOUT;
    if (nlos == 0 || (!F_out && !peak_idx && !peak_abs && !phi_peak)) return RMS_OK;

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return RMS_ERR_CUDA;
    if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess) return RMS_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int8_t *rexp = nullptr;
    cudaError_t e = rexp_address(p->device, &rexp);
    // calls on one plan share its split-operand scratch: order them on the device
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->last, 0);
    if (e == cudaSuccess) e = launch_row_exponent(*p, Q, U, nlos, layout, rexp, s);
    if (e == cudaSuccess) e = launch_umma(*p, Q, U, nlos, layout, F_out, peak_idx, peak_abs, phi_peak, rexp, s);
    if (e == cudaSuccess) e = cudaEventRecord(p->last, s);
    if (prev != p->device) cudaSetDevice(prev);
    if (e == cudaErrorMemoryAllocation) return RMS_ERR_OOM;
    return e == cudaSuccess ? RMS_OK : RMS_ERR_CUDA;
}
