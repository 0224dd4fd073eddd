// Self-test of the device-side failure path: a kernel whose bounded mbarrier wait
// cannot complete (nothing ever arrives on the barrier).  The wait must give up
// after the plan's limit, record RMS_DEVERR_TIMEOUT in the plan's mapped error
// word and let the kernel return, leaving the context usable -- the same helper
// every pipeline wait of the tensor-core kernels uses.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rms_internal.h"

namespace {

#include "tc_ptx.cuh"

__global__ void __launch_bounds__(32, 1) stuck_wait_kernel(int *err, int64_t limit_ns, int *done)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);   // expects one arrival that never comes
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = warp_wait(smem_u32(&bar), 0, &abort_flag, err, limit_ns);
    if (threadIdx.x == 0) *done = ok ? 1 : 2;
}

}  // namespace

extern "C" rms_status rms_selftest_wait_timeout(rms_plan_t p, int64_t limit_ns, int32_t *outcome)
{
    if (!p || limit_ns <= 0 || limit_ns > 10000000000LL || !outcome) return RMS_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->device && cudaSetDevice(p->device) != cudaSuccess) return RMS_ERR_CUDA;
    int *d_done = nullptr;
    cudaError_t e = cudaMalloc(&d_done, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d_done, 0, sizeof(int));
    if (e == cudaSuccess) {
        stuck_wait_kernel<<<1, 32>>>(p->d_err, limit_ns, d_done);
        e = cudaGetLastError();
    }
    int done = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&done, d_done, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d_done);
    if (prev >= 0 && prev != p->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return RMS_ERR_CUDA;
    *outcome = done;
    return RMS_OK;
}
