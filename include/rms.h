/*
 * rms.h -- C ABI of a GB300 (sm_103a) library for Faraday rotation measure (RM)
 * synthesis, after Sridhar, Heald & van der Hulst, "cuFFS: A GPU-accelerated code
 * for Fast Faraday Rotation Measure Synthesis" (Astronomy & Computing).
 *
 * For every line of sight (LOS) of a Stokes Q/U cube the library computes
 *
 *     F(phi_k) = K sum_j w_j (Q_j + i U_j) exp(-2 i phi_k (lambda_j^2 - lambda_0^2))   (Sec. 2.2, Eq. Fsum)
 *     K        = 1 / sum_j w_j                                                      (Eq. Ksum)
 *     lambda_0^2 = sum_j w_j lambda_j^2 / sum_j w_j       (Sec. 2.2 "mean of lambda_i^2", weighted)
 *
 * plus the RMSF R(phi) (Eq. Rsum) and a per-LOS peak map: the index of
 * max_k |F(phi_k)| (Sec. 2.2, phi_peak), |F| there, and phi at that index.
 *
 * Conventions for every call:
 *  - Every pointer documented "device" is a CUDA device pointer on the plan's
 *    device; "host" pointers are ordinary CPU memory.  The caller owns every
 *    buffer it passes; the library never frees or retains them after the call.
 *  - Argument errors are detected before any work is queued and return
 *    RMS_ERR_INVALID_ARG; nothing is launched and no output is touched.
 *  - rms_synth is asynchronous on the caller's stream (a cudaStream_t passed
 *    as void*; NULL = legacy default stream).  A device-side failure (a bounded
 *    wait inside a kernel that ran out) is sticky on the plan: it is reported
 *    by rms_plan_sync and by the next rms_synth on that plan.
 *  - Nothing in the library calls exit(), abort() or a device trap.
 *  - Units: lambda^2 in m^2, frequency in Hz, phi in rad m^-2.
 *  - A plan may be used from several streams.  The tensor-core precisions keep
 *    a per-plan scratch for split operands, so every synthesis call on a plan
 *    waits on the device for the previous call on that plan (an event recorded
 *    by each call); use one plan per stream for concurrent work.
 *    rms_synth_host owns per-plan staging buffers and must not run
 *    concurrently with itself on one plan.
 */
#ifndef RMS_H
#define RMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rms_plan_s *rms_plan_t;

typedef enum {
    RMS_OK = 0,
    RMS_ERR_INVALID_ARG = 1,   /* bad pointer, size, enum or channel set */
    RMS_ERR_OOM = 2,           /* device or pinned host allocation failed */
    RMS_ERR_CUDA = 3,          /* a CUDA runtime/driver call failed */
    RMS_ERR_UNSUPPORTED = 4,   /* e.g. tensor-core precision on a non-sm_103 device */
    RMS_ERR_TIMEOUT = 5        /* a bounded wait inside a kernel gave up */
} rms_status;

/* Kind of the channel axis passed to rms_plan_create. */
enum { RMS_AXIS_LAMBDA2 = 0, RMS_AXIS_FREQ_HZ = 1 };

/* Cube layouts (Sec. 3.2): channel-major is the FITS plane order, LOS-major has
 * frequency as the fastest axis (a "rotated" cube). */
enum {
    RMS_CHAN_MAJOR = 0,        /* Q[c * nlos + l] */
    RMS_LOS_MAJOR = 1          /* Q[l * nchan + c] */
};

/* How the contraction is computed.  The phase argument is always formed and
 * reduced mod 2 pi in FP64 at plan time, except RMS_FP32_SIMT_FLY, which is the
 * paper's own per-element FP32 sin/cos method (Sec. 3). */
enum {
    RMS_FP32_SIMT_FLY = 0,     /* FP32 CUDA cores, sincosf of an FP32 argument per (channel, phi) */
    RMS_FP32_SIMT_TABLE = 1,   /* FP32 CUDA cores, FP32 phase table built in FP64 */
    RMS_BF16 = 2,              /* tcgen05 tensor cores, one BF16 product, FP32 accumulate */
    RMS_BF16X3 = 3,            /* tcgen05, split BF16 hi+lo: hi*hi + hi*lo + lo*hi */
    RMS_FP16X3 = 4             /* tcgen05, split FP16 hi+lo with per-LOS power-of-2 data scaling */
};

/*
 * Create a plan for one channel set and one phi grid (Sec. 2.3: K, 2 phi and
 * lambda^2 - lambda_0^2 "need to be computed only once").
 *
 *  plan      host, out: receives the new plan (set to NULL on failure).
 *  axis      host, [nchan] doubles: lambda^2 in m^2 (RMS_AXIS_LAMBDA2) or channel
 *            centre frequencies in Hz (RMS_AXIS_FREQ_HZ; lambda = c / nu,
 *            c = 299792458 m/s).  Must be finite (and > 0 for frequencies).
 *  nchan     1 .. 65536.
 *  weights   host, [nchan] doubles, or NULL for all 1.  w_j = W(lambda_j^2)
 *            (Sec. 2.1); 0 flags a channel, whose data is then never read into
 *            the sum (NaN there is harmless).  Must be finite, >= 0, sum > 0.
 *  phi       host, [nphi] doubles, Faraday depths; any finite values, any order.
 *  nphi      1 .. 1048576.
 *  precision one of RMS_FP32_SIMT_FLY .. RMS_FP16X3.
 *  device    CUDA device ordinal the plan lives on.
 *
 * Builds on the device: the FP64 phase matrix / table for the chosen precision
 * and the RMSF.  Synchronises the device before returning.
 * Returns RMS_ERR_INVALID_ARG for any invalid argument above, RMS_ERR_OOM when
 * an allocation fails, RMS_ERR_UNSUPPORTED for a tensor-core precision on a
 * device that is not compute capability 10.3, RMS_ERR_CUDA otherwise.
 */
rms_status rms_plan_create(rms_plan_t *plan, const double *axis, int32_t nchan, int32_t axis_kind,
                           const double *weights, const double *phi, int32_t nphi,
                           int32_t precision, int32_t device);

/*
 * RMSF and plan constants (Sec. 2.2, Eq. Rsum; resolution estimate of Sec. 2.2).
 *
 *  R_out      device, [2 * nphi] floats (re, im interleaved) = R(phi_k), or NULL.
 *  lambda0sq  host, out, or NULL: weighted mean lambda^2.
 *  K          host, out, or NULL: 1 / sum w.
 *  fwhm_meas  host, out, or NULL: FWHM of |R(phi)|'s main lobe, measured on R
 *             (evaluated in FP64 on the device, bracketed and refined).
 *  fwhm_est   host, out, or NULL: the paper's estimate 2 sqrt(3) / Delta lambda^2
 *             over the weighted channels.
 * Synchronous.  Returns RMS_ERR_INVALID_ARG for a NULL plan.
 */
rms_status rms_rmsf(rms_plan_t plan, float *R_out, double *lambda0sq, double *K,
                    double *fwhm_meas, double *fwhm_est);

/*
 * RM synthesis of a cube (Sec. 2.2, Eq. Fsum; Eqs. qPhi/uPhi for the real form)
 * with the fused peak map.
 *
 *  Q, U      device, nchan * nlos floats each, in `layout` (see above); 4-byte aligned.
 *  nlos      number of lines of sight, >= 0 (0 launches nothing).
 *  layout    RMS_CHAN_MAJOR or RMS_LOS_MAJOR.
 *  F_out     device, [nlos][nphi] complex64 (re, im floats, phi fastest, Sec. 3.2),
 *            8-byte aligned; or NULL to compute only the peak map.
 *  peak_idx  device, [nlos] int32: index k of max |F(phi_k)|, lowest k on ties,
 *            NaN never selected, -1 when no |F| is finite; or NULL.
 *  peak_abs  device, [nlos] float: |F| at peak_idx (NaN for -1); or NULL.
 *  phi_peak  device, [nlos] float: phi[peak_idx] (NaN for -1); or NULL.
 *  stream    cudaStream_t as void*.
 * |F| is sqrt(re*re + im*im) of the stored FP32 values, each product and the sum
 * rounded to FP32 separately, so the peak index can be recomputed bit-exactly
 * from F_out.  Asynchronous, no host sync.  The tensor-core precisions take a
 * per-call scratch from the device's default stream-ordered memory pool on
 * `stream` (cudaMallocAsync / cudaFreeAsync): the cube split into 16-bit
 * operands, 4 bytes per (LOS, contraction channel) (2 for RMS_BF16), and for
 * RMS_FP16X3 one exponent byte per LOS; creating a tensor-core plan sets that
 * pool to keep freed memory reserved.  The FP32 precisions allocate nothing.
 */
rms_status rms_synth(rms_plan_t plan, const float *Q, const float *U, int64_t nlos, int32_t layout,
                     float *F_out, int32_t *peak_idx, float *peak_abs, float *phi_peak, void *stream);

/*
 * rms_synth from HOST buffers: copies Q and U to the device, synthesises, copies
 * F and the peak map back, and synchronises.  Same arguments as rms_synth with
 * every array a host pointer (pinned memory gives full copy bandwidth).  The
 * plan keeps device staging buffers between calls (grown on demand, freed by
 * rms_plan_destroy).  Returns RMS_ERR_OOM when staging cannot be allocated.
 */
rms_status rms_synth_host(rms_plan_t plan, const float *Q, const float *U, int64_t nlos,
                          int32_t layout, float *F_out, int32_t *peak_idx, float *peak_abs,
                          float *phi_peak, void *stream);

/*
 * rms_synth for FP16X3 plans that allocates nothing.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory while
 * they process data -- a pipeline that reserves all of its GPU memory when an
 * observation starts and treats any later allocation as an error, or a host
 * framework whose own allocator owns the device's memory budget.  rms_synth on
 * an FP16X3 plan takes a one-byte-per-LOS scratch from the stream-ordered pool
 * for every call; here that scratch is a fixed device array of
 * RMS_NOALLOC_MAX_LOS bytes compiled into the library, which every GPU that
 * loads the library holds until the process exits.
 *
 * Same arguments and results as rms_synth.  Returns RMS_ERR_INVALID_ARG when
 * nlos > RMS_NOALLOC_MAX_LOS (nothing is launched) and RMS_ERR_UNSUPPORTED for a
 * plan of another precision (rms_synth allocates nothing for those already).
 * Calls no cudaMalloc, cudaFree or pool allocation.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  All calls in the process share the one
 * array and every call rewrites the entries it uses, so calls whose kernels
 * overlap on the GPU race: do not run two at once, on any plans or streams.
 */
#define RMS_NOALLOC_MAX_LOS (1 << 22)
rms_status rms_synth_noalloc(rms_plan_t plan, const float *Q, const float *U, int64_t nlos, int32_t layout,
                             float *F_out, int32_t *peak_idx, float *peak_abs, float *phi_peak, void *stream);

/* Wait for `stream` (void* cudaStream_t) and report sticky device errors of
 * this plan: RMS_ERR_TIMEOUT if a kernel's bounded wait gave up, RMS_ERR_CUDA
 * for an asynchronous CUDA error.  The sticky state is cleared by the call. */
rms_status rms_plan_sync(rms_plan_t plan, void *stream);

/* Plan facts for callers and tests. */
enum {
    RMS_INFO_NCHAN = 0, RMS_INFO_NCHAN_ACTIVE = 1, RMS_INFO_NPHI = 2, RMS_INFO_PRECISION = 3,
    RMS_INFO_KPAD = 4,        /* padded contraction length of the tensor-core operand */
    RMS_INFO_NPAD = 5,        /* padded rows (2 * nphi rounded up) of the phase matrix */
    RMS_INFO_TILE_N = 6,      /* phase-matrix rows per tensor-core tile */
    RMS_INFO_DEVICE = 7
};
rms_status rms_plan_info(rms_plan_t plan, int32_t what, int64_t *value);

/*
 * Copy plan-owned arrays to the host (for inspection and tests).
 *   RMS_GET_LAMBDA2  double[nchan]            lambda_j^2
 *   RMS_GET_ACTIVE   int32 [nchan_active]     indices of channels with w != 0
 *   RMS_GET_TABLE    float [nchan_active][nphi][2]  w_j (cos, sin)(theta_jk), FP32 table plans only
 *   RMS_GET_B_HI     uint16[npad][kpad]       tensor-core phase matrix, high part (bf16/fp16 bits)
 *   RMS_GET_B_LO     uint16[npad][kpad]       low part
 *   RMS_GET_RMSF64   double[nphi][2]          R(phi_k) accumulated in FP64
 * `bytes` must equal the array size exactly.  Synchronous.
 */
enum { RMS_GET_LAMBDA2 = 0, RMS_GET_ACTIVE = 1, RMS_GET_TABLE = 2, RMS_GET_B_HI = 3,
       RMS_GET_B_LO = 4, RMS_GET_RMSF64 = 5 };
rms_status rms_plan_get(rms_plan_t plan, int32_t what, void *host_dst, int64_t bytes);

/* Destroy a plan: synchronises the plan's device, frees everything it owns.
 * NULL is accepted and returns RMS_OK. */
rms_status rms_plan_destroy(rms_plan_t plan);

/* Static English text for a status code (never NULL). */
const char *rms_status_string(rms_status s);

/* Bounded-wait limit, in nanoseconds, used by the tensor-core kernel's barrier
 * waits (default 2e9).  A kernel whose wait runs out stops, records
 * RMS_ERR_TIMEOUT on the plan and returns. */
rms_status rms_plan_set_timeout(rms_plan_t plan, int64_t ns);

#ifdef __cplusplus
}
#endif

#endif /* RMS_H */
