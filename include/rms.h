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
 *  - Tuning knobs: environment variables read once per process, for measurement.
 *    None of them changes what is computed beyond FP32 rounding order, and unset
 *    (or out-of-range) means the documented default:
 *      RMS_MAX_TILE_N (16..208)    phase rows per single-CTA tile (plan creation);
 *      RMS_GEMM_PAIR=0 | 2         single CTAs by default | pairs wherever tiles allow;
 *      RMS_L2_BUDGET_MB (8..1024)  L2 budget of the contraction's schedule (80);
 *      RMS_GROUP_KBLOCKS (2..64)   K blocks per TMEM partial before the FP32 fold of
 *                                  the split precisions (16; more chained MMAs add
 *                                  accumulation error: per LOS on the 1536-channel
 *                                  MWA cube, BF16X3 4.6e-6 at 16 and 6.1e-6 at 32);
 *      RMS_GEMM_CTAS (1..SMs)      persistent CTAs of the contraction;
 *      RMS_HOST_CHUNK (>= 1024)    LOS per chunk of rms_synth_host.
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
    RMS_FP16X3 = 4,            /* tcgen05, split FP16 hi+lo with per-LOS power-of-2 data scaling */
    RMS_FP32_CHIRPZ = 5        /* FP32 FFTs (chirp-z), exact for channels uniform in lambda^2 */
};

/*
 * RMS_FP32_CHIRPZ evaluates Eq. Fsum with FFTs (Sec. 4 names FFTs as the route to
 * further speed).  With x_j = lambda_j^2 - lambda_0^2 = x_0 + j D (every channel,
 * flagged ones included) and phi_k = phi_0 + k d, 2 j k = j^2 + k^2 - (k - j)^2
 * turns the sum into a convolution, which FFTs of length M (a power of two,
 * 1024 <= M, nchan + nphi - 1 <= M <= 2048) compute exactly up to FP32
 * rounding:
 *     F_k = K e^{-i (2 phi_0 x_0 + 2 d x_0 k + d D k^2)} sum_j w_j P_j e^{-i (2 phi_0 D j + d D j^2)} e^{i d D (k - j)^2}.
 * rms_plan_create returns RMS_ERR_UNSUPPORTED for this precision unless both
 * axes are uniform -- each model's largest deviation times the other axis'
 * largest |value| moves no phase by more than 1e-8 rad -- and M <= 2048.
 */

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
 *  precision one of RMS_FP32_SIMT_FLY .. RMS_FP32_CHIRPZ.
 *  device    CUDA device ordinal the plan lives on.
 *
 * Builds on the device: the FP64 phase matrix / table for the chosen precision
 * and the RMSF.  Synchronises the device before returning.
 * Returns RMS_ERR_INVALID_ARG for any invalid argument above, RMS_ERR_OOM when
 * an allocation fails, RMS_ERR_UNSUPPORTED on a device that is not compute
 * capability 10.3 or for RMS_FP32_CHIRPZ on axes it cannot take, RMS_ERR_CUDA
 * otherwise.
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
 * `stream` (cudaMallocAsync / cudaFreeAsync): the cube split into 16-bit hi and
 * lo operands, 8 bytes per (LOS, contraction channel slot; the channels are
 * padded to a multiple of 16 per 128 LOS), and for RMS_FP16X3 one exponent
 * byte per LOS; creating a tensor-core plan sets that pool to keep freed
 * memory reserved.  The FP32 precisions allocate nothing.
 */
rms_status rms_synth(rms_plan_t plan, const float *Q, const float *U, int64_t nlos, int32_t layout,
                     float *F_out, int32_t *peak_idx, float *peak_abs, float *phi_peak, void *stream);

/*
 * rms_synth with the paper's full set of peak outputs (Sec. 2.2: the values of
 * Q~ and U~ where |F~| peaks, and the polarisation angle there).  Arguments as
 * rms_synth; the peak outputs come in a struct, every pointer a device [nlos]
 * array or NULL:
 *   peak_idx, peak_abs, phi_peak  as rms_synth;
 *   q_peak, u_peak  Re F and Im F (K-scaled, Eqs. qPhi, uPhi) at peak_idx;
 *   chi0            0.5 atan2(u_peak, q_peak) - phi_peak lambda_0^2 reduced to
 *                   [0, pi): the angle of the Sec. 2.2 relation (printed garbled
 *                   there; for a Faraday-thin source on the grid it is the
 *                   source's intrinsic chi0).  NaN where peak_idx = -1.
 * q_peak, u_peak and chi0 need a tensor-core precision or RMS_FP32_CHIRPZ
 * (RMS_ERR_UNSUPPORTED for the FP32 SIMT precisions).  RMS_ERR_INVALID_ARG for a NULL `out`.
 */
typedef struct {
    int32_t *peak_idx;
    float *peak_abs, *phi_peak;
    float *q_peak, *u_peak, *chi0;
} rms_peak_outputs;
rms_status rms_synth_peaks(rms_plan_t plan, const float *Q, const float *U, int64_t nlos, int32_t layout,
                           float *F_out, const rms_peak_outputs *out, void *stream);

/*
 * Sub-grid peak refinement (the paper reports the grid sample where |F| peaks,
 * Sec. 2.2; this interpolates between samples): for each LOS, the vertex of the
 * parabola through |F| at phi_{k-1}, phi_k, phi_{k+1}, k = peak_idx[l].  With
 * d0 = phi_{k-1} - phi_k, d2 = phi_{k+1} - phi_k and y = |F| (FP64 from the
 * stored FP32 values):
 *     a = ((y_{k-1} - y_k) / d0 - (y_{k+1} - y_k) / d2) / (d0 - d2)
 *     b = (y_{k-1} - y_k) / d0 - a d0,   t* = -b / (2a) clamped to [d0, d2]
 *     phi_ref = phi_k + t*,   abs_ref = y_k + b t* + a t*^2
 * computed in FP64, rounded to FP32.  Where that is undefined -- k at either end
 * of the grid, a >= 0, a NaN neighbour, or neighbours on the same side of phi_k
 * (a non-monotonic grid) -- phi_ref = phi_k and abs_ref = |F_k|.  NaN for both
 * where peak_idx is -1 (or out of range).
 *   F        device [nlos][nphi] complex64 from rms_synth (8-byte aligned)
 *   peak_idx device [nlos] int32 from the same call
 *   phi_ref, abs_ref  device [nlos] float, either may be NULL
 * Asynchronous on stream; allocates nothing.  RMS_ERR_INVALID_ARG for a NULL
 * plan, F or peak_idx, nlos < 0, or a misaligned F.
 */
rms_status rms_refine_peaks(rms_plan_t plan, const float *F, int64_t nlos, const int32_t *peak_idx,
                            float *phi_ref, float *abs_ref, void *stream);

/*
 * rms_synth from HOST buffers: copies Q and U to the device, synthesises, copies
 * F and the peak map back, and synchronises.  Same arguments as rms_synth with
 * every array a host pointer.  Large cubes are processed in chunks of LOS
 * (LOS-major: max(16384, nlos / 16); channel-major: max(65536, nlos / 8),
 * whose 2-D copies need long rows) through three device slots, with the
 * copies in on a plan-owned stream, the synthesis on `stream` and the copies
 * out on a second plan-owned stream, so that they overlap; a channel-major
 * chunk is copied as a 2-D sub-array.  The copies overlap only from pinned
 * (page-locked) host memory.  The plan keeps the device slots between calls
 * (grown on demand, freed by rms_plan_destroy).  Returns RMS_ERR_OOM when they
 * cannot be allocated.
 */
rms_status rms_synth_host(rms_plan_t plan, const float *Q, const float *U, int64_t nlos,
                          int32_t layout, float *F_out, int32_t *peak_idx, float *peak_abs,
                          float *phi_peak, void *stream);

/*
 * Page-locked host memory for rms_synth_host (the paper streams cubes that live
 * in host memory through the GPU, Sec. 3.2; this call has no counterpart
 * there).  rms_host_alloc maps `bytes` of anonymous memory, asks the kernel for
 * transparent huge pages on it (a hint), and registers it with CUDA
 * (cudaHostRegister, portable to every device), so that the copies of
 * rms_synth_host overlap and run at the host link's rate (on GB300 210 GB/s to
 * the device and 193 GB/s back).  Measured on GB300 after other processes had
 * used the host's memory: buffers from the CUDA host allocator (cudaHostAlloc,
 * behind torch's pin_memory) copied at 25-85 GB/s to the device while these
 * kept 210 GB/s, in the same process.
 *
 * *ptr receives the address (aligned to the host page size), or NULL on failure;
 * the memory is not initialised.  Release it with rms_host_free(ptr, bytes),
 * passing the same size.  Returns RMS_ERR_INVALID_ARG for bytes <= 0 or a NULL
 * ptr, RMS_ERR_OOM when the mapping or the registration fails for lack of
 * memory, RMS_ERR_CUDA for another registration failure.  Thread-safe.
 */
rms_status rms_host_alloc(int64_t bytes, void **ptr);
rms_status rms_host_free(void *ptr, int64_t bytes);

/*
 * rms_synth for FP16X3 plans that allocates nothing.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory while
 * they process data -- a pipeline that reserves all of its GPU memory when an
 * observation starts and treats any later allocation as an error, or a host
 * framework whose own allocator owns the device's memory budget.  rms_synth on
 * an FP16X3 plan takes a one-byte-per-LOS scratch from the stream-ordered pool
 * for every call; here that scratch is a fixed device array of
 * RMS_NOALLOC_MAX_LOS bytes compiled into the library.  It becomes resident on a
 * device, together with the code of the kernels this call launches, when the
 * first FP16X3 plan is created there (rms_plan_create looks up the array's
 * address with cudaGetSymbolAddress and loads the kernels, so that lazy module
 * loading cannot allocate during a call), and it stays until the process exits.
 *
 * Same arguments and checks as rms_synth.  Returns RMS_ERR_INVALID_ARG when
 * nlos > RMS_NOALLOC_MAX_LOS (nothing is launched) and RMS_ERR_UNSUPPORTED for a
 * plan of another precision (rms_synth allocates nothing for those already).
 * Calls no cudaMalloc, cudaFree or pool allocation.  All calls in the process
 * share the one array and every call rewrites the entries it uses, so calls
 * whose kernels overlap on the GPU race: do not run two at once, on any plans
 * or streams.  The kernel-timing hook (rms_plan_set_kernel_timing) records
 * nothing for these calls.
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
    RMS_INFO_DEVICE = 7,
    /* what the last tensor-core rms_synth / rms_synth_peaks / rms_synth_host call ran: */
    RMS_INFO_LAST_CTAS = 8,   /* persistent CTAs of the contraction kernel */
    RMS_INFO_LAST_PAIR = 9,   /* 1: CTA pairs (two SMs per 256-row MMA), 0: single CTAs */
    RMS_INFO_LAST_PANELS = 10, /* 0: each CTA ran all phase tiles of its lines of sight;
                                  k > 0: single-tile jobs in k panels of the phase matrix */
    RMS_INFO_LAST_KERNELS = 11 /* kernels the call launched */
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

/*
 * How the tensor-core contraction of a plan is scheduled (no paper counterpart;
 * for measurement and tuning -- none of these changes a result):
 *   RMS_OPT_CONTRACTION  RMS_CONTRACT_AUTO (default): CTA pairs when the plan's pair
 *                        tiles are wider than 208 phase rows (2 nphi > 832 or so),
 *                        single CTAs otherwise; RMS_CONTRACT_SINGLE: one CTA per
 *                        128-row MMA with tiles of up to 208 phase rows;
 *                        RMS_CONTRACT_PAIR: CTA pairs (256-row MMAs on two SMs, each
 *                        SM holding half of a tile of up to 256 phase rows), or
 *                        RMS_ERR_UNSUPPORTED when the tiles do not allow them.
 *   RMS_OPT_SCHEDULE     RMS_SCHEDULE_AUTO (default): single-tile jobs (one line-of-
 *                        sight tile against one phase tile), dealt round-robin in
 *                        panels of the phase matrix, the peak map merged afterwards --
 *                        except for rms_synth_peaks calls that want Q, U or chi0 at the
 *                        peak without F_out; RMS_SCHEDULE_WHOLE: every CTA runs all
 *                        phase tiles of its lines of sight.  Both give bit-identical
 *                        outputs.
 *   RMS_OPT_L2_BUDGET    bytes of L2 the job schedule may count on (0 = the default,
 *                        80 MiB): the fewest panels whose working set (the operands
 *                        of the line-of-sight tiles in flight plus one panel of the
 *                        phase matrix) fits.
 * The environment variables RMS_GEMM_PAIR=0 (or 2: pairs wherever the tiles allow)
 * and RMS_L2_BUDGET_MB=<MiB>, read once per process, change the defaults.  Synchronous; RMS_ERR_INVALID_ARG
 * for an unknown option or value.
 */
enum { RMS_OPT_CONTRACTION = 0, RMS_OPT_L2_BUDGET = 1, RMS_OPT_SCHEDULE = 2 };
enum { RMS_SCHEDULE_AUTO = 0, RMS_SCHEDULE_WHOLE = 1 };
enum { RMS_CONTRACT_AUTO = 0, RMS_CONTRACT_SINGLE = 1, RMS_CONTRACT_PAIR = 2 };
rms_status rms_plan_set_option(rms_plan_t plan, int32_t option, int64_t value);

/*
 * Kernel timing for measurement (the paper has no counterpart).  While enabled,
 * every tensor-core synthesis call on the plan records CUDA events on its
 * stream around its two kernels (the layout stage that splits the cube into
 * 16-bit operands, and the tensor-core contraction).  rms_plan_kernel_times
 * waits for the recorded events, returns the summed milliseconds of each kernel
 * and the number of calls timed (host outputs, each may be NULL), and forgets
 * them.  FP32 plans and calls made while disabled record nothing.  Timing adds
 * three event records per call; it is off by default.
 */
rms_status rms_plan_set_kernel_timing(rms_plan_t plan, int32_t enable);
rms_status rms_plan_kernel_times(rms_plan_t plan, double *split_ms, double *contract_ms, int64_t *calls);

/*
 * Self-test of the device failure path (the paper has no counterpart): launches
 * a kernel that waits, with the same bounded wait as every pipeline wait of the
 * tensor-core kernels, on a barrier nothing ever arrives on.  The wait gives up
 * after limit_ns (1 .. 1e10), records RMS_ERR_TIMEOUT on the plan (reported and
 * cleared by the next rms_plan_sync) and the kernel returns; the context stays
 * usable.  outcome (host): 2 when the wait gave up as it must, 1 if it
 * completed.  Synchronous.
 */
rms_status rms_selftest_wait_timeout(rms_plan_t plan, int64_t limit_ns, int32_t *outcome);

/* ==========================================================================
 * RM-CLEAN (named after synthesis in Sec. 2.2 and Sec. 4; the paper gives no
 * algorithm: this is the Hogbom form used for RM synthesis)
 *
 * For each LOS, starting from res = F (a dirty spectrum from rms_synth), repeat
 * at most max_iter times:
 *     j = argmax_k |res_k| (lowest index on ties; NaN never chosen)
 *     stop when |res_j| < threshold (or no |res| is finite)
 *     c = gain res_j;  comp_j += c;  res_k -= c R(phi_k - phi_j) for every k
 * then restore  clean_k = res_k + sum_{|d| <= W} comp_{k-d} exp(-4 ln2 (d dphi)^2 / fwhm^2),
 * W = ceil(3 fwhm / dphi) (at most nphi - 1).  The plan's phi grid must be
 * uniform (step dphi), with 2 <= nphi <= 2048.  The iteration runs in FP64, every
 * product and sum rounded separately, so that with the same R table the device
 * makes the same choices as the FP64 definition.
 * ========================================================================== */
typedef struct rms_clean_s *rms_clean_t;

/*
 * fwhm: the restoring beam's FWHM in rad m^-2 (<= 0: the plan's measured RMSF
 * FWHM).  R2_host: NULL to build R at the 2 nphi - 1 offsets (m - nphi + 1)
 * dphi on the device in FP64 (Eq. Rsum), or a host array of those values
 * [2 nphi - 1][2] (re, im) to use instead.  RMS_ERR_INVALID_ARG for a
 * non-uniform or too long grid.  Synchronous.  The plan must outlive the object.
 */
rms_status rms_clean_create(rms_clean_t *clean, rms_plan_t plan, double fwhm, const double *R2_host);
rms_status rms_clean_destroy(rms_clean_t clean);

/*
 * F: device [nlos][nphi] complex64 dirty spectra (8-byte aligned).  gain in
 * (0, 1]; threshold >= 0 in |F| units; max_iter >= 0.  Outputs (device, any may
 * be NULL): F_clean, residual, components [nlos][nphi] complex64 (rounded from
 * FP64); niter [nlos] int32, the iterations performed.  Asynchronous on stream.
 */
rms_status rms_clean(rms_clean_t clean, const float *F, int64_t nlos, float gain, int32_t max_iter,
                     float threshold, float *F_clean, float *residual, float *components, int32_t *niter,
                     void *stream);

/* ==========================================================================
 * Synthetic sources on the device (Sec. 2.1 source models)
 * ========================================================================== */

/*
 * Source model of rms_generate.  Per line of sight: a component count uniform
 * in [ncomp_min, ncomp_max] (1 <= min <= max <= 3); per component phi0 ~
 * U(phi0_min, phi0_max), p0 ~ U(p0_min, p0_max), chi0 ~ U(0, pi); with
 * probability slab_prob the component is a Burn slab of width W ~ U(0, slab_w)
 * centred on phi0, else Faraday thin:
 *     P(lambda^2) = p0 exp(2i (chi0 + phi0 lambda^2)) [sin(W lambda^2) / (W lambda^2)]
 * (Eqs. PAdefn, Pdefn; the slab factor integrates Eq. Predefn over the slab).
 * Gaussian noise of standard deviation sigma is added to Q and to U; when
 * snr_min > 0, sigma is instead drawn per LOS so that max p0 / sigma_F ~
 * U(snr_min, snr_max), sigma_F = sigma sqrt(sum w^2) / sum w (the noise of F).
 * All draws are counter based on (seed, LOS index, draw number) -- see
 * csrc/generate.cu for the exact definition -- so one LOS can be regenerated
 * alone.
 */
typedef struct {
    uint64_t seed;
    int32_t ncomp_min, ncomp_max;
    double phi0_min, phi0_max;   /* rad m^-2 */
    double p0_min, p0_max;
    double slab_prob, slab_w;    /* slab_w in rad m^-2 */
    double sigma;                /* used when snr_min <= 0 */
    double snr_min, snr_max;
} rms_source_model;

/*
 * Write Q and U (device, nchan * nlos floats each, in `layout`) for lines of
 * sight los0 .. los0 + nlos - 1 of the source model, on the plan's channels
 * (lambda^2 and weights of the plan).  Asynchronous on `stream`.  Returns
 * RMS_ERR_INVALID_ARG for a NULL pointer, nlos < 0, los0 < 0 or a model outside
 * the ranges above.
 */
rms_status rms_generate(rms_plan_t plan, const rms_source_model *model, int64_t los0, int64_t nlos,
                        int32_t layout, float *Q, float *U, void *stream);

/* ==========================================================================
 * Learned peak proposal (not in the paper)
 *
 * A small network looks at one LOS's Q/U spectrum and proposes the bin of the
 * full phi grid that holds max |F|; exact synthesis (Eq. Fsum) then runs only
 * on a narrow window of a twice finer grid around the proposal, and the LOS
 * falls back to the full grid when the proposal is not confident or the
 * window's maximum lands on its edge.  Everything here runs on the plan's
 * device in the library's own kernels.
 *
 * Network: input x = [Q_a0, U_a0, Q_a1, U_a1, ...] / s over the plan's active
 * channels, s = RMS of |P| over them (1 for an all-zero spectrum);
 * h = relu(W1 x + b1) (W1: [hidden][2 nact]); logits z = W2 h + b2
 * (W2: [nbins][hidden], nbins = the plan's nphi).  BF16 weights and
 * activations, FP32 accumulation, FP32 master weights and AdamW moments.
 * Parameters are one flat FP32 array: W1 (row-major), b1, W2 (row-major), b2.
 * ========================================================================== */

typedef struct rms_net_s *rms_net_t;
typedef struct rms_window_s *rms_window_t;

/*
 * Create a network for `plan` (a tensor-core plan: RMS_BF16, RMS_BF16X3 or
 * RMS_FP16X3 -- else RMS_ERR_UNSUPPORTED -- with nphi <= 512).  hidden: 16 ..
 * 256, a multiple of 16.  max_batch: 1 .. 65536, the largest nlos of
 * rms_net_grad / rms_train_step (their scratch is allocated here).  Weights are
 * drawn from seed (uniform, fan-in scaled), biases 0.  The network refers to
 * the plan, which must outlive it.  Synchronous.
 */
rms_status rms_net_create(rms_net_t *net, rms_plan_t plan, int32_t hidden, int32_t max_batch, uint64_t seed);

/* Destroy a network (synchronises its device); NULL is accepted. */
rms_status rms_net_destroy(rms_net_t net);

enum { RMS_NET_NPARAMS = 0, RMS_NET_NIN = 1, RMS_NET_HIDDEN = 2, RMS_NET_NBINS = 3, RMS_NET_MAX_BATCH = 4,
       RMS_NET_STEPS = 5 };
rms_status rms_net_info(rms_net_t net, int32_t what, int64_t *value);

/*
 * Copy the flat FP32 parameters (RMS_NET_PARAMS) or the last gradients
 * (RMS_NET_GRADS) to `host` (set = 0), or load parameters from `host`
 * (set = 1, RMS_NET_PARAMS only; also resets the AdamW moments and step).
 * count must equal RMS_NET_NPARAMS.  Synchronous.
 */
enum { RMS_NET_PARAMS = 0, RMS_NET_GRADS = 1 };
rms_status rms_net_params(rms_net_t net, int32_t which, float *host, int64_t count, int32_t set);

/*
 * Run the network on a cube (arguments as rms_synth).  Outputs (device, any may
 * be NULL): logits [nlos][nbins] floats; bin [nlos] int32, argmax of the
 * logits (lowest on ties); conf [nlos] float, the softmax mass of the bins
 * within conf_halfwidth of bin (conf_halfwidth < 0: the largest probability).
 * Takes per-call scratch from the stream-ordered pool (2 bytes per (LOS,
 * contraction channel) plus 2 * hidden bytes per LOS).  Asynchronous.
 */
rms_status rms_propose(rms_net_t net, const float *Q, const float *U, int64_t nlos, int32_t layout,
                       int32_t conf_halfwidth, float *logits, int32_t *bin, float *conf, void *stream);

/*
 * Mean cross-entropy of the network on a batch with labels `label` (device
 * [nlos] int32 in 0 .. nbins - 1), and its gradient w.r.t. every parameter,
 * kept in the network (read with rms_net_params(RMS_NET_GRADS)).  1 <= nlos <=
 * max_batch.  loss: device float, or NULL.  Asynchronous.  Labels out of range
 * give undefined gradients (they are not checked on the device).
 */
rms_status rms_net_grad(rms_net_t net, const float *Q, const float *U, int64_t nlos, int32_t layout,
                        const int32_t *label, float *loss, void *stream);

/*
 * One training step: rms_net_grad, then AdamW on the FP32 master weights
 * (decoupled weight decay on W1 and W2 only, bias-corrected moments) and a
 * refresh of the BF16 weight copies.  Asynchronous.
 */
rms_status rms_train_step(rms_net_t net, const float *Q, const float *U, int64_t nlos, int32_t layout,
                          const int32_t *label, float lr, float beta1, float beta2, float eps, float weight_decay,
                          float *loss, void *stream);

/*
 * A window of `width` points (8 .. 128, a multiple of 8) on the fine grid
 * phi_0 + n D / 2 of a plan whose phi grid is uniform with step D (n = 0 ..
 * 2 (nphi - 1)).  The plan must be RMS_BF16 or RMS_BF16X3 (else
 * RMS_ERR_UNSUPPORTED) with a uniform grid (else RMS_ERR_INVALID_ARG).  Builds
 * the rotation table T[n][j] = exp(-2i phi_n (lambda_j^2 - lambda_0^2)) (argument
 * reduced in FP64) and the window's phase matrix for the offsets m D / 2,
 * m = -width/2 .. width/2 - 1, so that for every LOS
 *     F(phi_n + m D / 2) = K sum_j w_j (P_j T[n][j]) exp(-2i (m D / 2)(lambda_j^2 - lambda_0^2)),
 * an exact identity of Eq. Fsum.  Synchronous.  The plan must outlive it.
 */
rms_status rms_window_create(rms_window_t *win, rms_plan_t plan, int32_t width);
rms_status rms_window_destroy(rms_window_t win);

/*
 * The window centre rms_peakmap_learned uses for each proposal: fine point
 * 2 bin[l], clamped into width/2 .. 2 (nphi - 1) - width/2 + 1 so that the whole
 * window lies on the fine grid.  bin, centre: device [nlos] int32.
 * Asynchronous on stream; allocates nothing.  RMS_ERR_INVALID_ARG for a NULL
 * window or array, or nlos < 0.
 */
rms_status rms_window_centres(rms_window_t win, const int32_t *bin, int64_t nlos, int32_t *centre, void *stream);

/*
 * Exact synthesis on one window per LOS.  centre: device [nlos] int32, the
 * fine-grid index n of each window's centre, width/2 <= n <= 2 (nphi - 1) -
 * width/2 + 1 (checked on the device: an out-of-range centre is clamped).  The
 * window covers fine points n - width/2 .. n + width/2 - 1.  Outputs (device,
 * any may be NULL): F_out [nlos][width] complex64; widx [nlos] int32, index in
 * the window of max |F| (lowest on ties, -1 if none finite); wabs [nlos] float,
 * |F| there; wphi [nlos] float, phi there.  Other arguments as rms_synth.
 * Asynchronous; per-call scratch as rms_synth.
 */
rms_status rms_synth_window(rms_window_t win, const float *Q, const float *U, int64_t nlos, int32_t layout,
                            const int32_t *centre, float *F_out, int32_t *widx, float *wabs, float *wphi,
                            void *stream);

/*
 * The learned peak map: rms_propose (confidence = softmax mass within
 * width/4 - 2 bins of the proposal), a window centred on fine point 2 bin
 * (clamped into the grid), and a full-grid fallback for every LOS whose
 * confidence is below tau or NaN, whose window maximum is the window's first
 * or last point, or whose window holds no finite |F|.  Outputs (device, any
 * may be NULL): phi_peak, peak_abs [nlos] floats (as rms_synth; from the
 * window or the full grid); fallback [nlos] int32, 1 where the full grid was
 * used; nfallback: device int64, the number of fallbacks.  net and win must
 * belong to the same plan.  Asynchronous; per-call scratch from the stream-
 * ordered pool: two split operand images (as rms_synth's, the second for the
 * fallback rows), 2 x hidden bytes of activations and 44 bytes per LOS.
 */
rms_status rms_peakmap_learned(rms_window_t win, rms_net_t net, const float *Q, const float *U, int64_t nlos,
                               int32_t layout, float tau, float *phi_peak, float *peak_abs, int32_t *fallback,
                               int64_t *nfallback, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RMS_H */
