// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/rms.h"

// Device-side error codes written to the plan's error word.
enum { RMS_DEVERR_NONE = 0, RMS_DEVERR_TIMEOUT = 1 };

// Tensor-core tiling constants.
constexpr int kTileM = 128;        // LOS rows per tile (UMMA M)
constexpr int kChanPerKBlock = 16; // active channels per pipeline stage
constexpr int kKBlock = 32;        // K values (Q and U interleaved) per stage = 64 bytes of bf16
constexpr int kMaxTileN = 208;     // phase-matrix rows per tile: each of the two epilogue warps
                                   // sharing a row keeps tile_n / 2 FP32 sums in registers
constexpr int kMaxTileNPair = 256; // CTA pairs: the largest N of a 256-row MMA
constexpr int kGroupKBlocks = 16;  // K blocks accumulated in TMEM before the FP32 register fold (split precisions):
                                   // per-LOS error on the MWA cube 4.6e-6 (BF16x3) / 3.8e-6 (FP16x3) at 16,
                                   // 4.4e-6 / 1.8e-6 at 8, 6.1e-6 / 8.3e-6 at 32

struct rms_plan_s {
    int device = 0;
    int32_t nchan = 0, nact = 0, nphi = 0, precision = 0;
    double K = 0, lambda0sq = 0, wmax = 0, fwhm_meas = 0, fwhm_est = 0;
    std::vector<double> lambda2, weights, phi;
    std::vector<int32_t> active;

    // device arrays
    int32_t *d_active = nullptr;   // [nact] channel index of each active channel
    double *d_dl2 = nullptr;       // [nact] lambda_j^2 - lambda_0^2 (FP64)
    double *d_wact = nullptr;      // [nact] w_j
    double *d_phi = nullptr;       // [nphi]
    float *d_phi32 = nullptr;      // [nphi] phi rounded to FP32 (peak output)
    float *d_l2x32 = nullptr;      // [nact] 2 (lambda_j^2 - lambda_0^2) in FP32 (FP32 on-the-fly path)
    float *d_w32 = nullptr;        // [nact] w_j in FP32
    float2 *d_table = nullptr;     // [nact][nphi] w_j (cos, sin) FP32 (table path)
    uint16_t *d_bhi = nullptr;     // [npad][kpad] tensor-core phase matrix, high part
    uint16_t *d_blo = nullptr;     // [npad][kpad] low part
    double *d_R64 = nullptr;       // [nphi][2]
    float2 *d_czt = nullptr;       // chirp-z constants: H [M], twiddles [2 M], g [nchan], v [nphi]
    int32_t czt_M = 0;             // chirp-z FFT length
    int32_t kpad = 0, npad = 0, tile_n = 0, ntiles_n = 0, tile_n_last = 0, kblocks = 0;
    // the tiling of the two-CTA contraction: up to 256 phase rows per tile (npad covers both)
    int32_t tile_n2 = 0, ntiles_n2 = 0, tile_n_last2 = 0;
    CUtensorMap tmap_bhi;   // CUtensorMap is 64-byte aligned by its own declaration
    CUtensorMap tmap_blo;
    // LOS-major cubes contract over all channels (flagged ones zeroed in the
    // converter, zero rows in B), so their data tiles are contiguous boxes
    double *d_dl2_all = nullptr;   // [nchan]
    double *d_lambda2_all = nullptr;  // [nchan] lambda_j^2 (source generator)
    double *d_w_all = nullptr;     // [nchan]
    uint16_t *d_bhi_raw = nullptr, *d_blo_raw = nullptr;   // [npad][kpad_raw]; alias d_bhi/d_blo if no flags
    uint16_t *d_kbmask = nullptr;  // [kblocks_raw] bit i: channel 16 kb + i is active
    int32_t kpad_raw = 0, kblocks_raw = 0;
    CUtensorMap tmap_bhi_raw;
    CUtensorMap tmap_blo_raw;
    // the same matrices in boxes of tile_n / 2 rows: each CTA of a two-CTA
    // contraction loads its half of a tile
    CUtensorMap tmap2_bhi, tmap2_blo, tmap2_bhi_raw, tmap2_blo_raw;
    bool pair_maps = false;

    // sticky device error word, mapped host memory (readable without a sync)
    int *h_err = nullptr;
    int *d_err = nullptr;
    int64_t timeout_ns = 2000000000LL;
    int num_sms = 0;

    // rms_synth_host staging: slots of LOS chunks, copy streams and their events
    size_t stage_bytes = 0;
    void *d_stage = nullptr;
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t hev[9] = {};

    // tensor paths: per-CTA split-A scratch, [num_sms][max kblocks][128][128 B]
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    // calls on one plan are ordered on the device through this event (they share the scratch)
    cudaEvent_t last = nullptr;

    // FP16X3: per-LOS exponent scratch
    size_t rexp_cap = 0;
    int8_t *d_rexp = nullptr;

    // what the last tensor-core synthesis call ran (rms_plan_info): persistent CTAs of
    // the contraction, 1 if it ran as CTA pairs, N panels of the split schedule (0:
    // whole schedule), kernels launched by the call
    mutable int32_t last_ctas = 0, last_pair = 0, last_panels = 0, last_kernels = 0;
    // scheduling options (rms_plan_set_option): RMS_CONTRACT_*, L2 budget in bytes (0: default)
    int32_t contraction = 0, schedule = 0;
    int64_t l2_budget = 0;

    // optional kernel timing (rms_plan_set_kernel_timing): events around the layout
    // stage and the contraction of each tensor-core synthesis call
    bool timing = false;
    std::vector<cudaEvent_t> tev;   // triples: before split, after split, after contraction
};

// phase.cu
cudaError_t launch_phase_table(const rms_plan_s &p, cudaStream_t s);
cudaError_t launch_phase_bsplit(const rms_plan_s &p, const double *dl2, const double *w, int32_t nk,
                                int32_t kpad, uint16_t *bhi, uint16_t *blo, bool fp16, cudaStream_t s);
cudaError_t launch_rotation_table(const double *dl2, int32_t nk, int32_t ld, double phi0, double step,
                                  int32_t ncentre, float2 *T, cudaStream_t s);
cudaError_t launch_rmsf(const rms_plan_s &p, const double *d_phi, int32_t n, double *d_R64,
                        float *d_R32, cudaStream_t s);

// simt.cu
cudaError_t launch_simt(const rms_plan_s &p, bool fly, const float *Q, const float *U, int64_t nlos,
                        int layout, float *F, int32_t *pidx, float *pabs, float *pphi,
                        cudaStream_t s);
rms_status czt_plan_build(rms_plan_s *p);
cudaError_t launch_czt(const rms_plan_s &p, const float *Q, const float *U, int64_t nlos, int layout, float *F,
                       int32_t *pidx, float *pabs, float *pphi, float *pq, float *pu, float *pchi, cudaStream_t s);

// umma.cu
cudaError_t launch_umma(const rms_plan_s &p, const float *Q, const float *U, int64_t nlos,
                        int layout, float *F, int32_t *pidx, float *pabs, float *pphi,
                        const int8_t *rexp, cudaStream_t s);
cudaError_t launch_row_exponent(const rms_plan_s &p, const float *Q, const float *U, int64_t nlos,
                                int layout, int8_t *rexp, cudaStream_t s);
// loads umma.cu's kernels on the current device (cudaFuncGetAttributes) and checks the register split
cudaError_t umma_prepare();

// noalloc.cu: loads what rms_synth_noalloc needs on the current device (plan creation, FP16X3)
cudaError_t noalloc_prepare(int device);

// api.cu: argument checks shared by the synthesis entry points
rms_status check_synth_args(rms_plan_t p, const float *Q, const float *U, int64_t nlos, int32_t layout, float *F);

// gemm.cu: split kernel (layout stage) + contraction kernel
// Split operand image: [ceil(rows / 128)][kblocks][16 KB], K blocks of 16 channels
// (kblocks of the plan for channel-major cubes, kblocks_raw for LOS-major ones).
size_t split_operand_bytes(const rms_plan_s &p, int64_t nlos, int layout);
struct SplitOpts {
    const float *Q = nullptr, *U = nullptr;
    int64_t nlos_src = 0;              // lines of sight in the cube
    int layout = RMS_CHAN_MAJOR;
    int64_t nout = 0;                  // rows of the image (grid size)
    const int64_t *rows = nullptr;     // optional gather: image row r <- cube row rows[r]
    const int64_t *count = nullptr;    // optional device count of image rows to fill
    int mode = -1;                     // -1: the plan's precision; 0 BF16 (hi only)
    uint8_t *A = nullptr;
    int8_t *rexp = nullptr;            // FP16X3 per-row exponents
    float *rscale = nullptr;           // optional per-row 1 / RMS of |P| over the active channels
};
struct GemmOpts {
    const uint8_t *A = nullptr;
    int64_t nlos = 0;                  // image rows
    const int64_t *count = nullptr;    // optional device count (<= nlos) of live rows
    const int64_t *rows = nullptr;     // optional scatter of results: row r -> rows[r]
    int layout = RMS_CHAN_MAJOR;
    float *F = nullptr;
    int32_t *pidx = nullptr;
    float *pabs = nullptr, *pphi = nullptr;
    float *pq = nullptr, *pu = nullptr, *pchi = nullptr;   // F at the peak, chi0
    const int8_t *rexp = nullptr;
    // window plans: rotate row r by T[clamp(centre[r], cmin, cmax)][.] ([.][ldT] float2)
    const int32_t *centre = nullptr;
    const float2 *T = nullptr;
    int32_t ldT = 0, cmin = 0, cmax = 0;
    // optional scratch of nlos 64-bit peak keys: lets the contraction use its split
    // schedule (needed on cubes whose operands do not stay in L2; see gemm.cu)
    unsigned long long *keys = nullptr;
};
cudaError_t launch_split(const rms_plan_s &p, const SplitOpts &o, cudaStream_t s);
cudaError_t launch_gemm(const rms_plan_s &p, const GemmOpts &o, cudaStream_t s);
cudaError_t launch_image_gather(const rms_plan_s &p, int layout, const uint8_t *src, const int64_t *rows,
                                const int64_t *count, int64_t nmax, uint8_t *dst, cudaStream_t s);
cudaError_t launch_split_gemm(const rms_plan_s &p, const float *Q, const float *U, int64_t nlos, int layout,
                              float *F, int32_t *pidx, float *pabs, float *pphi, uint8_t *A, int8_t *rexp,
                              cudaStream_t s, cudaEvent_t ev_mid = nullptr, float *pq = nullptr,
                              float *pu = nullptr, float *pchi = nullptr, unsigned long long *keys = nullptr);

// generate.cu
cudaError_t launch_generate(const rms_plan_s &p, const rms_source_model &m, int64_t los0, int64_t nlos,
                            int32_t layout, float *Q, float *U, cudaStream_t s);

// net.cu: the learned proposal's network
struct rms_net_s {
    rms_plan_s *plan = nullptr;
    int device = 0;
    int32_t nin = 0, hidden = 0, nbins = 0, nbp = 0, max_batch = 0, ldb = 0;
    int64_t nparams = 0, oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, steps = 0;
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;   // flat FP32 (W1, b1, W2, b2)
    uint16_t *d_W1c = nullptr;   // [hidden][kpad]: W1 in the column order of channel-major operand images
    uint16_t *d_W1r = nullptr;   // [hidden][kpad_raw]: LOS-major images (zero columns for flagged channels)
    uint16_t *d_W2 = nullptr;    // [nbins][hidden]
    uint16_t *d_W2T = nullptr;   // [hidden][nbp]
    int32_t *d_colmap_c = nullptr, *d_colmap_r = nullptr;   // image column -> W1 column, -1 for none
    CUtensorMap tm_W1c, tm_W1r, tm_W2, tm_W2T;
    // training scratch for max_batch lines of sight
    uint8_t *d_img = nullptr;
    float *d_rs = nullptr, *d_dz32 = nullptr, *d_da32 = nullptr, *d_loss = nullptr;
    uint16_t *d_h = nullptr, *d_hT = nullptr, *d_dz = nullptr, *d_dzT = nullptr, *d_da1T = nullptr, *d_XT = nullptr;
    cudaEvent_t last = nullptr;
};
// Network forward from a split image (hi parts) and its per-row 1/RMS: bin and
// confidence (window mass within halfwin bins; < 0: largest probability), logits
// optional.  h: [nlos][hidden] BF16 scratch.
cudaError_t net_forward_image(const rms_net_s &n, const uint8_t *img, int layout, const float *rscale, int64_t nlos,
                              uint16_t *h, float *logits, int32_t *bin, float *conf, int32_t halfwin,
                              cudaStream_t s);

// api.cu: plan creation with a cap on phase rows per tensor-core tile (window
// plans use 128, the rotating kernel's limit)
rms_status plan_create_internal(rms_plan_t *out, const double *axis, int32_t nchan, int32_t axis_kind,
                                const double *weights, const double *phi, int32_t nphi, int32_t precision,
                                int32_t device, int32_t max_tile_cap);

// api.cu: cuTensorMapEncodeTiled through the runtime's driver entry point
bool encode_tensor_map(CUtensorMap *map, CUtensorMapDataType type, void *base, const cuuint64_t *dims,
                       const cuuint64_t *strides, const cuuint32_t *box, const cuuint32_t *estr,
                       CUtensorMapSwizzle swizzle, int rank = 2);
