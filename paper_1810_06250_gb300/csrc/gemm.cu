// Tensor-core RM synthesis in two kernels: a streaming split of the cube into
// 16-bit operands, then a tcgen05 contraction that only moves tiles.
//
// split_kernel (the layout stage): one CTA per 128-LOS M tile, one thread per
// LOS.  It reads FP32 Q/U in either cube layout once, zeroes flagged and padding
// channels (killing NaN there), and writes each K block of 16 channels as the
// exact shared-memory image the MMA reads: 128 rows x 64 bytes of hi parts, then
// of lo parts, 16-byte chunks swizzled in 64-byte rows (chunk c of row m at
// m * 64 + ((c ^ ((m >> 1) & 3)) << 4)).  For FP16X3 it first finds the row's
// largest |value| and stores the power-of-two exponent that brings it into
// [2^14, 2^15).
//
// gemm_kernel: C[l][2k + {0,1}] = sum over K of A[l][.] B[2k + {0,1}][.] with the
// phase matrix B of phase.cu (see umma.cu for the real form of Eq. Fsum).  A CTA
// is persistent over jobs: a job is one M tile (or M-tile pair) with all of its N
// tiles (whole schedule), or one (N panel, M tile, N tile) triple dealt
// round-robin (job schedule, see GemmParams).
//   warp 0      producer: the split A stage and TMA of the B hi/lo tiles  -> full
//   warp 1      TMEM allocator, single-thread MMA issuer          -> empty, tfull
//   warps 4-11  epilogue: warp w owns TMEM lane quarter w % 4 and column half
//               (w - 4) / 4; folds partials, scales, peak, stores F  -> tempty
// The PAIR variant runs on clusters of two CTAs (two SMs) with tcgen05's
// cta_group::2: every MMA is 256 rows (two M tiles, one per CTA) by tile_n, and
// each CTA's shared memory holds its own 128 A rows and half of the B tile
// (tile_n / 2 phase rows), so a stage carries half the phase-matrix bytes of the
// single-CTA kernel for the same MMA work.  Each CTA issues the TMA loads of its
// own stage, and the cta_group::2 form of the copies signals completion on the
// even CTA's full barrier, which alone expects both halves' bytes; the even CTA's
// warp 1 issues the MMAs.  Commits go to the barriers of both CTAs (multicast),
// and the epilogue warps of both CTAs release a TMEM partial on the even CTA's
// barrier.
// MMAs run in groups of up to 16 K blocks into one of two TMEM partials and the
// epilogue folds each partial into FP32 registers with round-to-nearest adds,
// because the tensor core's own FP32 accumulation does not round to nearest.
// Every wait is bounded: a wait that runs out aborts the CTA, records
// RMS_DEVERR_TIMEOUT, drains in-flight copies and MMAs and frees TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <limits.h>

#include <cstdlib>
#include <cstring>

#include "rms_internal.h"

namespace {

#include "tc_ptx.cuh"

constexpr int kThreads = 384;
constexpr int kEpiWarp0 = 4, kNumEpiWarps = 8;
constexpr int kRowBytes = kKBlock * 2;            // 64 B per operand row per stage
constexpr int kStageA = kTileM * kRowBytes;       // 8 KB per A part
constexpr int kTmemCols = 512;
constexpr int kAccStride = 256;
constexpr int kHalf = kMaxTileN / 2;              // 104 columns per epilogue thread
constexpr int kHalfWide = 128;                    // CTA pairs: tiles of up to 256 phase rows
constexpr int kRegsLaunch = 168, kRegsCtl = 56, kRegsEpi = 224;   // setmaxnreg split of the wide variant
static_assert(128 * kRegsCtl + 256 * kRegsEpi == kThreads * kRegsLaunch, "register split must fill the launch");
constexpr int kHalfRot = 64;                      // rotating (window) kernel: tile_n <= 128
constexpr int kEpiCols = 8;                       // staging chunk: 8 columns x 32 rows per warp
constexpr int kEpiLd = kEpiCols + 1;
constexpr int kEpiStageBytes = kNumEpiWarps * 32 * kEpiLd * 4;
constexpr int kSmemLimit = 227 * 1024;

enum { MODE_BF16 = 0, MODE_BF16X3 = 1, MODE_FP16X3 = 2 };

// ----------------------------------------------------------------------------
// split_kernel
// ----------------------------------------------------------------------------
struct SplitParams {
    const float *Q, *U;
    int64_t nlos_src;           // lines of sight in the cube (channel-major row stride)
    int64_t nout;               // output rows (the grid covers them)
    const int64_t *rows;        // optional: output row r reads cube row rows[r]
    const int64_t *count;       // optional device count: rows >= *count are left as padding
    int32_t nchan, layout, nk, kblocks, mode;
    int32_t kpg;                // K blocks per CTA: blockIdx.y covers K blocks [y kpg, (y + 1) kpg)
    int32_t vec4;               // LOS-major rows are 16-byte aligned: vector loads
    const int32_t *active;      // channel-major: active channel list
    const uint16_t *kbmask;     // LOS-major: per K block, bit i = channel 16 kb + i active
    uint8_t *A;                 // [nmt][kblocks][16 KB]
    int8_t *rexp;               // [nout] (FP16X3)
    float *rscale;              // optional [nout]: 1 / RMS of |P| over the nact_norm active channels
    int32_t nact_norm;
};

__device__ __forceinline__ void load_kblock(const SplitParams &P, int64_t src, bool valid, int kb, float (&q)[16],
                                            float (&u)[16])
{
    const int c0 = kb * kChanPerKBlock;
    if (P.layout == RMS_CHAN_MAJOR) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            q[i] = 0.f;
            u[i] = 0.f;
            if (c0 + i < P.nk && valid) {
                const int64_t off = (int64_t)__ldg(P.active + c0 + i) * P.nlos_src + src;
                q[i] = __ldg(P.Q + off);
                u[i] = __ldg(P.U + off);
            }
        }
    } else {
        const uint32_t live = __ldg(P.kbmask + kb);
        if (P.vec4 && valid && c0 + 16 <= P.nchan) {
            // 16 contiguous channels of this row: four 16-byte loads per array
            const float4 *q4 = reinterpret_cast<const float4 *>(P.Q + src * P.nchan + c0);
            const float4 *u4 = reinterpret_cast<const float4 *>(P.U + src * P.nchan + c0);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float4 a = __ldg(q4 + v), b = __ldg(u4 + v);
                q[4 * v] = a.x; q[4 * v + 1] = a.y; q[4 * v + 2] = a.z; q[4 * v + 3] = a.w;
                u[4 * v] = b.x; u[4 * v + 1] = b.y; u[4 * v + 2] = b.z; u[4 * v + 3] = b.w;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (!((live >> i) & 1u)) { q[i] = 0.f; u[i] = 0.f; }   // flagged: also kills NaN
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                q[i] = 0.f;
                u[i] = 0.f;
                if (((live >> i) & 1u) && valid) {
                    q[i] = __ldg(P.Q + src * P.nchan + c0 + i);
                    u[i] = __ldg(P.U + src * P.nchan + c0 + i);
                }
            }
        }
    }
}

// PAIRS: LOS-major rows with 16-byte aligned channels, two K blocks per load
// batch (a separate instantiation: its extra registers would cost the
// channel-major split occupancy).
template <bool PAIRS>
__global__ void __launch_bounds__(128) split_kernel(const SplitParams P)
{
    const int m = threadIdx.x;
    const int64_t mt = blockIdx.x;
    const int64_t row = mt * kTileM + m;
    const int64_t n_eff = P.count ? min(*P.count, P.nout) : P.nout;
    if (mt * kTileM >= n_eff) return;          // tiles past a device-side count stay untouched
    const bool valid = row < n_eff;
    const int64_t src = valid ? (P.rows ? P.rows[row] : row) : 0;
    const int sw = (m >> 1) & 3;
    // this CTA's K blocks (all of them whenever a whole-row pass is needed: FP16X3, rscale)
    const int kb0 = (int)blockIdx.y * P.kpg, kb1 = min(P.kblocks, kb0 + P.kpg);
    float scale = 1.0f;
    if (P.mode == MODE_FP16X3) {
        // the row's largest |value| sets its power-of-two scale: a first pass
        float mx = 0.f;
        for (int kb = 0; kb < P.kblocks; ++kb) {
            float q[16], u[16];
            load_kblock(P, src, valid, kb, q, u);
#pragma unroll
            for (int i = 0; i < 16; ++i) mx = fmaxf(mx, fmaxf(fabsf(q[i]), fabsf(u[i])));
        }
        int e = 0;
        if (mx > 0.f && isfinite(mx)) { frexpf(mx, &e); e = 15 - e; }
        e = max(-100, min(100, e));
        scale = ldexpf(1.0f, e);
        if (valid) P.rexp[row] = (int8_t)e;
    }
    float ss = 0.f;
    uint8_t *const dst0 = P.A + (size_t)mt * P.kblocks * (2 * kStageA);
    // write K block kb of this row: hi and lo chunks at their swizzled places
    auto emit = [&](int kb, const float *q, const float *u) {
        uint8_t *dst = dst0 + (size_t)kb * (2 * kStageA);
        if (P.rscale) {
#pragma unroll
            for (int i = 0; i < 16; ++i) ss = fmaf(q[i], q[i], fmaf(u[i], u[i], ss));
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = 4 * c + j;
                if (P.mode == MODE_FP16X3) split_pair_fp16(q[i] * scale, u[i] * scale, hi[j], lo[j]);
                else split_pair_bf16(q[i], u[i], hi[j], lo[j]);
            }
            const uint32_t off = (uint32_t)m * kRowBytes + ((uint32_t)(c ^ sw) << 4);
            *reinterpret_cast<uint4 *>(dst + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            if (P.mode != MODE_BF16)
                *reinterpret_cast<uint4 *>(dst + kStageA + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    };
    if (!PAIRS) {
        uint8_t *dst = dst0 + (size_t)kb0 * (2 * kStageA);
        for (int kb = kb0; kb < kb1; ++kb, dst += 2 * kStageA) {
            float q[16], u[16];
            load_kblock(P, src, valid, kb, q, u);
            if (P.rscale) {
#pragma unroll
                for (int i = 0; i < 16; ++i) ss = fmaf(q[i], q[i], fmaf(u[i], u[i], ss));
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int i = 4 * c + j;
                    if (P.mode == MODE_FP16X3) split_pair_fp16(q[i] * scale, u[i] * scale, hi[j], lo[j]);
                    else split_pair_bf16(q[i], u[i], hi[j], lo[j]);
                }
                const uint32_t off = (uint32_t)m * kRowBytes + ((uint32_t)(c ^ sw) << 4);
                *reinterpret_cast<uint4 *>(dst + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                if (P.mode != MODE_BF16)
                    *reinterpret_cast<uint4 *>(dst + kStageA + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
        }
    } else {
        for (int kb = kb0; kb < kb1;) {
            if (valid && kb + 1 < kb1 && (kb + 2) * kChanPerKBlock <= P.nchan) {
                // two K blocks at once: 128 contiguous bytes of the row per array, whole lines
                const int c0 = kb * kChanPerKBlock;
                const uint32_t live = __ldg(P.kbmask + kb) | ((uint32_t)__ldg(P.kbmask + kb + 1) << 16);
                const float4 *q4 = reinterpret_cast<const float4 *>(P.Q + src * P.nchan + c0);
                const float4 *u4 = reinterpret_cast<const float4 *>(P.U + src * P.nchan + c0);
                float q[32], u[32];
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const float4 a = __ldg(q4 + v), b = __ldg(u4 + v);
                    q[4 * v] = a.x; q[4 * v + 1] = a.y; q[4 * v + 2] = a.z; q[4 * v + 3] = a.w;
                    u[4 * v] = b.x; u[4 * v + 1] = b.y; u[4 * v + 2] = b.z; u[4 * v + 3] = b.w;
                }
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (!((live >> i) & 1u)) { q[i] = 0.f; u[i] = 0.f; }   // flagged: also kills NaN
                emit(kb, q, u);
                emit(kb + 1, q + 16, u + 16);
                kb += 2;
            } else {
                float q[16], u[16];
                load_kblock(P, src, valid, kb, q, u);
                emit(kb, q, u);
                kb += 1;
            }
        }
    }
    if (P.rscale && valid) {
        const float rms = sqrtf(ss / (float)P.nact_norm);
        P.rscale[row] = rms > 0.f ? 1.0f / rms : 1.0f;
    }
}

// Copy whole operand rows between split images: output row j <- image row
// rows[j], re-swizzled for its new position; rows at or past *count are not
// written.  One thread per (row, K block).
__global__ void __launch_bounds__(128) image_gather_kernel(const uint8_t *src, uint8_t *dst, int32_t kblocks,
                                                           const int64_t *rows, const int64_t *count,
                                                           int64_t nmax, int32_t parts)
{
    const int m = threadIdx.x;
    const int kb = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * kTileM + m;
    const int64_t n = min(*count, nmax);
    if ((int64_t)blockIdx.x * kTileM >= n) return;
    if (j >= n) return;
    const int64_t r = rows[j];
    const int ms = (int)(r % kTileM), swd = (m >> 1) & 3, sws = (ms >> 1) & 3;
    const uint8_t *sb = src + ((size_t)(r / kTileM) * kblocks + kb) * (2 * kStageA);
    uint8_t *db = dst + ((size_t)blockIdx.x * kblocks + kb) * (2 * kStageA);
    uint4 v[2][4];
#pragma unroll
    for (int part = 0; part < 2; ++part)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (part < parts)
                v[part][c] = *reinterpret_cast<const uint4 *>(sb + part * kStageA + ms * kRowBytes + ((c ^ sws) << 4));
#pragma unroll
    for (int part = 0; part < 2; ++part)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (part < parts)
                *reinterpret_cast<uint4 *>(db + part * kStageA + m * kRowBytes + ((c ^ swd) << 4)) = v[part][c];
}

// ----------------------------------------------------------------------------
// gemm_kernel
// ----------------------------------------------------------------------------
struct GemmParams {
    const uint8_t *A;           // split operand, [nmt][kblocks][16 KB]
    int64_t nlos;               // operand rows
    const int64_t *count;       // optional device count (<= nlos) of live rows
    const int64_t *rows;        // optional: results of row r go to output row rows[r]
    int32_t kblocks, group;
    int32_t nphi, ntiles_n, tile_n, tile_n_last;
    float *F;
    int32_t *pidx;
    float *pabs, *pphi;
    float *pq, *pu, *pchi;      // optional: Re, Im of F at the peak and the angle chi0 there
    const float *phi32;
    const double *phi64;
    double lambda0sq;
    float out_scale;
    int32_t mode;
    const int8_t *rexp;
    int *err;
    int64_t timeout_ns;
    int32_t stages;
    // schedule: jobs_split = 0: one job per M tile (or M-tile pair) covering every N
    // tile, peaks written directly; 1: one job per (N panel, M tile, N tile), ordered
    // panel by panel, M tile by M tile, and dealt round-robin to the persistent CTAs,
    // so that the CTAs working at any moment share a few M tiles' operands and one
    // panel of the phase matrix in L2; each job's per-row peak goes into keys[row]
    // with a 64-bit atomicMax and peak_finalize_kernel writes the peak outputs
    int32_t jobs_split, npanels;
    unsigned long long *keys;
    int32_t b_rows;             // phase rows of a B stage in this CTA's shared memory (tile_n, or tile_n / 2 in pairs)
    // window rotation (rotating kernel only): row r's operand is multiplied by
    // T[clamp(centre[r], cmin, cmax)][channel] before it enters the MMA
    const int32_t *centre;
    const float2 *T;
    int32_t ldT, cmin, cmax;
};

// One pipeline stage: the A part(s) then the B part(s) of b_rows phase rows each.
__host__ __device__ __forceinline__ uint32_t gemm_stage_bytes(int b_rows, int mode)
{
    const uint32_t parts = mode == MODE_BF16 ? 1u : 2u;
    return parts * kStageA + parts * (uint32_t)b_rows * kRowBytes;
}

struct GSmem {
    uint8_t *ring;
    uint32_t stage_bytes;
    float *epi, *pk_m, *pk_re, *pk_im;
    int *pk_i;
    uint64_t *full, *empty, *conv, *tfull, *tempty, *pkfull, *pkempty, *mma_done;   // conv: rotated stage (ROT)
    uint32_t *tmem_slot;
    volatile int *abort_flag;
};

__device__ __forceinline__ GSmem gcarve(uint8_t *base, const GemmParams &P)
{
    GSmem s;
    s.stage_bytes = gemm_stage_bytes(P.b_rows, P.mode);
    s.ring = base;
    s.epi = reinterpret_cast<float *>(s.ring + (size_t)P.stages * s.stage_bytes);
    s.pk_m = s.epi + kEpiStageBytes / 4;
    s.pk_i = reinterpret_cast<int *>(s.pk_m + 2 * 4 * 32);
    s.pk_re = reinterpret_cast<float *>(s.pk_i + 2 * 4 * 32);
    s.pk_im = s.pk_re + 2 * 4 * 32;
    uint64_t *b = reinterpret_cast<uint64_t *>(s.pk_im + 2 * 4 * 32);
    s.full = b;
    s.empty = s.full + P.stages;
    s.conv = s.empty + P.stages;
    s.tfull = s.conv + P.stages;
    s.tempty = s.tfull + 2;
    s.pkfull = s.tempty + 2;
    s.pkempty = s.pkfull + 8;
    s.mma_done = s.pkempty + 8;
    s.tmem_slot = reinterpret_cast<uint32_t *>(s.mma_done + 1);
    s.abort_flag = reinterpret_cast<volatile int *>(s.tmem_slot + 1);
    return s;
}

constexpr int kConvWarp0 = 12;   // rotating kernel: warps 12-15 rotate the A operand in place

// Job j of the schedule -> (work item it: an M tile, or an M-tile pair; N tiles [nt0, nt1)).
__device__ __forceinline__ void job_of(const GemmParams &P, int64_t nit, int64_t j, int64_t &it, int &nt0, int &nt1)
{
    if (!P.jobs_split) {
        it = j;
        nt0 = 0;
        nt1 = P.ntiles_n;
        return;
    }
    // panel p holds N tiles [p ntiles_n / npanels, (p + 1) ntiles_n / npanels) and the
    // jobs nit x (those tiles), M-major
    int lo = 0, hi = P.ntiles_n;
    for (int p = 0; p < P.npanels; ++p) {
        lo = (int)((int64_t)p * P.ntiles_n / P.npanels);
        hi = (int)((int64_t)(p + 1) * P.ntiles_n / P.npanels);
        if (j < nit * hi) break;
    }
    const int64_t r = j - nit * lo;
    const int len = hi - lo;
    it = r / len;
    nt0 = lo + (int)(r % len);
    nt1 = nt0 + 1;
}

// HALF: columns of the tile per epilogue thread (tile_n <= 2 HALF).  ROT: the
// window variant, 512 threads, whose converter warps rotate each stage's A
// rows in shared memory before the MMA reads them.  PAIR: the two-CTA variant
// (launched in clusters of two; not combined with ROT).
template <int HALF, bool ROT, bool PAIR>
__global__ void __launch_bounds__(ROT ? 512 : kThreads, 1)
gemm_kernel(const __grid_constant__ GemmParams P, const __grid_constant__ CUtensorMap tmB_hi,
            const __grid_constant__ CUtensorMap tmB_lo, const __grid_constant__ CUtensorMap tmA)
{
    static_assert(!(ROT && PAIR), "the rotating variant is single-CTA");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const GSmem S = gcarve(base, P);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nlos = P.count ? min(*P.count, P.nlos) : P.nlos;
    const int64_t nmt = (nlos + kTileM - 1) / kTileM;
    // work items: M tiles, or pairs of M tiles (even tile in the even CTA)
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const bool leader = rank == 0;
    const int64_t nit = PAIR ? (nmt + 1) / 2 : nmt;
    const int64_t it0 = PAIR ? (int64_t)(blockIdx.x >> 1) : (int64_t)blockIdx.x;
    const int64_t istride = PAIR ? (int64_t)(gridDim.x >> 1) : (int64_t)gridDim.x;
    const int64_t njobs = P.jobs_split ? nit * P.ntiles_n : nit;
    const bool split = P.mode != MODE_BF16;
    const int ngroups = (P.kblocks + P.group - 1) / P.group;
    const uint32_t a_bytes = split ? 2 * kStageA : kStageA;
    const uint32_t b_bytes = (uint32_t)P.b_rows * kRowBytes;
    // a wait that gives up in one CTA of a pair also stops the other one
    const uint32_t peer_abort = PAIR ? mapa_shared(smem_u32((const void *)S.abort_flag), rank ^ 1u) : 0u;
    auto stop_peer = [&]() {
        if constexpr (PAIR) st_cluster_u32(peer_abort, 1u);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.stages; ++s) {
            mbar_init(smem_u32(&S.full[s]), 1);
            mbar_init(smem_u32(&S.empty[s]), 1);
            mbar_init(smem_u32(&S.conv[s]), 4);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&S.tfull[b]), 1);
            mbar_init(smem_u32(&S.tempty[b]), PAIR ? 2 * kNumEpiWarps : kNumEpiWarps);
        }
        for (int i = 0; i < 8; ++i) {
            mbar_init(smem_u32(&S.pkfull[i]), 1);
            mbar_init(smem_u32(&S.pkempty[i]), 1);
        }
        mbar_init(smem_u32(S.mma_done), 1);
        *S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        __syncwarp();
        if constexpr (PAIR) tmem_alloc_pair(smem_u32(S.tmem_slot), kTmemCols);
        else tmem_alloc(smem_u32(S.tmem_slot), kTmemCols);
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync_all();   // the peer's barriers exist before anything targets them
    tc_fence_after();
    const uint32_t tmem_base = *S.tmem_slot;

    // Each epilogue thread keeps HALF FP32 sums plus four rows' peaks, so (except in
    // the window variant) warpgroup 0 (producer, MMA issuer) hands registers to the
    // two epilogue warpgroups at the top of their branches; the shares add up to the
    // launch's 384 x 168 registers (checked on the host before the first launch).
    if (warp < 4) {
    if constexpr (!ROT) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsCtl));
    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB_hi)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB_lo)) : "memory");
            if (PAIR) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            // bytes one CTA loads per stage; in a pair both CTAs' loads complete on the
            // even CTA's full barrier, which alone expects them (twice this)
            const uint32_t tx = a_bytes + (split ? 2 * b_bytes : b_bytes);
            int s = 0;
            uint32_t ph = 0, pending = 0, pend_par = 0;
            bool ok = true;
            for (int64_t j = it0; j < njobs && ok; j += istride) {
                int64_t it;
                int nt0, nt1;
                job_of(P, nit, j, it, nt0, nt1);
                const int64_t mt = PAIR ? 2 * it + rank : it;
                const uint8_t *a_mt = P.A + (size_t)mt * P.kblocks * (2 * kStageA);
                for (int nt = nt0; nt < nt1 && ok; ++nt) {
                    // phase rows of this CTA's part of the tile: all of it, or the pair's half
                    int32_t y = nt * P.tile_n;
                    if (PAIR && !leader) y += ((nt == P.ntiles_n - 1) ? P.tile_n_last : P.tile_n) / 2;
                    for (int kb = 0; kb < P.kblocks; ++kb) {
                        if (!wait_bounded(smem_u32(&S.empty[s]), ph ^ 1, S.abort_flag, P.err, P.timeout_ns)) {
                            ok = false;
                            break;
                        }
                        const uint32_t st = smem_u32(S.ring + (size_t)s * S.stage_bytes);
                        const uint32_t bar = smem_u32(&S.full[s]);
                        if constexpr (PAIR) {
                            const uint32_t bar0 = mapa_shared(bar, 0u);
                            if (leader) mbar_arrive_expect_tx(bar, 2 * tx);
                            tma_load_3d_pair(st, &tmA, 0, 0, (int32_t)(mt * P.kblocks + kb), bar0);
                            tma_load_2d_pair(st + a_bytes, &tmB_hi, kb * kKBlock, y, bar0);
                            if (split) tma_load_2d_pair(st + a_bytes + b_bytes, &tmB_lo, kb * kKBlock, y, bar0);
                        } else {
                            mbar_arrive_expect_tx(bar, tx);
                            bulk_load(st, a_mt + (size_t)kb * (2 * kStageA), a_bytes, bar);
                            tma_load_2d(st + a_bytes, &tmB_hi, kb * kKBlock, y, bar);
                            if (split) tma_load_2d(st + a_bytes + b_bytes, &tmB_lo, kb * kKBlock, y, bar);
                        }
                        pending |= 1u << s;
                        pend_par = (pend_par & ~(1u << s)) | (ph << s);
                        if (++s == P.stages) { s = 0; ph ^= 1; }
                    }
                }
            }
            if (!ok) {
                stop_peer();
                if (!PAIR || leader) {
                    for (int i = 0; i < P.stages; ++i)
                        if (pending & (1u << i))
                            wait_bounded(smem_u32(&S.full[i]), (pend_par >> i) & 1, S.abort_flag, P.err,
                                         P.timeout_ns, false);
                } else {
                    // the odd CTA's copies complete on the even CTA's barriers: give any still in
                    // flight far longer than a copy takes before this CTA may leave
                    const uint64_t t0 = global_ns();
                    while (global_ns() - t0 < 200000ull) __nanosleep(1000);
                }
            } else if (PAIR) {
                // the MMAs' commits arrive on this CTA's barriers from the tensor core: wait
                // for the one that releases each slot's last fill before the CTA may exit
                for (int i = 0; i < P.stages; ++i)
                    if ((pending & (1u << i)) &&
                        !wait_bounded(smem_u32(&S.empty[i]), (pend_par >> i) & 1, S.abort_flag, P.err,
                                      P.timeout_ns)) {
                        stop_peer();
                        break;
                    }
            }
        }
    } else if (warp == 1) {
        if (PAIR && !leader) {
            // the even CTA's last commit: all MMAs that touch this CTA are complete
            if (lane == 0 && !wait_bounded(smem_u32(S.mma_done), 0, S.abort_flag, P.err, P.timeout_ns)) stop_peer();
        } else if (lane == 0) {
            // -------------------------------------------------------- MMA issuer
            const bool bf = P.mode != MODE_FP16X3;
            const int mrows = PAIR ? 2 * kTileM : kTileM;
            const uint32_t id_full = idesc_f16_m(mrows, P.tile_n, bf), id_last = idesc_f16_m(mrows, P.tile_n_last, bf);
            int s = 0;
            uint32_t ph = 0, tph = 0;
            int g_all = 0;
            bool ok = true, issued = false;
            for (int64_t j = it0; j < njobs && ok; j += istride) {
                int64_t it;
                int nt0, nt1;
                job_of(P, nit, j, it, nt0, nt1);
                for (int nt = nt0; nt < nt1 && ok; ++nt) {
                    const uint32_t idesc = (nt == P.ntiles_n - 1) ? id_last : id_full;
                    for (int g = 0; g < ngroups && ok; ++g, ++g_all) {
                        const int b = g_all & 1;
                        const bool got = PAIR ? wait_bounded_cluster(smem_u32(&S.tempty[b]), ((tph >> b) & 1) ^ 1,
                                                                     S.abort_flag, P.err, P.timeout_ns)
                                              : wait_bounded(smem_u32(&S.tempty[b]), ((tph >> b) & 1) ^ 1,
                                                             S.abort_flag, P.err, P.timeout_ns);
                        if (!got) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem_base + (uint32_t)(b * kAccStride);
                        const int kb0 = g * P.group, kb1 = min(P.kblocks, kb0 + P.group);
                        for (int kb = kb0; kb < kb1; ++kb) {
                            const uint64_t *ready = ROT ? &S.conv[s] : &S.full[s];
                            const bool in = PAIR ? wait_bounded_cluster(smem_u32(ready), ph, S.abort_flag, P.err,
                                                                        P.timeout_ns)
                                                 : wait_bounded(smem_u32(ready), ph, S.abort_flag, P.err, P.timeout_ns);
                            if (!in) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t st = smem_u32(S.ring + (size_t)s * S.stage_bytes);
                            const uint32_t a_hi = st, a_lo = st + kStageA;
                            const uint32_t b_hi = st + a_bytes, b_lo = b_hi + b_bytes;
#pragma unroll
                            for (int kk = 0; kk < kKBlock / 16; ++kk) {
                                const uint32_t ko = kk * 32;
                                const uint32_t acc = (kb > kb0 || kk > 0) ? 1u : 0u;
                                if constexpr (PAIR) {
                                    mma_f16_pair(d, sdesc_k64(a_hi + ko), sdesc_k64(b_hi + ko), idesc, acc);
                                    if (split) {
                                        mma_f16_pair(d, sdesc_k64(a_hi + ko), sdesc_k64(b_lo + ko), idesc, 1u);
                                        mma_f16_pair(d, sdesc_k64(a_lo + ko), sdesc_k64(b_hi + ko), idesc, 1u);
                                    }
                                } else {
                                    mma_f16(d, sdesc_k64(a_hi + ko), sdesc_k64(b_hi + ko), idesc, acc);
                                    if (split) {
                                        mma_f16(d, sdesc_k64(a_hi + ko), sdesc_k64(b_lo + ko), idesc, 1u);
                                        mma_f16(d, sdesc_k64(a_lo + ko), sdesc_k64(b_hi + ko), idesc, 1u);
                                    }
                                }
                            }
                            issued = true;
                            if constexpr (PAIR) mma_commit_pair_mc(smem_u32(&S.empty[s]), (uint16_t)3);
                            else mma_commit(smem_u32(&S.empty[s]));
                            if (++s == P.stages) { s = 0; ph ^= 1; }
                        }
                        if (!ok) break;
                        if constexpr (PAIR) mma_commit_pair_mc(smem_u32(&S.tfull[b]), (uint16_t)3);
                        else mma_commit(smem_u32(&S.tfull[b]));
                        tph ^= 1u << b;
                    }
                }
            }
            if (!ok) stop_peer();
            if constexpr (PAIR) {
                // both CTAs wait for this commit before they leave (the odd CTA in its warp 1)
                mma_commit_pair_mc(smem_u32(S.mma_done), (uint16_t)3);
                wait_bounded(smem_u32(S.mma_done), 0, S.abort_flag, P.err, P.timeout_ns, false);
            } else if (issued) {
                mma_commit(smem_u32(S.mma_done));
                wait_bounded(smem_u32(S.mma_done), 0, S.abort_flag, P.err, P.timeout_ns, false);
            }
        }
    }
    } else if (ROT && warp >= kConvWarp0) {
        // ------------------------------------------------------------ rotation
        // Thread r owns operand row r: P' = (hi + lo) T[centre][channel] in FP32,
        // split again and written back in place, before the MMA may read it.
        const int r = threadIdx.x - 32 * kConvWarp0;
        const int sw = (r >> 1) & 3;
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int64_t mt = blockIdx.x; mt < nmt && ok; mt += gridDim.x) {
            const int64_t row = mt * kTileM + r;
            const bool live = row < nlos;
            int c = P.cmin;
            if (live) c = max(P.cmin, min(P.cmax, P.centre[row]));
            const float4 *trow = reinterpret_cast<const float4 *>(P.T + (size_t)c * P.ldT);
            // T for the next K block is loaded while this one is rotated (L2 latency hidden)
            float4 t[8], tn[8];
#pragma unroll
            for (int v = 0; v < 8; ++v) t[v] = live ? __ldg(trow + v) : make_float4(1.f, 0.f, 1.f, 0.f);
            for (int nt = 0; nt < P.ntiles_n && ok; ++nt)
                for (int kb = 0; kb < P.kblocks; ++kb) {
                    const int kbn = kb + 1 < P.kblocks ? kb + 1 : 0;
#pragma unroll
                    for (int v = 0; v < 8; ++v) tn[v] = live ? __ldg(trow + kbn * 8 + v) : make_float4(1.f, 0.f, 1.f, 0.f);
                    if (!warp_wait(smem_u32(&S.full[s]), ph, S.abort_flag, P.err, P.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    if (live) {
                        uint8_t *st = S.ring + (size_t)s * S.stage_bytes;
#pragma unroll
                        for (int ch = 0; ch < 4; ++ch) {
                            const uint32_t off = (uint32_t)r * kRowBytes + ((uint32_t)(ch ^ sw) << 4);
                            uint4 hv = *reinterpret_cast<const uint4 *>(st + off);
                            uint4 lv = split ? *reinterpret_cast<const uint4 *>(st + kStageA + off) : make_uint4(0, 0, 0, 0);
                            uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
                            uint32_t nh[4], nl[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float q = __uint_as_float(hw[j] << 16) + __uint_as_float(lw[j] << 16);
                                const float u = __uint_as_float(hw[j] & 0xffff0000u) + __uint_as_float(lw[j] & 0xffff0000u);
                                const int ci = 4 * ch + j;
                                const float4 tv = t[ci >> 1];
                                const float tr = (ci & 1) ? tv.z : tv.x, ti = (ci & 1) ? tv.w : tv.y;
                                const float qr = fmaf(q, tr, -u * ti), ur = fmaf(q, ti, u * tr);
                                split_pair_bf16(qr, ur, nh[j], nl[j]);
                            }
                            *reinterpret_cast<uint4 *>(st + off) = make_uint4(nh[0], nh[1], nh[2], nh[3]);
                            if (split) *reinterpret_cast<uint4 *>(st + kStageA + off) = make_uint4(nl[0], nl[1], nl[2], nl[3]);
                        }
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&S.conv[s]));
                    if (++s == P.stages) { s = 0; ph ^= 1; }
#pragma unroll
                    for (int v = 0; v < 8; ++v) t[v] = tn[v];
                }
        }
    } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + kNumEpiWarps) {
        if constexpr (!ROT) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsEpi));
        if constexpr (!ROT) {
            // ------------------------------------------------------------ epilogue
            // 16x256b TMEM loads: in each 16-lane block l of the quarter, thread t holds
            // rows 16 l + t/4 and 16 l + t/4 + 8, complex column 4 g + t % 4 of every
            // 8-column group g of its half; F leaves straight from registers (four lanes
            // write 32 contiguous bytes of a row), and each lane ends up owning one row's
            // peak after a butterfly over the four lanes of its row group.
            constexpr int NG = HALF / 8;
            constexpr int LB = HALF > kHalf ? 2 : 4;   // 8-column loads per TMEM wait
            const int q = warp & 3;
            const int h = (warp - kEpiWarp0) >> 2;
            const int rq = lane >> 2, cq = lane & 3;
            const int64_t row_pitch = 2 * (int64_t)P.nphi;
            uint32_t tph = 0;
            int g_all = 0, mt_count = 0;
            bool ok = true;
            float master[2][NG][4];
            uint32_t tempty_addr[2];
            for (int b = 0; b < 2; ++b)
                tempty_addr[b] = PAIR ? mapa_shared(smem_u32(&S.tempty[b]), 0u) : smem_u32(&S.tempty[b]);
            for (int64_t j = it0; j < njobs && ok; j += istride, ++mt_count) {
                int64_t it;
                int nt0, nt1;
                job_of(P, nit, j, it, nt0, nt1);
                const int64_t mt = PAIR ? 2 * it + rank : it;
                // the thread's rows i = 2 l + s: row0 + 16 l + 8 s
                const int64_t row0 = mt * kTileM + 32 * q + rq;
                float scale[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int64_t r = row0 + 16 * (i >> 1) + 8 * (i & 1);
                    scale[i] = P.out_scale;
                    if (P.rexp != nullptr && r < nlos) scale[i] = ldexpf(scale[i], -(int)P.rexp[r]);
                }
                float bm[4], br[4], bim[4];
                int bi[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) { bm[i] = -1.0f; br[i] = 0.f; bim[i] = 0.f; bi[i] = INT_MAX; }
                for (int nt = nt0; nt < nt1 && ok; ++nt) {
                    for (int g = 0; g < ngroups; ++g, ++g_all) {
                        const int b = g_all & 1;
                        if (!warp_wait(smem_u32(&S.tfull[b]), (tph >> b) & 1, S.abort_flag, P.err, P.timeout_ns)) {
                            ok = false;
                            break;
                        }
                        tph ^= 1u << b;
                        tc_fence_after();
                        const uint32_t taddr =
                            tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kAccStride + h * HALF);
#pragma unroll
                        for (int l = 0; l < 2; ++l)
#pragma unroll
                            for (int g0 = 0; g0 < NG; g0 += LB) {
                                uint32_t r[LB][4];
#pragma unroll
                                for (int jj = 0; jj < LB; ++jj)
                                    if (g0 + jj < NG) tmem_ld16x256(taddr + ((uint32_t)(16 * l) << 16) + 8 * (g0 + jj), r[jj]);
                                tmem_wait_ld();
#pragma unroll
                                for (int jj = 0; jj < LB; ++jj)
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        if (g0 + jj < NG) {
                                            const float v = __uint_as_float(r[jj][e]);
                                            master[l][g0 + jj][e] = g == 0 ? v : __fadd_rn(master[l][g0 + jj][e], v);
                                        }
                            }
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) {
                            if constexpr (PAIR) mbar_arrive_cluster(tempty_addr[b]);
                            else mbar_arrive(tempty_addr[b]);
                        }
                    }
                    if (!ok) break;
                    const int ncols = ((nt == P.ntiles_n - 1) ? P.tile_n_last : P.tile_n) - h * HALF;
                    const int kbase = (nt * P.tile_n + h * HALF) >> 1;
#pragma unroll
                    for (int l = 0; l < 2; ++l)
#pragma unroll
                        for (int gg = 0; gg < NG; ++gg) {
                            const int k = kbase + 4 * gg + cq;
                            const bool colok = 2 * (4 * gg + cq) < ncols && k < P.nphi;
#pragma unroll
                            for (int sh = 0; sh < 2; ++sh) {
                                const int i = 2 * l + sh;
                                const float fr = master[l][gg][2 * sh] * scale[i];
                                const float fi = master[l][gg][2 * sh + 1] * scale[i];
                                if (colok) {
                                    const float m2 = __fadd_rn(__fmul_rn(fr, fr), __fmul_rn(fi, fi));
                                    if (m2 > bm[i]) { bm[i] = m2; bi[i] = k; br[i] = fr; bim[i] = fi; }
                                    const int64_t r = row0 + 16 * l + 8 * sh;
                                    if (P.F != nullptr && r < nlos) {
                                        const int64_t orow = P.rows ? P.rows[r] : r;
                                        // streaming store: F is written once and must not push the
                                        // operands out of L2
                                        __stcs(reinterpret_cast<float2 *>(P.F + orow * row_pitch + 2 * (int64_t)k),
                                               make_float2(fr, fi));
                                    }
                                }
                            }
                        }
                }
                if (!ok) break;
                // the four lanes of a row group hold disjoint columns of the same four rows:
                // a butterfly leaves every lane with all four rows' peaks (lowest index on ties)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int off = 1; off <= 2; off <<= 1) {
                        const float om = __shfl_xor_sync(0xffffffffu, bm[i], off);
                        const int oi = __shfl_xor_sync(0xffffffffu, bi[i], off);
                        const float ore = __shfl_xor_sync(0xffffffffu, br[i], off);
                        const float oim = __shfl_xor_sync(0xffffffffu, bim[i], off);
                        if (om > bm[i] || (om == bm[i] && oi < bi[i])) { bm[i] = om; bi[i] = oi; br[i] = ore; bim[i] = oim; }
                    }
                // lane (rq, cq) now owns row i = cq of its group
                float pm = bm[0], pre = br[0], pim = bim[0];
                int pi = bi[0];
#pragma unroll
                for (int i = 1; i < 4; ++i)
                    if (cq == i) { pm = bm[i]; pi = bi[i]; pre = br[i]; pim = bim[i]; }
                const int rowq = 16 * (cq >> 1) + rq + 8 * (cq & 1);
                const int64_t prow = mt * kTileM + 32 * q + rowq;
                // combine the two column halves of each row: half 1 publishes, half 0 writes
                const int par = mt_count & 1;
                const uint32_t pbar = smem_u32(&S.pkfull[par * 4 + q]);
                const uint32_t ebar = smem_u32(&S.pkempty[par * 4 + q]);
                const uint32_t use_par = (mt_count >> 1) & 1;
                if (h == 1) {
                    if (!warp_wait(ebar, use_par ^ 1, S.abort_flag, P.err, P.timeout_ns)) { ok = false; break; }
                    S.pk_m[(par * 4 + q) * 32 + rowq] = pm;
                    S.pk_i[(par * 4 + q) * 32 + rowq] = pi;
                    S.pk_re[(par * 4 + q) * 32 + rowq] = pre;
                    S.pk_im[(par * 4 + q) * 32 + rowq] = pim;
                    __syncwarp();
                    if (lane == 0) mbar_arrive(pbar);
                } else {
                    if (!warp_wait(pbar, use_par, S.abort_flag, P.err, P.timeout_ns)) { ok = false; break; }
                    const float om = S.pk_m[(par * 4 + q) * 32 + rowq];
                    const int oi = S.pk_i[(par * 4 + q) * 32 + rowq];
                    const float ore = S.pk_re[(par * 4 + q) * 32 + rowq], oim = S.pk_im[(par * 4 + q) * 32 + rowq];
                    __syncwarp();
                    if (lane == 0) mbar_arrive(ebar);
                    if (om > pm || (om == pm && oi < pi)) { pm = om; pi = oi; pre = ore; pim = oim; }
                    if (P.jobs_split) {
                        // this job's peak of the row: |F|^2 bits (monotonic for values >= 0) above
                        // the complement of the index, so the largest key is the largest |F|^2
                        // with the lowest index among equal ones; NaN never gets here
                        if (prow < nlos && pi != INT_MAX)
                            atomicMax(P.keys + prow, ((unsigned long long)__float_as_uint(pm) << 32) |
                                                         (unsigned long long)(0xFFFFFFFFu - (uint32_t)pi));
                    } else if (prow < nlos) {
                        const int64_t porow = P.rows ? P.rows[prow] : prow;
                        const bool found = pi != INT_MAX;
                        if (P.pidx) P.pidx[porow] = found ? pi : -1;
                        if (P.pabs) P.pabs[porow] = found ? sqrtf(pm) : __int_as_float(0x7fc00000);
                        if (P.pphi) P.pphi[porow] = found ? P.phi32[pi] : __int_as_float(0x7fc00000);
                        if (P.pq) P.pq[porow] = found ? pre : __int_as_float(0x7fc00000);
                        if (P.pu) P.pu[porow] = found ? pim : __int_as_float(0x7fc00000);
                        if (P.pchi) {
                            // chi0 = arg F(phi_peak) / 2 - phi_peak lambda_0^2, reduced to [0, pi)
                            float c = __int_as_float(0x7fc00000);
                            if (found) {
                                double x = 0.5 * atan2((double)pim, (double)pre) - P.phi64[pi] * P.lambda0sq;
                                x -= M_PI * floor(x / M_PI);
                                c = (float)x;
                            }
                            P.pchi[porow] = c;
                        }
                    }
                }
            }
        } else {
            // ------------------------------------------------------------ epilogue
            const int q = warp & 3;
            const int h = (warp - kEpiWarp0) >> 2;
            float *stg = S.epi + (warp - kEpiWarp0) * 32 * kEpiLd;
            const int64_t row_pitch = 2 * (int64_t)P.nphi;
            uint32_t tph = 0;
            int g_all = 0, mt_count = 0;
            bool ok = true;
            float master[HALF];
            // the even CTA's barrier that releases a TMEM partial (this CTA's own without pairs)
            uint32_t tempty_addr[2];
            for (int b = 0; b < 2; ++b)
                tempty_addr[b] = PAIR ? mapa_shared(smem_u32(&S.tempty[b]), 0u) : smem_u32(&S.tempty[b]);
            for (int64_t j = it0; j < njobs && ok; j += istride, ++mt_count) {
                int64_t it;
                int nt0, nt1;
                job_of(P, nit, j, it, nt0, nt1);
                const int64_t mt = PAIR ? 2 * it + rank : it;
                const int64_t row = mt * kTileM + 32 * q + lane;
                float scale = P.out_scale;
                if (P.rexp != nullptr && row < nlos) scale = ldexpf(scale, -(int)P.rexp[row]);
                float bm = -1.0f, br = 0.f, bim = 0.f;
                int bi = INT_MAX;
                for (int nt = nt0; nt < nt1 && ok; ++nt) {
                    for (int g = 0; g < ngroups; ++g, ++g_all) {
                        const int b = g_all & 1;
                        if (!warp_wait(smem_u32(&S.tfull[b]), (tph >> b) & 1, S.abort_flag, P.err, P.timeout_ns)) {
                            ok = false;
                            break;
                        }
                        tph ^= 1u << b;
                        tc_fence_after();
                        const uint32_t taddr =
                            tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kAccStride + h * HALF);
    #pragma unroll
                        for (int c0 = 0; c0 < HALF; c0 += 32) {
                            uint32_t r[4][8];
    #pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (c0 + 8 * j < HALF) tmem_ld8(taddr + c0 + 8 * j, r[j]);
                            tmem_wait_ld();
    #pragma unroll
                            for (int j = 0; j < 4; ++j)
    #pragma unroll
                                for (int e = 0; e < 8; ++e)
                                    if (c0 + 8 * j < HALF) {
                                        const float v = __uint_as_float(r[j][e]);
                                        master[c0 + 8 * j + e] = g == 0 ? v : __fadd_rn(master[c0 + 8 * j + e], v);
                                    }
                        }
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) {
                            if constexpr (PAIR) mbar_arrive_cluster(tempty_addr[b]);
                            else mbar_arrive(tempty_addr[b]);
                        }
                    }
                    if (!ok) break;
                    const int ncols = ((nt == P.ntiles_n - 1) ? P.tile_n_last : P.tile_n) - h * HALF;
                    const int kbase = (nt * P.tile_n + h * HALF) >> 1;
    #pragma unroll
                    for (int p = 0; p < HALF / 2; ++p) {
                        const float fr = master[2 * p] * scale, fi = master[2 * p + 1] * scale;
                        master[2 * p] = fr;
                        master[2 * p + 1] = fi;
                        const int k = kbase + p;
                        if (2 * p < ncols && k < P.nphi) {
                            const float m2 = __fadd_rn(__fmul_rn(fr, fr), __fmul_rn(fi, fi));
                            if (m2 > bm) {
                                bm = m2;
                                bi = k;
                                if constexpr (!ROT) {   // F at the peak (the window kernel has no use for it)
                                    br = fr;
                                    bim = fi;
                                }
                            }
                        }
                    }
                    if (P.F != nullptr) {
    #pragma unroll
                        for (int c0 = 0; c0 < HALF; c0 += kEpiCols) {
    #pragma unroll
                            for (int j = 0; j < kEpiCols; ++j)
                                if (c0 + j < HALF) stg[lane * kEpiLd + j] = master[c0 + j];
                            __syncwarp();
                            // 4 lanes per row (one complex each), 8 rows per store instruction
                            const int jj = (lane & 3) * 2;
                            const int kk = kbase + (c0 >> 1) + (lane & 3);
                            const bool colok = c0 + jj < min(ncols, HALF) && kk < P.nphi;
    #pragma unroll
                            for (int it = 0; it < 4; ++it) {
                                const int r = 8 * it + (lane >> 2);
                                const int64_t grow = mt * kTileM + 32 * q + r;
                                if (colok && grow < nlos) {
                                    const int64_t orow = P.rows ? P.rows[grow] : grow;
                                    const float2 val = make_float2(stg[r * kEpiLd + jj], stg[r * kEpiLd + jj + 1]);
                                    // streaming store: F is written once and must not push the
                                    // operands out of L2
                                    __stcs(reinterpret_cast<float2 *>(P.F + orow * row_pitch + 2 * (int64_t)kk), val);
                                }
                            }
                            __syncwarp();
                        }
                    }
                }
                if (!ok) break;
                // combine the two column halves of each row: half 1 publishes, half 0 writes
                const int par = mt_count & 1;
                const uint32_t pbar = smem_u32(&S.pkfull[par * 4 + q]);
                const uint32_t ebar = smem_u32(&S.pkempty[par * 4 + q]);
                const uint32_t use_par = (mt_count >> 1) & 1;
                if (h == 1) {
                    if (!warp_wait(ebar, use_par ^ 1, S.abort_flag, P.err, P.timeout_ns)) { ok = false; break; }
                    S.pk_m[(par * 4 + q) * 32 + lane] = bm;
                    S.pk_i[(par * 4 + q) * 32 + lane] = bi;
                    S.pk_re[(par * 4 + q) * 32 + lane] = br;
                    S.pk_im[(par * 4 + q) * 32 + lane] = bim;
                    __syncwarp();
                    if (lane == 0) mbar_arrive(pbar);
                } else {
                    if (!warp_wait(pbar, use_par, S.abort_flag, P.err, P.timeout_ns)) { ok = false; break; }
                    const float om = S.pk_m[(par * 4 + q) * 32 + lane];
                    const int oi = S.pk_i[(par * 4 + q) * 32 + lane];
                    const float ore = S.pk_re[(par * 4 + q) * 32 + lane], oim = S.pk_im[(par * 4 + q) * 32 + lane];
                    __syncwarp();
                    if (lane == 0) mbar_arrive(ebar);
                    if (om > bm || (om == bm && oi < bi)) { bm = om; bi = oi; br = ore; bim = oim; }
                    if (P.jobs_split) {
                        // this job's peak of the row: |F|^2 bits (monotonic for values >= 0) above
                        // the complement of the index, so the largest key is the largest |F|^2
                        // with the lowest index among equal ones; NaN never gets here
                        if (row < nlos && bi != INT_MAX)
                            atomicMax(P.keys + row, ((unsigned long long)__float_as_uint(bm) << 32) |
                                                        (unsigned long long)(0xFFFFFFFFu - (uint32_t)bi));
                    } else if (row < nlos) {
                        const int64_t orow = P.rows ? P.rows[row] : row;
                        const bool found = bi != INT_MAX;
                        if (P.pidx) P.pidx[orow] = found ? bi : -1;
                        if (P.pabs) P.pabs[orow] = found ? sqrtf(bm) : __int_as_float(0x7fc00000);
                        if (P.pphi) P.pphi[orow] = found ? P.phi32[bi] : __int_as_float(0x7fc00000);
                        if (P.pq) P.pq[orow] = found ? br : __int_as_float(0x7fc00000);
                        if (P.pu) P.pu[orow] = found ? bim : __int_as_float(0x7fc00000);
                        if (P.pchi) {
                            // chi0 = arg F(phi_peak) / 2 - phi_peak lambda_0^2, reduced to [0, pi)
                            float c = __int_as_float(0x7fc00000);
                            if (found) {
                                double x = 0.5 * atan2((double)bim, (double)br) - P.phi64[bi] * P.lambda0sq;
                                x -= M_PI * floor(x / M_PI);
                                c = (float)x;
                            }
                            P.pchi[orow] = c;
                        }
                    }
                }
            }

        }
    }

    if constexpr (PAIR) {
        if (*S.abort_flag) stop_peer();
    }
    tc_fence_before();
    __syncthreads();
    // in a pair, neither CTA leaves (or frees TMEM) while the other may still use its
    // shared memory, barriers or TMEM
    if constexpr (PAIR) cluster_sync_all();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        if constexpr (PAIR) tmem_dealloc_pair(tmem_base, kTmemCols);
        else tmem_dealloc(tmem_base, kTmemCols);
    }
}

// Peak outputs from the merged keys of the split schedule (one thread per image
// row): the same values the contraction's epilogue writes in the whole schedule --
// index, sqrt of the FP32 |F|^2, phi, and Re F, Im F and chi0 read back from the
// stored F at the peak.
__global__ void peak_finalize_kernel(const unsigned long long *__restrict__ keys, int64_t n, const int64_t *count,
                                     const int64_t *rows, const float *F, int32_t nphi, const float *phi32,
                                     const double *phi64, double lambda0sq, int32_t *pidx, float *pabs, float *pphi,
                                     float *pq, float *pu, float *pchi)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n_eff = count ? min(*count, n) : n;
    if (r >= n_eff) return;
    const unsigned long long key = keys[r];
    const int64_t orow = rows ? rows[r] : r;
    const bool found = key != 0ull;
    const int bi = found ? (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull)) : -1;
    const float bm = __uint_as_float((uint32_t)(key >> 32));
    const float nan = __int_as_float(0x7fc00000);
    if (pidx) pidx[orow] = bi;
    if (pabs) pabs[orow] = found ? sqrtf(bm) : nan;
    if (pphi) pphi[orow] = found ? phi32[bi] : nan;
    if (pq || pu || pchi) {
        float br = nan, bim = nan;
        if (found) {
            const float2 v = *reinterpret_cast<const float2 *>(F + orow * 2 * (int64_t)nphi + 2 * (int64_t)bi);
            br = v.x;
            bim = v.y;
        }
        if (pq) pq[orow] = br;
        if (pu) pu[orow] = bim;
        if (pchi) {
            // chi0 = arg F(phi_peak) / 2 - phi_peak lambda_0^2, reduced to [0, pi)
            float c = nan;
            if (found) {
                double x = 0.5 * atan2((double)bim, (double)br) - phi64[bi] * lambda0sq;
                x -= M_PI * floor(x / M_PI);
                c = (float)x;
            }
            pchi[orow] = c;
        }
    }
}

size_t gemm_fixed_smem() { return 1024 + kEpiStageBytes + 2 * 4 * 32 * 16 + 8 * 32 + 32; }

int gemm_stages(int b_rows, int mode)
{
    size_t st = gemm_stage_bytes(b_rows, mode);
    int s = (int)((kSmemLimit - gemm_fixed_smem()) / (st + 24));
    return s > 8 ? 8 : s;
}

bool split_mode(int mode) { return mode != MODE_BF16; }

int mode_of(int precision)
{
    return precision == RMS_BF16 ? MODE_BF16 : (precision == RMS_BF16X3 ? MODE_BF16X3 : MODE_FP16X3);
}

}  // namespace

size_t split_operand_bytes(const rms_plan_s &p, int64_t nlos, int layout)
{
    // an even number of M tiles: the two-CTA contraction reads M tiles in pairs (the
    // rows of a padding tile only ever reach rows of the result that are not stored)
    const int kb = layout == RMS_CHAN_MAJOR ? p.kblocks : p.kblocks_raw;
    const int64_t nmt = (nlos + kTileM - 1) / kTileM;
    return (size_t)((nmt + 1) & ~(int64_t)1) * kb * (2 * kStageA);
}

cudaError_t launch_split(const rms_plan_s &p, const SplitOpts &o, cudaStream_t s)
{
    const bool chan = o.layout == RMS_CHAN_MAJOR;
    const int64_t nmt = (o.nout + kTileM - 1) / kTileM;
    if (nmt < 1) return cudaSuccess;
    if (nmt > 0x7fffffff) return cudaErrorInvalidValue;
    SplitParams sp;
    sp.Q = o.Q;
    sp.U = o.U;
    sp.nlos_src = o.nlos_src;
    sp.nout = o.nout;
    sp.rows = o.rows;
    sp.count = o.count;
    sp.nchan = p.nchan;
    sp.layout = o.layout;
    sp.nk = chan ? p.nact : p.nchan;
    sp.kblocks = chan ? p.kblocks : p.kblocks_raw;
    sp.mode = o.mode >= 0 ? o.mode : mode_of(p.precision);
    sp.active = p.d_active;
    sp.kbmask = p.d_kbmask;
    sp.A = o.A;
    sp.rexp = o.rexp;
    sp.rscale = o.rscale;
    sp.nact_norm = p.nact;
    sp.vec4 = !chan && (p.nchan % 4 == 0) && !(reinterpret_cast<uintptr_t>(o.Q) & 15) &&
              !(reinterpret_cast<uintptr_t>(o.U) & 15);
    if (sp.mode == MODE_FP16X3 && !o.rexp) return cudaErrorInvalidValue;
    // A grid of one CTA per M tile leaves a partial last wave (the LOFAR cube's 2,048
    // tiles are 1.5 waves at 9 CTAs per SM), so the K blocks of a tile are shared out
    // over blockIdx.y until the grid is about 8 waves; FP16X3 (a row's largest value
    // sets its scale) and rscale (a row's RMS) need the whole row in one thread.
    int ngroups = 1;
    if (sp.mode != MODE_FP16X3 && !o.rscale) {
        const int64_t target = (int64_t)8 * 9 * p.num_sms;
        ngroups = (int)std::min<int64_t>(sp.kblocks, std::max<int64_t>(1, (target + nmt - 1) / nmt));
    }
    sp.kpg = (sp.kblocks + ngroups - 1) / ngroups;
    if (sp.vec4 && (sp.kpg & 1) && sp.kpg < sp.kblocks) ++sp.kpg;   // LOS-major pairs of K blocks stay whole
    ngroups = (sp.kblocks + sp.kpg - 1) / sp.kpg;
    const dim3 grid((unsigned)nmt, (unsigned)ngroups);
    if (!chan && sp.vec4) split_kernel<true><<<grid, 128, 0, s>>>(sp);
    else split_kernel<false><<<grid, 128, 0, s>>>(sp);
    return cudaGetLastError();
}

cudaError_t launch_gemm(const rms_plan_s &p, const GemmOpts &o, cudaStream_t s)
{
    const bool chan = o.layout == RMS_CHAN_MAJOR;
    const int mode = mode_of(p.precision);
    const int64_t nmt = (o.nlos + kTileM - 1) / kTileM;
    if (nmt < 1) return cudaSuccess;
    const bool rot = o.T != nullptr;
    if (rot && (mode == MODE_FP16X3 || p.tile_n > 2 * kHalfRot || !o.centre)) return cudaErrorInvalidValue;
    GemmParams P;
    P.A = o.A;
    P.nlos = o.nlos;
    P.count = o.count;
    P.rows = o.rows;
    P.kblocks = chan ? p.kblocks : p.kblocks_raw;
    // K blocks chained into one TMEM partial before the round-to-nearest fold: the
    // tensor core's accumulation error grows ~4e-8 per chained MMA, which matters for
    // the split precisions only; plain BF16 (error ~1e-3) folds once per N tile.
    // RMS_GROUP_KBLOCKS (2..64) overrides the split-precision group (a tuning knob).
    static const int group_split = [] {
        const char *v = std::getenv("RMS_GROUP_KBLOCKS");
        const int g = v ? std::atoi(v) : 0;
        return (g >= 2 && g <= 64) ? g : kGroupKBlocks;
    }();
    const int group_max = mode == MODE_BF16 ? P.kblocks : group_split;
    int ngroups = (P.kblocks + group_max - 1) / group_max;
    P.group = (P.kblocks + ngroups - 1) / ngroups;
    P.nphi = p.nphi;
    P.F = o.F;
    P.pidx = o.pidx;
    P.pabs = o.pabs;
    P.pphi = o.pphi;
    P.pq = o.pq;
    P.pu = o.pu;
    P.pchi = o.pchi;
    P.phi32 = p.d_phi32;
    P.phi64 = p.d_phi;
    P.lambda0sq = p.lambda0sq;
    P.out_scale = (float)(p.K * p.wmax);
    P.mode = mode;
    P.rexp = mode == MODE_FP16X3 ? o.rexp : nullptr;
    P.err = p.d_err;
    P.timeout_ns = p.timeout_ns;
    P.centre = o.centre;
    P.T = o.T;
    P.ldT = o.ldT;
    P.cmin = o.cmin;
    P.cmax = o.cmax;
    // the two-CTA contraction serves full-grid calls unless the plan asks for single
    // CTAs (rms_plan_set_option); in the environment RMS_GEMM_PAIR=0 makes single CTAs
    // the default and RMS_GEMM_PAIR=2 CTA pairs wherever the tiles allow them
    static const int pair_default = [] {
        const char *v = std::getenv("RMS_GEMM_PAIR");
        return v && v[0] == '0' ? 0 : (v && v[0] == '2' ? 2 : 1);
    }();
    // Automatic choice: pairs where their tiles exceed 208 phase rows; with narrower
    // tiles (a 256-row MMA with N <= 208 takes ~116 cycles against ~104 for the 128-row
    // one) only for split precisions under the job schedule, where the halved
    // shared-memory traffic wins (LOFAR cube, BF16x3: 0.68 against 0.70 ms
    // channel-major, 0.69 against 0.74 LOS-major; whole schedule 0.87 against 0.75;
    // plain BF16 0.53 against 0.50).
    const bool f_at_peak = o.pq || o.pu || o.pchi;
    auto pair_for = [&](bool with_jobs) {
        const bool wanted =
            p.contraction == RMS_CONTRACT_PAIR ||
            (p.contraction == RMS_CONTRACT_AUTO &&
             (pair_default == 2 ||
              (pair_default == 1 && (p.tile_n2 > 2 * kHalf || (with_jobs && split_mode(mode))))));
        return !rot && wanted && p.pair_maps;
    };
    int ctas = p.num_sms;
    if (const char *v = std::getenv("RMS_GEMM_CTAS")) {   // tuning knob: persistent CTAs
        int c = std::atoi(v);
        if (c >= 1 && c <= p.num_sms) ctas = c;
    }
    // L2 budget of the schedule choice (below): 80 MiB by default; rms_plan_set_option,
    // or RMS_L2_BUDGET_MB = 8 .. 1024 in the environment
    static const double budget_default = [] {
        const char *v = std::getenv("RMS_L2_BUDGET_MB");
        const int mb = v ? std::atoi(v) : 0;
        return (mb >= 8 && mb <= 1024 ? mb : 80) * 1048576.0;
    }();
    const double budget = p.l2_budget > 0 ? (double)p.l2_budget : budget_default;
    const double a_tile = (double)P.kblocks * (split_mode(mode) ? 2 * kStageA : kStageA);
    const double b_all = (double)p.npad * (chan ? p.kpad : p.kpad_raw) * 2.0 * (split_mode(mode) ? 2 : 1);
    bool jobs = !rot && o.keys && p.schedule != RMS_SCHEDULE_WHOLE && (o.F || !f_at_peak);
    if (jobs && !o.F && p.schedule == RMS_SCHEDULE_AUTO) {
        // Peak map only: with no F to store, the whole schedule's longer jobs win wherever
        // one panel holds the phase matrix (LOFAR band, peak map only, pairs or single
        // CTAs: 8.78 against 9.76 ms for 4,194,304 LOS, 0.58 against 0.60 ms for 262,144;
        // the MWA band, 2 panels, stays split: 95.0 against 100.5 ms)
        const bool pr = pair_for(true);
        const int64_t nitp = pr ? (nmt + 1) / 2 : nmt;
        const int64_t u = std::min<int64_t>(nitp, pr ? std::max(1, ctas / 2) : ctas);
        const int64_t nt = pr ? p.ntiles_n2 : p.ntiles_n;
        const double live = (double)((u + nt - 1) / nt + 1) * (pr ? 2.0 : 1.0) * a_tile + b_all;
        if (live <= budget) jobs = false;
    }
    const bool pair = pair_for(jobs);
    P.ntiles_n = pair ? p.ntiles_n2 : p.ntiles_n;
    P.tile_n = pair ? p.tile_n2 : p.tile_n;
    P.tile_n_last = pair ? p.tile_n_last2 : p.tile_n_last;
    const bool wide = pair && P.tile_n > 2 * kHalf;   // the pair kernel with 128 columns per epilogue thread
    P.b_rows = pair ? P.tile_n / 2 : P.tile_n;
    P.stages = gemm_stages(P.b_rows, mode);
    if (P.stages < 2) return cudaErrorInvalidConfiguration;
    size_t smem = gemm_fixed_smem() + (size_t)P.stages * gemm_stage_bytes(P.b_rows, mode) + 24 * (size_t)P.stages;
    const int64_t nit = pair ? (nmt + 1) / 2 : nmt;
    int maxunits = pair ? (ctas / 2 > 0 ? ctas / 2 : 1) : ctas;
    using KernelFn = void (*)(GemmParams, CUtensorMap, CUtensorMap, CUtensorMap);
    const KernelFn pair_kern = wide ? gemm_kernel<kHalfWide, false, true> : gemm_kernel<kHalf, false, true>;
    if (!rot) {
        // the setmaxnreg shares of the non-window variants add up to 384 x 168 registers:
        // launching one with any other register count would leave its epilogue
        // warpgroups waiting for registers, so check the build once
        static const cudaError_t regs_ok = [] {
            const KernelFn ks[3] = {gemm_kernel<kHalf, false, false>, gemm_kernel<kHalf, false, true>,
                                    gemm_kernel<kHalfWide, false, true>};
            for (const KernelFn k : ks) {
                cudaFuncAttributes fa;
                cudaError_t e1 = cudaFuncGetAttributes(&fa, k);
                if (e1 != cudaSuccess) return e1;
                if (fa.numRegs != kRegsLaunch) return cudaErrorInvalidConfiguration;
            }
            return cudaSuccess;
        }();
        if (regs_ok != cudaSuccess) return regs_ok;
    }
    if (pair) {
        // a pair needs two SMs of one TPC; TPCs with a disabled SM cannot host one, so
        // the persistent grid takes as many clusters as can be resident at once (more
        // would wait for a second wave)
        cudaError_t e0 = cudaFuncSetAttribute(pair_kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e0 != cudaSuccess) return e0;
        cudaLaunchConfig_t qc = {};
        qc.gridDim = dim3((unsigned)(2 * maxunits), 1, 1);
        qc.blockDim = dim3(kThreads, 1, 1);
        qc.dynamicSmemBytes = smem;
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = 2;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        qc.attrs = qa;
        qc.numAttrs = 1;
        int nclusters = 0;
        e0 = cudaOccupancyMaxActiveClusters(&nclusters, pair_kern, &qc);
        if (e0 != cudaSuccess) return e0;
        if (nclusters < 1) return cudaErrorInvalidConfiguration;
        if (nclusters < maxunits) maxunits = nclusters;
    }
    const int units = (int)(nit < maxunits ? nit : maxunits);
    // Schedule.  Whole: every CTA (pair) runs all N tiles of its M tile(s), re-reading
    // their operand once per N tile; those re-reads hit L2 only while the operands of
    // all M tiles in flight plus the whole phase matrix fit there.  Split (the default
    // when the caller provides key scratch): single-N-tile jobs in panels (see
    // GemmParams), with the smallest number of panels whose working set -- the
    // operands of the M tiles the CTAs share at one time plus one panel of the phase
    // matrix -- fits the budget.
    P.jobs_split = 0;
    P.npanels = 1;
    P.keys = nullptr;
    if (jobs) {
        const double tiles_per_unit = pair ? 2.0 : 1.0;
        // measured on the LOFAR cube: split jobs 0.70 ms against 0.75 ms for the whole
        // schedule although the latter's working set fits (finer jobs balance the CTAs
        // better), so the split schedule is the default wherever the call has the keys
        {
            int best = 1;
            double best_live = 1e300;
            for (int np = 1; np <= P.ntiles_n; ++np) {
                const int len = P.ntiles_n / np;
                const double live = ((units + len - 1) / len + 1) * tiles_per_unit * a_tile + b_all / np;
                if (live <= budget) { best = np; best_live = live; break; }
                if (live < best_live) { best = np; best_live = live; }
            }
            P.jobs_split = 1;
            P.npanels = best;
            P.keys = o.keys;
        }
    }
    cudaError_t e;
    if (P.jobs_split) {
        e = cudaMemsetAsync(P.keys, 0, (size_t)o.nlos * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    if (rot) {
        const CUtensorMap &bhi = chan ? p.tmap_bhi : p.tmap_bhi_raw, &blo = chan ? p.tmap_blo : p.tmap_blo_raw;
        auto kern = gemm_kernel<kHalfRot, true, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<units, 512, smem, s>>>(P, bhi, blo, bhi);   // (the last map is unused here)
    } else if (pair) {
        if (P.tile_n > 2 * kHalfWide || (P.tile_n & 15) || (P.tile_n_last & 15)) return cudaErrorInvalidValue;
        const CUtensorMap &bhi = chan ? p.tmap2_bhi : p.tmap2_bhi_raw, &blo = chan ? p.tmap2_blo : p.tmap2_blo_raw;
        const int pairs = units;
        // the operand image as a 3-D tensor for the pair's TMA loads: 64-byte rows, 256
        // rows (hi then lo parts) per 16 KB block, one block per (M tile, K block); a
        // stage is one block's first a_rows rows
        CUtensorMap tmA;
        {
            const int64_t nblocks = (((int64_t)o.nlos + 2 * kTileM - 1) / (2 * kTileM)) * 2 * P.kblocks;
            const cuuint64_t dims[3] = {(cuuint64_t)kKBlock, (cuuint64_t)(2 * kTileM), (cuuint64_t)nblocks};
            const cuuint64_t strides[2] = {(cuuint64_t)kRowBytes, (cuuint64_t)(2 * kStageA)};
            const cuuint32_t box[3] = {(cuuint32_t)kKBlock, (cuuint32_t)(split_mode(mode) ? 2 * kTileM : kTileM), 1};
            const cuuint32_t estr[3] = {1, 1, 1};
            if (nblocks > 0x7fffffff ||
                !encode_tensor_map(&tmA, CU_TENSOR_MAP_DATA_TYPE_UINT16, const_cast<uint8_t *>(o.A), dims, strides,
                                   box, estr, CU_TENSOR_MAP_SWIZZLE_NONE, 3))
                return cudaErrorInvalidValue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(2 * pairs), 1, 1);
        cfg.blockDim = dim3(kThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, pair_kern, P, bhi, blo, tmA);
        if (e != cudaSuccess) return e;
    } else {
        if (p.tile_n > 2 * kHalf) return cudaErrorInvalidValue;
        const CUtensorMap &bhi = chan ? p.tmap_bhi : p.tmap_bhi_raw, &blo = chan ? p.tmap_blo : p.tmap_blo_raw;
        auto kern = gemm_kernel<kHalf, false, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<units, kThreads, smem, s>>>(P, bhi, blo, bhi);   // (the last map is unused here)
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    p.last_ctas = pair ? 2 * units : units;
    p.last_pair = pair ? 1 : 0;
    p.last_panels = P.jobs_split ? P.npanels : 0;
    p.last_kernels = 1;
    if (P.jobs_split && (o.pidx || o.pabs || o.pphi || f_at_peak)) {
        p.last_kernels = 2;
        const int64_t nb = (o.nlos + 255) / 256;
        if (nb > 0x7fffffff) return cudaErrorInvalidValue;
        peak_finalize_kernel<<<(unsigned)nb, 256, 0, s>>>(P.keys, o.nlos, o.count, o.rows, o.F, p.nphi, p.d_phi32,
                                                          p.d_phi, p.lambda0sq, o.pidx, o.pabs, o.pphi, o.pq, o.pu,
                                                          o.pchi);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_image_gather(const rms_plan_s &p, int layout, const uint8_t *src, const int64_t *rows,
                                const int64_t *count, int64_t nmax, uint8_t *dst, cudaStream_t s)
{
    const int64_t nmt = (nmax + kTileM - 1) / kTileM;
    if (nmt < 1) return cudaSuccess;
    if (nmt > 0x7fffffff) return cudaErrorInvalidValue;
    const int kb = layout == RMS_CHAN_MAJOR ? p.kblocks : p.kblocks_raw;
    const int parts = p.precision == RMS_BF16 ? 1 : 2;
    if (kb > 65535) return cudaErrorInvalidValue;
    image_gather_kernel<<<dim3((unsigned)nmt, (unsigned)kb), 128, 0, s>>>(src, dst, kb, rows, count, nmax, parts);
    return cudaGetLastError();
}

cudaError_t launch_split_gemm(const rms_plan_s &p, const float *Q, const float *U, int64_t nlos, int layout,
                              float *F, int32_t *pidx, float *pabs, float *pphi, uint8_t *A, int8_t *rexp,
                              cudaStream_t s, cudaEvent_t ev_mid, float *pq, float *pu, float *pchi,
                              unsigned long long *keys)
{
    SplitOpts so;
    so.Q = Q;
    so.U = U;
    so.nlos_src = nlos;
    so.nout = nlos;
    so.layout = layout;
    so.A = A;
    so.rexp = rexp;
    cudaError_t e = launch_split(p, so, s);
    if (e != cudaSuccess) return e;
    if (ev_mid && (e = cudaEventRecord(ev_mid, s)) != cudaSuccess) return e;
    GemmOpts go;
    go.A = A;
    go.nlos = nlos;
    go.layout = layout;
    go.F = F;
    go.pidx = pidx;
    go.pabs = pabs;
    go.pphi = pphi;
    go.pq = pq;
    go.pu = pu;
    go.pchi = pchi;
    go.rexp = rexp;
    go.keys = keys;
    e = launch_gemm(p, go, s);
    p.last_kernels += 1;   // the split
    return e;
}
