// Tensor-core RM synthesis for sm_103a: tcgen05.mma with TMEM accumulators,
// TMA-fed operands, FP32 data split into 16-bit operands on the fly.
//
// Eq. Fsum in its real form (Eqs. qPhi, uPhi) is a real GEMM
//     C[l][2k + {0,1}] = sum_a ( Q_la B[2k+{0,1}][2a] + U_la B[2k+{0,1}][2a+1] )
// with the phase block B = (w_a / w_max) [[c, s], [-s, c]] built at plan time in
// FP64 (phase.cu), so row l of C is F(phi) as interleaved complex64, up to the
// factor K w_max applied in the epilogue.  M = lines of sight, N = 2 nphi,
// K = 2 x (active channels for channel-major cubes | all channels for LOS-major).
//
// Precision.  A (data) and B (phase) are split into hi + lo 16-bit parts and
// hi*hi + hi*lo + lo*hi are accumulated (BF16X3, FP16X3), or hi*hi only (BF16).
// FP16 data are scaled per line of sight by a power of two (largest |value| in
// [2^14, 2^15)).  The tensor core adds each MMA's result into the FP32
// accumulator without round-to-nearest, and that error grows with the number
// of MMAs chained into one accumulator; so MMAs run in groups of a few K blocks
// into one of two TMEM partial accumulators, and the epilogue warps fold every
// finished partial into FP32 registers with round-to-nearest adds.
//
// CTA = 16 warps (4 warpgroups), persistent over 128-row M tiles; each M tile
// runs its N tiles in order so each row's running peak stays in registers.
//   warp 0       data producer: TMA of FP32 Q/U tiles (gather4 of active channel
//                rows for channel-major cubes, 2-D boxes for LOS-major)  -> fullD
//   warp 1       TMEM allocator, single-thread MMA issuer                -> emptyM, tfull
//   warp 2       phase producer: TMA of B hi/lo tiles                     -> fullB
//   warps 4..7   converters: FP32 -> split 16-bit A tile (64-byte swizzled
//                K-major layout), flagged / padded channels zeroed        -> fullA, emptyD
//   warps 8..15  epilogue: warp w owns TMEM lane quarter w % 4 and column half
//                (w - 8) / 4; folds partials, scales, peak, stores F      -> tempty
// The split A tile of an M tile is converted once, on its first N tile, and kept
// in a per-CTA scratch region (L2-resident for LOFAR-sized cubes) from which the
// converters reload it for the remaining N tiles.
// Without TMA-compatible strides the converters load FP32 directly instead.
// Every mbarrier wait is bounded by a wall-clock limit; a wait that runs out
// raises a CTA-wide abort flag and the device error word, every role leaves
// its loop, in-flight TMA copies and MMAs are drained with bounded waits, and
// TMEM is freed before the CTA exits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <limits.h>

#include <cstdlib>
#include <cstring>

#include "rms_internal.h"

namespace {

// K blocks per TMEM partial before the FP32 register fold in this kernel
constexpr int kUmmaGroupKBlocks = 6;

constexpr int kThreads = 512;
constexpr int kConvWarp0 = 4, kNumConvWarps = 4;
constexpr int kEpiWarp0 = 8, kNumEpiWarps = 8;
constexpr int kRowBytes = kKBlock * 2;              // 64 B per operand row per stage
constexpr int kStageA = kTileM * kRowBytes;         // 8 KB per A part
constexpr int kStageD = kTileM * kChanPerKBlock * 4; // 8 KB of FP32 per Q or U
constexpr int kTmemCols = 512;
constexpr int kAccStride = 256;                     // TMEM columns per partial
constexpr int kHalf = kMaxTileN / 2;                // 104 columns per epilogue thread
constexpr int kEpiLd = 17;                          // 16-column staging chunks
constexpr int kEpiStageBytes = kNumEpiWarps * 32 * kEpiLd * 4;
constexpr int kSmemLimit = 227 * 1024;
constexpr int kRegsLow = 96, kRegsHigh = 160;       // setmaxnreg split: 256*96 + 256*160 = 512*128

enum { MODE_BF16 = 0, MODE_BF16X3 = 1, MODE_FP16X3 = 2 };

struct UmmaParams {
    const float *Q, *U;
    int64_t nlos;
    int32_t nchan, layout, use_tma;
    const int32_t *active;      // channel-major: active channel list
    const uint16_t *kbmask;     // LOS-major: per K block, bit i = channel 16 kb + i active
    int32_t nk, kblocks, group; // contraction channels, K blocks, K blocks per TMEM group
    int32_t nphi, ntiles_n, tile_n, tile_n_last;
    float *F;
    int32_t *pidx;
    float *pabs, *pphi;
    const float *phi32;
    float out_scale;
    int32_t mode;
    const int8_t *rexp;
    int *err;
    int64_t timeout_ns;
    int32_t sd, sa, sb;         // stages of the FP32 data, A and B rings
    int32_t reuse;              // 1: convert on the first N tile only, reload from scratch after
    uint4 *scratch;             // [grid][kblocks][16 KB]: split A stages of the current M tile (smem image)
};

#include "tc_ptx.cuh"

// Convert one row's 16 channels (K values Q0 U0 Q1 U1 ...) into the four 16-byte
// chunks of the hi tile (and of the lo tile).  Row m, chunk c of a 64-byte-
// swizzled K-major tile lives at m * 64 + ((c ^ ((m >> 1) & 3)) << 4).  When
// scr is set, the same bytes also go to the scratch image of this stage
// (hi part at scr, lo part at scr + 8 KB).
__device__ __forceinline__ void convert_row(const float (&q)[16], const float (&u)[16], float scale, int mode,
                                            uint8_t *a_hi, uint8_t *a_lo, int m, int sw, uint8_t *scr)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = 4 * c + j;
            if (mode == MODE_FP16X3) split_pair_fp16(q[i] * scale, u[i] * scale, hi[j], lo[j]);
            else split_pair_bf16(q[i], u[i], hi[j], lo[j]);
        }
        const uint32_t off = (uint32_t)m * kRowBytes + ((uint32_t)(c ^ sw) << 4);
        const uint4 vh = make_uint4(hi[0], hi[1], hi[2], hi[3]), vl = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        *reinterpret_cast<uint4 *>(a_hi + off) = vh;
        if (mode != MODE_BF16) *reinterpret_cast<uint4 *>(a_lo + off) = vl;
        if (scr) {
            *reinterpret_cast<uint4 *>(scr + off) = vh;
            if (mode != MODE_BF16) *reinterpret_cast<uint4 *>(scr + kStageA + off) = vl;
        }
    }
}

struct Smem {
    uint8_t *dring, *aring, *bring;
    uint32_t bstage;
    float *epi;
    float *pk_m;
    int *pk_i;
    uint64_t *fullD, *emptyD, *fullA, *emptyA, *fullB, *emptyB, *tfull, *tempty, *pkfull, *pkempty, *scr_ready,
        *mma_done;
    uint32_t *tmem_slot;
    volatile int *abort_flag;
    int *converted;     // converter warps done with their M tiles' first N tile (x4 per M tile)
};

__device__ __forceinline__ Smem carve(uint8_t *base, const UmmaParams &P)
{
    Smem s;
    s.bstage = 2 * (uint32_t)P.tile_n * kRowBytes;
    s.dring = base;
    s.aring = s.dring + (size_t)P.sd * 2 * kStageD;
    s.bring = s.aring + (size_t)P.sa * 2 * kStageA;
    s.epi = reinterpret_cast<float *>(s.bring + (size_t)P.sb * s.bstage);
    s.pk_m = s.epi + kEpiStageBytes / 4;
    s.pk_i = reinterpret_cast<int *>(s.pk_m + 2 * 4 * 32);
    uint64_t *b = reinterpret_cast<uint64_t *>(s.pk_i + 2 * 4 * 32);
    s.fullD = b;
    s.emptyD = s.fullD + P.sd;
    s.fullA = s.emptyD + P.sd;
    s.emptyA = s.fullA + P.sa;
    s.fullB = s.emptyA + P.sa;
    s.emptyB = s.fullB + P.sb;
    s.tfull = s.emptyB + P.sb;
    s.tempty = s.tfull + 2;
    s.pkfull = s.tempty + 2;      // [2 parities][4 quarters]
    s.pkempty = s.pkfull + 8;
    s.scr_ready = s.pkempty + 8;  // [2 parities]
    s.mma_done = s.scr_ready + 2;
    s.tmem_slot = reinterpret_cast<uint32_t *>(s.mma_done + 1);
    s.abort_flag = reinterpret_cast<volatile int *>(s.tmem_slot + 1);
    s.converted = const_cast<int *>(s.abort_flag) + 1;
    return s;
}

// Ring position: slot index and phase parity.
struct Ring {
    int s = 0;
    uint32_t ph = 0;
    __device__ __forceinline__ void next(int n)
    {
        if (++s == n) { s = 0; ph ^= 1; }
    }
};

// Wait (bounded) for every copy this thread issued into a ring to land.
__device__ __forceinline__ void drain(const uint64_t *full, int n, uint32_t pending, uint32_t pend_par,
                                      volatile int *abort_flag, int *err, int64_t limit)
{
    for (int i = 0; i < n; ++i)
        if (pending & (1u << i))
            wait_bounded(smem_u32(&full[i]), (pend_par >> i) & 1, abort_flag, err, limit, false);
}

// ----------------------------------------------------------------------------
// The kernel
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1)
umma_synth_kernel(const __grid_constant__ UmmaParams P, const __grid_constant__ CUtensorMap tmB_hi,
                  const __grid_constant__ CUtensorMap tmB_lo, const __grid_constant__ CUtensorMap tmQ,
                  const __grid_constant__ CUtensorMap tmU)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const Smem S = carve(base, P);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nmt = (P.nlos + kTileM - 1) / kTileM;
    const bool split = P.mode != MODE_BF16;
    const int ngroups = (P.kblocks + P.group - 1) / P.group;
    const uint32_t a_bytes = split ? 2 * kStageA : kStageA;   // one A stage (hi [+ lo])

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.sd; ++s) {
            mbar_init(smem_u32(&S.fullD[s]), 1);
            mbar_init(smem_u32(&S.emptyD[s]), kNumConvWarps);
        }
        for (int s = 0; s < P.sa; ++s) {
            mbar_init(smem_u32(&S.fullA[s]), kNumConvWarps);   // converters, or producer: 1 + tx + 3
            mbar_init(smem_u32(&S.emptyA[s]), 1);
        }
        for (int s = 0; s < P.sb; ++s) {
            mbar_init(smem_u32(&S.fullB[s]), 1);
            mbar_init(smem_u32(&S.emptyB[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&S.tfull[b]), 1);
            mbar_init(smem_u32(&S.tempty[b]), kNumEpiWarps);
            mbar_init(smem_u32(&S.scr_ready[b]), kNumConvWarps);
        }
        for (int i = 0; i < 8; ++i) {
            mbar_init(smem_u32(&S.pkfull[i]), 1);
            mbar_init(smem_u32(&S.pkempty[i]), 1);
        }
        mbar_init(smem_u32(S.mma_done), 1);
        *S.abort_flag = 0;
        *S.converted = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        __syncwarp();
        tmem_alloc(smem_u32(S.tmem_slot), kTmemCols);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *S.tmem_slot;

    // register split: warpgroups 0-1 (producers, MMA, converters) give registers
    // to warpgroups 2-3 (epilogue, which keeps tile_n / 2 FP32 sums per thread)
    if (warp < kEpiWarp0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsLow));
        if (warp == 0) {
            // -------------------------------------------------------- data / A producer
            // first N tile: FP32 Q/U tiles into the data ring (converters split them);
            // later N tiles: the split A tile written to scratch on the first N tile,
            // one bulk copy per stage straight into the A ring.
            if (lane == 0) {
                if (P.use_tma) {
                    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmQ)) : "memory");
                    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmU)) : "memory");
                }
                Ring rd, ra;
                uint32_t pendD = 0, parD = 0, pendA = 0, parA = 0;
                bool ok = true;
                int mt_count = 0;
                for (int64_t mt = blockIdx.x; mt < nmt && ok; mt += gridDim.x, ++mt_count)
                    for (int nt = 0; nt < P.ntiles_n && ok; ++nt) {
                        if (P.reuse && nt == 1 &&
                            !wait_bounded(smem_u32(&S.scr_ready[mt_count & 1]), (mt_count >> 1) & 1, S.abort_flag,
                                          P.err, P.timeout_ns)) {
                            ok = false;
                            break;
                        }
                        for (int kb = 0; kb < P.kblocks; ++kb) {
                            if (nt == 0 || !P.reuse) {
                                ra.next(P.sa);      // the converters fill this A slot
                                if (!P.use_tma) continue;
                                if (!wait_bounded(smem_u32(&S.emptyD[rd.s]), rd.ph ^ 1, S.abort_flag, P.err,
                                                  P.timeout_ns)) {
                                    ok = false;
                                    break;
                                }
                                const uint32_t dq = smem_u32(S.dring + (size_t)rd.s * 2 * kStageD), du = dq + kStageD;
                                const uint32_t bar = smem_u32(&S.fullD[rd.s]);
                                mbar_arrive_expect_tx(bar, 2 * kStageD);
                                const int32_t m0 = (int32_t)(mt * kTileM);
                                if (P.layout == RMS_CHAN_MAJOR) {
#pragma unroll
                                    for (int g = 0; g < 4; ++g) {
                                        int32_t y[4];
#pragma unroll
                                        for (int r = 0; r < 4; ++r) {
                                            const int a = kb * kChanPerKBlock + 4 * g + r;
                                            y[r] = __ldg(P.active + (a < P.nk ? a : P.nk - 1));
                                        }
                                        tma_gather4(dq + g * 4 * kTileM * 4, &tmQ, m0, y[0], y[1], y[2], y[3], bar);
                                        tma_gather4(du + g * 4 * kTileM * 4, &tmU, m0, y[0], y[1], y[2], y[3], bar);
                                    }
                                } else {
                                    tma_load_2d(dq, &tmQ, kb * kChanPerKBlock, m0, bar);
                                    tma_load_2d(du, &tmU, kb * kChanPerKBlock, m0, bar);
                                }
                                pendD |= 1u << rd.s;
                                parD = (parD & ~(1u << rd.s)) | (rd.ph << rd.s);
                                rd.next(P.sd);
                            } else {
                                if (!wait_bounded(smem_u32(&S.emptyA[ra.s]), ra.ph ^ 1, S.abort_flag, P.err,
                                                  P.timeout_ns)) {
                                    ok = false;
                                    break;
                                }
                                const uint32_t bar = smem_u32(&S.fullA[ra.s]);
                                mbar_arrive_expect_tx(bar, a_bytes);
                                bulk_load(smem_u32(S.aring + (size_t)ra.s * 2 * kStageA),
                                          P.scratch + ((size_t)blockIdx.x * P.kblocks + kb) * (2 * kStageA / 16),
                                          a_bytes, bar);
                                mbar_arrive_n(bar, kNumConvWarps - 1);
                                pendA |= 1u << ra.s;
                                parA = (parA & ~(1u << ra.s)) | (ra.ph << ra.s);
                                ra.next(P.sa);
                            }
                        }
                    }
                if (!ok) {
                    drain(S.fullD, P.sd, pendD, parD, S.abort_flag, P.err, P.timeout_ns);
                    drain(S.fullA, P.sa, pendA, parA, S.abort_flag, P.err, P.timeout_ns);
                }
            }
        } else if (warp == 2) {
            // -------------------------------------------------------- phase producer
            if (lane == 0) {
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB_hi)) : "memory");
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB_lo)) : "memory");
                const uint32_t b_bytes = (uint32_t)P.tile_n * kRowBytes;
                const uint32_t tx = split ? 2 * b_bytes : b_bytes;
                Ring rb;
                uint32_t pending = 0, pend_par = 0;
                bool ok = true;
                for (int64_t mt = blockIdx.x; mt < nmt && ok; mt += gridDim.x)
                    for (int nt = 0; nt < P.ntiles_n && ok; ++nt)
                        for (int kb = 0; kb < P.kblocks; ++kb) {
                            if (!wait_bounded(smem_u32(&S.emptyB[rb.s]), rb.ph ^ 1, S.abort_flag, P.err,
                                              P.timeout_ns)) {
                                ok = false;
                                break;
                            }
                            const uint32_t st = smem_u32(S.bring + (size_t)rb.s * S.bstage);
                            const uint32_t bar = smem_u32(&S.fullB[rb.s]);
                            mbar_arrive_expect_tx(bar, tx);
                            tma_load_2d(st, &tmB_hi, kb * kKBlock, nt * P.tile_n, bar);
                            if (split) tma_load_2d(st + b_bytes, &tmB_lo, kb * kKBlock, nt * P.tile_n, bar);
                            pending |= 1u << rb.s;
                            pend_par = (pend_par & ~(1u << rb.s)) | (rb.ph << rb.s);
                            rb.next(P.sb);
                        }
                if (!ok) drain(S.fullB, P.sb, pending, pend_par, S.abort_flag, P.err, P.timeout_ns);
            }
        } else if (warp == 1) {
            // -------------------------------------------------------- MMA issuer
            if (lane == 0) {
                const bool bf = P.mode != MODE_FP16X3;
                const uint32_t id_full = idesc_f16(P.tile_n, bf), id_last = idesc_f16(P.tile_n_last, bf);
                const uint32_t b_bytes = (uint32_t)P.tile_n * kRowBytes;
                Ring ra, rb;
                uint32_t tph = 0;   // bit b: parity of TMEM partial b
                int g_all = 0;
                bool ok = true, issued = false;
                for (int64_t mt = blockIdx.x; mt < nmt && ok; mt += gridDim.x)
                    for (int nt = 0; nt < P.ntiles_n && ok; ++nt) {
                        const uint32_t idesc = (nt == P.ntiles_n - 1) ? id_last : id_full;
                        for (int g = 0; g < ngroups && ok; ++g, ++g_all) {
                            const int b = g_all & 1;
                            if (!wait_bounded(smem_u32(&S.tempty[b]), ((tph >> b) & 1) ^ 1, S.abort_flag, P.err,
                                              P.timeout_ns)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t d = tmem_base + (uint32_t)(b * kAccStride);
                            const int kb0 = g * P.group, kb1 = min(P.kblocks, kb0 + P.group);
                            for (int kb = kb0; kb < kb1; ++kb) {
                                if (!wait_bounded(smem_u32(&S.fullA[ra.s]), ra.ph, S.abort_flag, P.err, P.timeout_ns) ||
                                    !wait_bounded(smem_u32(&S.fullB[rb.s]), rb.ph, S.abort_flag, P.err, P.timeout_ns)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                                const uint32_t a_hi = smem_u32(S.aring + (size_t)ra.s * 2 * kStageA), a_lo = a_hi + kStageA;
                                const uint32_t b_hi = smem_u32(S.bring + (size_t)rb.s * S.bstage), b_lo = b_hi + b_bytes;
#pragma unroll
                                for (int kk = 0; kk < kKBlock / 16; ++kk) {
                                    const uint32_t ko = kk * 32;   // 16 K values = 32 bytes along the row
                                    const uint32_t acc = (kb > kb0 || kk > 0) ? 1u : 0u;
                                    mma_f16(d, sdesc_k64(a_hi + ko), sdesc_k64(b_hi + ko), idesc, acc);
                                    if (split) {
                                        mma_f16(d, sdesc_k64(a_hi + ko), sdesc_k64(b_lo + ko), idesc, 1u);
                                        mma_f16(d, sdesc_k64(a_lo + ko), sdesc_k64(b_hi + ko), idesc, 1u);
                                    }
                                }
                                issued = true;
                                mma_commit(smem_u32(&S.emptyA[ra.s]));
                                mma_commit(smem_u32(&S.emptyB[rb.s]));
                                ra.next(P.sa);
                                rb.next(P.sb);
                            }
                            if (!ok) break;
                            mma_commit(smem_u32(&S.tfull[b]));
                            tph ^= 1u << b;
                        }
                    }
                if (issued) {
                    // all MMAs of this thread complete before TMEM is released
                    mma_commit(smem_u32(S.mma_done));
                    wait_bounded(smem_u32(S.mma_done), 0, S.abort_flag, P.err, P.timeout_ns, false);
                }
            }
        } else if (warp == 3) {
            // -------------------------------------------------------- L2 prefetcher
            // Once the converters have finished an M tile's first N tile, its FP32 input
            // is no longer needed and the next M tile's input is prefetched into L2, so
            // that the next first N tile streams from L2 instead of waiting on HBM:
            // channel-major: 512-byte row pieces (Q and U of every active channel),
            // LOS-major: the contiguous 128-row blocks of Q and U in 4 KB pieces.
            if (P.reuse && P.use_tma) {
                const int units = P.layout == RMS_CHAN_MAJOR ? 2 * P.nk
                                                             : 2 * (int)(((int64_t)kTileM * P.nchan * 4 + 4095) / 4096);
                int mt_count = 0;
                for (int64_t mt = blockIdx.x; mt + gridDim.x < nmt; mt += gridDim.x, ++mt_count) {
                    // a pure performance hint: on a stall or an abort, stop prefetching
                    const uint64_t t0 = global_ns();
                    bool go = true;
                    while (go && *reinterpret_cast<volatile int *>(S.converted) < kNumConvWarps * (mt_count + 1)) {
                        __nanosleep(256);
                        go = !*S.abort_flag && (int64_t)(global_ns() - t0) < P.timeout_ns / 4;
                    }
                    if (!__all_sync(0xffffffffu, go)) break;
                    const int64_t mn = mt + gridDim.x;
                    const int64_t rows = min((int64_t)kTileM, P.nlos - mn * kTileM);
                    for (int u = lane; u < units; u += 32) {
                        if (P.layout == RMS_CHAN_MAJOR) {
                            const float *src = (u & 1) ? P.U : P.Q;
                            const int64_t off = (int64_t)__ldg(P.active + (u >> 1)) * P.nlos + mn * kTileM;
                            prefetch_l2(src + off, (uint32_t)(rows * 4));
                        } else {
                            const int per = units / 2;
                            const int64_t b0 = (int64_t)(u % per) * 4096;
                            const int64_t avail = rows * P.nchan * 4 - b0;
                            if (avail > 0) {
                                const char *src = reinterpret_cast<const char *>((u / per) ? P.U : P.Q) +
                                                  mn * kTileM * P.nchan * 4 + b0;
                                prefetch_l2(src, (uint32_t)min((int64_t)4096, avail));
                            }
                        }
                    }
                }
            }
        } else if (warp >= kConvWarp0) {
            // -------------------------------------------------------- converters (first N tile only)
            const int m = threadIdx.x - 32 * kConvWarp0;       // tile row 0..127
            const int sw = (m >> 1) & 3;
            Ring rd, ra;
            bool ok = true;
            int mt_count = 0;
            for (int64_t mt = blockIdx.x; mt < nmt && ok; mt += gridDim.x, ++mt_count) {
                const int64_t row = mt * kTileM + m;
                float sc = 1.0f;
                if (P.mode == MODE_FP16X3 && P.rexp != nullptr && row < P.nlos) sc = ldexpf(1.0f, (int)P.rexp[row]);
                const int nconv = P.reuse ? 1 : P.ntiles_n;   // N tiles whose A tiles are converted here
                for (int kb_all = 0; kb_all < nconv * P.kblocks; ++kb_all) {
                    const int kb = kb_all % P.kblocks;
                    float q[16], u[16];
                    const int c0 = kb * kChanPerKBlock;
                    uint32_t live;   // bit i: channel i of this K block contributes
                    if (P.layout == RMS_CHAN_MAJOR) live = (P.nk - c0 >= 16) ? 0xffffu : ((1u << (P.nk - c0)) - 1u);
                    else live = __ldg(P.kbmask + kb);
                    if (P.use_tma) {
                        if (!warp_wait(smem_u32(&S.fullD[rd.s]), rd.ph, S.abort_flag, P.err, P.timeout_ns)) { ok = false; break; }
                        const float *dq = reinterpret_cast<const float *>(S.dring + (size_t)rd.s * 2 * kStageD);
                        const float *du = dq + kStageD / 4;
                        if (P.layout == RMS_CHAN_MAJOR) {
                            // [16 channels][128 LOS]
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                q[i] = dq[i * kTileM + m];
                                u[i] = du[i * kTileM + m];
                            }
                        } else {
                            // [128 rows][16 channels], 64-byte swizzled
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const float4 a = *reinterpret_cast<const float4 *>(dq + m * 16 + ((c ^ sw) << 2));
                                const float4 b = *reinterpret_cast<const float4 *>(du + m * 16 + ((c ^ sw) << 2));
                                q[4 * c] = a.x; q[4 * c + 1] = a.y; q[4 * c + 2] = a.z; q[4 * c + 3] = a.w;
                                u[4 * c] = b.x; u[4 * c + 1] = b.y; u[4 * c + 2] = b.z; u[4 * c + 3] = b.w;
                            }
                        }
                        // the slot is refilled by TMA (async proxy): order these generic-proxy
                        // reads before the release
                        fence_proxy_async_smem();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(&S.emptyD[rd.s]));
                        rd.next(P.sd);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            q[i] = 0.f;
                            u[i] = 0.f;
                            if (((live >> i) & 1u) && row < P.nlos) {
                                const int64_t off = P.layout == RMS_CHAN_MAJOR
                                                        ? (int64_t)__ldg(P.active + c0 + i) * P.nlos + row
                                                        : row * P.nchan + c0 + i;
                                q[i] = __ldg(P.Q + off);
                                u[i] = __ldg(P.U + off);
                            }
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (!((live >> i) & 1u)) { q[i] = 0.f; u[i] = 0.f; }   // flagged / padding: also kills NaN
                    if (!warp_wait(smem_u32(&S.emptyA[ra.s]), ra.ph ^ 1, S.abort_flag, P.err, P.timeout_ns)) { ok = false; break; }
                    uint8_t *st = S.aring + (size_t)ra.s * 2 * kStageA;
                    // the scratch copy of this stage has the A slot's exact layout
                    uint8_t *scr = P.reuse
                                       ? reinterpret_cast<uint8_t *>(P.scratch + ((size_t)blockIdx.x * P.kblocks + kb) *
                                                                                     (2 * kStageA / 16))
                                       : nullptr;
                    convert_row(q, u, sc, P.mode, st, st + kStageA, m, sw, scr);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&S.fullA[ra.s]));
                    ra.next(P.sa);
                }
                if (!ok) break;
                if (P.reuse) {
                    // the A slots of the remaining N tiles are filled from scratch by the
                    // producer's bulk copies: make the scratch writes visible to them
                    for (int i = 0; i < (P.ntiles_n - 1) * P.kblocks; ++i) ra.next(P.sa);
                    fence_proxy_async_global();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(smem_u32(&S.scr_ready[mt_count & 1]));
                        atomicAdd(S.converted, 1);
                    }
                }
            }
        }
    } else {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsHigh));
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;                         // TMEM lane quarter
        const int h = (warp - kEpiWarp0) >> 2;          // column half of the tile
        float *stg = S.epi + (warp - kEpiWarp0) * 32 * kEpiLd;
        const int64_t row_pitch = 2 * (int64_t)P.nphi;
        uint32_t tph = 0;
        int g_all = 0, mt_count = 0;
        bool ok = true;
        float master[kHalf];
        for (int64_t mt = blockIdx.x; mt < nmt && ok; mt += gridDim.x, ++mt_count) {
            const int64_t row = mt * kTileM + 32 * q + lane;
            float scale = P.out_scale;
            if (P.rexp != nullptr && row < P.nlos) scale = ldexpf(scale, -(int)P.rexp[row]);
            float bm = -1.0f;
            int bi = INT_MAX;
            for (int nt = 0; nt < P.ntiles_n && ok; ++nt) {
                for (int g = 0; g < ngroups; ++g, ++g_all) {
                    const int b = g_all & 1;
                    if (!warp_wait(smem_u32(&S.tfull[b]), (tph >> b) & 1, S.abort_flag, P.err, P.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    tph ^= 1u << b;
                    tc_fence_after();
                    const uint32_t taddr = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kAccStride + h * kHalf);
#pragma unroll
                    for (int c0 = 0; c0 < kHalf; c0 += 32) {
                        uint32_t r[4][8];
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (c0 + 8 * j < kHalf) tmem_ld8(taddr + c0 + 8 * j, r[j]);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 4; ++j)
#pragma unroll
                            for (int e = 0; e < 8; ++e)
                                if (c0 + 8 * j < kHalf) {
                                    const float v = __uint_as_float(r[j][e]);
                                    master[c0 + 8 * j + e] = g == 0 ? v : __fadd_rn(master[c0 + 8 * j + e], v);
                                }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&S.tempty[b]));
                }
                if (!ok) break;
                // this unit's F for my row, columns [h*104, h*104 + 104) of the tile
                const int ncols = ((nt == P.ntiles_n - 1) ? P.tile_n_last : P.tile_n) - h * kHalf;
                const int kbase = (nt * P.tile_n + h * kHalf) >> 1;   // phi index of master[0]
#pragma unroll
                for (int p = 0; p < kHalf / 2; ++p) {
                    const float fr = master[2 * p] * scale, fi = master[2 * p + 1] * scale;
                    master[2 * p] = fr;
                    master[2 * p + 1] = fi;
                    const int k = kbase + p;
                    if (2 * p < ncols && k < P.nphi) {
                        const float m2 = __fadd_rn(__fmul_rn(fr, fr), __fmul_rn(fi, fi));
                        if (m2 > bm) { bm = m2; bi = k; }
                    }
                }
                if (P.F != nullptr) {
                    // transpose 16-column chunks through shared memory: each store
                    // instruction then writes four contiguous 64-byte row segments
#pragma unroll
                    for (int c0 = 0; c0 < kHalf; c0 += 16) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < kHalf) stg[lane * kEpiLd + j] = master[c0 + j];
                        __syncwarp();
                        const int jj = (lane & 7) * 2;
                        const int kk = kbase + (c0 >> 1) + (lane & 7);
                        const bool colok = c0 + jj < min(ncols, kHalf) && kk < P.nphi;
#pragma unroll
                        for (int it = 0; it < 8; ++it) {
                            const int r = 4 * it + (lane >> 3);
                            const int64_t grow = mt * kTileM + 32 * q + r;
                            if (colok && grow < P.nlos) {
                                const float2 val = make_float2(stg[r * kEpiLd + jj], stg[r * kEpiLd + jj + 1]);
                                // streaming store: F is written once and must not push the
                                // operands out of L2
                                __stcs(reinterpret_cast<float2 *>(P.F + grow * row_pitch + 2 * (int64_t)kk), val);
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
                __syncwarp();
                if (lane == 0) mbar_arrive(pbar);
            } else {
                if (!warp_wait(pbar, use_par, S.abort_flag, P.err, P.timeout_ns)) { ok = false; break; }
                const float om = S.pk_m[(par * 4 + q) * 32 + lane];
                const int oi = S.pk_i[(par * 4 + q) * 32 + lane];
                __syncwarp();
                if (lane == 0) mbar_arrive(ebar);
                if (om > bm || (om == bm && oi < bi)) { bm = om; bi = oi; }
                if (row < P.nlos) {
                    const bool found = bi != INT_MAX;
                    if (P.pidx) P.pidx[row] = found ? bi : -1;
                    if (P.pabs) P.pabs[row] = found ? sqrtf(bm) : __int_as_float(0x7fc00000);
                    if (P.pphi) P.pphi[row] = found ? P.phi32[bi] : __int_as_float(0x7fc00000);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// Per-LOS power-of-two exponent e such that 2^e * max |Q|,|U| over the
// contributing channels lies in [2^14, 2^15) (0 for an all-zero or non-finite row).
__global__ void row_exponent_kernel(const float *__restrict__ Q, const float *__restrict__ U, int64_t nlos,
                                    int32_t nchan, int32_t layout, const int32_t *__restrict__ active,
                                    int32_t nact, int8_t *__restrict__ rexp)
{
    if (layout == RMS_CHAN_MAJOR) {
        int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (l >= nlos) return;
        float mx = 0.f;
        for (int a = 0; a < nact; ++a) {
            int64_t off = (int64_t)__ldg(active + a) * nlos + l;
            mx = fmaxf(mx, fmaxf(fabsf(__ldg(Q + off)), fabsf(__ldg(U + off))));
        }
        int e = 0;
        if (mx > 0.f && isfinite(mx)) { frexpf(mx, &e); e = 15 - e; }
        rexp[l] = (int8_t)max(-100, min(100, e));
    } else {
        int64_t l = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
        int lane = threadIdx.x & 31;
        if (l >= nlos) return;
        float mx = 0.f;
        for (int a = lane; a < nact; a += 32) {
            int64_t off = l * nchan + __ldg(active + a);
            mx = fmaxf(mx, fmaxf(fabsf(__ldg(Q + off)), fabsf(__ldg(U + off))));
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            int e = 0;
            if (mx > 0.f && isfinite(mx)) { frexpf(mx, &e); e = 15 - e; }
            rexp[l] = (int8_t)max(-100, min(100, e));
        }
    }
}

size_t fixed_smem() { return 1024 + kEpiStageBytes + 2 * 4 * 32 * 8 + 8 * 32 + 32; }

bool encode_data_map(CUtensorMap *map, const float *base, int64_t nlos, int32_t nchan, int layout)
{
    if (reinterpret_cast<uintptr_t>(base) & 15) return false;
    cuuint64_t dims[2], strides[1];
    cuuint32_t box[2], estr[2] = {1, 1};
    CUtensorMapSwizzle sw;
    if (layout == RMS_CHAN_MAJOR) {
        if ((nlos * 4) % 16 != 0 || nlos < kTileM) return false;
        dims[0] = (cuuint64_t)nlos;
        dims[1] = (cuuint64_t)nchan;
        strides[0] = (cuuint64_t)nlos * 4;
        box[0] = kTileM;
        box[1] = 1;
        sw = CU_TENSOR_MAP_SWIZZLE_NONE;
    } else {
        if ((nchan * 4) % 16 != 0 || nchan < kChanPerKBlock) return false;
        dims[0] = (cuuint64_t)nchan;
        dims[1] = (cuuint64_t)nlos;
        strides[0] = (cuuint64_t)nchan * 4;
        box[0] = kChanPerKBlock;
        box[1] = kTileM;
        sw = CU_TENSOR_MAP_SWIZZLE_64B;
    }
    return encode_tensor_map(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, const_cast<float *>(base), dims, strides, box,
                             estr, sw);
}

}  // namespace

// Data and A rings of 3 stages each; the B ring takes the rest of shared memory.
int umma_bstages(int tile_n, int sd, int sa)
{
    size_t bst = 2 * (size_t)tile_n * kRowBytes;
    size_t avail = kSmemLimit - fixed_smem() - (size_t)sd * 2 * kStageD - (size_t)sa * 2 * kStageA - 8 * 2 * (sd + sa);
    int s = (int)(avail / (bst + 16));
    return s > 8 ? 8 : s;
}

size_t umma_smem_bytes(int tile_n, int sd, int sa, int sb)
{
    size_t bst = 2 * (size_t)tile_n * kRowBytes;
    return fixed_smem() + (size_t)sd * 2 * kStageD + (size_t)sa * 2 * kStageA + (size_t)sb * bst +
           8 * 2 * (size_t)(sd + sa + sb);
}

cudaError_t launch_row_exponent(const rms_plan_s &p, const float *Q, const float *U, int64_t nlos, int layout,
                                int8_t *rexp, cudaStream_t s)
{
    if (nlos <= 0) return cudaSuccess;
    int64_t threads = layout == RMS_CHAN_MAJOR ? nlos : nlos * 32;
    int64_t blocks = (threads + 255) / 256;
    row_exponent_kernel<<<(unsigned)blocks, 256, 0, s>>>(Q, U, nlos, p.nchan, layout, p.d_active, p.nact, rexp);
    return cudaGetLastError();
}

cudaError_t umma_prepare()
{
    // setmaxnreg moves registers between warpgroups inside the block's launch
    // allotment (512 threads x registers per thread); the split used here adds up
    // to exactly 512 x 128, so refuse any build whose kernel was not given 128.
    // cudaFuncGetAttributes also loads this file's module on the current device.
    cudaFuncAttributes fa, fr;
    cudaError_t e = cudaFuncGetAttributes(&fa, umma_synth_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fr, row_exponent_kernel);
    if (e != cudaSuccess) return e;
    return (fa.numRegs == 128 && 256 * (kRegsLow + kRegsHigh) == kThreads * 128) ? cudaSuccess
                                                                                : cudaErrorInvalidConfiguration;
}

cudaError_t launch_umma(const rms_plan_s &p, const float *Q, const float *U, int64_t nlos, int layout, float *F,
                        int32_t *pidx, float *pabs, float *pphi, const int8_t *rexp, cudaStream_t s)
{
    const cudaError_t reg_check = umma_prepare();
    if (reg_check != cudaSuccess) return reg_check;

    const bool chan = layout == RMS_CHAN_MAJOR;
    UmmaParams P;
    P.Q = Q;
    P.U = U;
    P.nlos = nlos;
    P.nchan = p.nchan;
    P.layout = layout;
    P.active = p.d_active;
    P.kbmask = p.d_kbmask;
    P.nk = chan ? p.nact : p.nchan;
    P.kblocks = chan ? p.kblocks : p.kblocks_raw;
    int ngroups = (P.kblocks + kUmmaGroupKBlocks - 1) / kUmmaGroupKBlocks;
    P.group = (P.kblocks + ngroups - 1) / ngroups;
    P.nphi = p.nphi;
    P.ntiles_n = p.ntiles_n;
    P.tile_n = p.tile_n;
    P.tile_n_last = p.tile_n_last;
    P.F = F;
    P.pidx = pidx;
    P.pabs = pabs;
    P.pphi = pphi;
    P.phi32 = p.d_phi32;
    P.out_scale = (float)(p.K * p.wmax);
    P.mode = p.precision == RMS_BF16 ? MODE_BF16 : (p.precision == RMS_BF16X3 ? MODE_BF16X3 : MODE_FP16X3);
    P.rexp = P.mode == MODE_FP16X3 ? rexp : nullptr;
    P.err = p.d_err;
    P.timeout_ns = p.timeout_ns;
    P.scratch = reinterpret_cast<uint4 *>(p.d_scratch);

    CUtensorMap tq, tu;
    std::memset(&tq, 0, sizeof(tq));
    std::memset(&tu, 0, sizeof(tu));
    // TMA staging of the FP32 data needs 16-byte aligned bases and rows; otherwise
    // the converters load it directly from global memory
    P.use_tma = encode_data_map(&tq, Q, nlos, p.nchan, layout) && encode_data_map(&tu, U, nlos, p.nchan, layout);
    P.sd = P.use_tma ? 3 : 0;
    P.sa = 3;
    P.sb = umma_bstages(p.tile_n, P.sd, P.sa);
    // Reloading from scratch is safe when a converter's write of K block kb for the
    // next M tile is ordered after the bulk copy that last read it: the converter
    // waits for the A slot used sa stages earlier, which is at or after that copy's
    // stage when kblocks >= sa.
    P.reuse = (p.ntiles_n > 1 && P.kblocks >= P.sa && p.d_scratch != nullptr) ? 1 : 0;
    if (P.sb < 2) return cudaErrorInvalidConfiguration;
    size_t smem = umma_smem_bytes(p.tile_n, P.sd, P.sa, P.sb);
    cudaError_t e = cudaFuncSetAttribute(umma_synth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t nmt = (nlos + kTileM - 1) / kTileM;
    int grid = (int)(nmt < p.num_sms ? nmt : p.num_sms);
    if (grid < 1) return cudaSuccess;
    umma_synth_kernel<<<grid, kThreads, smem, s>>>(P, chan ? p.tmap_bhi : p.tmap_bhi_raw,
                                                    chan ? p.tmap_blo : p.tmap_blo_raw, tq, tu);
    return cudaGetLastError();
}
