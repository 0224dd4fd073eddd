// Tensor-core RM synthesis for sm_103a: tcgen05.mma with TMEM accumulators,
// phase matrix streamed by TMA, data converted to split 16-bit operands on the fly.
//
// The synthesis of Eq. Fsum in its real form (Eqs. qPhi, uPhi) is a real GEMM
//     C[l][2k + {0,1}] = sum_a ( Q_la * B[2k+{0,1}][2a] + U_la * B[2k+{0,1}][2a+1] )
// with the phase block B = (w_a / w_max) [[c, s], [-s, c]] built at plan time in
// FP64 (phase.cu), so C[l] is F(phi) as interleaved complex64, up to the factor
// K w_max applied in the epilogue.  M = lines of sight, N = 2 nphi,
// K = 2 * active channels.
//
// Precision: A (data) and B (phase) are each split into hi + lo 16-bit parts and
// three products hi*hi + hi*lo + lo*hi are accumulated in FP32 in TMEM
// (BF16X3, FP16X3), or only hi*hi (BF16).  FP16 data are scaled per line of
// sight by a power of two so that their largest value lies in [2^14, 2^15).
//
// CTA = 14 warps, persistent over 128-row M tiles; each M tile runs all its N
// tiles in order so the epilogue can keep each row's running peak in registers.
//   warp 0      : TMA producer of the B tiles (hi, lo)              -> fullB[s]
//   warp 1      : TMEM allocator and single-thread MMA issuer         -> empty[s], tfull[b]
//   warps 2..5  : epilogue, one TMEM lane quarter each               -> tempty[b]
//   warps 6..13 : converters: FP32 Q/U (either cube layout, flagged
//                 channels skipped) -> split 16-bit A tile in the
//                 64-byte-swizzled K-major layout the MMA reads      -> fullA[s]
// Every mbarrier wait is bounded by a wall-clock limit; a wait that runs out
// raises a CTA-wide abort flag and the device error word, every role leaves its
// loop, in-flight TMA copies and MMAs are drained with bounded waits, and TMEM
// is freed before the CTA exits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <limits.h>

#include "rms_internal.h"

namespace {

constexpr int kNumConvWarps = 8;
constexpr int kNumEpiWarps = 4;
constexpr int kFirstEpiWarp = 2;
constexpr int kFirstConvWarp = kFirstEpiWarp + kNumEpiWarps;
constexpr int kThreads = 32 * (kFirstConvWarp + kNumConvWarps);   // 448
constexpr int kRowBytes = kKBlock * 2;                            // 64 B per row per stage
constexpr int kStageA = kTileM * kRowBytes;                       // 8 KB per A part
constexpr int kTmemCols = 512;
constexpr int kAccStride = 256;                                   // TMEM columns per accumulator
constexpr int kEpiLd = 33;                                        // epilogue staging row pitch (floats)
constexpr int kEpiStageBytes = kNumEpiWarps * 32 * kEpiLd * 4;
constexpr int kCvtLd = 17;
constexpr int kCvtStageBytes = kNumConvWarps * 2 * 16 * kCvtLd * 4;
constexpr int kSmemLimit = 227 * 1024;

enum { MODE_BF16 = 0, MODE_BF16X3 = 1, MODE_FP16X3 = 2 };

struct UmmaParams {
    const float *Q, *U;
    int64_t nlos;
    int32_t nchan, layout;
    const int32_t *active;
    int32_t nact, kblocks;
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
    int32_t stages;
};

// ----------------------------------------------------------------------------
// PTX wrappers
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity.  Returns false when the CTA has been
// aborted or when this wait exceeded the time limit (which then aborts the CTA
// and records the timeout in the device error word).
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                             int *err, int64_t limit_ns, bool honour_abort = true)
{
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_ns();
    while (true) {
#pragma unroll 1
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (honour_abort && *abort_flag) return false;
        if ((int64_t)(global_ns() - t0) > limit_ns) {
            *abort_flag = 1;
            atomicExch(err, RMS_DEVERR_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor for a K-major operand in the 64-byte swizzle
// layout: rows of 64 bytes, 8-row groups 512 bytes apart (stride byte offset),
// leading byte offset unused for swizzled K-major (encoded as 1), descriptor
// version 1 (bits 46-47), swizzle mode 4 = 64B (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_k64(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A/B type
// (bits 7-9, 10-12: 0 = F16, 1 = BF16), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t idesc_f16(int n, bool bf16)
{
    uint32_t ab = bf16 ? 1u : 0u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, float (&v)[32])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
#pragma unroll
    for (int i = 16; i < 32; ++i) v[i] = 0.f;
}

// ----------------------------------------------------------------------------
// Converter: split one value into hi + lo 16-bit parts (bits returned).
// ----------------------------------------------------------------------------
__device__ __forceinline__ void split_bf16(float x, uint32_t &hi, uint32_t &lo)
{
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = (uint32_t)__bfloat16_as_ushort(h);
    lo = (uint32_t)__bfloat16_as_ushort(l);
}

__device__ __forceinline__ void split_fp16(float x, uint32_t &hi, uint32_t &lo)
{
    __half h = __float2half_rn(x);
    __half l = __float2half_rn(x - __half2float(h));
    hi = (uint32_t)__half_as_ushort(h);
    lo = (uint32_t)__half_as_ushort(l);
}

// Convert 8 channels (Q, U interleaved -> 16 K values) of one A row and store the
// two 16-byte chunks of the hi part (and of the lo part) into the swizzled tile.
// Row m, chunk c of a 64-byte-swizzled K-major tile lives at
//   m * 64 + ((c ^ ((m >> 1) & 3)) << 4).
__device__ __forceinline__ void convert_store(const float (&q)[8], const float (&u)[8], float scale, int mode,
                                              uint8_t *a_hi, uint8_t *a_lo, int m, int h)
{
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        uint32_t qh, ql, uh, ul;
        if (mode == MODE_FP16X3) {
            split_fp16(q[i] * scale, qh, ql);
            split_fp16(u[i] * scale, uh, ul);
        } else {
            split_bf16(q[i], qh, ql);
            split_bf16(u[i], uh, ul);
        }
        hi[i] = qh | (uh << 16);
        lo[i] = ql | (ul << 16);
    }
    const int sw = (m >> 1) & 3;
    const uint32_t off0 = (uint32_t)m * kRowBytes + ((uint32_t)((2 * h) ^ sw) << 4);
    const uint32_t off1 = (uint32_t)m * kRowBytes + ((uint32_t)((2 * h + 1) ^ sw) << 4);
    *reinterpret_cast<uint4 *>(a_hi + off0) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4 *>(a_hi + off1) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
    if (mode != MODE_BF16) {
        *reinterpret_cast<uint4 *>(a_lo + off0) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        *reinterpret_cast<uint4 *>(a_lo + off1) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
    }
}

__device__ __forceinline__ float row_scale_up(const int8_t *rexp, int64_t row, int64_t nlos)
{
    if (rexp == nullptr || row >= nlos) return 1.0f;
    return ldexpf(1.0f, (int)rexp[row]);
}

// ----------------------------------------------------------------------------
// The kernel
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1)
umma_synth_kernel(const __grid_constant__ UmmaParams P, const __grid_constant__ CUtensorMap tmB_hi,
                  const __grid_constant__ CUtensorMap tmB_lo)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);

    const int S = P.stages;
    const int tile_n = P.tile_n;
    const uint32_t b_bytes = (uint32_t)tile_n * kRowBytes;
    const uint32_t stage_bytes = 2 * kStageA + 2 * b_bytes;
    float *epi_stage = reinterpret_cast<float *>(smem + (size_t)S * stage_bytes);
    float *cvt_stage = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(epi_stage) + kEpiStageBytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(cvt_stage) + kCvtStageBytes);
    uint64_t *fullA = bars, *fullB = bars + S, *empty = bars + 2 * S;
    uint64_t *tfull = bars + 3 * S, *tempty = tfull + 2, *mma_done = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nmt = (P.nlos + kTileM - 1) / kTileM;
    const bool split = P.mode != MODE_BF16;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&fullA[s]), kNumConvWarps);
            mbar_init(smem_u32(&fullB[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), kNumEpiWarps);
        }
        mbar_init(smem_u32(mma_done), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB_hi)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB_lo)) : "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA producer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, pending = 0, pend_par = 0;
            const uint32_t tx = split ? 2 * b_bytes : b_bytes;
            bool ok = true;
            for (int64_t mt = blockIdx.x; mt < nmt && ok; mt += gridDim.x)
                for (int nt = 0; nt < P.ntiles_n && ok; ++nt)
                    for (int kb = 0; kb < P.kblocks; ++kb) {
                        if (!wait_bounded(smem_u32(&empty[s]), ph ^ 1, abort_flag, P.err, P.timeout_ns)) {
                            ok = false;
                            break;
                        }
                        uint8_t *st = smem + (size_t)s * stage_bytes;
                        mbar_arrive_expect_tx(smem_u32(&fullB[s]), tx);
                        tma_load_2d(smem_u32(st + 2 * kStageA), &tmB_hi, kb * kKBlock, nt * tile_n,
                                    smem_u32(&fullB[s]));
                        if (split)
                            tma_load_2d(smem_u32(st + 2 * kStageA + b_bytes), &tmB_lo, kb * kKBlock,
                                        nt * tile_n, smem_u32(&fullB[s]));
                        pending |= 1u << s;
                        pend_par = (pend_par & ~(1u << s)) | (ph << s);
                        if (++s == S) { s = 0; ph ^= 1; }
                    }
            if (!ok) {
                // drain: every TMA copy still in flight must land before the CTA exits
                for (int i = 0; i < S; ++i)
                    if (pending & (1u << i))
                        wait_bounded(smem_u32(&fullB[i]), (pend_par >> i) & 1, abort_flag, P.err, P.timeout_ns,
                                     false);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id_full = idesc_f16(tile_n, P.mode != MODE_FP16X3);
            const uint32_t id_last = idesc_f16(P.tile_n_last, P.mode != MODE_FP16X3);
            int s = 0;
            uint32_t ph = 0, tph0 = 0, tph1 = 0;
            int t = 0;
            bool ok = true, issued = false;
            for (int64_t mt = blockIdx.x; mt < nmt && ok; mt += gridDim.x)
                for (int nt = 0; nt < P.ntiles_n && ok; ++nt, ++t) {
                    const int buf = t & 1;
                    if (!wait_bounded(smem_u32(&tempty[buf]), (buf ? tph1 : tph0) ^ 1, abort_flag, P.err,
                                      P.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + (uint32_t)(buf * kAccStride);
                    const uint32_t idesc = (nt == P.ntiles_n - 1) ? id_last : id_full;
                    for (int kb = 0; kb < P.kblocks; ++kb) {
                        if (!wait_bounded(smem_u32(&fullA[s]), ph, abort_flag, P.err, P.timeout_ns) ||
                            !wait_bounded(smem_u32(&fullB[s]), ph, abort_flag, P.err, P.timeout_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
                        const uint32_t a_hi = st, a_lo = st + kStageA;
                        const uint32_t b_hi = st + 2 * kStageA, b_lo = b_hi + b_bytes;
#pragma unroll
                        for (int kk = 0; kk < kKBlock / 16; ++kk) {
                            const uint32_t ko = kk * 32;   // 16 K values = 32 bytes along the row
                            const uint32_t acc = (kb | kk) ? 1u : 0u;
                            mma_f16(d, sdesc_k64(a_hi + ko), sdesc_k64(b_hi + ko), idesc, acc);
                            if (split) {
                                mma_f16(d, sdesc_k64(a_hi + ko), sdesc_k64(b_lo + ko), idesc, 1u);
                                mma_f16(d, sdesc_k64(a_lo + ko), sdesc_k64(b_hi + ko), idesc, 1u);
                            }
                        }
                        issued = true;
                        mma_commit(smem_u32(&empty[s]));
                        if (++s == S) { s = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    mma_commit(smem_u32(&tfull[buf]));
                    if (buf) tph1 ^= 1; else tph0 ^= 1;
                }
            if (issued) {
                // all MMAs of this thread complete before TMEM is released
                mma_commit(smem_u32(mma_done));
                wait_bounded(smem_u32(mma_done), 0, abort_flag, P.err, P.timeout_ns, false);
            }
        }
    } else if (warp < kFirstConvWarp) {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;                       // TMEM lane quarter this warp may access
        float *stg = epi_stage + (warp - kFirstEpiWarp) * 32 * kEpiLd;
        const int64_t row_pitch = 2 * (int64_t)P.nphi;
        uint32_t tph0 = 0, tph1 = 0;
        int t = 0;
        bool ok = true;
        for (int64_t mt = blockIdx.x; mt < nmt && ok; mt += gridDim.x) {
            const int64_t row = mt * kTileM + 32 * q + lane;
            float scale = P.out_scale;
            if (P.rexp != nullptr && row < P.nlos) scale = ldexpf(scale, -(int)P.rexp[row]);
            float bm = -1.0f;
            int bi = INT_MAX;
            for (int nt = 0; nt < P.ntiles_n; ++nt, ++t) {
                const int buf = t & 1;
                bool w = wait_bounded(smem_u32(&tfull[buf]), buf ? tph1 : tph0, abort_flag, P.err, P.timeout_ns);
                if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                if (buf) tph1 ^= 1; else tph0 ^= 1;
                tc_fence_after();
                const int ncols = (nt == P.ntiles_n - 1) ? P.tile_n_last : tile_n;
                const int64_t col0 = (int64_t)nt * tile_n;         // first C column of this tile
                for (int c = 0; c < ncols; c += 32) {
                    float v[32];
                    const uint32_t taddr = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * kAccStride + c);
                    if (ncols - c >= 32) tmem_ld_x32(taddr, v);
                    else tmem_ld_x16(taddr, v);
                    const int kbase = (int)((col0 + c) >> 1);      // phi index of v[0]
#pragma unroll
                    for (int p = 0; p < 16; ++p) {
                        const float fr = v[2 * p] * scale, fi = v[2 * p + 1] * scale;
                        v[2 * p] = fr;
                        v[2 * p + 1] = fi;
                        const int k = kbase + p;
                        if (2 * p < ncols - c && k < P.nphi) {
                            const float m2 = __fadd_rn(__fmul_rn(fr, fr), __fmul_rn(fi, fi));
                            if (m2 > bm) { bm = m2; bi = k; }
                        }
                    }
                    if (P.F != nullptr) {
                        // transpose through shared memory: each store instruction then
                        // writes two contiguous 128-byte row segments
#pragma unroll
                        for (int j = 0; j < 32; ++j) stg[lane * kEpiLd + j] = v[j];
                        __syncwarp();
                        const int jj = (lane & 15) * 2;
                        const int kk = kbase + (lane & 15);
#pragma unroll 4
                        for (int it = 0; it < 16; ++it) {
                            const int r = 2 * it + (lane >> 4);
                            const int64_t grow = mt * kTileM + 32 * q + r;
                            if (grow < P.nlos && jj < ncols - c && kk < P.nphi) {
                                float2 val = make_float2(stg[r * kEpiLd + jj], stg[r * kEpiLd + jj + 1]);
                                *reinterpret_cast<float2 *>(P.F + grow * row_pitch + col0 + c + jj) = val;
                            }
                        }
                        __syncwarp();
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[buf]));
            }
            if (!ok) break;
            if (row < P.nlos) {
                const bool found = bi != INT_MAX;
                if (P.pidx) P.pidx[row] = found ? bi : -1;
                if (P.pabs) P.pabs[row] = found ? sqrtf(bm) : __int_as_float(0x7fc00000);
                if (P.pphi) P.pphi[row] = found ? P.phi32[bi] : __int_as_float(0x7fc00000);
            }
        }
    } else {
        // ------------------------------------------------------------ converters
        const int cw = warp - kFirstConvWarp;         // 0..7
        const int ct = threadIdx.x - 32 * kFirstConvWarp;   // 0..255
        float *cq = cvt_stage + cw * (2 * 16 * kCvtLd);
        float *cu = cq + 16 * kCvtLd;
        int s = 0;
        uint32_t ph = 0;
        bool ok = true;
        for (int64_t mt = blockIdx.x; mt < nmt && ok; mt += gridDim.x)
            for (int nt = 0; nt < P.ntiles_n && ok; ++nt)
                for (int kb = 0; kb < P.kblocks; ++kb) {
                    float q[8], u[8];
                    int m, h;
                    const int a0 = kb * kChanPerKBlock;
                    if (P.layout == RMS_CHAN_MAJOR) {
                        // thread -> (row m, 8 channels): lanes run along LOS, loads coalesce
                        m = ct & 127;
                        h = ct >> 7;
                        const int64_t row = mt * kTileM + m;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int a = a0 + 8 * h + i;
                            q[i] = 0.f;
                            u[i] = 0.f;
                            if (a < P.nact && row < P.nlos) {
                                const int64_t off = (int64_t)__ldg(P.active + a) * P.nlos + row;
                                q[i] = __ldg(P.Q + off);
                                u[i] = __ldg(P.U + off);
                            }
                        }
                    } else {
                        // lanes run along channels of two rows at a time; transpose via smem
                        const int rr = lane >> 4, c = lane & 15;
                        const int a = a0 + c;
                        const int64_t choff = a < P.nact ? __ldg(P.active + a) : 0;
#pragma unroll
                        for (int it = 0; it < 8; ++it) {
                            const int64_t row = mt * kTileM + 16 * cw + 2 * it + rr;
                            q[it] = 0.f;
                            u[it] = 0.f;
                            if (a < P.nact && row < P.nlos) {
                                q[it] = __ldg(P.Q + row * P.nchan + choff);
                                u[it] = __ldg(P.U + row * P.nchan + choff);
                            }
                        }
                        m = 16 * cw + (lane & 15);
                        h = lane >> 4;
                    }
                    bool w = wait_bounded(smem_u32(&empty[s]), ph ^ 1, abort_flag, P.err, P.timeout_ns);
                    if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                    if (P.layout != RMS_CHAN_MAJOR) {
                        const int rr = lane >> 4, c = lane & 15;
#pragma unroll
                        for (int it = 0; it < 8; ++it) {
                            cq[(2 * it + rr) * kCvtLd + c] = q[it];
                            cu[(2 * it + rr) * kCvtLd + c] = u[it];
                        }
                        __syncwarp();
                        const int r = lane & 15;
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            q[i] = cq[r * kCvtLd + 8 * h + i];
                            u[i] = cu[r * kCvtLd + 8 * h + i];
                        }
                    }
                    const float sc = (P.mode == MODE_FP16X3) ? row_scale_up(P.rexp, mt * kTileM + m, P.nlos) : 1.0f;
                    uint8_t *st = smem + (size_t)s * stage_bytes;
                    convert_store(q, u, sc, P.mode, st, st + kStageA, m, h);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&fullA[s]));
                    if (++s == S) { s = 0; ph ^= 1; }
                }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// Per-LOS power-of-two exponent e such that 2^e * max |Q|,|U| over the active
// channels lies in [2^14, 2^15) (0 for an all-zero or non-finite row).
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

}  // namespace

int umma_stages(int tile_n)
{
    size_t stage = 2 * (size_t)kStageA + 2 * (size_t)tile_n * kRowBytes;
    size_t fixed = 1024 + kEpiStageBytes + kCvtStageBytes + 8 * (3 * 8 + 5) + 16;
    int s = (int)((kSmemLimit - fixed) / stage);
    return s > 6 ? 6 : s;
}

size_t umma_smem_bytes(int tile_n, int stages)
{
    size_t stage = 2 * (size_t)kStageA + 2 * (size_t)tile_n * kRowBytes;
    return 1024 + stages * stage + kEpiStageBytes + kCvtStageBytes + 8 * (3 * stages + 5) + 16;
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

cudaError_t launch_umma(const rms_plan_s &p, const float *Q, const float *U, int64_t nlos, int layout, float *F,
                        int32_t *pidx, float *pabs, float *pphi, const int8_t *rexp, cudaStream_t s)
{
    UmmaParams P;
    P.Q = Q;
    P.U = U;
    P.nlos = nlos;
    P.nchan = p.nchan;
    P.layout = layout;
    P.active = p.d_active;
    P.nact = p.nact;
    P.kblocks = p.kblocks;
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
    P.stages = umma_stages(p.tile_n);
    size_t smem = umma_smem_bytes(p.tile_n, P.stages);
    cudaError_t e = cudaFuncSetAttribute(umma_synth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t nmt = (nlos + kTileM - 1) / kTileM;
    int grid = (int)(nmt < p.num_sms ? nmt : p.num_sms);
    if (grid < 1) return cudaSuccess;
    umma_synth_kernel<<<grid, kThreads, smem, s>>>(P, p.tmap_bhi, p.tmap_blo);
    return cudaGetLastError();
}
