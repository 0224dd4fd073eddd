// The learned peak proposal's network: a two-layer perceptron on one line of
// sight's Q/U spectrum that proposes the bin of the phi grid holding max |F|.
// Nothing here is in the paper.
//
//   x = [Q_a0, U_a0, Q_a1, U_a1, ...] / s   (active channels; s = RMS of |P|)
//   h = relu(W1 x + b1),  z = W2 h + b2,  loss = mean -log softmax(z)[label]
//
// Every product runs in one tcgen05 kernel, net_gemm_kernel: C[M][N] = A[M][K]
// B[N][K]^T with BF16 operands staged by TMA in the 64-byte swizzle (or, for the
// first layer, bulk copies of the split operand image that the synthesis path
// writes: its hi parts are BF16 Q/U in exactly the interleaved column order
// above), FP32 accumulators in TMEM and one of four fused epilogues:
//   RELU     h = relu(acc * rowscale + b) -> BF16 h (and h^T for training)
//   SOFTMAX  z = acc + b over the whole row (<= 512 bins in one tile): argmax,
//            softmax, confidence = mass within a window of bins; with labels the
//            cross-entropy and dz = (softmax - onehot) / batch in BF16 (row- and
//            column-major) and FP32
//   DRELU    da = acc * [h > 0] -> BF16 (da * rowscale)^T and FP32 da
//   ACC      split-K partial sums added into FP32 gradients (optionally through a
//            column map from image columns to weight columns)
//   warp 0      TMA / bulk producer                        -> full
//   warp 1      TMEM allocator, single-thread MMA issuer   -> empty, tfull
//   warps 4-11  epilogue: warp w owns TMEM lane quarter w % 4 and column half
//               (w - 4) / 4 of each accumulator row          -> tempty
// Every wait is bounded (abort flag, device error word, drain, TMEM freed).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "rms_internal.h"

namespace {

#include "tc_ptx.cuh"

typedef __nv_bfloat16 bf16;

enum { EPI_RELU = 0, EPI_SOFTMAX = 1, EPI_DRELU = 2, EPI_ACC = 3 };
constexpr int kNetThreads = 384;
constexpr int kNetEpiWarp0 = 4;    // warps 4-11: two per TMEM lane quarter, one per column half
constexpr int kNetTmemCols = 512;
constexpr int kNetStageA = kTileM * 64;       // 8 KB: 128 rows x 32 BF16
constexpr int kImageKBlockBytes = 2 * kNetStageA;   // split image: hi then lo per K block
constexpr int kNetSmemLimit = 227 * 1024;
constexpr int kNetXchFloats = 4 * kTileM;     // (max, sum, argmax, z_label) per row
constexpr int kNetBiasMax = 512;               // bias staged in shared memory (N <= 512 when a bias is used)
constexpr int kNetFixedSmem = 1024 + 256 + (kNetXchFloats + kNetBiasMax) * 4;

struct NetGemmParams {
    int32_t M, N, kblocks, kb_per_split, ksplit, mtiles, ntiles;
    int32_t BN, tile_n, nsub, nbuf, stages, epi;
    const uint8_t *a_image;     // non-null: A = hi parts of a split image, [mtiles][a_image_kb][16 KB]
    int32_t a_image_kb;
    const float *row_scale;     // [M] or null
    const float *bias;          // [N] or null
    bf16 *out;
    int64_t ldo;
    bf16 *outT;
    int64_t ldt;
    float *outf;
    int64_t ldf;
    const bf16 *hmask;
    int64_t ldh;
    const int32_t *colmap;
    const int32_t *label;
    int32_t *bin;
    float *conf;
    int32_t halfwin;
    float *loss;
    float inv_batch;
    int *err;
    int64_t timeout_ns;
};

struct NSmem {
    uint8_t *ring;
    uint32_t stage_bytes;
    uint64_t *full, *empty, *tfull, *tempty, *mma_done;
    uint32_t *tmem_slot;
    volatile int *abort_flag;
    float *xch;                 // softmax: per-row values exchanged between the two column halves
};

__device__ __forceinline__ NSmem ncarve(uint8_t *base, const NetGemmParams &P)
{
    NSmem s;
    s.stage_bytes = kNetStageA + (uint32_t)P.BN * 64;
    s.ring = base;
    uint64_t *b = reinterpret_cast<uint64_t *>(base + (size_t)P.stages * s.stage_bytes);
    s.full = b;
    s.empty = s.full + P.stages;
    s.tfull = s.empty + P.stages;
    s.tempty = s.tfull + 2;
    s.mma_done = s.tempty + 2;
    s.tmem_slot = reinterpret_cast<uint32_t *>(s.mma_done + 1);
    s.abort_flag = reinterpret_cast<volatile int *>(s.tmem_slot + 1);
    s.xch = reinterpret_cast<float *>(const_cast<int *>(s.abort_flag) + 2);
    return s;
}

__device__ __forceinline__ void item_coords(const NetGemmParams &P, int64_t it, int &mt, int &nt, int &kb0, int &kb1)
{
    const int ks = (int)(it % P.ksplit);
    const int64_t t = it / P.ksplit;
    nt = (int)(t % P.ntiles);
    mt = (int)(t / P.ntiles);
    kb0 = ks * P.kb_per_split;
    kb1 = min(P.kblocks, kb0 + P.kb_per_split);
}

// 32 accumulator columns of this thread's row, starting at column c0 (fewer before column end).
__device__ __forceinline__ void load32(uint32_t taddr, int c0, int end, float (&v)[32])
{
    uint32_t r[4][8];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (c0 + 8 * j < end) tmem_ld8(taddr + c0 + 8 * j, r[j]);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 8; ++e) v[8 * j + e] = (c0 + 8 * j < end) ? __uint_as_float(r[j][e]) : 0.f;
}

// The two warps that share a TMEM lane quarter (64 threads, named barrier 1 + q).
__device__ __forceinline__ void pair_sync(int q) { asm volatile("bar.sync %0, 64;" ::"r"(1 + q) : "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// One accumulator row per thread; the warp pair of a lane quarter splits the
// columns in halves [c_lo, c_hi).  bias_s: the bias in shared memory.
template <int EPI>
__device__ void epilogue(const NetGemmParams &P, const NSmem &SM, const float *bias_s, uint32_t tacc, int mt, int nt,
                         int q, int h, int lane)
{
    const int r = 32 * q + lane;
    const int64_t m = (int64_t)mt * kTileM + r;
    const bool valid = m < P.M;
    const float rs = (P.row_scale && valid) ? P.row_scale[m] : 1.0f;
    const int n_base = nt * P.BN;
    const int half = P.BN / 2;
    const int c_lo = h * half, c_hi = c_lo + half;
    float v[32];
    if constexpr (EPI != EPI_SOFTMAX) {
        for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
            load32(tacc, c0, c_hi, v);
            if (!valid) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n0 = n_base + c0 + 8 * j;
                if (c0 + 8 * j >= c_hi || n0 >= P.N) continue;
                if constexpr (EPI == EPI_RELU) {
                    float o[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int n = n0 + e;
                        o[e] = n < P.N ? fmaxf(fmaf(v[8 * j + e], rs, bias_s ? bias_s[n] : 0.f), 0.f) : 0.f;
                    }
                    if (n0 + 8 <= P.N) {
                        *reinterpret_cast<uint4 *>(P.out + m * P.ldo + n0) =
                            make_uint4(pack_bf16(o[0], o[1]), pack_bf16(o[2], o[3]), pack_bf16(o[4], o[5]),
                                       pack_bf16(o[6], o[7]));
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (n0 + e < P.N) P.out[m * P.ldo + n0 + e] = __float2bfloat16_rn(o[e]);
                    }
                    if (P.outT) {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (n0 + e < P.N) P.outT[(int64_t)(n0 + e) * P.ldt + m] = __float2bfloat16_rn(o[e]);
                    }
                } else if constexpr (EPI == EPI_DRELU) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int n = n0 + e;
                        if (n >= P.N) continue;
                        const float hv = __bfloat162float(P.hmask[m * P.ldh + n]);
                        const float da = hv > 0.f ? v[8 * j + e] : 0.f;
                        P.outT[(int64_t)n * P.ldt + m] = __float2bfloat16_rn(da * rs);
                        P.outf[m * P.ldf + n] = da;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int n = n0 + e;
                        if (n >= P.N) continue;
                        const int col = P.colmap ? P.colmap[n] : n;
                        if (col >= 0) atomicAdd(P.outf + m * P.ldf + col, v[8 * j + e]);
                    }
                }
            }
        }
        return;
    } else {
        // One pass per half: running max, argmax (lowest index on ties) and the sum
        // of exp(z - max), rescaled once per 32-column chunk; the halves then combine
        // through shared memory.  Missing columns read as -inf (exp gives 0).
        const bool train = P.label != nullptr;
        const int y = (train && valid) ? P.label[m] : -1;
        const int lim = min(c_hi, P.N);
        float mx = -INFINITY, S = 0.f, zy = 0.f;
        int bi = -1;
        for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
            load32(tacc, c0, c_hi, v);
            float cm = -INFINITY;
            int ci = -1;
            if (c0 + 32 <= lim) {
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const float z = v[e] + bias_s[c0 + e];
                    v[e] = z;
                    if (z > cm) { cm = z; ci = c0 + e; }
                }
            } else {
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const float z = c0 + e < lim ? v[e] + bias_s[c0 + e] : -INFINITY;
                    v[e] = z;
                    if (z > cm) { cm = z; ci = c0 + e; }
                }
            }
            if (train) {
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    if (c0 + e == y) zy = v[e];
            } else if (P.outf && valid) {
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    if (c0 + e < lim) P.outf[m * P.ldf + c0 + e] = v[e];
            }
            if (cm > mx) {
                S *= __expf(mx - cm);
                mx = cm;
                bi = ci;
            }
            if (mx > -INFINITY) {
#pragma unroll
                for (int e = 0; e < 32; ++e) S += __expf(v[e] - mx);
            }
        }
        float *X = SM.xch;   // [4][128]: max, sum, argmax, z_label
        if (h == 1) {
            X[r] = mx;
            X[kTileM + r] = S;
            X[2 * kTileM + r] = __int_as_float(bi);
            X[3 * kTileM + r] = zy;
        }
        pair_sync(q);
        if (h == 0) {
            const float m1 = X[r], s1 = X[kTileM + r], z1 = X[3 * kTileM + r];
            const int b1 = __float_as_int(X[2 * kTileM + r]);
            const float M = fmaxf(mx, m1);
            const float St =
                (mx > -INFINITY ? S * __expf(mx - M) : 0.f) + (m1 > -INFINITY ? s1 * __expf(m1 - M) : 0.f);
            if (m1 > mx) bi = b1;
            if (y >= c_hi) zy = z1;
            mx = M;
            S = St;
            X[r] = mx;
            X[kTileM + r] = S;
            X[2 * kTileM + r] = __int_as_float(bi);
        }
        pair_sync(q);
        if (h == 1) {
            mx = X[r];
            S = X[kTileM + r];
            bi = __float_as_int(X[2 * kTileM + r]);
        }
        // window mass: columns within halfwin of the argmax that lie in this half.  The
        // TMEM loads are warp-collective (.sync.aligned), so every lane walks the same
        // 8-column groups -- those that meet any lane's window -- and masks its own.
        float Sw = 0.f;
        if (P.halfwin >= 0) {
            const bool has = bi >= 0;
            const int w0 = has ? max(c_lo, bi - P.halfwin) : c_hi;
            const int w1 = has ? min(lim, bi + P.halfwin + 1) : c_lo;
            int g0 = w0, g1 = w1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                g0 = min(g0, __shfl_xor_sync(0xffffffffu, g0, o));
                g1 = max(g1, __shfl_xor_sync(0xffffffffu, g1, o));
            }
            for (int c0 = g0 & ~7; c0 < g1; c0 += 8) {
                uint32_t rr[8];
                tmem_ld8(tacc + c0, rr);
                tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int n = c0 + e;
                    if (n >= w0 && n < w1) Sw += __expf(__uint_as_float(rr[e]) + bias_s[n] - mx);
                }
            }
        }
        pair_sync(q);
        if (h == 1) X[r] = Sw;
        pair_sync(q);
        if (h == 0) {
            Sw += X[r];
            if (valid) {
                if (P.bin) P.bin[m] = max(bi, 0);
                if (P.conf) P.conf[m] = P.halfwin >= 0 ? Sw / S : 1.0f / S;
            }
            if (train) {
                float lrow = valid ? (logf(S) + mx - zy) : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) lrow += __shfl_xor_sync(0xffffffffu, lrow, o);
                if (lane == 0 && P.loss) atomicAdd(P.loss, lrow * P.inv_batch);
            }
        }
        pair_sync(q);   // the exchange buffer is reused by the next tile
        if (!train) return;
        const float invS = 1.0f / S;
        for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
            load32(tacc, c0, c_hi, v);
            if (!valid) continue;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int n = c0 + e;
                if (n < lim) {
                    const float z = v[e] + bias_s[n];
                    const float d = (__expf(z - mx) * invS - (n == y ? 1.f : 0.f)) * P.inv_batch;
                    P.out[m * P.ldo + n] = __float2bfloat16_rn(d);
                    P.outT[(int64_t)n * P.ldt + m] = __float2bfloat16_rn(d);
                    P.outf[m * P.ldf + n] = d;
                }
            }
        }
    }
}

template <int EPI>
__global__ void __launch_bounds__(kNetThreads, 1)
net_gemm_kernel(const __grid_constant__ NetGemmParams P, const __grid_constant__ CUtensorMap tmA,
                const __grid_constant__ CUtensorMap tmB)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const NSmem S = ncarve(base, P);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t items = (int64_t)P.mtiles * P.ntiles * P.ksplit;

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.stages; ++s) {
            mbar_init(smem_u32(&S.full[s]), 1);
            mbar_init(smem_u32(&S.empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&S.tfull[b]), 1);
            mbar_init(smem_u32(&S.tempty[b]), 8);
        }
        mbar_init(smem_u32(S.mma_done), 1);
        *S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        __syncwarp();
        tmem_alloc(smem_u32(S.tmem_slot), kNetTmemCols);
    }
    float *bias_s = nullptr;
    if (P.bias && P.N <= kNetBiasMax) {
        bias_s = S.xch + kNetXchFloats;
        for (int i = threadIdx.x; i < P.N; i += blockDim.x) bias_s[i] = P.bias[i];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *S.tmem_slot;
    const uint32_t b_bytes = (uint32_t)P.tile_n * 64;

    if (warp == 0) {
        if (lane == 0) {
            if (!P.a_image) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            const uint32_t tx = kNetStageA + (uint32_t)P.nsub * b_bytes;
            int s = 0;
            uint32_t ph = 0, pending = 0, pend_par = 0;
            bool ok = true;
            for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
                int mt, nt, kb0, kb1;
                item_coords(P, it, mt, nt, kb0, kb1);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!wait_bounded(smem_u32(&S.empty[s]), ph ^ 1, S.abort_flag, P.err, P.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = smem_u32(S.ring + (size_t)s * S.stage_bytes);
                    const uint32_t bar = smem_u32(&S.full[s]);
                    mbar_arrive_expect_tx(bar, tx);
                    if (P.a_image)
                        bulk_load(st, P.a_image + ((size_t)mt * P.a_image_kb + kb) * kImageKBlockBytes, kNetStageA,
                                  bar);
                    else
                        tma_load_2d(st, &tmA, kb * kKBlock, mt * kTileM, bar);
                    for (int j = 0; j < P.nsub; ++j)
                        tma_load_2d(st + kNetStageA + j * b_bytes, &tmB, kb * kKBlock, nt * P.BN + j * P.tile_n, bar);
                    pending |= 1u << s;
                    pend_par = (pend_par & ~(1u << s)) | (ph << s);
                    if (++s == P.stages) { s = 0; ph ^= 1; }
                }
            }
            if (!ok)
                for (int i = 0; i < P.stages; ++i)
                    if (pending & (1u << i))
                        wait_bounded(smem_u32(&S.full[i]), (pend_par >> i) & 1, S.abort_flag, P.err, P.timeout_ns,
                                     false);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(P.tile_n, true);
            int s = 0;
            uint32_t ph = 0, tph = 0;
            int t = 0;
            bool ok = true, issued = false;
            for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x, ++t) {
                int mt, nt, kb0, kb1;
                item_coords(P, it, mt, nt, kb0, kb1);
                const int b = t % P.nbuf;
                if (!wait_bounded(smem_u32(&S.tempty[b]), ((tph >> b) & 1) ^ 1, S.abort_flag, P.err, P.timeout_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(b * P.BN);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!wait_bounded(smem_u32(&S.full[s]), ph, S.abort_flag, P.err, P.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = smem_u32(S.ring + (size_t)s * S.stage_bytes);
#pragma unroll
                    for (int kk = 0; kk < kKBlock / 16; ++kk)
                        for (int j = 0; j < P.nsub; ++j) {
                            const uint32_t acc = (kb > kb0 || kk > 0) ? 1u : 0u;
                            mma_f16(d + (uint32_t)(j * P.tile_n), sdesc_k64(st + kk * 32),
                                    sdesc_k64(st + kNetStageA + j * b_bytes + kk * 32), idesc, acc);
                        }
                    issued = true;
                    mma_commit(smem_u32(&S.empty[s]));
                    if (++s == P.stages) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                mma_commit(smem_u32(&S.tfull[b]));
                tph ^= 1u << b;
            }
            if (issued) {
                mma_commit(smem_u32(S.mma_done));
                wait_bounded(smem_u32(S.mma_done), 0, S.abort_flag, P.err, P.timeout_ns, false);
            }
        }
    } else if (warp >= kNetEpiWarp0) {
        const int q = warp & 3, h = (warp - kNetEpiWarp0) >> 2;
        uint32_t tph = 0;
        int t = 0;
        for (int64_t it = blockIdx.x; it < items; it += gridDim.x, ++t) {
            int mt, nt, kb0, kb1;
            item_coords(P, it, mt, nt, kb0, kb1);
            const int b = t % P.nbuf;
            if (!warp_wait(smem_u32(&S.tfull[b]), (tph >> b) & 1, S.abort_flag, P.err, P.timeout_ns)) break;
            tph ^= 1u << b;
            tc_fence_after();
            epilogue<EPI>(P, S, bias_s, tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * P.BN), mt, nt, q, h,
                          lane);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&S.tempty[b]));
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, kNetTmemCols);
    }
}

// ----------------------------------------------------------------------------
// small kernels
// ----------------------------------------------------------------------------
// X^T[k][m] = hi part of the split image, column k of row m (training's B operand of dW1).
__global__ void __launch_bounds__(128) image_transpose_kernel(const uint8_t *img, int32_t kblocks, int64_t rows,
                                                              bf16 *XT, int64_t ldt)
{
    const int64_t m = (int64_t)blockIdx.x * kTileM + threadIdx.x;
    const int chunk = blockIdx.y;   // 8 columns
    if (m >= rows) return;
    const int kb = chunk >> 2, c = chunk & 3, r = threadIdx.x;
    const uint8_t *src = img + ((size_t)blockIdx.x * kblocks + kb) * kImageKBlockBytes + r * 64 +
                         ((c ^ ((r >> 1) & 3)) << 4);
    const uint4 v = *reinterpret_cast<const uint4 *>(src);
    const uint16_t *h = reinterpret_cast<const uint16_t *>(&v);
    uint16_t *dst = reinterpret_cast<uint16_t *>(XT);
#pragma unroll
    for (int e = 0; e < 8; ++e) dst[(int64_t)(kb * kKBlock + c * 8 + e) * ldt + m] = h[e];
}

// out[n] += sum over rows of X[r][n] (FP32), a column chunk per thread, rows split over blockIdx.y.
__global__ void __launch_bounds__(128) colsum_kernel(const float *X, int64_t ld, int64_t rows, int32_t cols,
                                                     int64_t rows_per, float *out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= cols) return;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per, r1 = min(rows, r0 + rows_per);
    float s = 0.f;
    for (int64_t r = r0; r < r1; ++r) s += X[r * ld + n];
    atomicAdd(out + n, s);
}

struct AdamParams {
    float *p;
    const float *g;
    float *m, *v;
    int64_t n, ob1, oW2, ob2;
    float lr, b1, b2, eps, wd, bc1, bc2;
    int32_t update;
    int32_t nin, H, nbp, kpad_c, kpad_r;
    const int32_t *active;
    uint16_t *W1c, *W1r, *W2, *W2T;
};

// AdamW (decoupled weight decay on W1 and W2) on the FP32 masters, then the BF16
// copies the GEMMs read; update = 0 only refreshes the copies.
__global__ void __launch_bounds__(256) adamw_publish_kernel(const AdamParams A)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    float w = A.p[i];
    const bool is_w = i < A.ob1 || (i >= A.oW2 && i < A.ob2);
    if (A.update) {
        const float g = A.g[i];
        const float m = A.b1 * A.m[i] + (1.f - A.b1) * g;
        const float v = A.b2 * A.v[i] + (1.f - A.b2) * g * g;
        A.m[i] = m;
        A.v[i] = v;
        const float mh = m / A.bc1, vh = v / A.bc2;
        w -= A.lr * (mh / (sqrtf(vh) + A.eps) + (is_w ? A.wd * w : 0.f));
        A.p[i] = w;
    }
    const __nv_bfloat16 wb = __float2bfloat16_rn(w);
    const uint16_t bits = *reinterpret_cast<const uint16_t *>(&wb);
    if (i < A.ob1) {
        const int64_t h = i / A.nin, k = i % A.nin;
        A.W1c[h * A.kpad_c + k] = bits;
        A.W1r[h * A.kpad_r + 2 * (int64_t)A.active[k >> 1] + (k & 1)] = bits;
    } else if (i >= A.oW2 && i < A.ob2) {
        const int64_t r = (i - A.oW2) / A.H, h = (i - A.oW2) % A.H;
        A.W2[r * A.H + h] = bits;
        A.W2T[h * A.nbp + r] = bits;
    }
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
struct NetGemm {
    const void *A = nullptr;        // row-major [M][K] BF16 (TMA), or
    int64_t lda = 0;
    const uint8_t *a_image = nullptr;   // split image hi parts, a_image_kb K blocks per M tile
    int32_t a_image_kb = 0;
    const CUtensorMap *mapB = nullptr;  // prebuilt B map, or
    const void *B = nullptr;        // row-major [N][K] BF16
    int64_t ldb = 0;
    int32_t M = 0, N = 0, K = 0, epi = EPI_RELU;
    const float *row_scale = nullptr, *bias = nullptr;
    bf16 *out = nullptr;
    int64_t ldo = 0;
    bf16 *outT = nullptr;
    int64_t ldt = 0;
    float *outf = nullptr;
    int64_t ldf = 0;
    const bf16 *hmask = nullptr;
    int64_t ldh = 0;
    const int32_t *colmap = nullptr, *label = nullptr;
    int32_t *bin = nullptr;
    float *conf = nullptr;
    int32_t halfwin = -1;
    float *loss = nullptr;
    float inv_batch = 1.f;
};

void tile_shape(int N, int epi, int &ntiles, int &tile_n, int &nsub)
{
    if (epi == EPI_SOFTMAX) {
        ntiles = 1;
        nsub = N > 256 ? 2 : 1;
        tile_n = ((N + nsub - 1) / nsub + 15) / 16 * 16;
    } else {
        ntiles = (N + 255) / 256;
        nsub = 1;
        tile_n = ((N + ntiles - 1) / ntiles + 15) / 16 * 16;
    }
}

bool encode_bf16(CUtensorMap *map, const void *base, int64_t cols, int64_t rows, int64_t ld, int box_rows)
{
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kKBlock, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return encode_tensor_map(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, const_cast<void *>(base), dims, strides, box,
                             estr, CU_TENSOR_MAP_SWIZZLE_64B);
}

cudaError_t net_gemm(const rms_plan_s &p, const NetGemm &g, cudaStream_t s)
{
    if (g.M <= 0 || g.N <= 0 || g.K <= 0) return cudaSuccess;
    NetGemmParams P;
    std::memset(&P, 0, sizeof(P));
    P.M = g.M;
    P.N = g.N;
    P.epi = g.epi;
    int ntiles, tile_n, nsub;
    tile_shape(g.N, g.epi, ntiles, tile_n, nsub);
    P.ntiles = ntiles;
    P.tile_n = tile_n;
    P.nsub = nsub;
    P.BN = tile_n * nsub;
    if (P.BN > kNetTmemCols || tile_n > 256) return cudaErrorInvalidValue;
    P.nbuf = 2 * P.BN <= kNetTmemCols ? 2 : 1;
    P.mtiles = (g.M + kTileM - 1) / kTileM;
    P.kblocks = g.a_image ? g.a_image_kb : (g.K + kKBlock - 1) / kKBlock;
    int ksplit = 1;
    if (g.epi == EPI_ACC) {
        const int tiles = P.mtiles * P.ntiles;
        ksplit = std::max(1, std::min(P.kblocks, p.num_sms / std::max(1, tiles)));
    }
    P.kb_per_split = (P.kblocks + ksplit - 1) / ksplit;
    P.ksplit = (P.kblocks + P.kb_per_split - 1) / P.kb_per_split;
    const uint32_t stage = kNetStageA + (uint32_t)P.BN * 64;
    P.stages = std::min(8, (int)((kNetSmemLimit - kNetFixedSmem) / (stage + 16)));
    if (P.stages < 2) return cudaErrorInvalidConfiguration;
    P.a_image = g.a_image;
    P.a_image_kb = g.a_image_kb;
    P.row_scale = g.row_scale;
    P.bias = g.bias;
    P.out = g.out;
    P.ldo = g.ldo;
    P.outT = g.outT;
    P.ldt = g.ldt;
    P.outf = g.outf;
    P.ldf = g.ldf;
    P.hmask = g.hmask;
    P.ldh = g.ldh;
    P.colmap = g.colmap;
    P.label = g.label;
    P.bin = g.bin;
    P.conf = g.conf;
    P.halfwin = g.halfwin;
    P.loss = g.loss;
    P.inv_batch = g.inv_batch;
    P.err = p.d_err;
    P.timeout_ns = p.timeout_ns;

    CUtensorMap tmA, tmB;
    if (g.mapB) {
        tmB = *g.mapB;
    } else if (!encode_bf16(&tmB, g.B, g.K, g.N, g.ldb, tile_n)) {
        return cudaErrorInvalidValue;
    }
    if (g.a_image) {
        tmA = tmB;   // unused
    } else if (!encode_bf16(&tmA, g.A, g.K, g.M, g.lda, kTileM)) {
        return cudaErrorInvalidValue;
    }
    const size_t smem = kNetFixedSmem + (size_t)P.stages * (stage + 16);
    if (g.bias && g.N > kNetBiasMax) return cudaErrorInvalidValue;
    const int64_t items = (int64_t)P.mtiles * P.ntiles * P.ksplit;
    const int grid = (int)std::min<int64_t>(items, p.num_sms);
    auto kern = g.epi == EPI_RELU ? net_gemm_kernel<EPI_RELU>
              : g.epi == EPI_SOFTMAX ? net_gemm_kernel<EPI_SOFTMAX>
              : g.epi == EPI_DRELU ? net_gemm_kernel<EPI_DRELU> : net_gemm_kernel<EPI_ACC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kNetThreads, smem, s>>>(P, tmA, tmB);
    return cudaGetLastError();
}

cudaError_t publish(rms_net_s &n, bool update, float lr, float b1, float b2, float eps, float wd, cudaStream_t s)
{
    AdamParams A;
    A.p = n.d_p;
    A.g = n.d_g;
    A.m = n.d_m;
    A.v = n.d_v;
    A.n = n.nparams;
    A.ob1 = n.ob1;
    A.oW2 = n.oW2;
    A.ob2 = n.ob2;
    A.lr = lr;
    A.b1 = b1;
    A.b2 = b2;
    A.eps = eps;
    A.wd = wd;
    A.update = update ? 1 : 0;
    A.bc1 = update ? (float)(1.0 - std::pow((double)b1, (double)n.steps)) : 1.f;
    A.bc2 = update ? (float)(1.0 - std::pow((double)b2, (double)n.steps)) : 1.f;
    A.nin = n.nin;
    A.H = n.hidden;
    A.nbp = n.nbp;
    A.kpad_c = n.plan->kpad;
    A.kpad_r = n.plan->kpad_raw;
    A.active = n.plan->d_active;
    A.W1c = n.d_W1c;
    A.W1r = n.d_W1r;
    A.W2 = n.d_W2;
    A.W2T = n.d_W2T;
    adamw_publish_kernel<<<(unsigned)((n.nparams + 255) / 256), 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t colsum(const float *X, int64_t ld, int64_t rows, int32_t cols, float *out, cudaStream_t s)
{
    const int64_t per = 256;
    const int64_t gy = (rows + per - 1) / per;
    if (gy < 1) return cudaSuccess;
    dim3 grid((unsigned)((cols + 127) / 128), (unsigned)gy);
    colsum_kernel<<<grid, 128, 0, s>>>(X, ld, rows, cols, per, out);
    return cudaGetLastError();
}

rms_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return RMS_OK;
    if (e == cudaErrorMemoryAllocation) return RMS_ERR_OOM;
    return RMS_ERR_CUDA;
}

void free_net(rms_net_s *n)
{
    if (!n) return;
    void *ptrs[] = {n->d_p, n->d_g, n->d_m, n->d_v, n->d_W1c, n->d_W1r, n->d_W2, n->d_W2T, n->d_colmap_c,
                    n->d_colmap_r, n->d_img, n->d_rs, n->d_dz32, n->d_da32, n->d_loss, n->d_h, n->d_hT,
                    n->d_dz, n->d_dzT, n->d_da1T, n->d_XT};
    for (void *q : ptrs) cudaFree(q);
    if (n->last) cudaEventDestroy(n->last);
    delete n;
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

bool is_tensor_plan(const rms_plan_s *p)
{
    return p->precision == RMS_BF16 || p->precision == RMS_BF16X3 || p->precision == RMS_FP16X3;
}

rms_status check_cube(const rms_net_s *n, const float *Q, const float *U, int64_t nlos, int32_t layout)
{
    if (!n || !Q || !U || nlos < 0) return RMS_ERR_INVALID_ARG;
    if (layout != RMS_CHAN_MAJOR && layout != RMS_LOS_MAJOR) return RMS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(Q) & 3) || (reinterpret_cast<uintptr_t>(U) & 3)) return RMS_ERR_INVALID_ARG;
    if (nlos > ((int64_t)1 << 31) - kTileM) return RMS_ERR_INVALID_ARG;
    return RMS_OK;
}

// One SplitMix64 draw in [-1, 1) for weight initialisation.
double init_uniform(uint64_t seed, uint64_t i)
{
    uint64_t x = seed * 0x9E3779B97F4A7C15ull + i * 0xD1B54A32D192ED03ull + 0x632BE59BD9B4E019ull;
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Backward pass of one batch into n.d_g (see rms_net_grad).
cudaError_t net_grad(rms_net_s &n, const float *Q, const float *U, int64_t B, int32_t layout, const int32_t *label,
                     cudaStream_t s)
{
    const rms_plan_s &p = *n.plan;
    const bool chan = layout == RMS_CHAN_MAJOR;
    const int kb = chan ? p.kblocks : p.kblocks_raw;
    const int kpad = kb * kKBlock;
    cudaError_t e = cudaMemsetAsync(n.d_g, 0, n.nparams * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(n.d_loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    SplitOpts so;
    so.Q = Q;
    so.U = U;
    so.nlos_src = B;
    so.layout = layout;
    so.nout = B;
    so.mode = 0;   // BF16 hi parts only
    so.A = n.d_img;
    so.rscale = n.d_rs;
    if ((e = launch_split(p, so, s)) != cudaSuccess) return e;
    bf16 *h = reinterpret_cast<bf16 *>(n.d_h), *hT = reinterpret_cast<bf16 *>(n.d_hT);
    bf16 *dz = reinterpret_cast<bf16 *>(n.d_dz), *dzT = reinterpret_cast<bf16 *>(n.d_dzT);
    bf16 *da1T = reinterpret_cast<bf16 *>(n.d_da1T), *XT = reinterpret_cast<bf16 *>(n.d_XT);
    const float invB = 1.0f / (float)B;
    {   // h = relu(W1 x + b1), also h^T
        NetGemm g;
        g.a_image = n.d_img;
        g.a_image_kb = kb;
        g.mapB = chan ? &n.tm_W1c : &n.tm_W1r;
        g.M = (int32_t)B;
        g.N = n.hidden;
        g.K = kpad;
        g.epi = EPI_RELU;
        g.row_scale = n.d_rs;
        g.bias = n.d_p + n.ob1;
        g.out = h;
        g.ldo = n.hidden;
        g.outT = hT;
        g.ldt = n.ldb;
        if ((e = net_gemm(p, g, s)) != cudaSuccess) return e;
    }
    {   // softmax cross-entropy: loss, dz, dz^T, dz (FP32)
        NetGemm g;
        g.A = h;
        g.lda = n.hidden;
        g.mapB = &n.tm_W2;
        g.M = (int32_t)B;
        g.N = n.nbins;
        g.K = n.hidden;
        g.epi = EPI_SOFTMAX;
        g.bias = n.d_p + n.ob2;
        g.label = label;
        g.loss = n.d_loss;
        g.inv_batch = invB;
        g.out = dz;
        g.ldo = n.nbp;
        g.outT = dzT;
        g.ldt = n.ldb;
        g.outf = n.d_dz32;
        g.ldf = n.nbp;
        if ((e = net_gemm(p, g, s)) != cudaSuccess) return e;
    }
    {   // dW2 = dz^T h
        NetGemm g;
        g.A = dzT;
        g.lda = n.ldb;
        g.B = hT;
        g.ldb = n.ldb;
        g.M = n.nbins;
        g.N = n.hidden;
        g.K = (int32_t)B;
        g.epi = EPI_ACC;
        g.outf = n.d_g + n.oW2;
        g.ldf = n.hidden;
        if ((e = net_gemm(p, g, s)) != cudaSuccess) return e;
    }
    if ((e = colsum(n.d_dz32, n.nbp, B, n.nbins, n.d_g + n.ob2, s)) != cudaSuccess) return e;
    {   // da1 = (dz W2) * [h > 0]: (da1 / s)^T for dW1, da1 for db1
        NetGemm g;
        g.A = dz;
        g.lda = n.nbp;
        g.mapB = &n.tm_W2T;
        g.M = (int32_t)B;
        g.N = n.hidden;
        g.K = n.nbins;
        g.epi = EPI_DRELU;
        g.row_scale = n.d_rs;
        g.hmask = h;
        g.ldh = n.hidden;
        g.outT = da1T;
        g.ldt = n.ldb;
        g.outf = n.d_da32;
        g.ldf = n.hidden;
        if ((e = net_gemm(p, g, s)) != cudaSuccess) return e;
    }
    if ((e = colsum(n.d_da32, n.hidden, B, n.hidden, n.d_g + n.ob1, s)) != cudaSuccess) return e;
    {   // X^T from the image, then dW1 = (da1 / s)^T X_raw in W1's column order
        dim3 grid((unsigned)((B + kTileM - 1) / kTileM), (unsigned)(kb * 4));
        image_transpose_kernel<<<grid, 128, 0, s>>>(n.d_img, kb, B, XT, n.ldb);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        NetGemm g;
        g.A = da1T;
        g.lda = n.ldb;
        g.B = XT;
        g.ldb = n.ldb;
        g.M = n.hidden;
        g.N = kpad;
        g.K = (int32_t)B;
        g.epi = EPI_ACC;
        g.colmap = chan ? n.d_colmap_c : n.d_colmap_r;
        g.outf = n.d_g + n.oW1;
        g.ldf = n.nin;
        if ((e = net_gemm(p, g, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t net_forward_image(const rms_net_s &n, const uint8_t *img, int layout, const float *rscale, int64_t nlos,
                              uint16_t *h, float *logits, int32_t *bin, float *conf, int32_t halfwin,
                              cudaStream_t s)
{
    const rms_plan_s &p = *n.plan;
    const bool chan = layout == RMS_CHAN_MAJOR;
    const int kb = chan ? p.kblocks : p.kblocks_raw;
    NetGemm g1;
    g1.a_image = img;
    g1.a_image_kb = kb;
    g1.mapB = chan ? &n.tm_W1c : &n.tm_W1r;
    g1.M = (int32_t)nlos;
    g1.N = n.hidden;
    g1.K = kb * kKBlock;
    g1.epi = EPI_RELU;
    g1.row_scale = rscale;
    g1.bias = n.d_p + n.ob1;
    g1.out = reinterpret_cast<bf16 *>(h);
    g1.ldo = n.hidden;
    cudaError_t e = net_gemm(p, g1, s);
    if (e != cudaSuccess) return e;
    NetGemm g2;
    g2.A = h;
    g2.lda = n.hidden;
    g2.mapB = &n.tm_W2;
    g2.M = (int32_t)nlos;
    g2.N = n.nbins;
    g2.K = n.hidden;
    g2.epi = EPI_SOFTMAX;
    g2.bias = n.d_p + n.ob2;
    g2.outf = logits;
    g2.ldf = n.nbins;
    g2.bin = bin;
    g2.conf = conf;
    g2.halfwin = halfwin;
    return net_gemm(p, g2, s);
}

extern "C" {

rms_status rms_net_create(rms_net_t *out, rms_plan_t plan, int32_t hidden, int32_t max_batch, uint64_t seed)
{
    if (!out) return RMS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plan || hidden < 16 || hidden > 256 || hidden % 16 || max_batch < 1 || max_batch > 65536)
        return RMS_ERR_INVALID_ARG;
    if (!is_tensor_plan(plan) || plan->nphi > 512) return RMS_ERR_UNSUPPORTED;
    Guard guard(plan->device);
    if (!guard.ok) return RMS_ERR_CUDA;
    rms_net_s *n = new (std::nothrow) rms_net_s();
    if (!n) return RMS_ERR_OOM;
    const rms_plan_s &p = *plan;
    n->plan = plan;
    n->device = plan->device;
    n->nin = 2 * p.nact;
    n->hidden = hidden;
    n->nbins = p.nphi;
    n->nbp = (p.nphi + 7) / 8 * 8;
    n->max_batch = max_batch;
    n->ldb = (max_batch + 7) / 8 * 8;
    n->oW1 = 0;
    n->ob1 = (int64_t)hidden * n->nin;
    n->oW2 = n->ob1 + hidden;
    n->ob2 = n->oW2 + (int64_t)p.nphi * hidden;
    n->nparams = n->ob2 + p.nphi;
    const int kpad_max = std::max(p.kpad, p.kpad_raw);
    const size_t img = std::max(split_operand_bytes(p, max_batch, RMS_CHAN_MAJOR),
                                split_operand_bytes(p, max_batch, RMS_LOS_MAJOR));
    const size_t B = (size_t)max_batch, L = (size_t)n->ldb;
    cudaError_t e = cudaSuccess;
    std::vector<float> h0(n->nparams, 0.0f);
    std::vector<int32_t> cm_c(p.kpad, -1), cm_r(p.kpad_raw, -1);
#define NET_TRY(x)                       \
    do {                                 \
        e = (x);                         \
        if (e != cudaSuccess) goto fail; \
    } while (0)
    NET_TRY(cudaMalloc(&n->d_p, n->nparams * sizeof(float)));
    NET_TRY(cudaMalloc(&n->d_g, n->nparams * sizeof(float)));
    NET_TRY(cudaMalloc(&n->d_m, n->nparams * sizeof(float)));
    NET_TRY(cudaMalloc(&n->d_v, n->nparams * sizeof(float)));
    NET_TRY(cudaMalloc(&n->d_W1c, (size_t)hidden * p.kpad * 2));
    NET_TRY(cudaMalloc(&n->d_W1r, (size_t)hidden * p.kpad_raw * 2));
    NET_TRY(cudaMalloc(&n->d_W2, (size_t)p.nphi * hidden * 2));
    NET_TRY(cudaMalloc(&n->d_W2T, (size_t)hidden * n->nbp * 2));
    NET_TRY(cudaMalloc(&n->d_colmap_c, p.kpad * sizeof(int32_t)));
    NET_TRY(cudaMalloc(&n->d_colmap_r, p.kpad_raw * sizeof(int32_t)));
    NET_TRY(cudaMalloc(&n->d_img, img));
    NET_TRY(cudaMalloc(&n->d_rs, B * sizeof(float)));
    NET_TRY(cudaMalloc(&n->d_dz32, B * n->nbp * sizeof(float)));
    NET_TRY(cudaMalloc(&n->d_da32, B * hidden * sizeof(float)));
    NET_TRY(cudaMalloc(&n->d_loss, sizeof(float)));
    NET_TRY(cudaMalloc(&n->d_h, B * hidden * 2));
    NET_TRY(cudaMalloc(&n->d_hT, (size_t)hidden * L * 2));
    NET_TRY(cudaMalloc(&n->d_dz, B * n->nbp * 2));
    NET_TRY(cudaMalloc(&n->d_dzT, (size_t)p.nphi * L * 2));
    NET_TRY(cudaMalloc(&n->d_da1T, (size_t)hidden * L * 2));
    NET_TRY(cudaMalloc(&n->d_XT, (size_t)kpad_max * L * 2));
    NET_TRY(cudaMemset(n->d_W1c, 0, (size_t)hidden * p.kpad * 2));
    NET_TRY(cudaMemset(n->d_W1r, 0, (size_t)hidden * p.kpad_raw * 2));
    NET_TRY(cudaMemset(n->d_W2T, 0, (size_t)hidden * n->nbp * 2));
    NET_TRY(cudaMemset(n->d_m, 0, n->nparams * sizeof(float)));
    NET_TRY(cudaMemset(n->d_v, 0, n->nparams * sizeof(float)));
    NET_TRY(cudaMemset(n->d_g, 0, n->nparams * sizeof(float)));
    // uniform init scaled by fan-in: sqrt(6 / fan_in) for the ReLU layer, sqrt(3 / fan_in) for the head
    for (int64_t i = 0; i < n->ob1; ++i)
        h0[i] = (float)(init_uniform(seed, (uint64_t)i) * std::sqrt(6.0 / n->nin));
    for (int64_t i = n->oW2; i < n->ob2; ++i)
        h0[i] = (float)(init_uniform(seed, (uint64_t)i) * std::sqrt(3.0 / hidden));
    NET_TRY(cudaMemcpy(n->d_p, h0.data(), n->nparams * sizeof(float), cudaMemcpyHostToDevice));
    for (int k = 0; k < n->nin; ++k) cm_c[k] = k;
    for (int a = 0; a < p.nact; ++a) {
        cm_r[2 * p.active[a]] = 2 * a;
        cm_r[2 * p.active[a] + 1] = 2 * a + 1;
    }
    NET_TRY(cudaMemcpy(n->d_colmap_c, cm_c.data(), p.kpad * sizeof(int32_t), cudaMemcpyHostToDevice));
    NET_TRY(cudaMemcpy(n->d_colmap_r, cm_r.data(), p.kpad_raw * sizeof(int32_t), cudaMemcpyHostToDevice));
    {
        int nt, tn, ns;
        tile_shape(hidden, EPI_RELU, nt, tn, ns);
        const int tile_w1 = tn;
        tile_shape(p.nphi, EPI_SOFTMAX, nt, tn, ns);
        const int tile_w2 = tn;
        tile_shape(hidden, EPI_DRELU, nt, tn, ns);
        if (!encode_bf16(&n->tm_W1c, n->d_W1c, p.kpad, hidden, p.kpad, tile_w1) ||
            !encode_bf16(&n->tm_W1r, n->d_W1r, p.kpad_raw, hidden, p.kpad_raw, tile_w1) ||
            !encode_bf16(&n->tm_W2, n->d_W2, hidden, p.nphi, hidden, tile_w2) ||
            !encode_bf16(&n->tm_W2T, n->d_W2T, p.nphi, hidden, n->nbp, tn)) {
            free_net(n);
            return RMS_ERR_CUDA;
        }
    }
    NET_TRY(publish(*n, false, 0.f, 0.f, 0.f, 0.f, 0.f, 0));
    NET_TRY(cudaEventCreateWithFlags(&n->last, cudaEventDisableTiming));
    NET_TRY(cudaDeviceSynchronize());
#undef NET_TRY
    *out = n;
    return RMS_OK;
fail:
    cudaGetLastError();
    free_net(n);
    return from_cuda(e);
}

rms_status rms_net_destroy(rms_net_t n)
{
    if (!n) return RMS_OK;
    Guard guard(n->device);
    cudaDeviceSynchronize();
    free_net(n);
    return RMS_OK;
}

rms_status rms_net_info(rms_net_t n, int32_t what, int64_t *value)
{
    if (!n || !value) return RMS_ERR_INVALID_ARG;
    switch (what) {
    case RMS_NET_NPARAMS: *value = n->nparams; break;
    case RMS_NET_NIN: *value = n->nin; break;
    case RMS_NET_HIDDEN: *value = n->hidden; break;
    case RMS_NET_NBINS: *value = n->nbins; break;
    case RMS_NET_MAX_BATCH: *value = n->max_batch; break;
    case RMS_NET_STEPS: *value = n->steps; break;
    default: return RMS_ERR_INVALID_ARG;
    }
    return RMS_OK;
}

rms_status rms_net_params(rms_net_t n, int32_t which, float *host, int64_t count, int32_t set)
{
    if (!n || !host || count != n->nparams) return RMS_ERR_INVALID_ARG;
    if (which != RMS_NET_PARAMS && which != RMS_NET_GRADS) return RMS_ERR_INVALID_ARG;
    if (set && which != RMS_NET_PARAMS) return RMS_ERR_INVALID_ARG;
    Guard guard(n->device);
    if (!guard.ok) return RMS_ERR_CUDA;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return from_cuda(e);
    const size_t bytes = n->nparams * sizeof(float);
    if (!set) return from_cuda(cudaMemcpy(host, which == RMS_NET_PARAMS ? n->d_p : n->d_g, bytes, cudaMemcpyDeviceToHost));
    e = cudaMemcpy(n->d_p, host, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->d_m, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(n->d_v, 0, bytes);
    n->steps = 0;
    if (e == cudaSuccess) e = publish(*n, false, 0.f, 0.f, 0.f, 0.f, 0.f, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return from_cuda(e);
}

rms_status rms_propose(rms_net_t n, const float *Q, const float *U, int64_t nlos, int32_t layout,
                       int32_t conf_halfwidth, float *logits, int32_t *bin, float *conf, void *stream)
{
    rms_status st = check_cube(n, Q, U, nlos, layout);
    if (st != RMS_OK) return st;
    if (*n->plan->h_err) return RMS_ERR_TIMEOUT;
    if (nlos == 0 || (!logits && !bin && !conf)) return RMS_OK;
    Guard guard(n->device);
    if (!guard.ok) return RMS_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const rms_plan_s &p = *n->plan;
    const size_t ib = split_operand_bytes(p, nlos, layout);
    const size_t hb = (size_t)nlos * n->hidden * 2, rb = (size_t)nlos * sizeof(float);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    uint8_t *scr = nullptr;
    cudaError_t e = cudaStreamWaitEvent(s, n->last, 0);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&scr), up(ib) + up(hb) + up(rb), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
    }
    uint8_t *img = scr;
    uint16_t *h = reinterpret_cast<uint16_t *>(scr + up(ib));
    float *rs = reinterpret_cast<float *>(scr + up(ib) + up(hb));
    SplitOpts so;
    so.Q = Q;
    so.U = U;
    so.nlos_src = nlos;
    so.layout = layout;
    so.nout = nlos;
    so.mode = 0;
    so.A = img;
    so.rscale = rs;
    e = launch_split(p, so, s);
    if (e == cudaSuccess) e = net_forward_image(*n, img, layout, rs, nlos, h, logits, bin, conf, conf_halfwidth, s);
    cudaError_t e2 = cudaFreeAsync(scr, s);
    if (e == cudaSuccess) e = e2;
    e2 = cudaEventRecord(n->last, s);
    if (e == cudaSuccess) e = e2;
    return from_cuda(e);
}

rms_status rms_net_grad(rms_net_t n, const float *Q, const float *U, int64_t nlos, int32_t layout,
                        const int32_t *label, float *loss, void *stream)
{
    rms_status st = check_cube(n, Q, U, nlos, layout);
    if (st != RMS_OK) return st;
    if (!label || nlos < 1 || nlos > n->max_batch) return RMS_ERR_INVALID_ARG;
    if (*n->plan->h_err) return RMS_ERR_TIMEOUT;
    Guard guard(n->device);
    if (!guard.ok) return RMS_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamWaitEvent(s, n->last, 0);
    if (e == cudaSuccess) e = net_grad(*n, Q, U, nlos, layout, label, s);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, n->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaError_t e2 = cudaEventRecord(n->last, s);
    if (e == cudaSuccess) e = e2;
    return from_cuda(e);
}

rms_status rms_train_step(rms_net_t n, const float *Q, const float *U, int64_t nlos, int32_t layout,
                          const int32_t *label, float lr, float beta1, float beta2, float eps, float weight_decay,
                          float *loss, void *stream)
{
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) ||
        !(weight_decay >= 0.f))
        return RMS_ERR_INVALID_ARG;
    rms_status st = rms_net_grad(n, Q, U, nlos, layout, label, loss, stream);
    if (st != RMS_OK) return st;
    Guard guard(n->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    n->steps += 1;
    cudaError_t e = publish(*n, true, lr, beta1, beta2, eps, weight_decay, s);
    cudaError_t e2 = cudaEventRecord(n->last, s);
    if (e == cudaSuccess) e = e2;
    return from_cuda(e);
}

}  // extern "C"
