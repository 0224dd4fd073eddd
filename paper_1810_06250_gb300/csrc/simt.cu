// FP32 CUDA-core RM synthesis with the fused peak map.
//
// The paper's kernel (Sec. 3) gives each thread one Faraday depth and loops
// over channels, computing sin/cos per (channel, phi) in FP32.  Here a block
// owns 64 lines of sight and walks all phi in tiles of 64; per channel chunk
// the 32 x 64 (cos, sin) tile is shared by the block's 64 lines of sight, and
// each thread accumulates a 4 LOS x 4 phi register tile (16 complex MACs =
// 64 FMAs per channel for 4 shared-memory vector loads).
//   FLY   : (cos, sin) = sincosf(phi_k * 2(lambda_j^2 - lambda_0^2)) in FP32
//           (the paper's method, argument and reduction in FP32);
//   TABLE : (cos, sin) read from the plan's FP32 table built in FP64.
// The peak of |F| (Sec. 2.2) is reduced in registers over the block's phi
// tiles, so F never has to be re-read.
#include <limits.h>

#include "rms_internal.h"

namespace {

constexpr int TL = 64;    // lines of sight per block
constexpr int TP = 64;    // phi per tile
constexpr int CH = 32;    // channels per chunk
constexpr int LDQ = TL + 4;

struct SimtArgs {
    const float *Q, *U;
    int64_t nlos;
    int32_t nchan, nact, nphi;
    const int32_t *active;
    const float *l2x;      // [nact] 2 (lambda^2 - lambda_0^2), FP32
    const float *w32;      // [nact]
    const float *phi32;    // [nphi]
    const float2 *table;   // [nact][nphi]
    float scale;           // K
    float *F;
    int32_t *pidx;
    float *pabs, *pphi;
};

__device__ __forceinline__ bool better(float m, int i, float bm, int bi)
{
    return m > bm || (m == bm && i < bi);
}

template <bool FLY, int LAYOUT>
__global__ void __launch_bounds__(256) simt_kernel(const SimtArgs a)
{
    __shared__ __align__(16) float sQ[CH][LDQ];
    __shared__ __align__(16) float sU[CH][LDQ];
    __shared__ __align__(16) float sC[CH][TP];
    __shared__ __align__(16) float sS[CH][TP];

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t l0 = (int64_t)blockIdx.x * TL;

    float bm[4];
    int bi[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { bm[i] = -1.0f; bi[i] = INT_MAX; }

    for (int p0 = 0; p0 < a.nphi; p0 += TP) {
        float re[4][4], im[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) { re[i][j] = 0.f; im[i][j] = 0.f; }

        for (int c0 = 0; c0 < a.nact; c0 += CH) {
            __syncthreads();
            // data tile: sQ[c][m] = Q of active channel c0 + c, LOS l0 + m
            if (LAYOUT == RMS_CHAN_MAJOR) {
#pragma unroll 4
                for (int i = tid; i < CH * TL; i += 256) {
                    int c = i / TL, m = i % TL;
                    int64_t l = l0 + m;
                    float q = 0.f, u = 0.f;
                    if (c0 + c < a.nact && l < a.nlos) {
                        int64_t off = (int64_t)__ldg(a.active + c0 + c) * a.nlos + l;
                        q = __ldg(a.Q + off);
                        u = __ldg(a.U + off);
                    }
                    sQ[c][m] = q;
                    sU[c][m] = u;
                }
            } else {
#pragma unroll 4
                for (int i = tid; i < CH * TL; i += 256) {
                    int c = i % CH, m = i / CH;
                    int64_t l = l0 + m;
                    float q = 0.f, u = 0.f;
                    if (c0 + c < a.nact && l < a.nlos) {
                        int64_t off = l * a.nchan + __ldg(a.active + c0 + c);
                        q = __ldg(a.Q + off);
                        u = __ldg(a.U + off);
                    }
                    sQ[c][m] = q;
                    sU[c][m] = u;
                }
            }
            // phase tile: (w cos, w sin) for channel c0 + c and phi p0 + k
#pragma unroll 2
            for (int i = tid; i < CH * TP; i += 256) {
                int c = i / TP, k = i % TP;
                float cv = 0.f, sv = 0.f;
                if (c0 + c < a.nact && p0 + k < a.nphi) {
                    if (FLY) {
                        float th = a.phi32[p0 + k] * a.l2x[c0 + c];
                        float sn, cs;
                        sincosf(th, &sn, &cs);
                        float w = a.w32[c0 + c];
                        cv = w * cs;
                        sv = w * sn;
                    } else {
                        float2 t = __ldg(a.table + (int64_t)(c0 + c) * a.nphi + p0 + k);
                        cv = t.x;
                        sv = t.y;
                    }
                }
                sC[c][k] = cv;
                sS[c][k] = sv;
            }
            __syncthreads();
#pragma unroll 4
            for (int c = 0; c < CH; ++c) {
                float4 q = *reinterpret_cast<const float4 *>(&sQ[c][4 * ty]);
                float4 u = *reinterpret_cast<const float4 *>(&sU[c][4 * ty]);
                float4 cs = *reinterpret_cast<const float4 *>(&sC[c][4 * tx]);
                float4 sn = *reinterpret_cast<const float4 *>(&sS[c][4 * tx]);
                const float qv[4] = {q.x, q.y, q.z, q.w}, uv[4] = {u.x, u.y, u.z, u.w};
                const float cv[4] = {cs.x, cs.y, cs.z, cs.w}, sv[4] = {sn.x, sn.y, sn.z, sn.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        // (q + iu)(c - is): Re += q c + u s, Im += u c - q s  (Eqs. qPhi, uPhi)
                        re[i][j] = fmaf(qv[i], cv[j], re[i][j]);
                        re[i][j] = fmaf(uv[i], sv[j], re[i][j]);
                        im[i][j] = fmaf(uv[i], cv[j], im[i][j]);
                        im[i][j] = fmaf(-qv[i], sv[j], im[i][j]);
                    }
            }
        }

        // epilogue for this phi tile: scale by K, store, update the running peak
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int64_t l = l0 + 4 * ty + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int k = p0 + 4 * tx + j;
                float fr = re[i][j] * a.scale, fi = im[i][j] * a.scale;
                if (k < a.nphi) {
                    float m2 = __fadd_rn(__fmul_rn(fr, fr), __fmul_rn(fi, fi));
                    if (m2 > bm[i]) { bm[i] = m2; bi[i] = k; }
                    if (a.F != nullptr && l < a.nlos)
                        *reinterpret_cast<float2 *>(a.F + (l * a.nphi + k) * 2) = make_float2(fr, fi);
                }
            }
        }
    }

    // reduce the peak over the 16 threads (tx) that share each line of sight
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float m = bm[i];
        int k = bi[i];
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) {
            float mo = __shfl_xor_sync(0xffffffffu, m, off);
            int ko = __shfl_xor_sync(0xffffffffu, k, off);
            if (better(mo, ko, m, k)) { m = mo; k = ko; }
        }
        int64_t l = l0 + 4 * ty + i;
        if (tx == 0 && l < a.nlos) {
            bool ok = k != INT_MAX;
            if (a.pidx) a.pidx[l] = ok ? k : -1;
            if (a.pabs) a.pabs[l] = ok ? sqrtf(m) : __int_as_float(0x7fc00000);
            if (a.pphi) a.pphi[l] = ok ? a.phi32[k] : __int_as_float(0x7fc00000);
        }
    }
}

}  // namespace

cudaError_t launch_simt(const rms_plan_s &p, bool fly, const float *Q, const float *U, int64_t nlos,
                        int layout, float *F, int32_t *pidx, float *pabs, float *pphi,
                        cudaStream_t s)
{
    SimtArgs a;
    a.Q = Q;
    a.U = U;
    a.nlos = nlos;
    a.nchan = p.nchan;
    a.nact = p.nact;
    a.nphi = p.nphi;
    a.active = p.d_active;
    a.l2x = p.d_l2x32;
    a.w32 = p.d_w32;
    a.phi32 = p.d_phi32;
    a.table = p.d_table;
    a.scale = (float)p.K;
    a.F = F;
    a.pidx = pidx;
    a.pabs = pabs;
    a.pphi = pphi;
    int64_t blocks = (nlos + TL - 1) / TL;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    dim3 g((unsigned)blocks);
    if (fly) {
        if (layout == RMS_CHAN_MAJOR) simt_kernel<true, RMS_CHAN_MAJOR><<<g, 256, 0, s>>>(a);
        else simt_kernel<true, RMS_LOS_MAJOR><<<g, 256, 0, s>>>(a);
    } else {
        if (layout == RMS_CHAN_MAJOR) simt_kernel<false, RMS_CHAN_MAJOR><<<g, 256, 0, s>>>(a);
        else simt_kernel<false, RMS_LOS_MAJOR><<<g, 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}
