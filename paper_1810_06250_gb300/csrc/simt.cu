// FP32 CUDA-core RM synthesis with the fused peak map.
//
// The paper's kernel (Sec. 3) gives each thread one Faraday depth and loops
// over channels, computing sin/cos per (channel, phi) in FP32.  Here a block
// owns 256 lines of sight and walks all phi in tiles of 64; per chunk of 16
// channels the 16 x 64 (cos, sin) tile is shared by the block's 256 lines of
// sight, and each thread accumulates an 8 LOS x 8 phi register tile: 64 complex
// MACs = 256 FMAs per channel for 8 shared-memory vector loads, so the FMA pipe,
// not shared-memory bandwidth, sets the rate.  The chunks stream through a
// two-stage cp.async pipeline, so the next chunk's loads overlap this one's FMAs.
//   FLY   : (cos, sin) = sincosf(phi_k * 2(lambda_j^2 - lambda_0^2)) in FP32
//           (the paper's method, argument and reduction in FP32);
//   TABLE : (cos, sin) read from the plan's FP32 table built in FP64.
// The peak of |F| (Sec. 2.2) is reduced in registers over the block's phi
// tiles, so F never has to be re-read.
#include <limits.h>

#include "rms_internal.h"

namespace {

constexpr int TL = 256;   // lines of sight per block (32 thread rows x 8)
constexpr int TP = 64;    // phi per tile (8 thread columns x 8, as 4 pairs at stride 16)
constexpr int CH = 16;    // channels per chunk
constexpr int LDQ = TL + 4;

// one pipeline stage in shared memory: the chunk's data and phase tiles
struct Stage {
    float q[CH][LDQ];
    float u[CH][LDQ];
    float2 cs[CH][TP];     // (w cos, w sin)
};
constexpr size_t kSimtSmem = 2 * sizeof(Stage);

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

// asynchronous global -> shared copy of 4 or 8 bytes; a false predicate
// writes zeros and reads nothing (the source is then any valid address)
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES),
                 "r"(ok ? BYTES : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ void load8(const float *p, float (&v)[8])
{
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Each thread copies one channel of every chunk: ISSUE_CH(tid) is that channel's
// slot in the chunk, and its active-channel index is loaded one chunk ahead
// (act), so no global load latency sits in front of the copies.
template <int LAYOUT>
__device__ __forceinline__ int issue_ch(int tid)
{
    return LAYOUT == RMS_CHAN_MAJOR ? tid / (256 / CH) : tid % CH;
}

template <int LAYOUT>
__device__ __forceinline__ int32_t load_active(const SimtArgs &a, int c0, int tid)
{
    const int c = c0 + issue_ch<LAYOUT>(tid);
    return c < a.nact ? __ldg(a.active + c) : -1;
}

// fill stage st with channel chunk c0 and phi tile p0 of the block's lines of sight
template <bool FLY, int LAYOUT>
__device__ __forceinline__ void issue(const SimtArgs &a, Stage &st, int64_t l0, int c0, int p0, int32_t act,
                                      int tid)
{
    const int c = issue_ch<LAYOUT>(tid);
    if (LAYOUT == RMS_CHAN_MAJOR) {
        // 16 threads per channel, each 16 LOS at stride 16 (64-byte runs along LOS)
#pragma unroll 4
        for (int r = 0; r < TL / (256 / CH); ++r) {
            const int m = tid % (256 / CH) + r * (256 / CH);
            const bool ok = act >= 0 && l0 + m < a.nlos;
            const int64_t off = ok ? (int64_t)act * a.nlos + l0 + m : 0;
            cp_async<4>(&st.q[c][m], a.Q + off, ok);
            cp_async<4>(&st.u[c][m], a.U + off, ok);
        }
    } else {
        // consecutive threads take consecutive channels of one LOS
#pragma unroll 4
        for (int r = 0; r < TL / (256 / CH); ++r) {
            const int m = tid / CH + r * (256 / CH);
            const bool ok = act >= 0 && l0 + m < a.nlos;
            const int64_t off = ok ? (l0 + m) * a.nchan + act : 0;
            cp_async<4>(&st.q[c][m], a.Q + off, ok);
            cp_async<4>(&st.u[c][m], a.U + off, ok);
        }
    }
    if (!FLY) {
#pragma unroll
        for (int i = tid; i < CH * TP; i += 256) {
            const int c = i / TP, k = i % TP;
            const bool ok = c0 + c < a.nact && p0 + k < a.nphi;
            const int64_t off = ok ? (int64_t)(c0 + c) * a.nphi + p0 + k : 0;
            cp_async<8>(&st.cs[c][k], a.table + off, ok);
        }
    }
}

// on-the-fly phases: the operands of a thread's CH * TP / 256 phase-tile
// entries are loaded one chunk ahead and turned into (w cos, w sin) after the
// current chunk's accumulation, so their load latency is hidden behind it
constexpr int kFlyPer = CH * TP / 256;
struct FlyOps {
    float ph[kFlyPer], l2[kFlyPer], w[kFlyPer];
};

__device__ __forceinline__ void fly_load(const SimtArgs &a, FlyOps &o, int c0, int p0, int tid)
{
#pragma unroll
    for (int r = 0; r < kFlyPer; ++r) {
        const int i = tid + 256 * r, c = i / TP, k = i % TP;
        const bool ok = c0 + c < a.nact && p0 + k < a.nphi;
        // a padded entry gets weight 0 (and phase 0), hence (0, 0)
        o.ph[r] = ok ? __ldg(a.phi32 + p0 + k) : 0.f;
        o.l2[r] = ok ? __ldg(a.l2x + c0 + c) : 0.f;
        o.w[r] = ok ? __ldg(a.w32 + c0 + c) : 0.f;
    }
}

__device__ __forceinline__ void fly_store(Stage &st, const FlyOps &o, int tid)
{
#pragma unroll
    for (int r = 0; r < kFlyPer; ++r) {
        const int i = tid + 256 * r, c = i / TP, k = i % TP;
        float sn, cs;
        sincosf(o.ph[r] * o.l2[r], &sn, &cs);
        st.cs[c][k] = make_float2(o.w[r] * cs, o.w[r] * sn);
    }
}

// Pipeline state carried from one phi tile to the next.
struct Pipe {
    int t;          // (phi tile, channel chunk) pair being accumulated
    int total, nck;
    int32_t act;    // active-channel index for the next copy
};

// One phi tile starting at p0: accumulate all channel chunks, then scale, store
// and update the running peak.  JJ: phi pairs-of-16 of the tile that hold grid
// points (4 for a full tile; the last, partial tile drops the columns beyond).
template <int JJ, bool FLY, int LAYOUT>
__device__ __forceinline__ void phi_tile(const SimtArgs &a, Stage *stage, int64_t l0, int p0, Pipe &pp, FlyOps &fo,
                                         float (&bm)[8], int (&bi)[8])
{
    constexpr int NJ = 2 * JJ;
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    float re[8][NJ], im[8][NJ];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j) { re[i][j] = 0.f; im[i][j] = 0.f; }

    for (int ck = 0; ck < pp.nck; ++ck, ++pp.t) {
        const int n = pp.t + 1;
        if (n < pp.total) {
            issue<FLY, LAYOUT>(a, stage[n & 1], l0, (n % pp.nck) * CH, (n / pp.nck) * TP, pp.act, tid);
            if (FLY) fly_load(a, fo, (n % pp.nck) * CH, (n / pp.nck) * TP, tid);
            if (n + 1 < pp.total) pp.act = load_active<LAYOUT>(a, ((n + 1) % pp.nck) * CH, tid);
        }
        cp_commit();
        cp_wait_prev();
        __syncthreads();
        const Stage &st = stage[pp.t & 1];
#pragma unroll 2
        for (int c = 0; c < CH; ++c) {
            float qv[8], uv[8], cv[NJ], sv[NJ];
            load8(&st.q[c][8 * ty], qv);
            load8(&st.u[c][8 * ty], uv);
            // thread tx owns phi pairs 16 jj + 2 tx + {0, 1}: the 8 threads of a
            // row read 128 contiguous bytes per vector load (no bank conflict)
#pragma unroll
            for (int j = 0; j < NJ; j += 2) {
                const float4 v = *reinterpret_cast<const float4 *>(&st.cs[c][8 * j + 2 * tx]);
                cv[j] = v.x; sv[j] = v.y; cv[j + 1] = v.z; sv[j + 1] = v.w;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    // (q + iu)(c - is): Re += q c + u s, Im += u c - q s  (Eqs. qPhi, uPhi)
                    re[i][j] = fmaf(qv[i], cv[j], re[i][j]);
                    re[i][j] = fmaf(uv[i], sv[j], re[i][j]);
                    im[i][j] = fmaf(uv[i], cv[j], im[i][j]);
                    im[i][j] = fmaf(-qv[i], sv[j], im[i][j]);
                }
        }
        // stage n & 1 was last read before the previous trailing barrier
        if (FLY && n < pp.total) fly_store(stage[n & 1], fo, tid);
        __syncthreads();
    }

    // epilogue for this phi tile: scale by K, store, update the running peak
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t l = l0 + 8 * ty + i;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int k = p0 + 16 * (j >> 1) + 2 * tx + (j & 1);
            const float fr = re[i][j] * a.scale, fi = im[i][j] * a.scale;
            if (k < a.nphi) {
                const float m2 = __fadd_rn(__fmul_rn(fr, fr), __fmul_rn(fi, fi));
                if (m2 > bm[i]) { bm[i] = m2; bi[i] = k; }
                if (a.F != nullptr && l < a.nlos)
                    *reinterpret_cast<float2 *>(a.F + (l * a.nphi + k) * 2) = make_float2(fr, fi);
            }
        }
    }
}

template <bool FLY, int LAYOUT>
__global__ void __launch_bounds__(256, 1) simt_kernel(const SimtArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Stage *stage = reinterpret_cast<Stage *>(smem_raw);

    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int64_t l0 = (int64_t)blockIdx.x * TL;
    Pipe pp;
    pp.nck = (a.nact + CH - 1) / CH;
    pp.total = pp.nck * ((a.nphi + TP - 1) / TP);
    pp.t = 0;

    float bm[8];
    int bi[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { bm[i] = -1.0f; bi[i] = INT_MAX; }

    // two-stage pipeline over (phi tile, channel chunk) pairs t: the copies of
    // pair t + 1 are in flight while pair t is accumulated
    FlyOps fo;
    issue<FLY, LAYOUT>(a, stage[0], l0, 0, 0, load_active<LAYOUT>(a, 0, tid), tid);
    cp_commit();
    pp.act = pp.total > 1 ? load_active<LAYOUT>(a, (1 % pp.nck) * CH, tid) : -1;
    if (FLY) {
        fly_load(a, fo, 0, 0, tid);
        fly_store(stage[0], fo, tid);
    }
    const int full = a.nphi / TP, rem = a.nphi - full * TP;
    for (int it = 0; it < full; ++it) phi_tile<4, FLY, LAYOUT>(a, stage, l0, it * TP, pp, fo, bm, bi);
    // the last, partial tile computes only the pairs-of-16 that hold grid points
    switch ((rem + 15) / 16) {
    case 1: phi_tile<1, FLY, LAYOUT>(a, stage, l0, full * TP, pp, fo, bm, bi); break;
    case 2: phi_tile<2, FLY, LAYOUT>(a, stage, l0, full * TP, pp, fo, bm, bi); break;
    case 3: phi_tile<3, FLY, LAYOUT>(a, stage, l0, full * TP, pp, fo, bm, bi); break;
    case 4: phi_tile<4, FLY, LAYOUT>(a, stage, l0, full * TP, pp, fo, bm, bi); break;
    default: break;
    }

    // reduce the peak over the 8 threads (tx) that share each line of sight
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float m = bm[i];
        int k = bi[i];
#pragma unroll
        for (int off = 4; off >= 1; off >>= 1) {
            const float mo = __shfl_xor_sync(0xffffffffu, m, off);
            const int ko = __shfl_xor_sync(0xffffffffu, k, off);
            if (better(mo, ko, m, k)) { m = mo; k = ko; }
        }
        const int64_t l = l0 + 8 * ty + i;
        if (tx == 0 && l < a.nlos) {
            const bool ok = k != INT_MAX;
            if (a.pidx) a.pidx[l] = ok ? k : -1;
            if (a.pabs) a.pabs[l] = ok ? sqrtf(m) : __int_as_float(0x7fc00000);
            if (a.pphi) a.pphi[l] = ok ? a.phi32[k] : __int_as_float(0x7fc00000);
        }
    }
}

template <bool FLY, int LAYOUT>
cudaError_t launch_one(const SimtArgs &a, dim3 g, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(simt_kernel<FLY, LAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSimtSmem);
    if (e != cudaSuccess) return e;
    simt_kernel<FLY, LAYOUT><<<g, 256, kSimtSmem, s>>>(a);
    return cudaGetLastError();
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
    if (fly)
        return layout == RMS_CHAN_MAJOR ? launch_one<true, RMS_CHAN_MAJOR>(a, g, s)
                                        : launch_one<true, RMS_LOS_MAJOR>(a, g, s);
    return layout == RMS_CHAN_MAJOR ? launch_one<false, RMS_CHAN_MAJOR>(a, g, s)
                                    : launch_one<false, RMS_LOS_MAJOR>(a, g, s);
}
