// Chirp-z synthesis: Eq. Fsum evaluated with FFTs when the channels are
// uniform in lambda^2 and the phi grid is uniform (Sec. 4 names FFTs as the
// route to further speed; they are exact in this case).  With x_j = lambda_j^2 - lambda_0^2 = x_0 + j D and
// phi_k = phi_0 + k d, the phase of term (j, k) is
//     2 phi_k x_j = 2 phi_0 x_0 + 2 phi_0 D j + 2 d x_0 k + 2 d D j k,
// and 2 j k = j^2 + k^2 - (k - j)^2 turns the sum into a convolution:
//     F_k = v_k sum_j a_j h_{k-j},   a_j = w_j P_j g_j,
//     g_j = exp(-i (2 phi_0 D j + d D j^2)),   h_m = exp(+i d D m^2),
//     v_k = K exp(-i (2 phi_0 x_0 + 2 d x_0 k + d D k^2)).
// The linear convolution of the nchan inputs with h on m = -(nchan-1) .. nphi-1
// is a circular one of length M >= nchan + nphi - 1: c = IFFT(FFT(a) H), with
// H = FFT of h wrapped mod M (built on the host in FP64) and 1/M folded into v.
// This is exact: only the rounding of the FP32 FFT separates it from Eq. Fsum.
//
// One warp transforms one line of sight; M = 32 R (R = 32 or 64).  Element n of
// a length-M sequence is held by lane n % 32 in register n / 32.  Forward:
// an R-point DFT per lane in registers (radix 4), a twiddle, a transpose through
// shared memory, then 32-point DFTs per lane (the four-step FFT); the product with H;
// the inverse runs the same steps backwards, so its output comes back in the
// input's layout and the warp writes 32 consecutive phi per store.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <limits.h>
#include <vector>

#include "rms_internal.h"

namespace {

// warps per block: 16 for M = 1024 (one block of 512 threads per SM, 128
// registers each), 8 for M = 2048 (255 registers)
template <int R>
struct Warps {
    static constexpr int value = R == 32 ? 16 : 8;
};
// The per-warp transpose buffer holds R rows of kLd float2: the one-element pad
// lets a row written by 32 lanes and a column read by 32 lanes both take the
// minimum two shared-memory wavefronts.
constexpr int kLd = 33;
__device__ __forceinline__ int tidx(int row, int col) { return row * kLd + col; }

// W_64^m = exp(-2 pi i m / 64), m < 64: the twiddles of every in-register DFT
__constant__ float2 c_w64[64];

struct CztParams {
    const float *Q, *U;
    int64_t nlos;
    int32_t nchan, nphi, layout;
    const float2 *g;      // [nchan] w_j g_j (0 for flagged channels)
    const float2 *H;      // [M]
    const float2 *tw;     // [2 M]: T1[k1][lane] = W_M^(lane k1), then T2[s][n][lane] = W_M^(n (lane + 32 s))
    const float2 *v;      // [nphi] v_k / M
    const float *phi32;   // [nphi]
    const double *phi64;  // [nphi]
    double lambda0sq;
    float *F;
    int32_t *pidx;
    float *pabs, *pphi, *pq, *pu, *pchi;
};

// Output position of frequency k after the radix-4 (and, for N = 32, final
// radix-2) decimation-in-frequency stages: k = m1 + 4 m2 + 16 m3 sits at
// (N / 4) m1 + (N / 16) m2 + m3.
__host__ __device__ constexpr int digitrev(int k, int n)
{
    return (n / 4) * (k % 4) + (n / 16) * ((k / 4) % 4) + k / 16;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 cmulc(float2 a, float2 b)   // a * conj(b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// d * W_64^m (forward) or d * conj(W_64^m) (inverse); m a compile-time value
template <bool INV>
__device__ __forceinline__ float2 twiddle64(float2 d, int m)
{
    if (m == 0) return d;
    if (m == 32) return make_float2(-d.x, -d.y);
    if (m == 16) return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);   // -i, or +i inverse
    if (m == 48) return INV ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);   // +i, or -i inverse
    return INV ? cmulc(d, c_w64[m]) : cmul(d, c_w64[m]);
}

// In-register N-point DFT, N = 32 or 64, natural order in and out:
// v_k <- sum_n v_n W_N^(+-nk).  Radix-4 decimation in frequency (a last radix-2
// stage for N = 32), then the digit-reversal permutation, which is a renaming
// of registers once unrolled.  Per radix-4 butterfly on a span of L points:
//     t0 = a + c, t1 = a - c, t2 = b + d, t3 = -+i (b - d)
//     outputs t0 + t2, (t1 + t3) W_L^j, (t0 - t2) W_L^2j, (t1 - t3) W_L^3j.
template <int N, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[N])
{
#pragma unroll
    for (int L = N; L >= 4; L /= 4) {
        const int q = L / 4;
#pragma unroll
        for (int base = 0; base < N; base += L) {
#pragma unroll
            for (int j = 0; j < q; ++j) {
                const float2 a = v[base + j], b = v[base + j + q], c = v[base + j + 2 * q], d = v[base + j + 3 * q];
                const float2 t0 = make_float2(a.x + c.x, a.y + c.y), t1 = make_float2(a.x - c.x, a.y - c.y);
                const float2 t2 = make_float2(b.x + d.x, b.y + d.y);
                const float2 t3 = INV ? make_float2(d.y - b.y, b.x - d.x) : make_float2(b.y - d.y, d.x - b.x);
                v[base + j] = make_float2(t0.x + t2.x, t0.y + t2.y);
                v[base + j + q] = twiddle64<INV>(make_float2(t1.x + t3.x, t1.y + t3.y), j * 64 / L);
                v[base + j + 2 * q] = twiddle64<INV>(make_float2(t0.x - t2.x, t0.y - t2.y), 2 * j * 64 / L);
                v[base + j + 3 * q] = twiddle64<INV>(make_float2(t1.x - t3.x, t1.y - t3.y), 3 * j * 64 / L);
            }
        }
    }
    if (N == 32) {
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const float2 a = v[i], b = v[i + 1];
            v[i] = make_float2(a.x + b.x, a.y + b.y);
            v[i + 1] = make_float2(a.x - b.x, a.y - b.y);
        }
    }
    float2 t[N];
#pragma unroll
    for (int i = 0; i < N; ++i) t[i] = v[digitrev(i, N)];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = t[i];
}

__device__ __forceinline__ bool better(float m, int i, float bm, int bi)
{
    return m > bm || (m == bm && i < bi);
}

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Shared memory of one block, in float2 units: H [M], T1 [M], T2 [M] (only when
// R = 64: for R = 32 it equals T1), g [nchan], v [nphi], the W warps' transpose
// buffers [R][kLd], then with PF the block's input stage: Q and U of its W LOS,
// [W][2][nchan + 1] floats.
inline size_t czt_smem_floats2(int R, int W, int nchan, int nphi, bool pf)
{
    const size_t M = 32 * (size_t)R;
    return M * (R == 32 ? 2 : 3) + (size_t)nchan + (size_t)nphi + (size_t)W * R * kLd +
           (pf ? (size_t)W * (nchan + 1) : 0);
}

// Copy Q and U of LOS l0 .. l0 + W - 1 (those < nlos) into the stage; the
// block's threads split the elements so that each warp-wide copy reads
// contiguous runs: W LOS of 32 / W channels (channel-major), or 32 channels of
// a LOS (LOS-major).
template <int W>
__device__ __forceinline__ void stage_issue(const CztParams &P, float *st, int64_t l0)
{
    const int ld = P.nchan + 1;
    auto copy = [&](int i, int c) {
        const int64_t l = l0 + i;
        if (l < P.nlos) {
            const int64_t off = P.layout == RMS_CHAN_MAJOR ? (int64_t)c * P.nlos + l : l * P.nchan + c;
            cp_async4(st + (size_t)i * 2 * ld + c, P.Q + off);
            cp_async4(st + (size_t)i * 2 * ld + ld + c, P.U + off);
        }
    };
    if (P.layout == RMS_CHAN_MAJOR) {
        for (int e = threadIdx.x; e < W * P.nchan; e += blockDim.x) copy(e % W, e / W);
    } else {
        for (int i = 0; i < W; ++i)
            for (int c = threadIdx.x; c < P.nchan; c += blockDim.x) copy(i, c);
    }
}

// PF: the block copies the next W LOS into its shared stage with
// cp.async while its warps transform the current ones (the loads' latency is
// hidden behind the FFTs); without PF each warp loads its inputs directly.
// HALF: nchan <= M / 2 and nphi <= M / 2, so only the first R / 2 registers
// hold inputs and only the first R / 2 hold wanted outputs: the others are
// compile-time zeros or dead, and the compiler drops the work on them.
template <int R, bool PF, bool HALF>
__global__ void __launch_bounds__(32 * Warps<R>::value, 1) czt_kernel(const CztParams P)
{
    constexpr int M = 32 * R, r = R / 32, W = Warps<R>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sH = reinterpret_cast<float2 *>(smem_raw);
    float2 *sT1 = sH + M;
    float2 *sT2 = r == 1 ? sT1 : sT1 + M;
    float2 *sG = sT1 + (r == 1 ? M : 2 * M);
    float2 *sV = sG + P.nchan;
    float2 *bufs = sV + P.nphi;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *buf = bufs + warp * R * kLd;
    float *stage = reinterpret_cast<float *>(bufs + W * R * kLd);
    const int ld = P.nchan + 1;
    const float *mine = stage + (size_t)warp * 2 * ld;

    for (int i = threadIdx.x; i < M; i += blockDim.x) sH[i] = P.H[i];
    for (int i = threadIdx.x; i < r * M; i += blockDim.x) sT1[i] = P.tw[i];
    if (r == 2)
        for (int i = threadIdx.x; i < M; i += blockDim.x) sT2[i] = P.tw[M + i];
    for (int i = threadIdx.x; i < P.nchan; i += blockDim.x) sG[i] = P.g[i];
    for (int i = threadIdx.x; i < P.nphi; i += blockDim.x) sV[i] = P.v[i];
    __syncthreads();

    auto offset = [&](int j, int64_t l) {
        return P.layout == RMS_CHAN_MAJOR ? (int64_t)j * P.nlos + l : l * P.nchan + j;
    };
    // the warps of a block take consecutive LOS; the loop runs the same number of
    // times in every warp, so the block's barriers are reached by all of them
    const int64_t stride = (int64_t)gridDim.x * W;
    int64_t l0 = (int64_t)blockIdx.x * W;
    if (PF) {
        if (l0 < P.nlos) stage_issue<W>(P, stage, l0);
        cp_commit();
    }
    for (; l0 < P.nlos; l0 += stride) {
        const int64_t l = l0 + warp;
        float2 x[R];
        // a_j = w_j g_j (Q_j + i U_j), j = 32 n1 + lane; flagged channels (g_j = 0)
        // and the zero padding give 0, whatever the data holds there
        if (PF) {
            cp_wait_all();
            __syncthreads();
        }
#pragma unroll
        for (int n1 = 0; n1 < R; ++n1) {
            if (HALF && n1 >= R / 2) {
                x[n1] = make_float2(0.f, 0.f);
                continue;
            }
            const int j = 32 * n1 + lane;
            float2 a = make_float2(0.f, 0.f);
            if (j < P.nchan && l < P.nlos) {
                const float2 g = sG[j];
                const float2 d = PF ? make_float2(mine[j], mine[ld + j])
                                    : make_float2(__ldg(P.Q + offset(j, l)), __ldg(P.U + offset(j, l)));
                if (g.x != 0.f || g.y != 0.f) a = cmul(d, g);
            }
            x[n1] = a;
        }
        if (PF) {
            __syncthreads();
            if (l0 + stride < P.nlos) stage_issue<W>(P, stage, l0 + stride);
            cp_commit();
        }
        if (l >= P.nlos) continue;

        // forward: R-point DFTs over n1, twiddle W_M^(lane k1), transpose
        dft_reg<R, false>(x);
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) buf[tidx(k1, lane)] = cmul(x[k1], sT1[k1 * 32 + lane]);
        __syncwarp();
        // lane holds Y[k1][n2] for k1 = lane + 32 s; 32-point DFTs over n2 give
        // X[k1 + R k2]; times H; 32-point inverse DFTs over k2 give Z[k1][n]
#pragma unroll
        for (int s = 0; s < r; ++s) {
            float2 y[32];
            const int k1 = lane + 32 * s;
#pragma unroll
            for (int n2 = 0; n2 < 32; ++n2) y[n2] = buf[tidx(k1, n2)];
            dft_reg<32, false>(y);
#pragma unroll
            for (int k2 = 0; k2 < 32; ++k2) y[k2] = cmul(y[k2], sH[k1 + R * k2]);
            dft_reg<32, true>(y);
#pragma unroll
            for (int n = 0; n < 32; ++n) x[32 * s + n] = cmulc(y[n], sT2[(s * 32 + n) * 32 + lane]);
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < r; ++s)
#pragma unroll
            for (int n = 0; n < 32; ++n) buf[tidx(lane + 32 * s, n)] = x[32 * s + n];
        __syncwarp();
        // lane n holds Z[k1][n] for every k1; R-point inverse DFTs give c[n + 32 nb]
#pragma unroll
        for (int k1 = 0; k1 < R; ++k1) x[k1] = buf[tidx(k1, lane)];
        __syncwarp();
        dft_reg<R, true>(x);

        // F_k = v_k c_k for k = lane + 32 nb; the peak of |F| over the row
        float bm = -1.f, bre = 0.f, bim = 0.f;
        int bi = INT_MAX;
#pragma unroll
        for (int nb = 0; nb < (HALF ? R / 2 : R); ++nb) {
            const int k = lane + 32 * nb;
            if (k < P.nphi) {
                const float2 f = cmul(x[nb], sV[k]);
                const float m2 = __fadd_rn(__fmul_rn(f.x, f.x), __fmul_rn(f.y, f.y));
                if (m2 > bm) { bm = m2; bi = k; bre = f.x; bim = f.y; }
                if (P.F) reinterpret_cast<float2 *>(P.F)[l * P.nphi + k] = f;
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const float om = __shfl_xor_sync(0xffffffffu, bm, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            const float ore = __shfl_xor_sync(0xffffffffu, bre, off);
            const float oim = __shfl_xor_sync(0xffffffffu, bim, off);
            if (better(om, oi, bm, bi)) { bm = om; bi = oi; bre = ore; bim = oim; }
        }
        if (lane == 0) {
            const bool found = bi != INT_MAX;
            const float qnan = __int_as_float(0x7fc00000);
            if (P.pidx) P.pidx[l] = found ? bi : -1;
            if (P.pabs) P.pabs[l] = found ? sqrtf(bm) : qnan;
            if (P.pphi) P.pphi[l] = found ? P.phi32[bi] : qnan;
            if (P.pq) P.pq[l] = found ? bre : qnan;
            if (P.pu) P.pu[l] = found ? bim : qnan;
            if (P.pchi) {
                // chi0 = arg F(phi_peak) / 2 - phi_peak lambda_0^2, reduced to [0, pi)
                float c = qnan;
                if (found) {
                    double a = 0.5 * atan2((double)bim, (double)bre) - P.phi64[bi] * P.lambda0sq;
                    a -= M_PI * floor(a / M_PI);
                    c = (float)a;
                }
                P.pchi[l] = c;
            }
        }
    }
    if (PF) cp_wait_all();
}


// largest |v - (v_0 + i step)| over a sequence, step from its end points
double uniform_residual(const std::vector<double> &v, double *v0, double *step)
{
    const size_t n = v.size();
    *v0 = v[0];
    *step = n > 1 ? (v[n - 1] - v[0]) / (double)(n - 1) : 0.0;
    double worst = 0.0;
    for (size_t i = 0; i < n; ++i) worst = std::max(worst, std::fabs(v[i] - (v[0] + (double)i * *step)));
    return worst;
}

std::complex<double> expi(double a) { return std::complex<double>(std::cos(a), std::sin(a)); }

}  // namespace

// Plan-time constants of the chirp-z path, built in FP64 on the host.  Returns
// RMS_ERR_UNSUPPORTED unless the channels are uniform in lambda^2 and phi is
// uniform (each model's largest deviation, times the largest conjugate
// coordinate, moves no phase by more than 1e-8 rad) and nchan + nphi - 1 <= 2048.
rms_status czt_plan_build(rms_plan_s *p)
{
    const int nc = p->nchan, nk = p->nphi;
    std::vector<double> x(nc);
    double xmax = 0.0, phimax = 0.0;
    for (int j = 0; j < nc; ++j) {
        x[j] = p->lambda2[j] - p->lambda0sq;
        xmax = std::max(xmax, std::fabs(x[j]));
    }
    for (int k = 0; k < nk; ++k) phimax = std::max(phimax, std::fabs(p->phi[k]));
    double x0, D, phi0, d;
    const double ex = uniform_residual(x, &x0, &D), ep = uniform_residual(p->phi, &phi0, &d);
    if (2.0 * ex * phimax > 1e-8 || 2.0 * ep * xmax > 1e-8) return RMS_ERR_UNSUPPORTED;
    int M = 1024;
    while (M < nc + nk - 1) M *= 2;
    if (M > 2048) return RMS_ERR_UNSUPPORTED;
    const double dD = d * D;
    const double two_pi = 2.0 * M_PI;

    // g_j (times w_j), v_k (times K / M)
    std::vector<float2> g(nc), v(nk), H(M), tw(2 * M);
    for (int j = 0; j < nc; ++j) {
        const std::complex<double> e = p->weights[j] * expi(-(2.0 * phi0 * D * j + dD * (double)j * j));
        g[j] = make_float2((float)e.real(), (float)e.imag());
    }
    for (int k = 0; k < nk; ++k) {
        const std::complex<double> e = (p->K / M) * expi(-(2.0 * phi0 * x0 + 2.0 * d * x0 * k + dD * (double)k * k));
        v[k] = make_float2((float)e.real(), (float)e.imag());
    }
    // H_k = sum_n h~_n W_M^(n k), h~ = h wrapped mod M; W_M^m from one table, m = n k mod M
    std::vector<std::complex<double>> W(M), h(M, 0.0);
    for (int m = 0; m < M; ++m) W[m] = expi(-two_pi * m / M);
    for (int m = -(nc - 1); m <= nk - 1; ++m) h[(m + M) % M] = expi(dD * (double)m * m);
    for (int k = 0; k < M; ++k) {
        std::complex<double> s = 0.0;
        for (int n = 0; n < M; ++n)
            if (h[n] != 0.0) s += h[n] * W[(int)(((int64_t)n * k) % M)];
        H[k] = make_float2((float)s.real(), (float)s.imag());
    }
    const int R = M / 32;
    for (int k1 = 0; k1 < R; ++k1)
        for (int ln = 0; ln < 32; ++ln) {
            const std::complex<double> t = W[(ln * k1) % M];
            tw[k1 * 32 + ln] = make_float2((float)t.real(), (float)t.imag());
        }
    for (int s = 0; s < R / 32; ++s)
        for (int n = 0; n < 32; ++n)
            for (int ln = 0; ln < 32; ++ln) {
                const std::complex<double> t = W[(n * (ln + 32 * s)) % M];
                tw[M + (s * 32 + n) * 32 + ln] = make_float2((float)t.real(), (float)t.imag());
            }
    float2 w64[64];
    for (int m = 0; m < 64; ++m) {
        const std::complex<double> t = expi(-two_pi * m / 64.0);
        w64[m] = make_float2((float)t.real(), (float)t.imag());
    }

    cudaError_t e = cudaMemcpyToSymbol(c_w64, w64, sizeof(w64));
    const size_t n_all = (size_t)nc + nk + 3 * (size_t)M;
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&p->d_czt), n_all * sizeof(float2));
    if (e == cudaSuccess) {
        float2 *b = p->d_czt;
        e = cudaMemcpy(b, H.data(), M * sizeof(float2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b + M, tw.data(), 2 * M * sizeof(float2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b + 3 * M, g.data(), nc * sizeof(float2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b + 3 * M + nc, v.data(), nk * sizeof(float2), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? RMS_ERR_OOM : RMS_ERR_CUDA;
    }
    p->czt_M = M;
    return RMS_OK;
}

cudaError_t launch_czt(const rms_plan_s &p, const float *Q, const float *U, int64_t nlos, int layout, float *F,
                       int32_t *pidx, float *pabs, float *pphi, float *pq, float *pu, float *pchi, cudaStream_t s)
{
    const int M = p.czt_M;
    CztParams P;
    P.Q = Q;
    P.U = U;
    P.nlos = nlos;
    P.nchan = p.nchan;
    P.nphi = p.nphi;
    P.layout = layout;
    P.H = p.d_czt;
    P.tw = p.d_czt + M;
    P.g = p.d_czt + 3 * M;
    P.v = p.d_czt + 3 * M + p.nchan;
    P.phi32 = p.d_phi32;
    P.phi64 = p.d_phi;
    P.lambda0sq = p.lambda0sq;
    P.F = F;
    P.pidx = pidx;
    P.pabs = pabs;
    P.pphi = pphi;
    P.pq = pq;
    P.pu = pu;
    P.pchi = pchi;
    // one block per SM; the prefetching kernel where its stage fits
    const int R = M / 32, W = R == 32 ? Warps<32>::value : Warps<64>::value;
    constexpr size_t kSmemMax = 227 * 1024;
    const size_t s_pf = czt_smem_floats2(R, W, p.nchan, p.nphi, true) * sizeof(float2);
    const size_t s_np = czt_smem_floats2(R, W, p.nchan, p.nphi, false) * sizeof(float2);
    const bool pf = s_pf <= kSmemMax;
    const size_t smem = pf ? s_pf : s_np;
    if (smem > kSmemMax) return cudaErrorInvalidValue;
    const int64_t want = (nlos + W - 1) / W;
    const unsigned blocks = (unsigned)std::min<int64_t>(want, p.num_sms);
    auto go = [&](auto kern) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) kern<<<blocks, 32 * W, smem, s>>>(P);
        return err;
    };
    cudaError_t e;
    const bool half = 2 * p.nchan <= M && 2 * p.nphi <= M;
    if (R == 32) {
        if (half) e = pf ? go(czt_kernel<32, true, true>) : go(czt_kernel<32, false, true>);
        else e = pf ? go(czt_kernel<32, true, false>) : go(czt_kernel<32, false, false>);
    } else {
        if (half) e = pf ? go(czt_kernel<64, true, true>) : go(czt_kernel<64, false, true>);
        else e = pf ? go(czt_kernel<64, true, false>) : go(czt_kernel<64, false, false>);
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
}
