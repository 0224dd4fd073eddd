// Seeded synthetic Stokes Q/U on the device: the training-data generator of the
// learned peak proposal, and the way large synthetic cubes are made without a
// host round trip.
//
// Source model (Sec. 2.1): per line of sight 1-3 components, each Faraday thin,
//     P(lambda^2) = p0 exp(2i (chi0 + phi0 lambda^2))            (Eqs. PAdefn, Pdefn)
// or a Burn slab of width W (F = p0 e^{2i chi0} / W on [phi0 - W/2, phi0 + W/2]),
//     P(lambda^2) = p0 exp(2i (chi0 + phi0 lambda^2)) sin(W lambda^2) / (W lambda^2),
// plus independent Gaussian noise on Q and U.  Random numbers are counter based:
// the SplitMix64 finaliser (Steele, Lea & Flood 2014) of
// seed * 0x9E3779B97F4A7C15 + los * 0xD1B54A32D192ED03 + draw * 0x8CB92BA72F3D8DD7,
// top 53 bits mapped to (0, 1]; normals by the Box-Muller cosine branch from
// draws 2^32 + 2 d and 2^32 + 2 d + 1.  Draw numbers: 0 component count; 1 + 8 c
// + {0 slab?, 1 phi0, 2 p0, 3 chi0, 4 W} for component c; 30 the SNR; noise on
// channel j: normal draws 2 j (Q) and 2 j + 1 (U).  The same definition is
// implemented independently on the host for the CPU checks, so any line of
// sight can be regenerated there.
#include <math.h>

#include <cmath>

#include "rms_internal.h"

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x)
{
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return x;
}

__device__ __forceinline__ double uni(uint64_t seed, uint64_t los, uint64_t draw)
{
    const uint64_t x = seed * 0x9E3779B97F4A7C15ull + los * 0xD1B54A32D192ED03ull + draw * 0x8CB92BA72F3D8DD7ull;
    return ((double)(mix64(x) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double normal(uint64_t seed, uint64_t los, uint64_t draw)
{
    const uint64_t base = (1ull << 32) + 2ull * draw;
    const double u1 = uni(seed, los, base), u2 = uni(seed, los, base + 1);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

struct GenParams {
    rms_source_model m;
    int64_t los0, nlos;
    int32_t nchan, layout;
    const double *lambda2;
    double noise_gain;          // sqrt(sum w^2) / sum w
    float *Q, *U;
};

// One thread per (line of sight, channel); the fast grid axis runs along the
// output's contiguous dimension.
__global__ void __launch_bounds__(256) generate_kernel(const GenParams P)
{
    const bool los_major = P.layout == RMS_LOS_MAJOR;
    const int64_t fast = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t slow = blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
    const int64_t l = los_major ? slow : fast;
    const int32_t j = (int32_t)(los_major ? fast : slow);
    if (l >= P.nlos || j >= P.nchan) return;
    const uint64_t seed = P.m.seed, los = (uint64_t)(P.los0 + l);
    const int span = P.m.ncomp_max - P.m.ncomp_min;
    const int ncomp = P.m.ncomp_min + min((int)(uni(seed, los, 0) * (span + 1)), span);
    const double l2 = P.lambda2[j];
    double q = 0.0, u = 0.0, pmax = 0.0;
    for (int c = 0; c < 3; ++c) {
        const uint64_t d = 1 + 8 * c;
        const bool present = c < ncomp;
        const bool slab = uni(seed, los, d) < P.m.slab_prob;
        const double phi0 = P.m.phi0_min + (P.m.phi0_max - P.m.phi0_min) * uni(seed, los, d + 1);
        const double p0 = present ? P.m.p0_min + (P.m.p0_max - P.m.p0_min) * uni(seed, los, d + 2) : 0.0;
        const double chi0 = M_PI * uni(seed, los, d + 3);
        const double W = slab ? P.m.slab_w * uni(seed, los, d + 4) : 0.0;
        const double wl = W * l2;
        const double env = wl == 0.0 ? 1.0 : sin(wl) / wl;
        const double amp = p0 * env;
        const double ang = 2.0 * (chi0 + phi0 * l2);
        q += amp * cos(ang);
        u += amp * sin(ang);
        pmax = fmax(pmax, p0);
    }
    double sigma = P.m.sigma;
    if (P.m.snr_min > 0.0) {
        const double snr = P.m.snr_min + (P.m.snr_max - P.m.snr_min) * uni(seed, los, 30);
        sigma = pmax / (snr * P.noise_gain);
    }
    if (sigma != 0.0) {
        q += sigma * normal(seed, los, 2ull * (uint64_t)j);
        u += sigma * normal(seed, los, 2ull * (uint64_t)j + 1);
    }
    const int64_t off = los_major ? l * P.nchan + j : (int64_t)j * P.nlos + l;
    P.Q[off] = (float)q;
    P.U[off] = (float)u;
}

}  // namespace

cudaError_t launch_generate(const rms_plan_s &p, const rms_source_model &m, int64_t los0, int64_t nlos,
                            int32_t layout, float *Q, float *U, cudaStream_t s)
{
    GenParams P;
    P.m = m;
    P.los0 = los0;
    P.nlos = nlos;
    P.nchan = p.nchan;
    P.layout = layout;
    P.lambda2 = p.d_lambda2_all;
    double sw = 0.0, sw2 = 0.0;
    for (double w : p.weights) {
        sw += w;
        sw2 += w * w;
    }
    P.noise_gain = std::sqrt(sw2) / sw;
    P.Q = Q;
    P.U = U;
    const bool los_major = layout == RMS_LOS_MAJOR;
    const int64_t nfast = los_major ? p.nchan : nlos;
    const int64_t nslow = los_major ? nlos : p.nchan;
    const int64_t gx = (nfast + 255) / 256;
    const int64_t gz = (nslow + 65535 - 1) / 65535;
    if (gx > 0x7fffffff || gz > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)gx, (unsigned)(nslow < 65535 ? nslow : 65535), (unsigned)gz);
    generate_kernel<<<grid, 256, 0, s>>>(P);
    return cudaGetLastError();
}

extern "C" rms_status rms_generate(rms_plan_t plan, const rms_source_model *model, int64_t los0, int64_t nlos,
                                   int32_t layout, float *Q, float *U, void *stream)
{
    if (!plan || !model || !Q || !U || los0 < 0 || nlos < 0) return RMS_ERR_INVALID_ARG;
    if (layout != RMS_CHAN_MAJOR && layout != RMS_LOS_MAJOR) return RMS_ERR_INVALID_ARG;
    const rms_source_model &m = *model;
    if (m.ncomp_min < 1 || m.ncomp_max > 3 || m.ncomp_min > m.ncomp_max) return RMS_ERR_INVALID_ARG;
    const double vals[] = {m.phi0_min, m.phi0_max, m.p0_min, m.p0_max, m.slab_prob, m.slab_w, m.sigma, m.snr_min,
                           m.snr_max};
    for (double v : vals)
        if (!std::isfinite(v)) return RMS_ERR_INVALID_ARG;
    if (m.slab_w < 0 || m.sigma < 0 || (m.snr_min > 0 && !(m.snr_max >= m.snr_min))) return RMS_ERR_INVALID_ARG;
    if (nlos == 0) return RMS_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != plan->device && cudaSetDevice(plan->device) != cudaSuccess) return RMS_ERR_CUDA;
    cudaError_t e = launch_generate(*plan, m, los0, nlos, layout, Q, U, reinterpret_cast<cudaStream_t>(stream));
    if (prev >= 0 && prev != plan->device) cudaSetDevice(prev);
    return e == cudaSuccess ? RMS_OK : RMS_ERR_CUDA;
}
