// C ABI of the RM-synthesis library: plan creation, RMSF, synthesis dispatch,
// host-buffer synthesis, sticky device errors.  See include/rms.h for the
// contract of every entry point.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>

#include <sys/mman.h>

#include "rms_internal.h"

namespace {

constexpr double kCLight = 299792458.0;   // m/s, exact

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

rms_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return RMS_OK;
    if (e == cudaErrorMemoryAllocation) return RMS_ERR_OOM;
    return RMS_ERR_CUDA;
}

bool is_tensor(int prec) { return prec == RMS_BF16 || prec == RMS_BF16X3 || prec == RMS_FP16X3; }

template <typename T>
cudaError_t dalloc(T **p, size_t n)
{
    if (n == 0) n = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T));
}

void free_plan(rms_plan_s *p)
{
    if (!p) return;
    cudaFree(p->d_active);
    cudaFree(p->d_dl2);
    cudaFree(p->d_wact);
    cudaFree(p->d_phi);
    cudaFree(p->d_phi32);
    cudaFree(p->d_l2x32);
    cudaFree(p->d_w32);
    cudaFree(p->d_table);
    cudaFree(p->d_bhi);
    cudaFree(p->d_blo);
    cudaFree(p->d_R64);
    cudaFree(p->d_czt);
    cudaFree(p->d_dl2_all);
    cudaFree(p->d_lambda2_all);
    cudaFree(p->d_w_all);
    if (p->d_bhi_raw != p->d_bhi) cudaFree(p->d_bhi_raw);
    if (p->d_blo_raw != p->d_blo) cudaFree(p->d_blo_raw);
    cudaFree(p->d_kbmask);
    cudaFree(p->d_stage);
    cudaFree(p->d_rexp);
    cudaFree(p->d_scratch);
    for (cudaEvent_t x : p->tev) cudaEventDestroy(x);
    for (cudaEvent_t x : p->hev)
        if (x) cudaEventDestroy(x);
    if (p->s_h2d) cudaStreamDestroy(p->s_h2d);
    if (p->s_d2h) cudaStreamDestroy(p->s_d2h);
    if (p->last) cudaEventDestroy(p->last);
    if (p->h_err) cudaFreeHost(p->h_err);
    delete p;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

bool encode_b_map(CUtensorMap *map, void *base, int kpad, int npad, int tile_n)
{
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)npad};
    cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
    cuuint32_t box[2] = {(cuuint32_t)kKBlock, (cuuint32_t)tile_n};
    cuuint32_t estr[2] = {1, 1};
    return encode_tensor_map(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_SWIZZLE_64B);
}

// FWHM of |R|'s main lobe: |R| is even in phi, so find the first phi > 0 where
// |R(phi)| <= 1/2 by evaluating R on 1024-point grids on the device, three
// rounds of bracketing, then linear interpolation inside the last bracket.
double measure_fwhm(rms_plan_s *p)
{
    const int n = 1024;
    double *d_phi = nullptr, *d_R = nullptr;
    if (cudaMalloc(&d_phi, n * sizeof(double)) != cudaSuccess) return NAN;
    if (cudaMalloc(&d_R, 2 * n * sizeof(double)) != cudaSuccess) { cudaFree(d_phi); return NAN; }
    std::vector<double> phi(n), R(2 * n);
    double lo = 0.0, hi = 8.0 * p->fwhm_est;
    double result = NAN;
    bool found = false;
    for (int expand = 0; expand < 4 && !found; ++expand) {
        for (int round = 0; round < 3; ++round) {
            for (int i = 0; i < n; ++i) phi[i] = lo + (hi - lo) * i / (n - 1);
            if (cudaMemcpy(d_phi, phi.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
                launch_rmsf(*p, d_phi, n, d_R, nullptr, 0) != cudaSuccess ||
                cudaMemcpy(R.data(), d_R, 2 * n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
                goto out;
            int first = -1;
            for (int i = 1; i < n; ++i)
                if (std::hypot(R[2 * i], R[2 * i + 1]) <= 0.5) { first = i; break; }
            if (first < 0) {
                if (round > 0) goto out;
                break;
            }
            lo = phi[first - 1];
            hi = phi[first];
            if (round == 2) {
                double a = std::hypot(R[2 * (first - 1)], R[2 * (first - 1) + 1]);
                double b = std::hypot(R[2 * first], R[2 * first + 1]);
                double t = (a - 0.5) / (a - b);
                result = 2.0 * (lo + t * (hi - lo));
                found = true;
            }
        }
        if (!found) { lo = 0.0; hi *= 8.0; }
    }
out:
    cudaFree(d_phi);
    cudaFree(d_R);
    return result;
}

}  // namespace

bool encode_tensor_map(CUtensorMap *map, CUtensorMapDataType type, void *base, const cuuint64_t *dims,
                       const cuuint64_t *strides, const cuuint32_t *box, const cuuint32_t *estr,
                       CUtensorMapSwizzle swizzle, int rank)
{
    auto enc = get_encode();
    if (!enc) return false;
    CUresult r = enc(map, type, (cuuint32_t)rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

extern "C" {

const char *rms_status_string(rms_status s)
{
    switch (s) {
    case RMS_OK: return "success";
    case RMS_ERR_INVALID_ARG: return "invalid argument";
    case RMS_ERR_OOM: return "out of memory";
    case RMS_ERR_CUDA: return "CUDA error";
    case RMS_ERR_UNSUPPORTED: return "unsupported device or precision";
    case RMS_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

}  // extern "C"

rms_status plan_create_internal(rms_plan_t *out, const double *axis, int32_t nchan, int32_t axis_kind,
                                const double *weights, const double *phi, int32_t nphi, int32_t precision,
                                int32_t device, int32_t max_tile_cap)
{
    if (!out) return RMS_ERR_INVALID_ARG;
    *out = nullptr;
    if (!axis || !phi || nchan < 1 || nchan > 65536 || nphi < 1 || nphi > (1 << 20)) return RMS_ERR_INVALID_ARG;
    if (axis_kind != RMS_AXIS_LAMBDA2 && axis_kind != RMS_AXIS_FREQ_HZ) return RMS_ERR_INVALID_ARG;
    if (precision < RMS_FP32_SIMT_FLY || precision > RMS_FP32_CHIRPZ) return RMS_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return RMS_ERR_CUDA;
    if (device < 0 || device >= ndev) return RMS_ERR_INVALID_ARG;

    // plan constants (Sec. 2.2): lambda^2, K = 1/sum w, lambda_0^2 = weighted mean
    std::vector<double> lam2(nchan), w(nchan);
    double sw = 0.0, swl = 0.0, wmax = 0.0;
    for (int i = 0; i < nchan; ++i) {
        double a = axis[i];
        if (!std::isfinite(a)) return RMS_ERR_INVALID_ARG;
        if (axis_kind == RMS_AXIS_FREQ_HZ) {
            if (!(a > 0.0)) return RMS_ERR_INVALID_ARG;
            double lam = kCLight / a;
            lam2[i] = lam * lam;
        } else {
            lam2[i] = a;
        }
        double wi = weights ? weights[i] : 1.0;
        if (!std::isfinite(wi) || wi < 0.0) return RMS_ERR_INVALID_ARG;
        w[i] = wi;
        sw += wi;
        swl += wi * lam2[i];
        if (wi > wmax) wmax = wi;
    }
    if (!(sw > 0.0)) return RMS_ERR_INVALID_ARG;
    for (int k = 0; k < nphi; ++k)
        if (!std::isfinite(phi[k])) return RMS_ERR_INVALID_ARG;

    DeviceGuard guard(device);
    if (!guard.ok) return RMS_ERR_CUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return RMS_ERR_CUDA;
    // the library's device code is built for sm_103a only
    if (!(prop.major == 10 && prop.minor == 3)) return RMS_ERR_UNSUPPORTED;

    rms_plan_s *p = new (std::nothrow) rms_plan_s();
    if (!p) return RMS_ERR_OOM;
    p->device = device;
    p->nchan = nchan;
    p->nphi = nphi;
    p->precision = precision;
    p->K = 1.0 / sw;
    p->lambda0sq = swl / sw;
    p->wmax = wmax;
    p->lambda2 = lam2;
    p->weights = w;
    p->phi.assign(phi, phi + nphi);
    p->num_sms = prop.multiProcessorCount;
    std::vector<double> dl2, wact;
    double lmin = INFINITY, lmax = -INFINITY;
    for (int i = 0; i < nchan; ++i)
        if (w[i] != 0.0) {
            p->active.push_back(i);
            dl2.push_back(lam2[i] - p->lambda0sq);
            wact.push_back(w[i]);
            lmin = std::fmin(lmin, lam2[i]);
            lmax = std::fmax(lmax, lam2[i]);
        }
    p->nact = (int32_t)p->active.size();
    p->fwhm_est = lmax > lmin ? 2.0 * std::sqrt(3.0) / (lmax - lmin) : INFINITY;
    std::vector<float> phi32(nphi), l2x32(p->nact), w32(p->nact);
    for (int k = 0; k < nphi; ++k) phi32[k] = (float)phi[k];
    for (int a = 0; a < p->nact; ++a) {
        l2x32[a] = (float)(2.0 * dl2[a]);
        w32[a] = (float)wact[a];
    }

    cudaError_t e = cudaSuccess;
#define RMS_TRY(x)                   \
    do {                             \
        e = (x);                     \
        if (e != cudaSuccess) goto fail; \
    } while (0)
    RMS_TRY(cudaHostAlloc(reinterpret_cast<void **>(&p->h_err), sizeof(int), cudaHostAllocMapped));
    *p->h_err = 0;
    RMS_TRY(cudaHostGetDevicePointer(reinterpret_cast<void **>(&p->d_err), p->h_err, 0));
    RMS_TRY(dalloc(&p->d_active, p->nact));
    RMS_TRY(dalloc(&p->d_dl2, p->nact));
    RMS_TRY(dalloc(&p->d_wact, p->nact));
    RMS_TRY(dalloc(&p->d_phi, nphi));
    RMS_TRY(dalloc(&p->d_phi32, nphi));
    RMS_TRY(dalloc(&p->d_l2x32, p->nact));
    RMS_TRY(dalloc(&p->d_w32, p->nact));
    RMS_TRY(dalloc(&p->d_R64, 2 * (size_t)nphi));
    RMS_TRY(dalloc(&p->d_lambda2_all, nchan));
    RMS_TRY(cudaMemcpy(p->d_lambda2_all, lam2.data(), nchan * sizeof(double), cudaMemcpyHostToDevice));
    RMS_TRY(cudaMemcpy(p->d_active, p->active.data(), p->nact * sizeof(int32_t), cudaMemcpyHostToDevice));
    RMS_TRY(cudaMemcpy(p->d_dl2, dl2.data(), p->nact * sizeof(double), cudaMemcpyHostToDevice));
    RMS_TRY(cudaMemcpy(p->d_wact, wact.data(), p->nact * sizeof(double), cudaMemcpyHostToDevice));
    RMS_TRY(cudaMemcpy(p->d_phi, phi, nphi * sizeof(double), cudaMemcpyHostToDevice));
    RMS_TRY(cudaMemcpy(p->d_phi32, phi32.data(), nphi * sizeof(float), cudaMemcpyHostToDevice));
    RMS_TRY(cudaMemcpy(p->d_l2x32, l2x32.data(), p->nact * sizeof(float), cudaMemcpyHostToDevice));
    RMS_TRY(cudaMemcpy(p->d_w32, w32.data(), p->nact * sizeof(float), cudaMemcpyHostToDevice));

    if (precision == RMS_FP32_SIMT_TABLE) {
        RMS_TRY(dalloc(&p->d_table, (size_t)p->nact * nphi));
        RMS_TRY(launch_phase_table(*p, 0));
    } else if (precision == RMS_FP32_CHIRPZ) {
        const rms_status cst = czt_plan_build(p);
        if (cst != RMS_OK) {
            free_plan(p);
            return cst;
        }
    } else if (is_tensor(precision)) {
        const int N = 2 * nphi;
        // RMS_MAX_TILE_N (16..208, multiple of 16) in the environment lowers the phase
        // rows per tensor-core tile (a tuning knob: smaller tiles leave shared memory
        // for more pipeline stages)
        int max_tile = max_tile_cap;
        if (const char *v = std::getenv("RMS_MAX_TILE_N")) {
            int t = std::atoi(v);
            if (t >= 16 && t <= max_tile_cap && t % 16 == 0) max_tile = t;
        }
        // balanced tiles of at most max_tile rows, each a multiple of 16 (the last one
        // rounded up to 16 as well)
        auto tiling = [N](int cap, int32_t &ntiles, int32_t &tile, int32_t &last) {
            ntiles = (N + cap - 1) / cap;
            const int per = (N + ntiles - 1) / ntiles;
            tile = (per + 15) / 16 * 16;
            last = (N - (ntiles - 1) * tile + 15) / 16 * 16;
        };
        tiling(max_tile, p->ntiles_n, p->tile_n, p->tile_n_last);
        // CTA pairs take tiles of up to 256 rows (plans for the single-CTA window kernel keep theirs)
        if (max_tile_cap == kMaxTileN) tiling(kMaxTileNPair, p->ntiles_n2, p->tile_n2, p->tile_n_last2);
        else { p->ntiles_n2 = p->ntiles_n; p->tile_n2 = p->tile_n; p->tile_n_last2 = p->tile_n_last; }
        p->npad = std::max(p->ntiles_n * p->tile_n, p->ntiles_n2 * p->tile_n2);
        p->kblocks = (p->nact + kChanPerKBlock - 1) / kChanPerKBlock;
        p->kpad = p->kblocks * kKBlock;
        const bool fp16 = precision == RMS_FP16X3;
        RMS_TRY(dalloc(&p->d_bhi, (size_t)p->npad * p->kpad));
        RMS_TRY(dalloc(&p->d_blo, (size_t)p->npad * p->kpad));
        RMS_TRY(launch_phase_bsplit(*p, p->d_dl2, p->d_wact, p->nact, p->kpad, p->d_bhi, p->d_blo, fp16, 0));
        // LOS-major cubes contract over every channel (zero rows where flagged)
        p->kblocks_raw = (nchan + kChanPerKBlock - 1) / kChanPerKBlock;
        p->kpad_raw = p->kblocks_raw * kKBlock;
        std::vector<uint16_t> kbmask(p->kblocks_raw, 0);
        for (int i = 0; i < nchan; ++i)
            if (w[i] != 0.0) kbmask[i / kChanPerKBlock] |= (uint16_t)(1u << (i % kChanPerKBlock));
        RMS_TRY(dalloc(&p->d_kbmask, p->kblocks_raw));
        RMS_TRY(cudaMemcpy(p->d_kbmask, kbmask.data(), p->kblocks_raw * sizeof(uint16_t), cudaMemcpyHostToDevice));
        if (p->nact == nchan) {
            p->d_bhi_raw = p->d_bhi;
            p->d_blo_raw = p->d_blo;
        } else {
            std::vector<double> dl2_all(nchan);
            for (int i = 0; i < nchan; ++i) dl2_all[i] = lam2[i] - p->lambda0sq;
            RMS_TRY(dalloc(&p->d_dl2_all, nchan));
            RMS_TRY(dalloc(&p->d_w_all, nchan));
            RMS_TRY(cudaMemcpy(p->d_dl2_all, dl2_all.data(), nchan * sizeof(double), cudaMemcpyHostToDevice));
            RMS_TRY(cudaMemcpy(p->d_w_all, w.data(), nchan * sizeof(double), cudaMemcpyHostToDevice));
            RMS_TRY(dalloc(&p->d_bhi_raw, (size_t)p->npad * p->kpad_raw));
            RMS_TRY(dalloc(&p->d_blo_raw, (size_t)p->npad * p->kpad_raw));
            RMS_TRY(launch_phase_bsplit(*p, p->d_dl2_all, p->d_w_all, nchan, p->kpad_raw, p->d_bhi_raw,
                                        p->d_blo_raw, fp16, 0));
        }
        p->scratch_bytes = (size_t)p->num_sms * (size_t)std::max(p->kblocks, p->kblocks_raw) * kTileM * 128;
        RMS_TRY(cudaMalloc(&p->d_scratch, p->scratch_bytes));
        if (!encode_b_map(&p->tmap_bhi, p->d_bhi, p->kpad, p->npad, p->tile_n) ||
            !encode_b_map(&p->tmap_blo, p->d_blo, p->kpad, p->npad, p->tile_n) ||
            !encode_b_map(&p->tmap_bhi_raw, p->d_bhi_raw, p->kpad_raw, p->npad, p->tile_n) ||
            !encode_b_map(&p->tmap_blo_raw, p->d_blo_raw, p->kpad_raw, p->npad, p->tile_n)) {
            free_plan(p);
            return RMS_ERR_CUDA;
        }
        // half-tile boxes for the two-CTA contraction (tile_n a multiple of 16, so a
        // half is whole 8-row swizzle groups)
        if (p->tile_n2 % 16 == 0 && p->tile_n_last2 % 16 == 0) {
            const int h = p->tile_n2 / 2;
            p->pair_maps = encode_b_map(&p->tmap2_bhi, p->d_bhi, p->kpad, p->npad, h) &&
                           encode_b_map(&p->tmap2_blo, p->d_blo, p->kpad, p->npad, h) &&
                           encode_b_map(&p->tmap2_bhi_raw, p->d_bhi_raw, p->kpad_raw, p->npad, h) &&
                           encode_b_map(&p->tmap2_blo_raw, p->d_blo_raw, p->kpad_raw, p->npad, h);
        }
    }
    RMS_TRY(cudaEventCreateWithFlags(&p->last, cudaEventDisableTiming));
    // rms_synth_noalloc on this plan must find its array and kernels loaded on the device
    if (precision == RMS_FP16X3) RMS_TRY(noalloc_prepare(device));
    if (is_tensor(precision)) {
        // rms_synth takes per-call scratch from the device's default stream-ordered
        // pool; keep freed blocks reserved there so calls do not go back to the driver
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    RMS_TRY(launch_rmsf(*p, p->d_phi, nphi, p->d_R64, nullptr, 0));
    RMS_TRY(cudaDeviceSynchronize());
    p->fwhm_meas = measure_fwhm(p);
    RMS_TRY(cudaDeviceSynchronize());
#undef RMS_TRY
    *out = p;
    return RMS_OK;
fail:
    cudaGetLastError();
    free_plan(p);
    return from_cuda(e);
}

extern "C" {

rms_status rms_plan_create(rms_plan_t *out, const double *axis, int32_t nchan, int32_t axis_kind,
                           const double *weights, const double *phi, int32_t nphi, int32_t precision,
                           int32_t device)
{
    return plan_create_internal(out, axis, nchan, axis_kind, weights, phi, nphi, precision, device, kMaxTileN);
}

rms_status rms_plan_destroy(rms_plan_t p)
{
    if (!p) return RMS_OK;
    DeviceGuard guard(p->device);
    cudaDeviceSynchronize();
    free_plan(p);
    return RMS_OK;
}

rms_status rms_rmsf(rms_plan_t p, float *R_out, double *lambda0sq, double *K, double *fwhm_meas,
                    double *fwhm_est)
{
    if (!p) return RMS_ERR_INVALID_ARG;
    if (lambda0sq) *lambda0sq = p->lambda0sq;
    if (K) *K = p->K;
    if (fwhm_meas) *fwhm_meas = p->fwhm_meas;
    if (fwhm_est) *fwhm_est = p->fwhm_est;
    if (R_out) {
        DeviceGuard guard(p->device);
        cudaError_t e = launch_rmsf(*p, p->d_phi, p->nphi, nullptr, R_out, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return from_cuda(e);
    }
    return RMS_OK;
}

// Optional peak outputs beyond index, |F| and phi (tensor-core precisions only).
struct PeakExtras {
    float *q = nullptr, *u = nullptr, *chi = nullptr;
};

static rms_status synth_launch(rms_plan_t p, const float *Q, const float *U, int64_t nlos, int32_t layout,
                               float *F, int32_t *pidx, float *pabs, float *pphi, cudaStream_t s,
                               const PeakExtras &x);

static rms_status synth_device(rms_plan_t p, const float *Q, const float *U, int64_t nlos, int32_t layout,
                               float *F, int32_t *pidx, float *pabs, float *pphi, cudaStream_t s,
                               const PeakExtras &x = PeakExtras())
{
    // the plan's scratch is shared by its calls: order them on the device
    cudaError_t e = cudaStreamWaitEvent(s, p->last, 0);
    if (e != cudaSuccess) return from_cuda(e);
    rms_status st = synth_launch(p, Q, U, nlos, layout, F, pidx, pabs, pphi, s, x);
    e = cudaEventRecord(p->last, s);
    if (st == RMS_OK && e != cudaSuccess) st = from_cuda(e);
    return st;
}

static rms_status synth_launch(rms_plan_t p, const float *Q, const float *U, int64_t nlos, int32_t layout,
                               float *F, int32_t *pidx, float *pabs, float *pphi, cudaStream_t s,
                               const PeakExtras &x)
{
    cudaError_t e = cudaSuccess;
    switch (p->precision) {
    case RMS_FP32_SIMT_FLY:
    case RMS_FP32_SIMT_TABLE:
        e = launch_simt(*p, p->precision == RMS_FP32_SIMT_FLY, Q, U, nlos, layout, F, pidx, pabs, pphi, s);
        break;
    case RMS_FP32_CHIRPZ:
        e = launch_czt(*p, Q, U, nlos, layout, F, pidx, pabs, pphi, x.q, x.u, x.chi, s);
        break;
    case RMS_BF16:
    case RMS_BF16X3:
    case RMS_FP16X3: {
        // the split operand (and FP16X3's per-LOS exponents): stream-ordered scratch
        // and 8 bytes of peak key per LOS (the contraction's split schedule)
        const size_t abytes = split_operand_bytes(*p, nlos, layout);
        const size_t rbytes = p->precision == RMS_FP16X3 ? (size_t)((nlos + 255) & ~(int64_t)255) : 0;
        const size_t kbytes = (size_t)((nlos * 8 + 255) & ~(int64_t)255);
        uint8_t *scr = nullptr;
        e = cudaMallocAsync(reinterpret_cast<void **>(&scr), abytes + rbytes + kbytes, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return from_cuda(e);
        }
        cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
        if (p->timing) {
            for (auto &x : ev)
                if (cudaEventCreate(&x) != cudaSuccess) x = nullptr;
            if (ev[0] && ev[1] && ev[2]) {
                cudaEventRecord(ev[0], s);
            } else {
                for (auto &x : ev)
                    if (x) cudaEventDestroy(x);
                ev[0] = ev[1] = ev[2] = nullptr;
            }
            cudaGetLastError();
        }
        e = launch_split_gemm(*p, Q, U, nlos, layout, F, pidx, pabs, pphi, scr,
                              rbytes ? reinterpret_cast<int8_t *>(scr + abytes) : nullptr, s, ev[1], x.q, x.u, x.chi,
                              reinterpret_cast<unsigned long long *>(scr + abytes + rbytes));
        if (ev[2]) {
            if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);
            p->tev.insert(p->tev.end(), ev, ev + 3);
        }
        cudaError_t e2 = cudaFreeAsync(scr, s);
        if (e == cudaSuccess) e = e2;
        break;
    }
    default:
        return RMS_ERR_INVALID_ARG;
    }
    return from_cuda(e);
}

extern "C++" {
rms_status check_synth_args(rms_plan_t p, const float *Q, const float *U, int64_t nlos, int32_t layout,
                            float *F)
{
    if (!p || !Q || !U || nlos < 0) return RMS_ERR_INVALID_ARG;
    if (layout != RMS_CHAN_MAJOR && layout != RMS_LOS_MAJOR) return RMS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(Q) & 3) || (reinterpret_cast<uintptr_t>(U) & 3)) return RMS_ERR_INVALID_ARG;
    if (F && (reinterpret_cast<uintptr_t>(F) & 7)) return RMS_ERR_INVALID_ARG;
    if (nlos > ((int64_t)1 << 40) / ((int64_t)p->nchan + p->nphi)) return RMS_ERR_INVALID_ARG;
    return RMS_OK;
}
}  // extern "C++"

rms_status rms_synth(rms_plan_t p, const float *Q, const float *U, int64_t nlos, int32_t layout, float *F_out,
                     int32_t *peak_idx, float *peak_abs, float *phi_peak, void *stream)
{
    rms_status st = check_synth_args(p, Q, U, nlos, layout, F_out);
    if (st != RMS_OK) return st;
    if (*p->h_err) return RMS_ERR_TIMEOUT;
    if (nlos == 0 || (!F_out && !peak_idx && !peak_abs && !phi_peak)) return RMS_OK;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RMS_ERR_CUDA;
    return synth_device(p, Q, U, nlos, layout, F_out, peak_idx, peak_abs, phi_peak,
                        reinterpret_cast<cudaStream_t>(stream));
}

rms_status rms_synth_peaks(rms_plan_t p, const float *Q, const float *U, int64_t nlos, int32_t layout, float *F_out,
                           const rms_peak_outputs *out, void *stream)
{
    rms_status st = check_synth_args(p, Q, U, nlos, layout, F_out);
    if (st != RMS_OK) return st;
    if (!out) return RMS_ERR_INVALID_ARG;
    if (!is_tensor(p->precision) && p->precision != RMS_FP32_CHIRPZ && (out->q_peak || out->u_peak || out->chi0))
        return RMS_ERR_UNSUPPORTED;
    if (*p->h_err) return RMS_ERR_TIMEOUT;
    if (nlos == 0 ||
        (!F_out && !out->peak_idx && !out->peak_abs && !out->phi_peak && !out->q_peak && !out->u_peak && !out->chi0))
        return RMS_OK;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RMS_ERR_CUDA;
    PeakExtras x;
    x.q = out->q_peak;
    x.u = out->u_peak;
    x.chi = out->chi0;
    return synth_device(p, Q, U, nlos, layout, F_out, out->peak_idx, out->peak_abs, out->phi_peak,
                        reinterpret_cast<cudaStream_t>(stream), x);
}

rms_status rms_synth_host(rms_plan_t p, const float *Q, const float *U, int64_t nlos, int32_t layout, float *F_out,
                          int32_t *peak_idx, float *peak_abs, float *phi_peak, void *stream)
{
    rms_status st = check_synth_args(p, Q, U, nlos, layout, F_out);
    if (st != RMS_OK) return st;
    if (*p->h_err) return RMS_ERR_TIMEOUT;
    if (nlos == 0 || (!F_out && !peak_idx && !peak_abs && !phi_peak)) return RMS_OK;
    DeviceGuard guard(p->device);
    if (!guard.ok) return RMS_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // Chunks of LOS flow through kSlots device slots: copy in (stream h2d), synthesis
    // (the caller's stream), copy out (stream d2h), so the three overlap.  A cube of
    // fewer than two chunks runs as one chunk.
    constexpr int kSlots = 3;
    // Chunk sizes measured on GB300 (pinned memory): LOS-major chunks are contiguous, and
    // 16 of them pipeline best (LOFAR cube); a channel-major chunk is a 2-D copy of one
    // row per channel, efficient only when rows are >= 256 KB (65536 LOS), and at least 8
    // chunks keep the pipeline's fill and drain short (MWA cube, 1M LOS: 205 ms per call
    // with 8 chunks, 260 ms with 4; the 33.6 GB of F leaving over the host link set ~196 ms).
    // RMS_HOST_CHUNK (LOS, >= 1024) overrides the chunk size (a tuning knob).
    static const int64_t knob = [] {
        const char *v = std::getenv("RMS_HOST_CHUNK");
        const long long c = v ? std::atoll(v) : 0;
        return c >= 1024 ? (int64_t)c : (int64_t)0;
    }();
    const int64_t chunk = knob ? knob
                               : layout == RMS_LOS_MAJOR ? std::max<int64_t>(16384, (nlos + 15) / 16)
                                                         : std::max<int64_t>(65536, (nlos + 7) / 8);
    const int64_t nchunks = (nlos + chunk - 1) / chunk;
    const int slots = (int)std::min<int64_t>(kSlots, nchunks);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t in_b = (size_t)chunk * p->nchan * sizeof(float);
    const size_t f_b = F_out ? (size_t)chunk * p->nphi * 2 * sizeof(float) : 0;
    const size_t pk_b = (size_t)chunk * sizeof(float);
    const size_t slot_bytes = 2 * up(in_b) + up(f_b) + 3 * up(pk_b);
    const size_t need = slots * slot_bytes;
    if (need > p->stage_bytes) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return from_cuda(e);
        cudaFree(p->d_stage);
        p->d_stage = nullptr;
        p->stage_bytes = 0;
        if (cudaMalloc(&p->d_stage, need) != cudaSuccess) {
            cudaGetLastError();
            return RMS_ERR_OOM;
        }
        p->stage_bytes = need;
    }
    if (!p->s_h2d && cudaStreamCreateWithFlags(&p->s_h2d, cudaStreamNonBlocking) != cudaSuccess) return RMS_ERR_CUDA;
    if (!p->s_d2h && cudaStreamCreateWithFlags(&p->s_d2h, cudaStreamNonBlocking) != cudaSuccess) return RMS_ERR_CUDA;
    for (int k = 0; k < 3 * kSlots; ++k)
        if (!p->hev[k] && cudaEventCreateWithFlags(&p->hev[k], cudaEventDisableTiming) != cudaSuccess)
            return RMS_ERR_CUDA;
    cudaEvent_t *ev_in = p->hev, *ev_syn = p->hev + kSlots, *ev_out = p->hev + 2 * kSlots;
    // the staging slots may still be read by an earlier call's copies: start after them
    cudaError_t e = cudaStreamSynchronize(p->s_d2h);
    for (int64_t i = 0; i < nchunks && e == cudaSuccess && st == RMS_OK; ++i) {
        const int k = (int)(i % slots);
        const int64_t r0 = i * chunk, n = std::min(chunk, nlos - r0);
        char *b = static_cast<char *>(p->d_stage) + k * slot_bytes;
        float *dQ = reinterpret_cast<float *>(b);
        float *dU = reinterpret_cast<float *>(b + up(in_b));
        float *dF = F_out ? reinterpret_cast<float *>(b + 2 * up(in_b)) : nullptr;
        char *pk = b + 2 * up(in_b) + up(f_b);
        int32_t *dI = peak_idx ? reinterpret_cast<int32_t *>(pk) : nullptr;
        float *dA = peak_abs ? reinterpret_cast<float *>(pk + up(pk_b)) : nullptr;
        float *dP = phi_peak ? reinterpret_cast<float *>(pk + 2 * up(pk_b)) : nullptr;
        // copy in, once this slot's previous copy-out has finished
        if (i >= slots) e = cudaStreamWaitEvent(p->s_h2d, ev_out[k], 0);
        if (e != cudaSuccess) break;
        if (layout == RMS_LOS_MAJOR) {
            e = cudaMemcpyAsync(dQ, Q + r0 * p->nchan, (size_t)n * p->nchan * sizeof(float), cudaMemcpyHostToDevice,
                                p->s_h2d);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dU, U + r0 * p->nchan, (size_t)n * p->nchan * sizeof(float),
                                    cudaMemcpyHostToDevice, p->s_h2d);
        } else {   // channel-major: the chunk is n columns of every channel row
            e = cudaMemcpy2DAsync(dQ, n * sizeof(float), Q + r0, nlos * sizeof(float), n * sizeof(float), p->nchan,
                                  cudaMemcpyHostToDevice, p->s_h2d);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(dU, n * sizeof(float), U + r0, nlos * sizeof(float), n * sizeof(float),
                                      p->nchan, cudaMemcpyHostToDevice, p->s_h2d);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_in[k], p->s_h2d);
        // synthesis on the caller's stream
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_in[k], 0);
        if (e != cudaSuccess) break;
        st = synth_device(p, dQ, dU, n, layout, dF, dI, dA, dP, s);
        if (st != RMS_OK) break;
        e = cudaEventRecord(ev_syn[k], s);
        // copy out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_d2h, ev_syn[k], 0);
        if (e == cudaSuccess && F_out)
            e = cudaMemcpyAsync(F_out + r0 * p->nphi * 2, dF, (size_t)n * p->nphi * 2 * sizeof(float),
                                cudaMemcpyDeviceToHost, p->s_d2h);
        if (e == cudaSuccess && dI)
            e = cudaMemcpyAsync(peak_idx + r0, dI, n * sizeof(int32_t), cudaMemcpyDeviceToHost, p->s_d2h);
        if (e == cudaSuccess && dA)
            e = cudaMemcpyAsync(peak_abs + r0, dA, n * sizeof(float), cudaMemcpyDeviceToHost, p->s_d2h);
        if (e == cudaSuccess && dP)
            e = cudaMemcpyAsync(phi_peak + r0, dP, n * sizeof(float), cudaMemcpyDeviceToHost, p->s_d2h);
        if (e == cudaSuccess) e = cudaEventRecord(ev_out[k], p->s_d2h);
    }
    cudaError_t e2 = cudaStreamSynchronize(p->s_d2h);
    if (e == cudaSuccess) e = e2;
    e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (st != RMS_OK) return st;
    if (e != cudaSuccess) return from_cuda(e);
    return *p->h_err ? RMS_ERR_TIMEOUT : RMS_OK;
}

rms_status rms_host_alloc(int64_t bytes, void **ptr)
{
    if (!ptr) return RMS_ERR_INVALID_ARG;
    *ptr = nullptr;
    if (bytes <= 0) return RMS_ERR_INVALID_ARG;
    void *m = mmap(nullptr, (size_t)bytes, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (m == MAP_FAILED) return RMS_ERR_OOM;
#ifdef MADV_HUGEPAGE
    madvise(m, (size_t)bytes, MADV_HUGEPAGE);   // a hint: without huge pages the memory still works
#endif
    const cudaError_t e = cudaHostRegister(m, (size_t)bytes, cudaHostRegisterPortable);
    if (e != cudaSuccess) {
        cudaGetLastError();
        munmap(m, (size_t)bytes);
        return from_cuda(e);
    }
    *ptr = m;
    return RMS_OK;
}

rms_status rms_host_free(void *ptr, int64_t bytes)
{
    if (!ptr || bytes <= 0) return RMS_ERR_INVALID_ARG;
    const cudaError_t e = cudaHostUnregister(ptr);
    if (e != cudaSuccess) cudaGetLastError();
    if (munmap(ptr, (size_t)bytes) != 0) return RMS_ERR_INVALID_ARG;
    return e == cudaSuccess ? RMS_OK : RMS_ERR_CUDA;
}

rms_status rms_plan_sync(rms_plan_t p, void *stream)
{
    if (!p) return RMS_ERR_INVALID_ARG;
    DeviceGuard guard(p->device);
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaGetLastError();
    int err = *p->h_err;
    *p->h_err = 0;
    if (e != cudaSuccess) return RMS_ERR_CUDA;
    return err ? RMS_ERR_TIMEOUT : RMS_OK;
}

rms_status rms_plan_set_kernel_timing(rms_plan_t p, int32_t enable)
{
    if (!p) return RMS_ERR_INVALID_ARG;
    p->timing = enable != 0;
    return RMS_OK;
}

rms_status rms_plan_kernel_times(rms_plan_t p, double *split_ms, double *contract_ms, int64_t *calls)
{
    if (!p) return RMS_ERR_INVALID_ARG;
    DeviceGuard guard(p->device);
    double a = 0.0, b = 0.0;
    int64_t n = 0;
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i + 2 < p->tev.size(); i += 3) {
        float t0 = 0.f, t1 = 0.f;
        if (e == cudaSuccess) e = cudaEventSynchronize(p->tev[i + 2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, p->tev[i], p->tev[i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, p->tev[i + 1], p->tev[i + 2]);
        a += t0;
        b += t1;
        ++n;
    }
    for (cudaEvent_t x : p->tev) cudaEventDestroy(x);
    p->tev.clear();
    if (split_ms) *split_ms = a;
    if (contract_ms) *contract_ms = b;
    if (calls) *calls = n;
    return from_cuda(e);
}

rms_status rms_plan_set_timeout(rms_plan_t p, int64_t ns)
{
    if (!p || ns <= 0) return RMS_ERR_INVALID_ARG;
    p->timeout_ns = ns;
    return RMS_OK;
}

rms_status rms_plan_set_option(rms_plan_t p, int32_t option, int64_t value)
{
    if (!p) return RMS_ERR_INVALID_ARG;
    switch (option) {
    case RMS_OPT_CONTRACTION:
        if (value < RMS_CONTRACT_AUTO || value > RMS_CONTRACT_PAIR) return RMS_ERR_INVALID_ARG;
        if (value == RMS_CONTRACT_PAIR && !p->pair_maps) return RMS_ERR_UNSUPPORTED;
        p->contraction = (int32_t)value;
        return RMS_OK;
    case RMS_OPT_L2_BUDGET:
        if (value < 0) return RMS_ERR_INVALID_ARG;
        p->l2_budget = value;
        return RMS_OK;
    case RMS_OPT_SCHEDULE:
        if (value < RMS_SCHEDULE_AUTO || value > RMS_SCHEDULE_WHOLE) return RMS_ERR_INVALID_ARG;
        p->schedule = (int32_t)value;
        return RMS_OK;
    default: return RMS_ERR_INVALID_ARG;
    }
}

rms_status rms_plan_info(rms_plan_t p, int32_t what, int64_t *value)
{
    if (!p || !value) return RMS_ERR_INVALID_ARG;
    switch (what) {
    case RMS_INFO_NCHAN: *value = p->nchan; break;
    case RMS_INFO_NCHAN_ACTIVE: *value = p->nact; break;
    case RMS_INFO_NPHI: *value = p->nphi; break;
    case RMS_INFO_PRECISION: *value = p->precision; break;
    case RMS_INFO_KPAD: *value = p->kpad; break;
    case RMS_INFO_NPAD: *value = p->npad; break;
    case RMS_INFO_TILE_N: *value = p->tile_n; break;
    case RMS_INFO_DEVICE: *value = p->device; break;
    case RMS_INFO_LAST_CTAS: *value = p->last_ctas; break;
    case RMS_INFO_LAST_PAIR: *value = p->last_pair; break;
    case RMS_INFO_LAST_PANELS: *value = p->last_panels; break;
    case RMS_INFO_LAST_KERNELS: *value = p->last_kernels; break;
    default: return RMS_ERR_INVALID_ARG;
    }
    return RMS_OK;
}

rms_status rms_plan_get(rms_plan_t p, int32_t what, void *dst, int64_t bytes)
{
    if (!p || !dst) return RMS_ERR_INVALID_ARG;
    const void *src = nullptr;
    size_t n = 0;
    bool host = false;
    switch (what) {
    case RMS_GET_LAMBDA2: src = p->lambda2.data(); n = p->lambda2.size() * sizeof(double); host = true; break;
    case RMS_GET_ACTIVE: src = p->active.data(); n = p->active.size() * sizeof(int32_t); host = true; break;
    case RMS_GET_TABLE: src = p->d_table; n = (size_t)p->nact * p->nphi * sizeof(float2); break;
    case RMS_GET_B_HI: src = p->d_bhi; n = (size_t)p->npad * p->kpad * sizeof(uint16_t); break;
    case RMS_GET_B_LO: src = p->d_blo; n = (size_t)p->npad * p->kpad * sizeof(uint16_t); break;
    case RMS_GET_RMSF64: src = p->d_R64; n = (size_t)p->nphi * 2 * sizeof(double); break;
    default: return RMS_ERR_INVALID_ARG;
    }
    if (!src || (int64_t)n != bytes) return RMS_ERR_INVALID_ARG;
    if (host) {
        std::memcpy(dst, src, n);
        return RMS_OK;
    }
    DeviceGuard guard(p->device);
    return from_cuda(cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost));
}

}  // extern "C"
