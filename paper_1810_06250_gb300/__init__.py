"""GB300-native Faraday rotation measure synthesis.

The compute lives in librms.so (CUDA, sm_103a; C ABI in include/rms.h).  This
package is its thin Python binding (_binding: the C names, argument
marshalling only), a convenience Plan wrapper, the build script, and the seeded
synthetic-cube generator (inputs).  Importing the package does not load the
library; the first call does, and raises if it has not been built.
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    EXPORTS, LAYOUTS, PRECISIONS, RmsError,
    RMS_AXIS_FREQ_HZ, RMS_AXIS_LAMBDA2, RMS_BF16, RMS_BF16X3, RMS_CHAN_MAJOR, RMS_ERR_CUDA,
    RMS_ERR_INVALID_ARG, RMS_ERR_OOM, RMS_ERR_TIMEOUT, RMS_ERR_UNSUPPORTED, RMS_FP16X3, RMS_FP32_CHIRPZ,
    RMS_FP32_SIMT_FLY, RMS_FP32_SIMT_TABLE, RMS_GET_ACTIVE, RMS_GET_B_HI, RMS_GET_B_LO,
    RMS_GET_LAMBDA2, RMS_GET_RMSF64, RMS_GET_TABLE, RMS_INFO_DEVICE, RMS_INFO_KPAD,
    RMS_INFO_NCHAN, RMS_INFO_NCHAN_ACTIVE, RMS_INFO_NPAD, RMS_INFO_NPHI, RMS_INFO_PRECISION,
    RMS_INFO_TILE_N, RMS_INFO_LAST_CTAS, RMS_INFO_LAST_PAIR, RMS_INFO_LAST_PANELS, RMS_INFO_LAST_KERNELS,
    RMS_LOS_MAJOR, RMS_OK,
    RMS_NOALLOC_MAX_LOS, load, rms_plan_create, rms_plan_destroy, rms_plan_get, rms_plan_info, rms_plan_set_timeout,
    rms_plan_sync, rms_rmsf, rms_status_string, rms_synth, rms_synth_host, rms_synth_noalloc,
    RMS_NET_GRADS, RMS_NET_HIDDEN, RMS_NET_MAX_BATCH, RMS_NET_NBINS, RMS_NET_NIN, RMS_NET_NPARAMS, RMS_NET_PARAMS,
    RMS_NET_STEPS, rms_source_model, rms_generate, rms_net_create, rms_net_destroy, rms_net_info, rms_net_params,
    rms_propose, rms_net_grad, rms_train_step, rms_window_create, rms_window_destroy, rms_synth_window,
    rms_peakmap_learned, rms_plan_set_kernel_timing, rms_plan_kernel_times, rms_peak_outputs, rms_synth_peaks,
    rms_selftest_wait_timeout, rms_clean_create, rms_clean_destroy, rms_clean, rms_refine_peaks,
    rms_window_centres, rms_plan_set_option, RMS_OPT_CONTRACTION, RMS_OPT_L2_BUDGET, RMS_OPT_SCHEDULE, RMS_SCHEDULE_AUTO,
    RMS_SCHEDULE_WHOLE, RMS_CONTRACT_AUTO,
    RMS_CONTRACT_SINGLE, RMS_CONTRACT_PAIR, rms_host_alloc, rms_host_free, HostBuffer,
)


class Plan:
    """Owns one rms_plan_t; frees it on close() / context exit / garbage collection."""

    def __init__(self, axis, phi, precision="bf16x3", weights=None, axis_kind=RMS_AXIS_FREQ_HZ, device=0):
        self.handle = rms_plan_create(axis, weights, phi, precision, axis_kind, device)
        self.nchan = rms_plan_info(self.handle, RMS_INFO_NCHAN)
        self.nact = rms_plan_info(self.handle, RMS_INFO_NCHAN_ACTIVE)
        self.nphi = rms_plan_info(self.handle, RMS_INFO_NPHI)
        self.device = device

    def synth(self, Q, U, nlos, layout="los", F_out=None, peak_idx=None, peak_abs=None, phi_peak=None,
              stream=None):
        rms_synth(self.handle, Q, U, nlos, layout, F_out, peak_idx, peak_abs, phi_peak, stream)

    def synth_host(self, Q, U, nlos, layout="los", F_out=None, peak_idx=None, peak_abs=None, phi_peak=None,
                   stream=None):
        rms_synth_host(self.handle, Q, U, nlos, layout, F_out, peak_idx, peak_abs, phi_peak, stream)

    def rmsf(self, R_out=None):
        return rms_rmsf(self.handle, R_out)

    def sync(self, stream=None):
        rms_plan_sync(self.handle, stream)

    def get(self, what):
        return rms_plan_get(self.handle, what)

    def close(self):
        if getattr(self, "handle", None):
            rms_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build(force: bool = False, verbose: bool = False) -> str:
    from .builder import build as _b
    return _b(force=force, verbose=verbose)
