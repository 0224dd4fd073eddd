"""ctypes binding of include/rms.h -- argument marshalling only.

Every function here has the name of the C entry point it calls and does
nothing but convert arguments (torch tensors -> device pointers, numpy arrays
-> host pointers, the current torch stream -> cudaStream_t) and turn a
non-zero rms_status into an RmsError.  All arithmetic happens in librms.so.
There is no fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librms.so")

RMS_OK, RMS_ERR_INVALID_ARG, RMS_ERR_OOM, RMS_ERR_CUDA, RMS_ERR_UNSUPPORTED, RMS_ERR_TIMEOUT = range(6)
RMS_AXIS_LAMBDA2, RMS_AXIS_FREQ_HZ = 0, 1
RMS_CHAN_MAJOR, RMS_LOS_MAJOR = 0, 1
RMS_FP32_SIMT_FLY, RMS_FP32_SIMT_TABLE, RMS_BF16, RMS_BF16X3, RMS_FP16X3, RMS_FP32_CHIRPZ = range(6)
(RMS_INFO_NCHAN, RMS_INFO_NCHAN_ACTIVE, RMS_INFO_NPHI, RMS_INFO_PRECISION, RMS_INFO_KPAD,
 RMS_INFO_NPAD, RMS_INFO_TILE_N, RMS_INFO_DEVICE, RMS_INFO_LAST_CTAS, RMS_INFO_LAST_PAIR, RMS_INFO_LAST_PANELS,
 RMS_INFO_LAST_KERNELS) = range(12)
RMS_GET_LAMBDA2, RMS_GET_ACTIVE, RMS_GET_TABLE, RMS_GET_B_HI, RMS_GET_B_LO, RMS_GET_RMSF64 = range(6)

PRECISIONS = {"fp32_fly": RMS_FP32_SIMT_FLY, "fp32_table": RMS_FP32_SIMT_TABLE, "bf16": RMS_BF16,
              "bf16x3": RMS_BF16X3, "fp16x3": RMS_FP16X3, "fp32_czt": RMS_FP32_CHIRPZ}
LAYOUTS = {"chan": RMS_CHAN_MAJOR, "los": RMS_LOS_MAJOR}

# Every symbol include/rms.h declares (checked by the ABI test).
EXPORTS = ("rms_plan_create", "rms_rmsf", "rms_synth", "rms_synth_host", "rms_synth_noalloc",
           "rms_plan_sync", "rms_plan_info", "rms_plan_get", "rms_plan_destroy", "rms_status_string",
           "rms_plan_set_timeout", "rms_generate", "rms_net_create", "rms_net_destroy", "rms_net_info",
           "rms_net_params", "rms_propose", "rms_net_grad", "rms_train_step", "rms_window_create",
           "rms_window_destroy", "rms_synth_window", "rms_peakmap_learned", "rms_plan_set_kernel_timing",
           "rms_plan_kernel_times", "rms_synth_peaks", "rms_selftest_wait_timeout", "rms_clean_create",
           "rms_clean_destroy", "rms_clean", "rms_refine_peaks", "rms_window_centres", "rms_plan_set_option",
           "rms_host_alloc", "rms_host_free")
(RMS_NET_NPARAMS, RMS_NET_NIN, RMS_NET_HIDDEN, RMS_NET_NBINS, RMS_NET_MAX_BATCH, RMS_NET_STEPS) = range(6)
RMS_NET_PARAMS, RMS_NET_GRADS = 0, 1


class rms_peak_outputs(ctypes.Structure):
    """Mirror of the C struct rms_peak_outputs (include/rms.h)."""
    _fields_ = [("peak_idx", ctypes.c_void_p), ("peak_abs", ctypes.c_void_p), ("phi_peak", ctypes.c_void_p),
                ("q_peak", ctypes.c_void_p), ("u_peak", ctypes.c_void_p), ("chi0", ctypes.c_void_p)]


class rms_source_model(ctypes.Structure):
    """Mirror of the C struct rms_source_model (include/rms.h)."""
    _fields_ = [("seed", ctypes.c_uint64), ("ncomp_min", ctypes.c_int32), ("ncomp_max", ctypes.c_int32),
                ("phi0_min", ctypes.c_double), ("phi0_max", ctypes.c_double), ("p0_min", ctypes.c_double),
                ("p0_max", ctypes.c_double), ("slab_prob", ctypes.c_double), ("slab_w", ctypes.c_double),
                ("sigma", ctypes.c_double), ("snr_min", ctypes.c_double), ("snr_max", ctypes.c_double)]
RMS_NOALLOC_MAX_LOS = 1 << 22


class RmsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, rms_status_string(status), status))


_lock = threading.Lock()
_lib = None
_c_void_p = ctypes.c_void_p
_i32, _i64 = ctypes.c_int32, ctypes.c_int64


def load(path: str = LIB_PATH):
    """Load librms.so (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("librms.so is not built (%s); run paper_1810_06250_gb300.build()" % path)
        lib = ctypes.CDLL(path)
        P = _c_void_p
        sig = {
            "rms_plan_create": [ctypes.POINTER(P), P, _i32, _i32, P, P, _i32, _i32, _i32],
            "rms_rmsf": [P, P, P, P, P, P],
            "rms_synth": [P, P, P, _i64, _i32, P, P, P, P, P],
            "rms_synth_host": [P, P, P, _i64, _i32, P, P, P, P, P],
            "rms_synth_noalloc": [P, P, P, _i64, _i32, P, P, P, P, P],
            "rms_host_alloc": [_i64, ctypes.POINTER(P)],
            "rms_host_free": [P, _i64],
            "rms_plan_sync": [P, P],
            "rms_plan_info": [P, _i32, P],
            "rms_plan_get": [P, _i32, P, _i64],
            "rms_plan_destroy": [P],
            "rms_plan_set_timeout": [P, _i64],
            "rms_plan_set_option": [P, _i32, _i64],
            "rms_generate": [P, P, _i64, _i64, _i32, P, P, P],
            "rms_plan_set_kernel_timing": [P, _i32],
            "rms_synth_peaks": [P, P, P, _i64, _i32, P, P, P],
            "rms_selftest_wait_timeout": [P, _i64, P],
            "rms_refine_peaks": [P, P, _i64, P, P, P, P],
            "rms_clean_create": [ctypes.POINTER(P), P, ctypes.c_double, P],
            "rms_clean_destroy": [P],
            "rms_clean": [P, P, _i64, ctypes.c_float, _i32, ctypes.c_float, P, P, P, P, P],
            "rms_plan_kernel_times": [P, P, P, P],
            "rms_net_create": [ctypes.POINTER(P), P, _i32, _i32, ctypes.c_uint64],
            "rms_net_destroy": [P],
            "rms_net_info": [P, _i32, P],
            "rms_net_params": [P, _i32, P, _i64, _i32],
            "rms_propose": [P, P, P, _i64, _i32, _i32, P, P, P, P],
            "rms_net_grad": [P, P, P, _i64, _i32, P, P, P],
            "rms_train_step": [P, P, P, _i64, _i32, P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, ctypes.c_float, P, P],
            "rms_window_create": [ctypes.POINTER(P), P, _i32],
            "rms_window_destroy": [P],
            "rms_synth_window": [P, P, P, _i64, _i32, P, P, P, P, P, P],
            "rms_window_centres": [P, P, _i64, P, P],
            "rms_peakmap_learned": [P, P, P, P, _i64, _i32, ctypes.c_float, P, P, P, P, P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.rms_status_string.argtypes = [ctypes.c_int]
        lib.rms_status_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(st: int, where: str):
    if st != RMS_OK:
        raise RmsError(st, where)


def _dptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (or None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    return t.data_ptr()


def _hptr(a, dtype=None, name="array"):
    """Host pointer of a tensor/ndarray in CPU memory (or None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "is_cuda"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("%s must be a contiguous CPU tensor" % name)
        if dtype is not None and str(a.dtype) != "torch." + dtype:
            raise ValueError("%s must have dtype %s" % (name, dtype))
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("%s must be C-contiguous" % name)
    if dtype is not None and a.dtype != np.dtype(dtype):
        raise ValueError("%s must have dtype %s" % (name, dtype))
    return a.ctypes.data


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def rms_status_string(status: int) -> str:
    return load().rms_status_string(int(status)).decode()


def rms_plan_create(axis, weights, phi, precision, axis_kind=RMS_AXIS_FREQ_HZ, device=0) -> int:
    """Returns the opaque plan handle (an int).  See include/rms.h."""
    lib = load()
    axis = np.ascontiguousarray(axis, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    out = _c_void_p()
    st = lib.rms_plan_create(ctypes.byref(out), axis.ctypes.data, axis.shape[0], int(axis_kind),
                             None if w is None else w.ctypes.data, phi.ctypes.data, phi.shape[0],
                             int(precision), int(device))
    _check(st, "rms_plan_create")
    return out.value


def rms_plan_destroy(plan: int):
    _check(load().rms_plan_destroy(plan), "rms_plan_destroy")


def rms_rmsf(plan: int, R_out=None):
    """Returns (lambda0sq, K, fwhm_meas, fwhm_est); fills R_out (CUDA float32 [2*nphi]) if given."""
    lib = load()
    vals = [ctypes.c_double() for _ in range(4)]
    st = lib.rms_rmsf(plan, _dptr(R_out, None, "R_out"), *[ctypes.byref(v) for v in vals])
    _check(st, "rms_rmsf")
    return tuple(v.value for v in vals)


def _layout(layout):
    return LAYOUTS[layout] if isinstance(layout, str) else int(layout)


def rms_synth(plan: int, Q, U, nlos: int, layout, F_out=None, peak_idx=None, peak_abs=None,
              phi_peak=None, stream=None):
    """Asynchronous synthesis on CUDA tensors (see include/rms.h)."""
    import torch
    st = load().rms_synth(plan, _dptr(Q, torch.float32, "Q"), _dptr(U, torch.float32, "U"), int(nlos),
                          _layout(layout), _dptr(F_out, None, "F_out"),
                          _dptr(peak_idx, torch.int32, "peak_idx"), _dptr(peak_abs, torch.float32, "peak_abs"),
                          _dptr(phi_peak, torch.float32, "phi_peak"), _stream(stream))
    _check(st, "rms_synth")


def rms_synth_noalloc(plan: int, Q, U, nlos: int, layout, F_out=None, peak_idx=None, peak_abs=None,
                      phi_peak=None, stream=None):
    """rms_synth for FP16X3 plans with a fixed scratch array instead of a per-call
    pool allocation, for callers that must not allocate device memory while they
    process data (see include/rms.h: at most RMS_NOALLOC_MAX_LOS lines of sight,
    calls must not overlap on the GPU)."""
    import torch
    st = load().rms_synth_noalloc(plan, _dptr(Q, torch.float32, "Q"), _dptr(U, torch.float32, "U"), int(nlos),
                                  _layout(layout), _dptr(F_out, None, "F_out"),
                                  _dptr(peak_idx, torch.int32, "peak_idx"), _dptr(peak_abs, torch.float32, "peak_abs"),
                                  _dptr(phi_peak, torch.float32, "phi_peak"), _stream(stream))
    _check(st, "rms_synth_noalloc")


def rms_synth_host(plan: int, Q, U, nlos: int, layout, F_out=None, peak_idx=None, peak_abs=None,
                   phi_peak=None, stream=None):
    """Synthesis from host buffers (numpy arrays or CPU tensors, pinned for speed); synchronous."""
    st = load().rms_synth_host(plan, _hptr(Q, "float32", "Q"), _hptr(U, "float32", "U"), int(nlos),
                               _layout(layout), _hptr(F_out, None, "F_out"), _hptr(peak_idx, "int32", "peak_idx"),
                               _hptr(peak_abs, "float32", "peak_abs"), _hptr(phi_peak, "float32", "phi_peak"),
                               _stream(stream))
    _check(st, "rms_synth_host")


def rms_host_alloc(nbytes: int) -> int:
    """Page-locked host memory (huge-page backed where the kernel allows) for rms_synth_host."""
    p = _c_void_p()
    _check(load().rms_host_alloc(int(nbytes), ctypes.byref(p)), "rms_host_alloc")
    return int(p.value)


def rms_host_free(ptr: int, nbytes: int):
    _check(load().rms_host_free(ptr, int(nbytes)), "rms_host_free")


class HostBuffer:
    """A CPU torch tensor over rms_host_alloc memory; the memory is released by close()
    (or on leaving a with block), after which the tensor must not be used."""

    def __init__(self, shape, dtype="float32"):
        import torch
        shape = tuple(int(x) for x in (shape if isinstance(shape, (tuple, list)) else (shape,)))
        np_dtype = np.dtype(dtype)
        self.ptr = 0
        self.nbytes = max(1, int(np.prod(shape)) * np_dtype.itemsize)
        self.ptr = rms_host_alloc(self.nbytes)
        raw = (ctypes.c_uint8 * self.nbytes).from_address(self.ptr)
        arr = np.frombuffer(raw, dtype=np_dtype, count=int(np.prod(shape))).reshape(shape)
        self.tensor = torch.from_numpy(arr)

    def close(self):
        if self.ptr:
            self.tensor = None
            rms_host_free(self.ptr, self.nbytes)
            self.ptr = 0

    def __del__(self):
        try:
            self.close()
        except Exception:       # interpreter shutdown: the library may already be gone
            pass

    def __enter__(self):
        return self.tensor

    def __exit__(self, *exc):
        self.close()
        return False


def rms_plan_sync(plan: int, stream=None):
    _check(load().rms_plan_sync(plan, _stream(stream)), "rms_plan_sync")


RMS_OPT_CONTRACTION, RMS_OPT_L2_BUDGET, RMS_OPT_SCHEDULE = 0, 1, 2
RMS_SCHEDULE_AUTO, RMS_SCHEDULE_WHOLE = 0, 1
RMS_CONTRACT_AUTO, RMS_CONTRACT_SINGLE, RMS_CONTRACT_PAIR = 0, 1, 2


def rms_plan_set_option(plan: int, option: int, value: int):
    _check(load().rms_plan_set_option(plan, int(option), int(value)), "rms_plan_set_option")


def rms_plan_set_timeout(plan: int, ns: int):
    _check(load().rms_plan_set_timeout(plan, int(ns)), "rms_plan_set_timeout")


def rms_plan_info(plan: int, what: int) -> int:
    v = ctypes.c_int64()
    _check(load().rms_plan_info(plan, int(what), ctypes.byref(v)), "rms_plan_info")
    return v.value


def rms_plan_get(plan: int, what: int) -> np.ndarray:
    """Copy a plan-owned array to a new numpy array (shapes as in include/rms.h)."""
    nchan = rms_plan_info(plan, RMS_INFO_NCHAN)
    nact = rms_plan_info(plan, RMS_INFO_NCHAN_ACTIVE)
    nphi = rms_plan_info(plan, RMS_INFO_NPHI)
    kpad = rms_plan_info(plan, RMS_INFO_KPAD)
    npad = rms_plan_info(plan, RMS_INFO_NPAD)
    shapes = {
        RMS_GET_LAMBDA2: ((nchan,), np.float64),
        RMS_GET_ACTIVE: ((nact,), np.int32),
        RMS_GET_TABLE: ((nact, nphi, 2), np.float32),
        RMS_GET_B_HI: ((npad, kpad), np.uint16),
        RMS_GET_B_LO: ((npad, kpad), np.uint16),
        RMS_GET_RMSF64: ((nphi, 2), np.float64),
    }
    shape, dt = shapes[what]
    out = np.empty(shape, dtype=dt)
    _check(load().rms_plan_get(plan, int(what), out.ctypes.data, out.nbytes), "rms_plan_get")
    return out


def rms_generate(plan: int, model: rms_source_model, los0: int, nlos: int, layout, Q, U, stream=None):
    """Seeded synthetic Q/U on the device (include/rms.h); Q, U CUDA float32 tensors."""
    import torch
    st = load().rms_generate(plan, ctypes.byref(model), int(los0), int(nlos), _layout(layout),
                             _dptr(Q, torch.float32, "Q"), _dptr(U, torch.float32, "U"), _stream(stream))
    _check(st, "rms_generate")


def rms_net_create(plan: int, hidden: int, max_batch: int, seed: int) -> int:
    out = _c_void_p()
    _check(load().rms_net_create(ctypes.byref(out), plan, int(hidden), int(max_batch), int(seed)), "rms_net_create")
    return out.value


def rms_net_destroy(net: int):
    _check(load().rms_net_destroy(net), "rms_net_destroy")


def rms_net_info(net: int, what: int) -> int:
    v = _i64()
    _check(load().rms_net_info(net, int(what), ctypes.byref(v)), "rms_net_info")
    return v.value


def rms_net_params(net: int, which: int, host: np.ndarray, set: bool = False):
    """Copy parameters/gradients to (set=False) or parameters from (set=True) a float32 numpy array."""
    _check(load().rms_net_params(net, int(which), _hptr(host, "float32", "host"), host.size, 1 if set else 0),
           "rms_net_params")


def rms_propose(net: int, Q, U, nlos: int, layout, conf_halfwidth: int = -1, logits=None, bin=None, conf=None,
                stream=None):
    import torch
    st = load().rms_propose(net, _dptr(Q, torch.float32, "Q"), _dptr(U, torch.float32, "U"), int(nlos),
                            _layout(layout), int(conf_halfwidth), _dptr(logits, torch.float32, "logits"),
                            _dptr(bin, torch.int32, "bin"), _dptr(conf, torch.float32, "conf"), _stream(stream))
    _check(st, "rms_propose")


def rms_net_grad(net: int, Q, U, nlos: int, layout, label, loss=None, stream=None):
    import torch
    st = load().rms_net_grad(net, _dptr(Q, torch.float32, "Q"), _dptr(U, torch.float32, "U"), int(nlos),
                             _layout(layout), _dptr(label, torch.int32, "label"), _dptr(loss, torch.float32, "loss"),
                             _stream(stream))
    _check(st, "rms_net_grad")


def rms_train_step(net: int, Q, U, nlos: int, layout, label, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                   eps: float = 1e-8, weight_decay: float = 0.0, loss=None, stream=None):
    import torch
    st = load().rms_train_step(net, _dptr(Q, torch.float32, "Q"), _dptr(U, torch.float32, "U"), int(nlos),
                               _layout(layout), _dptr(label, torch.int32, "label"), float(lr), float(beta1),
                               float(beta2), float(eps), float(weight_decay), _dptr(loss, torch.float32, "loss"),
                               _stream(stream))
    _check(st, "rms_train_step")


def rms_window_create(plan: int, width: int) -> int:
    out = _c_void_p()
    _check(load().rms_window_create(ctypes.byref(out), plan, int(width)), "rms_window_create")
    return out.value


def rms_window_destroy(win: int):
    _check(load().rms_window_destroy(win), "rms_window_destroy")


def rms_window_centres(win: int, bin_, nlos: int, centre, stream=None):
    import torch
    st = load().rms_window_centres(win, _dptr(bin_, torch.int32, "bin"), int(nlos), _dptr(centre, torch.int32, "centre"),
                                   _stream(stream))
    _check(st, "rms_window_centres")


def rms_synth_window(win: int, Q, U, nlos: int, layout, centre, F_out=None, widx=None, wabs=None, wphi=None,
                     stream=None):
    import torch
    st = load().rms_synth_window(win, _dptr(Q, torch.float32, "Q"), _dptr(U, torch.float32, "U"), int(nlos),
                                 _layout(layout), _dptr(centre, torch.int32, "centre"), _dptr(F_out, None, "F_out"),
                                 _dptr(widx, torch.int32, "widx"), _dptr(wabs, torch.float32, "wabs"),
                                 _dptr(wphi, torch.float32, "wphi"), _stream(stream))
    _check(st, "rms_synth_window")


def rms_peakmap_learned(win: int, net: int, Q, U, nlos: int, layout, tau: float, phi_peak=None, peak_abs=None,
                        fallback=None, nfallback=None, stream=None):
    import torch
    st = load().rms_peakmap_learned(win, net, _dptr(Q, torch.float32, "Q"), _dptr(U, torch.float32, "U"),
                                    int(nlos), _layout(layout), float(tau), _dptr(phi_peak, torch.float32, "phi_peak"),
                                    _dptr(peak_abs, torch.float32, "peak_abs"),
                                    _dptr(fallback, torch.int32, "fallback"),
                                    _dptr(nfallback, torch.int64, "nfallback"), _stream(stream))
    _check(st, "rms_peakmap_learned")


def rms_plan_set_kernel_timing(plan: int, enable: bool):
    _check(load().rms_plan_set_kernel_timing(plan, 1 if enable else 0), "rms_plan_set_kernel_timing")


def rms_plan_kernel_times(plan: int):
    """(split_ms, contraction_ms, calls) summed over the calls timed since the last read."""
    a, b, n = ctypes.c_double(), ctypes.c_double(), _i64()
    _check(load().rms_plan_kernel_times(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)),
           "rms_plan_kernel_times")
    return a.value, b.value, n.value


def rms_synth_peaks(plan: int, Q, U, nlos: int, layout, F_out=None, peak_idx=None, peak_abs=None, phi_peak=None,
                    q_peak=None, u_peak=None, chi0=None, stream=None):
    """rms_synth with Q, U at the peak and the angle chi0 there (include/rms.h)."""
    import torch
    out = rms_peak_outputs(_dptr(peak_idx, torch.int32, "peak_idx"), _dptr(peak_abs, torch.float32, "peak_abs"),
                           _dptr(phi_peak, torch.float32, "phi_peak"), _dptr(q_peak, torch.float32, "q_peak"),
                           _dptr(u_peak, torch.float32, "u_peak"), _dptr(chi0, torch.float32, "chi0"))
    st = load().rms_synth_peaks(plan, _dptr(Q, torch.float32, "Q"), _dptr(U, torch.float32, "U"), int(nlos),
                                _layout(layout), _dptr(F_out, None, "F_out"), ctypes.byref(out), _stream(stream))
    _check(st, "rms_synth_peaks")


def rms_refine_peaks(plan: int, F, nlos: int, peak_idx, phi_ref=None, abs_ref=None, stream=None):
    """Parabolic sub-grid refinement of the peak (include/rms.h)."""
    import torch
    st = load().rms_refine_peaks(plan, _dptr(F, None, "F"), int(nlos), _dptr(peak_idx, torch.int32, "peak_idx"),
                                 _dptr(phi_ref, torch.float32, "phi_ref"), _dptr(abs_ref, torch.float32, "abs_ref"),
                                 _stream(stream))
    _check(st, "rms_refine_peaks")


def rms_selftest_wait_timeout(plan: int, limit_ns: int) -> int:
    """Run the bounded-wait self-test; returns 2 when the wait gave up (see include/rms.h)."""
    out = _i32()
    _check(load().rms_selftest_wait_timeout(plan, int(limit_ns), ctypes.byref(out)), "rms_selftest_wait_timeout")
    return out.value


def rms_clean_create(plan: int, fwhm: float = 0.0, R2_host=None) -> int:
    """RM-CLEAN object for a plan with a uniform phi grid (include/rms.h); R2_host: optional
    complex128 numpy array of R at the 2 nphi - 1 offsets."""
    out = _c_void_p()
    r2 = None
    if R2_host is not None:
        r2 = np.ascontiguousarray(np.stack([np.real(R2_host), np.imag(R2_host)], axis=-1), dtype=np.float64)
    _check(load().rms_clean_create(ctypes.byref(out), plan, float(fwhm), None if r2 is None else r2.ctypes.data),
           "rms_clean_create")
    return out.value


def rms_clean_destroy(c: int):
    _check(load().rms_clean_destroy(c), "rms_clean_destroy")


def rms_clean(c: int, F, nlos: int, gain: float, max_iter: int, threshold: float, F_clean=None, residual=None,
              components=None, niter=None, stream=None):
    import torch
    st = load().rms_clean(c, _dptr(F, None, "F"), int(nlos), float(gain), int(max_iter), float(threshold),
                          _dptr(F_clean, None, "F_clean"), _dptr(residual, None, "residual"),
                          _dptr(components, None, "components"), _dptr(niter, torch.int32, "niter"), _stream(stream))
    _check(st, "rms_clean")
