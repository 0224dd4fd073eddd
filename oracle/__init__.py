"""FP64 CPU oracle for RM synthesis -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct definition that the GPU
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import it; the product package never does,
and nothing here reads a value that the CUDA path produced.

The arithmetic lives in ``rms_oracle.c`` (plain C, double precision, OpenMP
over lines of sight).  This module compiles it with gcc, loads it with ctypes
and adds the host-side FWHM search of the RMSF main lobe.

Equations followed (Sridhar et al., cuFFS):
  * Eq. Fsum  F(phi) = K sum_i w_i P_i exp(-2i phi (lambda_i^2 - lambda_0^2))
  * Eq. Rsum  R(phi) = K sum_i w_i exp(-2i phi (lambda_i^2 - lambda_0^2))
  * Eq. Ksum  K = 1 / sum_i w_i
  * Sec. 2.2  lambda_0^2 = (weighted) mean of lambda_i^2; phi_peak = argmax |F|
  * Sec. 2.2  resolution estimate delta_phi ~ 2 sqrt(3) / Delta lambda^2
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rms_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

C_LIGHT = 299792458.0

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile rms_oracle.c into liboracle.so next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", _SRC, "-lm", "-o", tmp],
                       check=True)
        os.replace(tmp, _SO)
    return _SO


def _bind(path: str):
    lib = ctypes.CDLL(path)
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_plan.restype = ctypes.c_int
    lib.oracle_plan.argtypes = [_dp, ctypes.c_int32, ctypes.c_int32, _dp, _dp, _dp, _dp]
    lib.oracle_synth.restype = None
    lib.oracle_synth.argtypes = [ctypes.c_int64, ctypes.c_int32, _dp, _dp, _dp, _dp,
                                 ctypes.c_double, ctypes.c_double, _dp, ctypes.c_int32, _dp]
    lib.oracle_rmsf.restype = None
    lib.oracle_rmsf.argtypes = [ctypes.c_int32, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                _dp, ctypes.c_int32, _dp]
    lib.oracle_peak.restype = None
    lib.oracle_peak.argtypes = [ctypes.c_int64, ctypes.c_int32, _dp, _ip, _dp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_SO)
    return _lib


def compile_variant(src: str, out: str) -> str:
    """Compile another copy of the oracle source (used by tests that plant mistakes)."""
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", src, "-lm", "-o", out], check=True)
    return out


class use_library:
    """Context manager: route this module's calls through another compiled oracle."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self._saved = _lib
            _lib = _bind(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved
        return False


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().oracle_num_threads())


class Plan:
    """lambda^2, K and lambda_0^2 for one channel set (Sec. 2.2, Eq. Ksum)."""

    def __init__(self, lambda2, weights, K, lambda0sq):
        self.lambda2 = lambda2
        self.weights = weights
        self.K = K
        self.lambda0sq = lambda0sq

    @property
    def active(self):
        return np.nonzero(self.weights != 0.0)[0]


def plan(axis, kind: str = "freq", weights=None) -> Plan:
    """Plan constants.  kind='freq' (axis in Hz, lambda = c/nu) or 'lambda2' (m^2).

    Raises ValueError for a negative/non-finite weight, a non-positive weight sum
    or a non-finite axis value.
    """
    axis = _d(axis)
    n = axis.shape[0]
    w = np.ones(n) if weights is None else _d(weights)
    lam2 = np.empty(n)
    K = ctypes.c_double()
    l0 = ctypes.c_double()
    rc = _load().oracle_plan(_ptr(axis), n, 1 if kind == "freq" else 0, _ptr(w), _ptr(lam2),
                             ctypes.byref(K), ctypes.byref(l0))
    if rc != 0:
        raise ValueError("oracle_plan rejected the channel set (code %d)" % rc)
    return Plan(lam2, w, K.value, l0.value)


def synth(Q, U, p: Plan, phi) -> np.ndarray:
    """F(phi_k) for every line of sight, Eq. Fsum.  Q, U: [nlos][nchan] (LOS-major).

    Returns complex128 [nlos][nphi].
    """
    Q = _d(Q)
    U = _d(U)
    phi = _d(phi)
    if Q.ndim == 1:
        Q = Q[None, :]
        U = U[None, :]
    nlos, nchan = Q.shape
    F = np.empty((nlos, phi.shape[0], 2))
    _load().oracle_synth(nlos, nchan, _ptr(Q), _ptr(U), _ptr(_d(p.lambda2)), _ptr(_d(p.weights)),
                         p.lambda0sq, p.K, _ptr(phi), phi.shape[0], _ptr(F))
    return F[..., 0] + 1j * F[..., 1]


def rmsf(p: Plan, phi) -> np.ndarray:
    """R(phi_k), Eq. Rsum.  Returns complex128 [nphi]."""
    phi = _d(np.atleast_1d(phi))
    R = np.empty((phi.shape[0], 2))
    _load().oracle_rmsf(p.lambda2.shape[0], _ptr(_d(p.lambda2)), _ptr(_d(p.weights)), p.lambda0sq,
                        p.K, _ptr(phi), phi.shape[0], _ptr(R))
    return R[:, 0] + 1j * R[:, 1]


def peak(F):
    """argmax_k |F[l, k]| per row (lowest index on ties, NaN never chosen, -1 if none).

    Returns (idx int32 [nlos], |F| at the peak float64 [nlos]).
    """
    F = np.asarray(F)
    if F.ndim == 1:
        F = F[None, :]
    Fd = np.ascontiguousarray(np.stack([F.real, F.imag], axis=-1), dtype=np.float64)
    nlos, nphi = F.shape
    idx = np.empty(nlos, dtype=np.int32)
    a = np.empty(nlos)
    _load().oracle_peak(nlos, nphi, _ptr(Fd), _ptr(idx, _ip), _ptr(a))
    return idx, a


def fwhm_estimate(p: Plan) -> float:
    """Sec. 2.2 resolution estimate 2 sqrt(3) / Delta lambda^2 over the weighted channels."""
    lam = p.lambda2[p.weights != 0.0]
    return 2.0 * np.sqrt(3.0) / (lam.max() - lam.min())


def fwhm_measured(p: Plan) -> float:
    """Full width at half maximum of |R(phi)|'s main lobe, measured on the oracle RMSF.

    |R| is even in phi (R(-phi) = conj R(phi)), so the FWHM is twice the first
    phi > 0 where |R| drops to 1/2: stepped at 1/200 of the estimate, then bisected.
    """
    est = fwhm_estimate(p)
    h = est / 200.0
    lo, hi = 0.0, h
    while abs(rmsf(p, hi)[0]) > 0.5:
        lo, hi = hi, hi + h
        if hi > 50 * est:
            raise RuntimeError("RMSF main lobe never falls to half maximum")
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if abs(rmsf(p, mid)[0]) > 0.5:
            lo = mid
        else:
            hi = mid
    return 2.0 * 0.5 * (lo + hi)


def chi0(F_peak, phi_peak, lambda0sq):
    """Polarisation angle at the peak (Sec. 2.2): 0.5 arg F(phi_peak) - phi_peak lambda_0^2, in [0, pi).

    The printed relation is garbled (an angle times a complex factor); this is its
    reading from the thin-source identity F(phi0) = p0 exp(2i (chi0 + phi0 lambda_0^2)).
    """
    F_peak = np.asarray(F_peak)
    x = 0.5 * np.arctan2(F_peak.imag, F_peak.real) - np.asarray(phi_peak, dtype=np.float64) * lambda0sq
    return x - np.pi * np.floor(x / np.pi)


def refine_peak(F, phi, idx):
    """Sub-grid peak: the vertex of the parabola through |F| at phi[k-1], phi[k], phi[k+1], k = idx.

    The paper reports the grid sample where |F| peaks (Sec. 2.2); this
    interpolates between samples.  The parabola is the exact quadratic
    interpolant of the three points (numpy.polyfit of degree 2, in t = phi -
    phi[k]); its vertex t* = -c1 / (2 c2) is kept inside [phi[k-1], phi[k+1]].
    Where the vertex is undefined -- k at an end of the grid, an interpolant
    that is not concave (c2 >= 0), a non-finite neighbour, or both neighbours
    on one side of phi[k] -- the sample itself is returned.  NaN where idx < 0.

    F: complex [nlos][nphi]; phi: [nphi]; idx: int [nlos].
    Returns (phi_ref, abs_ref), float64 [nlos].
    """
    F = np.atleast_2d(np.asarray(F))
    phi = np.asarray(phi, dtype=np.float64)
    idx = np.asarray(idx)
    nlos, nphi = F.shape
    phi_ref = np.full(nlos, np.nan)
    abs_ref = np.full(nlos, np.nan)
    for l in range(nlos):
        k = int(idx[l])
        if k < 0 or k >= nphi:
            continue
        y = np.abs(F[l].astype(np.complex128))
        phi_ref[l], abs_ref[l] = phi[k], y[k]
        if k == 0 or k == nphi - 1:
            continue
        t = phi[k - 1:k + 2] - phi[k]
        yy = y[k - 1:k + 2]
        if not (t[0] * t[2] < 0.0) or not np.all(np.isfinite(yy)):
            continue
        c2, c1, c0 = np.polyfit(t, yy, 2)
        if not c2 < 0.0:
            continue
        ts = min(max(-c1 / (2.0 * c2), min(t[0], t[2])), max(t[0], t[2]))
        phi_ref[l] = phi[k] + ts
        abs_ref[l] = np.polyval([c2, c1, c0], ts)
    return phi_ref, abs_ref
