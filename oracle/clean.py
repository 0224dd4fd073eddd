"""FP64 CPU oracle of RM-CLEAN -- TEST INFRASTRUCTURE ONLY.

Only tests/ and the benchmark's CPU leg use this module.  RM-CLEAN deconvolves
a dirty Faraday spectrum F (Eq. Fsum) with the RMSF R (Eq. Rsum); the paper
names it as the next step after synthesis (Sec. 2.2, Sec. 4) without giving
the algorithm.  This is the Hogbom form used for RM synthesis: repeat

    j = argmax_k |res_k|               (lowest index on ties)
    stop if |res_j| < threshold
    c = gain * res_j;  comp_j += c;  res_k -= c * R(phi_k - phi_j)  for every k

at most max_iter times, on a uniform phi grid (so R(phi_k - phi_j) is R at
(k - j) dphi).  The clean spectrum restores the components with a real
Gaussian beam of the RMSF's FWHM, truncated at W = ceil(3 FWHM / dphi) bins:

    clean_k = res_k + sum_{|d| <= W} comp_{k-d} exp(-4 ln 2 (d dphi)^2 / FWHM^2)

The residual of a single Faraday-thin source on the grid is (1 - gain)^n F
exactly (res stays proportional to F, so its maximum stays put); the tests
pin that.
"""
from __future__ import annotations

import math

import numpy as np


def beam_halfwidth(fwhm, dphi):
    return int(math.ceil(3.0 * fwhm / dphi))


def clean(F, R2, gain, max_iter, threshold, fwhm, dphi):
    """F: complex [nlos][N] dirty spectra; R2: complex [2N - 1], R at (m - N + 1) dphi.

    Returns (clean, residual, components, niter)."""
    F = np.atleast_2d(np.asarray(F, dtype=np.complex128))
    nlos, N = F.shape
    W = min(N - 1, beam_halfwidth(fwhm, dphi))
    d = np.arange(-W, W + 1)
    beam = np.exp(-4.0 * math.log(2.0) * (d * dphi) ** 2 / fwhm ** 2)
    R2 = np.asarray(R2, dtype=np.complex128)
    Rr, Ri = np.ascontiguousarray(R2.real), np.ascontiguousarray(R2.imag)
    res = F.copy()
    comp = np.zeros_like(F)
    niter = np.zeros(nlos, dtype=np.int32)
    thr = float(threshold)
    thr2 = thr * thr
    g = float(gain)
    for l in range(nlos):
        # real and imaginary parts kept apart: every product and sum is one rounded
        # operation (no fused multiply-add), the arithmetic the definition states
        rr, ri = res[l].real.copy(), res[l].imag.copy()
        it = 0
        while it < max_iter:
            m2 = np.add(np.multiply(rr, rr), np.multiply(ri, ri))
            if np.all(np.isnan(m2)):
                break
            j = int(np.nanargmax(m2))        # first maximum
            if not m2[j] >= thr2:
                break
            cr, ci = g * rr[j], g * ri[j]
            comp[l, j] += complex(cr, ci)
            sr, si = Rr[N - 1 - j:2 * N - 1 - j], Ri[N - 1 - j:2 * N - 1 - j]
            rr = np.subtract(rr, np.subtract(np.multiply(cr, sr), np.multiply(ci, si)))
            ri = np.subtract(ri, np.add(np.multiply(cr, si), np.multiply(ci, sr)))
            it += 1
        res[l] = rr + 1j * ri
        niter[l] = it
    cl = res.copy()
    for l in range(nlos):
        for k in range(N):
            lo, hi = max(0, k - W), min(N - 1, k + W)
            cl[l, k] += np.sum(comp[l, lo:hi + 1] * beam[W - (k - np.arange(lo, hi + 1))])
    return cl, res, comp, niter
