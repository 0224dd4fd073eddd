"""Checks that pin the FP64 oracle to facts fixed by the paper and by mathematics.

Each check takes the ``oracle`` module and raises AssertionError on failure.
They are collected in PINS so that tests/test_oracle_mutations.py can run all
of them against copies of the oracle with a planted mistake and show that
every such mistake is caught by at least one of them.

What pins what (Sridhar et al., cuFFS):
  golden      hand-derived F, R, K, lambda_0^2 (Eqs. Fsum, Rsum, Ksum) and peaks
  rmsf        R(0) = 1 (Eq. Ksum), |R| <= 1, R(-phi) = conj R(phi),
              dR/dphi(0) = 0 for the weighted lambda_0^2
  thin        Faraday-thin source: F(phi) = p0 e^{2i(chi0 + phi0 lambda_0^2)} R(phi - phi0)
              (Eqs. Pdefn, Fsum, Rsum), peak at phi0 with |F| = p0 on the grid
  linearity   F is linear in (Q, U) (Eq. Fsum)
  flagged     channels with w = 0 have no effect, even with NaN data (Sec. 2.1)
  fft         uniform lambda^2 and phi grids turn Eq. Fsum into a DFT (Sec. 4 names FFT)
  fwhm        resolution 2 sqrt(3) / Delta lambda^2 (Sec. 2.2) and the exact
              sinc half-width for continuous uniform lambda^2 coverage
  realform    Eqs. qPhi, uPhi evaluated in 40-digit arithmetic
"""
from __future__ import annotations

import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hand_worked.json")


def _num(x):
    return float("nan") if x == "nan" else float(x)


def _cplx(rows):
    return np.array([complex(_num(r[0]), _num(r[1])) for r in rows])


def check_golden(o):
    g = json.load(open(GOLDEN))
    for case in g["cases"]:
        p = o.plan(case["lambda2"], kind="lambda2", weights=case["weights"])
        assert abs(p.K - case["K"]) <= 1e-15, (case["name"], p.K)
        assert abs(p.lambda0sq - case["lambda0sq"]) <= 1e-15, (case["name"], p.lambda0sq)
        phi = np.pi * np.array(case["phi_over_pi"])
        Q = np.array([_num(v) for v in case["Q"]])
        U = np.array([_num(v) for v in case["U"]])
        F = o.synth(Q[None], U[None], p, phi)[0]
        np.testing.assert_allclose(F, _cplx(case["F"]), rtol=0, atol=1e-14, err_msg=case["name"])
        R = o.rmsf(p, phi)
        np.testing.assert_allclose(R, _cplx(case["R"]), rtol=0, atol=1e-14, err_msg=case["name"])
    fa = g["frequency_axis"]
    p = o.plan(fa["freq_hz"], kind="freq")
    np.testing.assert_allclose(p.lambda2, fa["lambda2"], rtol=1e-15, atol=0)
    for row in g["peaks"]["rows"]:
        idx, _ = o.peak(_cplx(row["F"])[None])
        assert int(idx[0]) == row["idx"], (row, idx)


def _lofar_like(nchan=400, seed=7, flags=True):
    rng = np.random.default_rng(seed)
    freq = np.linspace(115e6, 178e6, nchan)
    w = rng.uniform(0.2, 2.0, nchan)
    if flags:
        w[rng.choice(nchan, nchan // 10, replace=False)] = 0.0
    return freq, w


def check_rmsf(o):
    freq, w = _lofar_like()
    p = o.plan(freq, "freq", w)
    R0 = o.rmsf(p, [0.0])[0]
    assert abs(R0 - 1.0) <= 1e-14, R0
    phi = np.linspace(-300, 300, 1201)
    R = o.rmsf(p, phi)
    assert np.all(np.abs(R) <= 1.0 + 1e-13)
    np.testing.assert_allclose(o.rmsf(p, -phi), np.conj(R), rtol=0, atol=1e-13)
    # Im R(h) = -K sum w sin(2 h (l2 - l0^2)) = -2h K sum w (l2 - l0^2) + O(h^3): zero slope
    lam = p.lambda2[w != 0]
    h = 1e-4 / (lam.max() - lam.min())
    slope = o.rmsf(p, [h])[0].imag / (2 * h * (lam.max() - lam.min()))
    assert abs(slope) < 1e-7, slope


def check_thin(o):
    freq, w = _lofar_like(seed=11)
    p = o.plan(freq, "freq", w)
    rng = np.random.default_rng(3)
    phi = np.linspace(-100, 100, 401)
    n = 24
    phi0 = rng.uniform(-60, 60, n)
    phi0[: n // 2] = phi[rng.integers(40, 360, n // 2)]      # half exactly on the grid
    p0 = rng.uniform(0.1, 1.0, n)
    chi0 = rng.uniform(0, np.pi, n)
    ang = 2.0 * (chi0[:, None] + phi0[:, None] * p.lambda2[None, :])
    Q = p0[:, None] * np.cos(ang)
    U = p0[:, None] * np.sin(ang)
    F = o.synth(Q, U, p, phi)
    for l in range(n):
        expect = p0[l] * np.exp(2j * (chi0[l] + phi0[l] * p.lambda0sq)) * o.rmsf(p, phi - phi0[l])
        np.testing.assert_allclose(F[l], expect, rtol=0, atol=1e-12)
    idx, a = o.peak(F[: n // 2])
    np.testing.assert_array_equal(phi[idx], phi0[: n // 2])
    np.testing.assert_allclose(a, p0[: n // 2], rtol=1e-12)


def check_linearity(o):
    freq, w = _lofar_like(nchan=64, seed=5)
    p = o.plan(freq, "freq", w)
    rng = np.random.default_rng(9)
    phi = np.linspace(-50, 50, 101)
    Q1, U1, Q2, U2 = rng.normal(size=(4, 5, 64))
    a, b = 0.7, -1.9
    F = o.synth(a * Q1 + b * Q2, a * U1 + b * U2, p, phi)
    G = a * o.synth(Q1, U1, p, phi) + b * o.synth(Q2, U2, p, phi)
    np.testing.assert_allclose(F, G, rtol=0, atol=1e-12)


def check_flagged(o):
    freq, w = _lofar_like(nchan=64, seed=13)
    rng = np.random.default_rng(2)
    Q, U = rng.normal(size=(2, 6, 64))
    Qn, Un = Q.copy(), U.copy()
    Qn[:, w == 0] = np.nan
    Un[:, w == 0] = np.inf
    phi = np.linspace(-50, 50, 101)
    F = o.synth(Qn, Un, o.plan(freq, "freq", w), phi)
    keep = w != 0
    G = o.synth(Q[:, keep], U[:, keep], o.plan(freq[keep], "freq", w[keep]), phi)
    assert np.array_equal(F, G)


def check_fft(o):
    # lambda_j^2 = a + j D, phi_k = phi_min + k d with 2 d D = 2 pi / M:
    # F_k = K exp(2i phi_k (lambda_0^2 - a)) DFT_M[w_j P_j exp(-2i phi_min j D)]_k
    rng = np.random.default_rng(21)
    N, M = 48, 64
    a, D = 0.9, 0.013
    lam2 = a + D * np.arange(N)
    w = rng.uniform(0.5, 1.5, N)
    w[[3, 17, 30]] = 0.0
    d = np.pi / (M * D)
    phi_min = -(M // 2) * d + 0.37 * d
    phi = phi_min + d * np.arange(M)
    p = o.plan(lam2, "lambda2", w)
    Q, U = rng.normal(size=(2, 3, N))
    F = o.synth(Q, U, p, phi)
    x = np.zeros((3, M), complex)
    x[:, :N] = w * (Q + 1j * U) * np.exp(-2j * phi_min * D * np.arange(N))
    G = p.K * np.exp(2j * phi * (p.lambda0sq - a))[None, :] * np.fft.fft(x, axis=1)
    np.testing.assert_allclose(F, G, rtol=0, atol=1e-12)


def check_fwhm(o):
    # continuous uniform lambda^2 coverage of width D: |R| = |sin(phi D) / (phi D)|,
    # half maximum at phi D = 1.895494267..., so FWHM = 3.790988534 / D
    lam2 = np.linspace(1.0, 3.0, 20001)
    p = o.plan(lam2, "lambda2")
    f = o.fwhm_measured(p)
    assert abs(f * 2.0 / 3.790988534067962 - 1.0) < 1e-3, f
    # Sec. 2.2: delta phi ~ 2 sqrt(3) / Delta lambda^2 (an estimate that assumes uniform
    # lambda^2 coverage; frequency-uniform channels crowd toward small lambda^2, so the
    # lobe is wider: within 30% for these fractional bandwidths, about 2x for 72-231 MHz)
    for nu0, nu1, n in ((120e6, 168e6, 64), (115e6, 178e6, 400), (110e6, 190e6, 800), (1e9, 2e9, 1000)):
        p = o.plan(np.linspace(nu0, nu1, n), "freq")
        ratio = o.fwhm_measured(p) / o.fwhm_estimate(p)
        assert 0.7 < ratio < 1.3, (nu0, nu1, ratio)


def check_realform(o):
    import mpmath as mp
    mp.mp.dps = 40
    rng = np.random.default_rng(31)
    nchan, nphi = 12, 9
    freq = np.sort(rng.uniform(110e6, 190e6, nchan))
    w = rng.uniform(0.0, 2.0, nchan)
    w[4] = 0.0
    phi = rng.uniform(-400, 400, nphi)
    Q, U = rng.normal(size=(2, 3, nchan))
    p = o.plan(freq, "freq", w)
    F = o.synth(Q, U, p, phi)
    c = mp.mpf(299792458)
    lam2 = [(c / mp.mpf(float(f))) ** 2 for f in freq]
    W = [mp.mpf(float(x)) for x in w]
    sw = sum(W)
    K = 1 / sw
    l0 = sum(W[i] * lam2[i] for i in range(nchan)) / sw
    for l in range(3):
        for k in range(nphi):
            qt = ut = mp.mpf(0)
            for i in range(nchan):
                th = 2 * mp.mpf(float(phi[k])) * (lam2[i] - l0)
                q = W[i] * mp.mpf(float(Q[l, i]))
                u = W[i] * mp.mpf(float(U[l, i]))
                qt += q * mp.cos(th) + u * mp.sin(th)      # Eq. qPhi
                ut += u * mp.cos(th) - q * mp.sin(th)      # Eq. uPhi
            assert abs(F[l, k].real - float(K * qt)) < 1e-12, (l, k)
            assert abs(F[l, k].imag - float(K * ut)) < 1e-12, (l, k)


PINS = {
    "golden": check_golden,
    "rmsf": check_rmsf,
    "thin": check_thin,
    "linearity": check_linearity,
    "flagged": check_flagged,
    "fft": check_fft,
    "fwhm": check_fwhm,
    "realform": check_realform,
}
