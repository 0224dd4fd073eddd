"""The FP64 oracle against what the paper and mathematics fix (no GPU)."""
import numpy as np
import pytest

import pins


@pytest.mark.parametrize("name", sorted(pins.PINS))
def test_oracle_pin(oracle_mod, name):
    pins.PINS[name](oracle_mod)


def test_plan_rejects(oracle_mod):
    import numpy as np
    freq = np.linspace(115e6, 178e6, 8)
    with pytest.raises(ValueError):
        oracle_mod.plan(freq, "freq", np.zeros(8))
    with pytest.raises(ValueError):
        oracle_mod.plan(freq, "freq", np.r_[-1.0, np.ones(7)])
    with pytest.raises(ValueError):
        oracle_mod.plan(freq, "freq", np.r_[np.nan, np.ones(7)])
    with pytest.raises(ValueError):
        oracle_mod.plan(np.r_[0.0, freq[1:]], "freq")


def test_chi0_of_thin_sources(oracle_mod):
    # Faraday-thin source on the grid: the peak is at phi0 and chi0 comes back exactly (mod pi)
    nu = np.linspace(115e6, 178e6, 200)
    p = oracle_mod.plan(nu, "freq")
    phi = np.linspace(-50, 50, 201)
    for phi0, c0 in ((10.0, 0.3), (-23.5, 3.1), (0.0, 0.0), (40.0, 1.5707)):
        lam2 = p.lambda2
        P = 0.9 * np.exp(2j * (c0 + phi0 * lam2))
        F = oracle_mod.synth(P.real, P.imag, p, phi)[0]
        k, _ = oracle_mod.peak(F)
        assert phi[k[0]] == phi0
        c = oracle_mod.chi0(F[k[0]], phi0, p.lambda0sq)
        d = (c - c0) % np.pi
        assert min(d, np.pi - d) < 1e-9


def test_chi0_rotates_with_the_data(oracle_mod):
    # multiplying P by exp(2i a) rotates every F by the same phase: chi0 moves by a (mod pi)
    rng = np.random.default_rng(4)
    nu = np.linspace(120e6, 168e6, 64)
    p = oracle_mod.plan(nu, "freq")
    phi = np.linspace(-50, 50, 101)
    Q, U = rng.normal(size=(2, 5, 64))
    F = oracle_mod.synth(Q, U, p, phi)
    k, _ = oracle_mod.peak(F)
    a = 0.7
    P2 = (Q + 1j * U) * np.exp(2j * a)
    F2 = oracle_mod.synth(P2.real, P2.imag, p, phi)
    k2, _ = oracle_mod.peak(F2)
    np.testing.assert_array_equal(k, k2)
    for i in range(5):
        c1 = oracle_mod.chi0(F[i, k[i]], phi[k[i]], p.lambda0sq)
        c2 = oracle_mod.chi0(F2[i, k[i]], phi[k[i]], p.lambda0sq)
        d = (c2 - c1 - a) % np.pi
        assert min(d, np.pi - d) < 1e-9


# ------------------------------------------------------------------- sub-grid peak refinement
def test_refine_recovers_an_exact_parabola(oracle_mod):
    # |F| sampled from y = A - B (phi - phi_v)^2 on a non-uniform grid: the vertex and height come back
    rng = np.random.default_rng(17)
    for _ in range(40):
        phi = np.cumsum(rng.uniform(0.2, 1.0, 9)) - 4.0
        k = int(rng.integers(1, 8))
        pv = rng.uniform(phi[k] - 0.45 * (phi[k] - phi[k - 1]), phi[k] + 0.45 * (phi[k + 1] - phi[k]))
        A, B = rng.uniform(5.0, 6.0), rng.uniform(0.1, 1.0)
        y = A - B * (phi - pv) ** 2
        F = y * np.exp(1j * rng.uniform(0, 2 * np.pi, 9))
        pr, ar = oracle_mod.refine_peak(F[None], phi, [k])
        assert abs(pr[0] - pv) < 1e-11 and abs(ar[0] - A) < 1e-11


def test_refine_matches_the_uniform_grid_formula(oracle_mod):
    # uniform step h: the vertex sits (y0 - y2) / (2 (y0 - 2 y1 + y2)) steps from the middle sample
    rng = np.random.default_rng(18)
    h = 0.5
    phi = -3.0 + h * np.arange(13)
    for _ in range(40):
        k = int(rng.integers(1, 12))
        y = rng.uniform(0.0, 1.0, 13)
        y[k] = 1.0 + rng.uniform(0.0, 0.5)
        y0, y1, y2 = y[k - 1], y[k], y[k + 1]
        delta = (y0 - y2) / (2.0 * (y0 - 2.0 * y1 + y2))
        height = y1 - 0.25 * (y0 - y2) * delta
        pr, ar = oracle_mod.refine_peak(y[None].astype(np.complex128), phi, [k])
        assert abs(pr[0] - (phi[k] + delta * h)) < 1e-12 and abs(ar[0] - height) < 1e-12


def test_refine_thin_source_midway_between_samples(oracle_mod):
    # |R| is even (R Hermitian), so a source midway between two samples gives two equal
    # samples and the parabola's vertex is exactly the midpoint, whichever of them is the argmax
    freq = np.linspace(115e6, 178e6, 400)
    p = oracle_mod.plan(freq, "freq")
    phi = np.arange(-20.0, 20.0 + 1e-9, 0.5)
    for phi0 in (-7.25, 0.25, 13.75):
        P = 0.8 * np.exp(2j * (0.4 + phi0 * p.lambda2))
        F = oracle_mod.synth(P.real[None].copy(), P.imag[None].copy(), p, phi)
        k, _ = oracle_mod.peak(F)
        pr, _ = oracle_mod.refine_peak(F, phi, k)
        assert abs(pr[0] - phi0) < 1e-9


def test_refine_moves_toward_off_grid_sources(oracle_mod):
    # Faraday-thin sources at random depths: the refined depth is much closer than the grid
    # sample (the RMSF main lobe is close to a parabola near its top), and the refined
    # height is closer to p0 than the sampled one
    freq = np.linspace(115e6, 178e6, 400)
    p = oracle_mod.plan(freq, "freq")
    fw = oracle_mod.fwhm_measured(p)
    rng = np.random.default_rng(19)
    phi0 = rng.uniform(-30.0, 30.0, 120)
    P = np.exp(2j * (0.3 + phi0[:, None] * p.lambda2[None, :]))
    for step, bound in ((fw / 2, 0.06), (fw / 8, 0.005)):
        phi = np.arange(-40.0, 40.0 + 1e-9, step)
        F = oracle_mod.synth(P.real.copy(), P.imag.copy(), p, phi)
        k, a = oracle_mod.peak(F)
        pr, ar = oracle_mod.refine_peak(F, phi, k)
        eg, er = np.abs(phi[k] - phi0), np.abs(pr - phi0)
        assert np.all(er <= 0.3 * eg + 1e-9)
        assert er.max() <= bound * step
        assert np.all(np.abs(ar - 1.0) <= np.abs(a - 1.0) + 1e-12)


def test_refine_undefined_cases_keep_the_sample(oracle_mod):
    phi = np.linspace(-2.0, 2.0, 5)
    y = np.array([[3.0, 1.0, 0.5, 1.0, 2.0],      # k = 0: grid end
                  [1.0, 2.0, 0.5, 1.0, 4.0],      # k = 4: grid end
                  [1.0, 0.5, 0.4, 0.5, 1.0],      # k = 2: convex, no vertex
                  [1.0, np.nan, 2.0, 1.0, 1.0],   # k = 2: NaN neighbour
                  [1.0, 1.0, 1.0, 1.0, 1.0]])     # k = -1: no peak
    k = np.array([0, 4, 2, 2, -1])
    pr, ar = oracle_mod.refine_peak(y.astype(np.complex128), phi, k)
    np.testing.assert_array_equal(pr[:4], phi[k[:4]])
    np.testing.assert_array_equal(ar[:4], y[np.arange(4), k[:4]])
    assert np.isnan(pr[4]) and np.isnan(ar[4])
    # both neighbours on one side of phi_k (a non-monotonic grid): the sample
    pr, ar = oracle_mod.refine_peak(np.array([[1.0, 2.0, 1.5]], dtype=np.complex128), [0.0, 1.0, 0.5], [1])
    assert pr[0] == 1.0 and ar[0] == 2.0


# ------------------------------------------------------------------- the paper's cost example
def test_unit_count_reproduces_the_papers_cost_example():
    # the benchmark's unit is one (LOS, channel, phi) triple; at the paper's 15 flop per unit
    # the WSRT-SINGS-shaped cube of Sec. 2.3 must come to its printed ~1.27 TFLOP
    import json
    import os
    from paper_1810_06250_gb300.inputs import CubeConfig
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_cost.json")))
    cfg = CubeConfig("wsrt_sings_shape", g["nlos"], g["nchan"], 1.3e9, 1.45e9, g["nphi"], -100.0, 100.0, seed=1)
    tflop = cfg.units * g["flop_per_unit"] / 1e12
    assert round(tflop, g["printed_digits"]) == g["tflop_printed"]


# ------------------------------------------------------------------- FFT (chirp-z) form of Eq. Fsum
def test_chirp_z_form_equals_the_direct_sum(oracle_mod):
    # with lambda^2 uniform (x_j = x_0 + j D) and phi uniform (phi_k = phi_0 + k d), 2 j k =
    # j^2 + k^2 - (k - j)^2 turns Eq. Fsum into a convolution that FFTs evaluate exactly, for any
    # d D (no relation to 2 pi / M is needed); the FFT synthesis path relies on this identity
    rng = np.random.default_rng(21)
    for nc, nk, l2lo, l2hi, phmax in ((64, 101, 2.8, 6.8, 50.0), (400, 401, 2.84, 6.8, 100.0),
                                      (120, 333, 1.7, 17.3, 900.0)):
        lam2 = np.linspace(l2hi, l2lo, nc)
        w = rng.uniform(0.5, 1.5, nc)
        w[rng.random(nc) < 0.1] = 0.0
        phi = np.linspace(-phmax, phmax, nk)
        Q, U = rng.normal(size=(3, nc)), rng.normal(size=(3, nc))
        p = oracle_mod.plan(lam2, "lambda2", w)
        Fo = oracle_mod.synth(Q, U, p, phi)
        x = lam2 - p.lambda0sq
        x0, D = x[0], (x[-1] - x[0]) / (nc - 1)
        p0, d = phi[0], (phi[-1] - phi[0]) / (nk - 1)
        j, k = np.arange(nc), np.arange(nk)
        M = int(2 ** np.ceil(np.log2(nc + nk - 1)))
        a = np.zeros((3, M), complex)
        a[:, :nc] = w * (Q + 1j * U) * np.exp(-1j * (2 * p0 * D * j + d * D * j * j))
        m = np.arange(-(nc - 1), nk)
        h = np.zeros(M, complex)
        h[m % M] = np.exp(1j * d * D * m * m)
        c = np.fft.ifft(np.fft.fft(a, axis=1) * np.fft.fft(h), axis=1)[:, :nk]
        F = p.K * np.exp(-1j * (2 * p0 * x0 + 2 * d * x0 * k + d * D * k * k)) * c
        assert np.abs(F - Fo).max() <= 1e-10 * np.abs(Fo).max()
