"""The FP64 RM-CLEAN oracle against closed forms (no GPU)."""
import numpy as np

from oracle import clean as oc

C = 299792458.0


def _setup(oracle_mod, nphi=201, phi_max=50.0):
    nu = np.linspace(115e6, 178e6, 200)
    p = oracle_mod.plan(nu, "freq")
    phi = np.linspace(-phi_max, phi_max, nphi)
    dphi = phi[1] - phi[0]
    R2 = oracle_mod.rmsf(p, (np.arange(2 * nphi - 1) - (nphi - 1)) * dphi)
    return p, phi, dphi, R2


def test_single_thin_source_closed_form(oracle_mod):
    # F = A R(phi - phi0) for a thin source on the grid, so every step removes the same
    # fraction: residual = (1 - g)^n F exactly, one component A (1 - (1 - g)^n) at phi0
    p, phi, dphi, R2 = _setup(oracle_mod)
    P = 0.8 * np.exp(2j * (0.4 + 12.5 * p.lambda2))
    F = oracle_mod.synth(P.real, P.imag, p, phi)
    g, n = 0.1, 37
    cl, res, comp, it = oc.clean(F, R2, g, n, 0.0, oracle_mod.fwhm_measured(p), dphi)
    assert it[0] == n
    np.testing.assert_allclose(res[0], (1 - g) ** n * F[0], atol=1e-12)
    k0 = int(np.argmin(np.abs(phi - 12.5)))
    nz = np.nonzero(np.abs(comp[0]) > 0)[0]
    np.testing.assert_array_equal(nz, [k0])
    A = F[0, k0]
    assert abs(comp[0, k0] - A * (1 - (1 - g) ** n)) < 1e-12
    assert abs(abs(A) - 0.8) < 1e-12                        # thin-source identity: |F(phi0)| = p0


def test_threshold_stops_at_the_predicted_step(oracle_mod):
    p, phi, dphi, R2 = _setup(oracle_mod)
    P = 1.0 * np.exp(2j * (0.1 - 20.0 * p.lambda2))
    F = oracle_mod.synth(P.real, P.imag, p, phi)
    g, t = 0.2, 0.05
    _, res, _, it = oc.clean(F, R2, g, 10000, t, oracle_mod.fwhm_measured(p), dphi)
    n = int(np.ceil(np.log(t / 1.0) / np.log(1 - g)))      # first n with (1 - g)^n < t
    assert it[0] == n
    assert np.abs(res[0]).max() < t <= np.abs(res[0]).max() / (1 - g)


def test_restore_adds_the_beam(oracle_mod):
    p, phi, dphi, R2 = _setup(oracle_mod)
    P = 0.5 * np.exp(2j * (1.0 + 5.0 * p.lambda2))
    F = oracle_mod.synth(P.real, P.imag, p, phi)
    fwhm = 1.0
    cl, res, comp, it = oc.clean(F, R2, 0.5, 3, 0.0, fwhm, dphi)
    k0 = int(np.nonzero(np.abs(comp[0]) > 0)[0][0])
    W = oc.beam_halfwidth(fwhm, dphi)
    for d in (-W, -1, 0, 2, W):
        want = res[0, k0 + d] + comp[0, k0] * np.exp(-4 * np.log(2) * (d * dphi) ** 2 / fwhm ** 2)
        assert abs(cl[0, k0 + d] - want) < 1e-14
    assert abs(cl[0, k0 + W + 1] - res[0, k0 + W + 1]) == 0      # outside the truncated beam


def test_nan_spectrum_does_nothing(oracle_mod):
    p, phi, dphi, R2 = _setup(oracle_mod)
    F = np.full((1, len(phi)), np.nan + 0j)
    _, _, comp, it = oc.clean(F, R2, 0.1, 10, 0.0, 1.0, dphi)
    assert it[0] == 0 and np.all(comp == 0)
