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
