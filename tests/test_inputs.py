"""The seeded synthetic inputs (no GPU): band layouts, flags, and that any LOS can be
regenerated alone (what lets the oracle check sampled rows of a device-generated cube)."""
import numpy as np

from paper_1810_06250_gb300 import inputs


def test_uniform_lambda2_band():
    cfg = inputs.CONFIGS["lofar_ul2"]
    f = inputs.frequencies(cfg)
    l2 = (inputs.C_LIGHT / f) ** 2
    assert abs(f[0] - cfg.nu0) < 1e-3 and abs(f[-1] - cfg.nu1) < 1e-3
    lin = np.linspace(l2[0], l2[-1], len(l2))
    assert np.abs(l2 - lin).max() <= 1e-14 * np.abs(l2).max()
    # the frequency-uniform LOFAR band is far from uniform in lambda^2
    g = inputs.frequencies(inputs.CONFIGS["lofar"])
    m2 = (inputs.C_LIGHT / g) ** 2
    assert np.abs(m2 - np.linspace(m2[0], m2[-1], len(m2))).max() > 0.1


def test_flags_and_phi_grid():
    cfg = inputs.CONFIGS["lofar"]
    w = inputs.weights(cfg)
    assert int((w == 0).sum()) == 40 and set(np.unique(w)) == {0.0, 1.0}
    np.testing.assert_array_equal(w, inputs.weights(cfg))            # seeded
    phi = inputs.phi_grid(cfg)
    assert len(phi) == 401 and phi[0] == -100.0 and abs(phi[-1] - 100.0) < 1e-12
    np.testing.assert_allclose(np.diff(phi), 0.5, rtol=0, atol=1e-12)


def test_any_los_regenerates_alone():
    cfg = inputs.CONFIGS["tiny"]
    Q, U = inputs.make_cube(cfg, 0, 200)
    Q2, U2 = inputs.make_cube(cfg, 137, 5)
    np.testing.assert_array_equal(Q[137:142], Q2)
    np.testing.assert_array_equal(U[137:142], U2)
    assert Q.dtype == np.float32 and Q.shape == (200, cfg.nchan)
