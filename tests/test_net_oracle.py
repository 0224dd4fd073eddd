"""The FP64 network oracle against finite differences, closed forms and special cases (no GPU)."""
import numpy as np

from oracle import net

C = 299792458.0


def _params(rng, nin=24, h=9, nb=7):
    return {"W1": rng.normal(0, 0.3, (h, nin)), "b1": rng.normal(0, 0.1, h),
            "W2": rng.normal(0, 0.3, (nb, h)), "b2": rng.normal(0, 0.1, nb)}


def _const_logits(nin, nb, z):
    """Parameters whose logits are z for every input: W1 = 0 gives h = 0, so z = b2."""
    return {"W1": np.zeros((4, nin)), "b1": np.zeros(4), "W2": np.zeros((nb, 4)), "b2": np.asarray(z, float)}


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    p = _params(rng)
    x = rng.normal(size=(5, 24))
    lab = rng.integers(0, 7, 5)
    loss, g = net.loss_and_grads(p, x, lab)
    eps = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        num = np.zeros_like(flat)
        for i in range(flat.size):
            old = flat[i]
            flat[i] = old + eps
            lp, _ = net.loss_and_grads(p, x, lab)
            flat[i] = old - eps
            lm, _ = net.loss_and_grads(p, x, lab)
            flat[i] = old
            num[i] = (lp - lm) / (2 * eps)
        np.testing.assert_allclose(g[name].reshape(-1), num, rtol=1e-6, atol=1e-9, err_msg=name)


def test_uniform_logits():
    # all-zero parameters: uniform softmax, loss = log(NB), max probability 1/NB, bin 0 (lowest on ties)
    p = _const_logits(6, 5, np.zeros(5))
    x = np.ones((3, 6))
    loss, _ = net.loss_and_grads(p, x, np.array([0, 2, 4]))
    assert abs(loss - np.log(5)) < 1e-15
    b, c = net.propose(p, x)
    assert np.all(b == 0) and np.allclose(c, 0.2)
    b, c = net.propose(p, x, halfwin=1)          # bins 0 and 1 (the range is clipped at 0)
    assert np.allclose(c, 0.4)


def test_window_mass_confidence():
    # softmax(log [1, 2, 3, 4]) = [0.1, 0.2, 0.3, 0.4]: bin 3; mass within 1 bin = 0.3 + 0.4
    p = _const_logits(2, 4, np.log([1.0, 2.0, 3.0, 4.0]))
    b, c = net.propose(p, np.zeros((1, 2)), halfwin=1)
    assert b[0] == 3 and abs(c[0] - 0.7) < 1e-15
    b, c = net.propose(p, np.zeros((1, 2)), halfwin=3)
    assert abs(c[0] - 1.0) < 1e-15


def test_normalise_interleaves_active_channels():
    Q = np.array([[3.0, 100.0, 0.0], [0.0, 0.0, 0.0]])
    U = np.array([[4.0, 7.0, 0.0], [0.0, 0.0, 0.0]])
    x = net.normalise(Q, U, active=[0, 2])        # channel 1 flagged: dropped
    s = np.sqrt((9 + 16 + 0) / 2)                 # RMS of |P| over the two active channels
    np.testing.assert_allclose(x[0], [3 / s, 4 / s, 0, 0])
    np.testing.assert_array_equal(x[1], np.zeros(4))   # all-zero row stays zero


def test_window_centre_and_fine_grid():
    phi = np.linspace(-100, 100, 401)
    assert net.fine_phi(phi, 1) == -99.75 and net.fine_phi(phi, 800) == 100.0
    c = net.window_centre([0, 200, 400], 401, 64)
    np.testing.assert_array_equal(c, [32, 400, 769])
    # windows c - 32 .. c + 31 stay on the fine grid 0 .. 800
    assert (c - 32).min() == 0 and (c + 31).max() == 800


def _thin(phi0, p0, chi0, lam2):
    P = p0 * np.exp(2j * (chi0 + phi0 * lam2))     # Faraday-thin source (Sec. 2.1)
    return P.real[None, :], P.imag[None, :]


def test_learned_peak_on_fine_grid_is_exact(oracle_mod):
    # A thin source at phi0 = 10.25, half-way between two coarse grid points.  With the
    # proposal on the coarse bin phi = 10 and full confidence, the window holds phi0 itself,
    # where |F| = p0 |R(0)| = p0 exactly (thin-source identity from Eqs. Fsum, Rsum).
    nu = np.linspace(115e6, 178e6, 64)
    lam2 = (C / nu) ** 2
    w = np.ones(64)
    phi = np.linspace(-100, 100, 401)
    Q, U = _thin(10.25, 0.7, 0.3, lam2)
    z = np.full(401, -50.0)
    z[220] = 50.0                                  # bin 220 is phi = 10
    p = _const_logits(128, 401, z)
    ph, a, fell = net.learned_peaks(oracle_mod, lam2, w, phi, p, Q, U, tau=0.5, width=64, halfwin=14)
    assert not fell[0]
    assert ph[0] == 10.25
    assert abs(a[0] - 0.7) < 1e-12
    # the full grid cannot represent phi0: it peaks on a neighbouring coarse point
    full_idx, _ = oracle_mod.peak(oracle_mod.synth(Q, U, oracle_mod.plan(lam2, "lambda2", w), phi))
    assert phi[full_idx[0]] in (10.0, 10.5)


def test_learned_fallbacks(oracle_mod):
    nu = np.linspace(115e6, 178e6, 64)
    lam2 = (C / nu) ** 2
    w = np.ones(64)
    phi = np.linspace(-100, 100, 401)
    Q, U = _thin(10.25, 0.7, 0.3, lam2)
    plan = oracle_mod.plan(lam2, "lambda2", w)
    full_idx, full_abs = oracle_mod.peak(oracle_mod.synth(Q, U, plan, phi))
    # (1) uniform logits: confidence 29/401 < tau -> the full-grid peak
    p = _const_logits(128, 401, np.zeros(401))
    ph, a, fell = net.learned_peaks(oracle_mod, lam2, w, phi, p, Q, U, tau=0.5, width=64, halfwin=14)
    assert fell[0] and ph[0] == phi[full_idx[0]] and a[0] == full_abs[0]
    # (2) confident proposal whose window ends just below the source: the window maximum
    # sits on its last point (the main lobe rising towards it) -> fallback
    z = np.full(401, -50.0)
    z[204] = 50.0                                  # centre 408: fine points 376 .. 439 (phi 9.75)
    p = _const_logits(128, 401, z)
    wphi = net.fine_phi(phi, 376 + np.arange(64))
    k, _ = oracle_mod.peak(oracle_mod.synth(Q, U, plan, wphi))
    assert k[0] == 63                              # brute force: the edge really holds the maximum
    ph, a, fell = net.learned_peaks(oracle_mod, lam2, w, phi, p, Q, U, tau=0.5, width=64, halfwin=14)
    assert fell[0] and ph[0] == phi[full_idx[0]]
    # (3) NaN in an active channel: no finite window maximum -> fallback (full grid gives -1)
    Qn = Q.copy()
    Qn[0, 5] = np.nan
    ph, a, fell = net.learned_peaks(oracle_mod, lam2, w, phi, p, Qn, U, tau=0.5, width=64, halfwin=14)
    assert fell[0] and np.isnan(ph[0])
