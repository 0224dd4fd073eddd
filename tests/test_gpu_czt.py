"""GPU parity of the chirp-z (FFT) synthesis, RMS_FP32_CHIRPZ, against the FP64
oracle's direct sum (Eq. Fsum).  The FFT form is exact for channels uniform in
lambda^2 on a uniform phi grid, so the oracle is the plain definition and the
gate is the same 1e-5 per LOS as the split-precision paths.  Inputs are the
seeded host generator's; expected values come from oracle/ only.
"""
import dataclasses

import numpy as np
import pytest

import gpu_helpers as gh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PATH = "fp32_czt"


@pytest.fixture(scope="module")
def rms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_06250_gb300 as rms
    rms.build()
    rms.load()
    return rms


@pytest.fixture(scope="module")
def inputs():
    from paper_1810_06250_gb300 import inputs
    return inputs


def ul2(inputs, name, **kw):
    """A config of the given shape and band with channels uniform in lambda^2."""
    return dataclasses.replace(inputs.CONFIGS[name], extra={"lambda2_uniform": True}, **kw)


def axes(inputs, cfg):
    return inputs.frequencies(cfg), inputs.weights(cfg), inputs.phi_grid(cfg)


def run(rms, inputs, cfg, Q, U, layout, n, extras=False):
    dev = torch.device("cuda")
    freq, w, phi = axes(inputs, cfg)
    q = torch.from_numpy(inputs.to_layout(Q, layout)).to(dev)
    u = torch.from_numpy(inputs.to_layout(U, layout)).to(dev)
    F = torch.full((n, cfg.nphi, 2), float("nan"), device=dev)
    out = [torch.full((n,), -7, dtype=torch.int32, device=dev)] + [torch.full((n,), -7.0, device=dev)
                                                                    for _ in range(5 if extras else 2)]
    with rms.Plan(freq, phi, PATH, weights=w) as plan:
        if extras:
            rms.rms_synth_peaks(plan.handle, q, u, n, layout, F, *out)
        else:
            plan.synth(q, u, n, layout, F, *out)
        plan.sync()
        l0 = plan.rmsf()[0]
    return F.cpu().numpy(), [t.cpu().numpy() for t in out], l0


# (config, LOS, overrides), covering every kernel variant: FFT length 1024 for
# tiny and LOFAR shapes, 2048 for 800 x 1001 and 1200 x 401; half-length inputs
# and outputs (nchan, nphi <= M / 2) or not (520 x 100, 1000 x 25, 1200 x 401);
# with the input stage or without it (1000 x 25 and the 2048-point cases); LOS
# counts that leave ragged warps and blocks
CASES = [("tiny", 256, {}), ("tiny", 13, {}), ("lofar", 2999, {}), ("precision", 1031, {}),
         ("lofar", 301, {"nchan": 520, "nphi": 100, "phi_min": -50.0, "phi_max": 50.0}),
         ("lofar", 517, {"nchan": 1000, "nphi": 25, "phi_min": -12.0, "phi_max": 12.0}),
         ("lofar", 203, {"nchan": 1200}),
         ("lofar", 64, {"nchan": 1048, "nphi": 1001, "phi_min": -250.0, "phi_max": 250.0})]   # M = 2048 exactly


@pytest.mark.parametrize("layout", ["chan", "los"])
@pytest.mark.parametrize("name,n,kw", CASES)
def test_czt_parity(rms, inputs, oracle_mod, name, n, kw, layout):
    cfg = ul2(inputs, name, nlos=n, **kw)
    freq, w, phi = axes(inputs, cfg)
    Q, U = inputs.make_cube(cfg, 0, n)
    F, (pidx, pabs, pphi), _ = run(rms, inputs, cfg, Q, U, layout, n)
    Fo = oracle_mod.synth(Q, U, oracle_mod.plan(freq, "freq", w), phi)
    ok, info = gh.gate(PATH, F[..., 0] + 1j * F[..., 1], Fo)
    print(info)
    assert ok, info
    gh.check_peaks_self(F, pidx, pabs, pphi, phi)
    gh.check_peaks_oracle(pidx, Fo, gh.TOL[PATH])


def test_czt_flagged_nan_and_thin_source(rms, inputs, oracle_mod):
    # NaN in flagged channels never reaches F; a thin source on the grid peaks at phi0 with |F| = p0
    cfg = ul2(inputs, "lofar", nlos=64)
    freq, w, phi = axes(inputs, cfg)
    lam2 = (inputs.C_LIGHT / freq) ** 2
    phi0 = phi[37 + np.arange(64)]
    P = 0.7 * np.exp(2j * (0.2 + phi0[:, None] * lam2[None, :]))
    Q, U = P.real.astype(np.float32), P.imag.astype(np.float32)
    Q[:, w == 0] = np.nan
    U[:, w == 0] = np.nan
    F, (pidx, pabs, pphi), _ = run(rms, inputs, cfg, Q, U, "chan", 64)
    assert np.all(np.isfinite(F))
    np.testing.assert_array_equal(pidx, 37 + np.arange(64))
    assert np.all(np.abs(pabs - 0.7) <= 1e-5)
    Qz, Uz = np.where(w == 0, 0, Q).astype(np.float32), np.where(w == 0, 0, U).astype(np.float32)
    Fo = oracle_mod.synth(Qz, Uz, oracle_mod.plan(freq, "freq", w), phi)
    ok, info = gh.gate(PATH, F[..., 0] + 1j * F[..., 1], Fo)
    assert ok, info


def test_czt_nan_and_zero_lines_of_sight(rms, inputs, oracle_mod):
    # a NaN in an active channel reaches every output of its LOS (the FFT mixes all
    # channels), so that LOS has no peak; an all-zero LOS peaks at index 0 (a tie)
    cfg = ul2(inputs, "lofar", nlos=40)
    freq, w, phi = axes(inputs, cfg)
    Q, U = inputs.make_cube(cfg, 0, 40)
    act = np.nonzero(w)[0]
    Q[5, act[3]] = np.nan
    Q[9] = 0.0
    U[9] = 0.0
    F, (pidx, pabs, pphi), _ = run(rms, inputs, cfg, Q, U, "chan", 40)
    assert np.all(np.isnan(F[5]))
    assert pidx[5] == -1 and np.isnan(pabs[5]) and np.isnan(pphi[5])
    assert np.all(F[9] == 0) and pidx[9] == 0 and pabs[9] == 0
    good = np.ones(40, dtype=bool)
    good[5] = False
    Fo = oracle_mod.synth(Q[good], U[good], oracle_mod.plan(freq, "freq", w), phi)
    ok, info = gh.gate(PATH, F[good, :, 0] + 1j * F[good, :, 1], Fo)
    assert ok, info
    gh.check_peaks_self(F, pidx, pabs, pphi, phi)


def test_czt_peak_outputs(rms, inputs, oracle_mod):
    cfg = ul2(inputs, "lofar", nlos=2000)
    freq, w, phi = axes(inputs, cfg)
    Q, U = inputs.make_cube(cfg, 77, 2000)
    F, (idx, ab, ph, qp, up, chi), l0 = run(rms, inputs, cfg, Q, U, "chan", 2000, extras=True)
    r = np.arange(2000)
    np.testing.assert_array_equal(qp, F[r, idx, 0])
    np.testing.assert_array_equal(up, F[r, idx, 1])
    op = oracle_mod.plan(freq, "freq", w)
    Fo = oracle_mod.synth(Q, U, op, phi)
    fo = Fo[r, idx]
    tol = gh.TOL[PATH] * np.abs(Fo).max(axis=1)
    assert np.all(np.abs(qp - fo.real) <= tol) and np.all(np.abs(up - fo.imag) <= tol)
    co = oracle_mod.chi0(fo, phi[idx], l0)
    d = np.abs(chi.astype(np.float64) - co) % np.pi
    d = np.minimum(d, np.pi - d)
    assert np.all(d <= tol / np.abs(fo) + 1e-6)


def test_czt_empty_call(rms, inputs):
    cfg = ul2(inputs, "tiny")
    freq, w, phi = axes(inputs, cfg)
    z = torch.zeros(cfg.nchan, device="cuda")
    with rms.Plan(freq, phi, PATH, weights=w) as plan:
        plan.synth(z, z, 0, "chan", None, None, None, None)
        plan.sync()


def test_czt_rejects_axes_it_cannot_take(rms, inputs):
    def status(freq, phi, w=None):
        with pytest.raises(rms.RmsError) as e:
            rms.Plan(freq, phi, PATH, weights=w)
        return e.value.status
    lof = inputs.CONFIGS["lofar"]
    # channels uniform in frequency, not in lambda^2
    assert status(inputs.frequencies(lof), inputs.phi_grid(lof)) == rms.RMS_ERR_UNSUPPORTED
    # a non-uniform phi grid
    cfg = ul2(inputs, "lofar")
    phi = inputs.phi_grid(cfg).copy()
    phi[7] += 1e-3
    assert status(inputs.frequencies(cfg), phi) == rms.RMS_ERR_UNSUPPORTED
    # nchan + nphi - 1 > 2048
    mwa = ul2(inputs, "mwa")
    assert status(inputs.frequencies(mwa), inputs.phi_grid(mwa)) == rms.RMS_ERR_UNSUPPORTED


@pytest.mark.parametrize("layout", ["chan", "los"])
def test_czt_full_lofar_shape(rms, inputs, oracle_mod, layout):
    """The full 512^2 x 400 x 401 uniform-lambda^2 cube, generated on the device
    by the seeded generator's twin, in the benchmark's launch configuration;
    sampled rows are regenerated on the host for the oracle."""
    from paper_1810_06250_gb300 import learned as Lm
    cfg = inputs.CONFIGS["lofar_ul2"]
    freq, w, phi = axes(inputs, cfg)
    dev = torch.device("cuda")
    F = torch.empty(cfg.nlos, cfg.nphi, 2, device=dev)
    pidx = torch.empty(cfg.nlos, dtype=torch.int32, device=dev)
    pabs, pphi = torch.empty(cfg.nlos, device=dev), torch.empty(cfg.nlos, device=dev)
    with rms.Plan(freq, phi, PATH, weights=w) as plan:
        q, u = Lm.generate(plan.handle, cfg, 0, cfg.nlos, layout)
        plan.synth(q, u, cfg.nlos, layout, F, pidx, pabs, pphi)
        plan.sync()
        rng = np.random.default_rng(99)
        starts = np.r_[0, np.sort(rng.choice(cfg.nlos // 64 - 1, 6, replace=False)) * 64 + 64, cfg.nlos - 64]
        rows = (starts[:, None] + np.arange(64)[None, :]).ravel()
        Qs, Us = zip(*(inputs.make_cube(cfg, int(s), 64) for s in starts))
        Fo = oracle_mod.synth(np.concatenate(Qs), np.concatenate(Us), oracle_mod.plan(freq, "freq", w), phi)
        sel = torch.from_numpy(rows).to(dev)
        Fs = F[sel].cpu().numpy()
        ok, info = gh.gate(PATH, Fs[..., 0] + 1j * Fs[..., 1], Fo)
        print(info)
        assert ok, info
        gh.check_peaks_self(Fs, pidx[sel].cpu().numpy(), pabs[sel].cpu().numpy(), pphi[sel].cpu().numpy(), phi)
        gh.check_peaks_oracle(pidx[sel].cpu().numpy(), Fo, gh.TOL[PATH])
    del F, q, u
    torch.cuda.empty_cache()
