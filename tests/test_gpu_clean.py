"""RM-CLEAN on the GPU (rms_clean) against the FP64 oracle (oracle/clean.py).

The dirty spectra are computed by the oracle (FP64 synthesis, rounded to FP32)
and given to both sides.  With the oracle's own R table the device must make the
same greedy choices and produce the same FP64 residual and components (compared
after rounding to FP32, bit for bit); with the device-built table the choices
may differ only at near-ties.
"""
import numpy as np
import pytest

from oracle import clean as oc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_06250_gb300 as rms
    rms.build()
    rms.load()
    return rms


def _case(oracle_mod, n=300):
    from paper_1810_06250_gb300 import inputs
    cfg = inputs.CONFIGS["lofar"]
    freq, w, phi = inputs.frequencies(cfg), inputs.weights(cfg), inputs.phi_grid(cfg)
    Q, U = inputs.make_cube(cfg, 2024, n)
    op = oracle_mod.plan(freq, "freq", w)
    F = oracle_mod.synth(Q, U, op, phi).astype(np.complex64)      # the dirty spectra both sides clean
    dphi = phi[1] - phi[0]
    R2 = oracle_mod.rmsf(op, (np.arange(2 * len(phi) - 1) - (len(phi) - 1)) * dphi)
    return cfg, freq, w, phi, op, F, dphi, R2


def _run(rms, plan, R2, F, fwhm, gain, niter, thr):
    n, N = F.shape
    c = rms.rms_clean_create(plan.handle, fwhm, R2)
    Fd = torch.from_numpy(np.ascontiguousarray(F).view(np.float32).reshape(n, N, 2)).cuda()
    outs = [torch.full((n, N, 2), float("nan"), device="cuda") for _ in range(3)]
    it = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rms.rms_clean(c, Fd, n, gain, niter, thr, outs[0], outs[1], outs[2], it)
    torch.cuda.synchronize()
    rms.rms_clean_destroy(c)
    cplx = [o.cpu().numpy().view(np.complex64)[..., 0] for o in outs]
    return cplx[0], cplx[1], cplx[2], it.cpu().numpy()


def test_clean_matches_oracle_bit_for_bit(rms, oracle_mod):
    cfg, freq, w, phi, op, F, dphi, R2 = _case(oracle_mod)
    fwhm = oracle_mod.fwhm_measured(op)
    g, t, n_it = np.float32(0.1), np.float32(0.02), 40
    with rms.Plan(freq, phi, "bf16x3", weights=w) as plan:
        cl, res, comp, it = _run(rms, plan, R2, F, fwhm, float(g), n_it, float(t))
    ocl, ores, ocomp, oit = oc.clean(F.astype(np.complex128), R2, float(g), n_it, float(t), fwhm, dphi)
    np.testing.assert_array_equal(it, oit)
    assert (it < n_it).any() and (it == n_it).any() and (it > 0).mean() > 0.5   # both stopping rules exercised
    np.testing.assert_array_equal(res, ores.astype(np.complex64))
    np.testing.assert_array_equal(comp, ocomp.astype(np.complex64))
    scale = np.abs(F).max(axis=1, keepdims=True)
    assert np.all(np.abs(cl - ocl) <= 1e-6 * scale)              # restore: summation order differs


def test_clean_with_device_rmsf(rms, oracle_mod):
    cfg, freq, w, phi, op, F, dphi, R2 = _case(oracle_mod, 200)
    fwhm = oracle_mod.fwhm_measured(op)
    with rms.Plan(freq, phi, "bf16x3", weights=w) as plan:
        cl, res, comp, it = _run(rms, plan, None, F, fwhm, 0.1, 300, 0.02)
    ocl, ores, ocomp, oit = oc.clean(F.astype(np.complex128), R2, float(np.float32(0.1)), 300,
                                     float(np.float32(0.02)), fwhm, dphi)
    same = (it == oit) & np.all((np.abs(comp) > 0) == (np.abs(ocomp) > 0), axis=1)
    assert same.mean() >= 0.98, same.mean()
    scale = np.abs(F).max(axis=1, keepdims=True)
    assert np.all(np.abs(res[same] - ores[same]) <= 1e-6 * scale[same])


def test_clean_single_thin_source(rms, oracle_mod):
    from paper_1810_06250_gb300 import inputs
    cfg = inputs.CONFIGS["lofar"]
    freq, w, phi = inputs.frequencies(cfg), inputs.weights(cfg), inputs.phi_grid(cfg)
    op = oracle_mod.plan(freq, "freq", w)
    P = 0.7 * np.exp(2j * (0.3 + 30.0 * op.lambda2))
    F = oracle_mod.synth(P.real, P.imag, op, phi).astype(np.complex64)
    with rms.Plan(freq, phi, "bf16x3", weights=w) as plan:
        cl, res, comp, it = _run(rms, plan, None, F, 0.0, 0.2, 25, 0.0)
    k0 = int(np.argmin(np.abs(phi - 30.0)))
    assert it[0] == 25
    np.testing.assert_array_equal(np.nonzero(np.abs(comp[0]) > 0)[0], [k0])
    np.testing.assert_allclose(res[0], 0.8 ** 25 * F[0].astype(np.complex128), atol=1e-6)
    assert abs(abs(comp[0, k0]) - 0.7 * (1 - 0.8 ** 25)) < 1e-5
