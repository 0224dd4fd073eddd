"""GPU parity: librms.so (through the C ABI) against the FP64 oracle.

Inputs are seeded synthetic cubes from paper_1810_06250_gb300.inputs generated
on the host; expected values come from oracle/ only.
"""
import numpy as np
import pytest

import gpu_helpers as gh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PATHS = ["fp32_fly", "fp32_table", "bf16", "bf16x3", "fp16x3"]


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


def run(rms, plan, Q, U, layout, nlos, want_F=True, stream=None):
    """Q, U: host float32 LOS-major [nlos][nchan]."""
    dev = torch.device("cuda")
    from paper_1810_06250_gb300.inputs import to_layout
    q = torch.from_numpy(to_layout(Q, layout)).to(dev)
    u = torch.from_numpy(to_layout(U, layout)).to(dev)
    F = torch.full((nlos, plan.nphi, 2), float("nan"), device=dev) if want_F else None
    pidx = torch.full((nlos,), -7, dtype=torch.int32, device=dev)
    pabs = torch.zeros(nlos, device=dev)
    pphi = torch.zeros(nlos, device=dev)
    plan.synth(q, u, nlos, layout, F, pidx, pabs, pphi, stream)
    plan.sync(stream)
    torch.cuda.synchronize()
    return (F.cpu().numpy() if want_F else None, pidx.cpu().numpy(), pabs.cpu().numpy(), pphi.cpu().numpy())


def axes(inputs, cfg):
    return inputs.frequencies(cfg), inputs.weights(cfg), inputs.phi_grid(cfg)


# ------------------------------------------------------------------- plan
@pytest.mark.parametrize("path", PATHS)
def test_plan_constants(rms, inputs, oracle_mod, path):
    cfg = inputs.CONFIGS["lofar"]
    freq, w, phi = axes(inputs, cfg)
    with rms.Plan(freq, phi, path, weights=w) as plan:
        op = oracle_mod.plan(freq, "freq", w)
        l0, K, fm, fe = plan.rmsf()
        assert abs(K - op.K) <= 1e-15 * op.K
        assert abs(l0 - op.lambda0sq) <= 1e-14 * op.lambda0sq
        np.testing.assert_allclose(plan.get(rms.RMS_GET_LAMBDA2), op.lambda2, rtol=1e-15)
        np.testing.assert_array_equal(plan.get(rms.RMS_GET_ACTIVE), op.active)
        R64 = plan.get(rms.RMS_GET_RMSF64)
        Ro = oracle_mod.rmsf(op, phi)
        np.testing.assert_allclose(R64[:, 0] + 1j * R64[:, 1], Ro, rtol=0, atol=1e-13)
        R32 = torch.empty(2 * cfg.nphi, device="cuda")
        plan.rmsf(R32)
        r = R32.cpu().numpy().reshape(-1, 2)
        np.testing.assert_allclose(r[:, 0] + 1j * r[:, 1], Ro, rtol=0, atol=2e-7)
        assert abs(fe - oracle_mod.fwhm_estimate(op)) <= 1e-12 * fe
        assert abs(fm - oracle_mod.fwhm_measured(op)) <= 1e-6 * fm


def test_phase_table(rms, inputs, oracle_mod):
    cfg = inputs.CONFIGS["mwa"]          # largest phases: |theta| up to ~7e4 rad
    freq, w, phi = axes(inputs, cfg)
    phi = phi[::7]
    with rms.Plan(freq, phi, "fp32_table", weights=w) as plan:
        op = oracle_mod.plan(freq, "freq", w)
        tab = plan.get(rms.RMS_GET_TABLE)
        act = op.active
        th = 2.0 * phi[None, :] * (op.lambda2[act, None] - op.lambda0sq)
        exp_c = w[act, None] * np.cos(th)
        exp_s = w[act, None] * np.sin(th)
        # FP32 rounding of an FP64 value accurate to ~1e-15
        np.testing.assert_allclose(tab[..., 0], exp_c, rtol=0, atol=6.1e-8)
        np.testing.assert_allclose(tab[..., 1], exp_s, rtol=0, atol=6.1e-8)


def _bits_to_float(b, fp16):
    if fp16:
        return b.view(np.float16).astype(np.float64)
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("path", ["bf16x3", "fp16x3"])
def test_phase_split_matrix(rms, inputs, oracle_mod, path):
    cfg = inputs.CONFIGS["mwa"]
    freq, w, phi = axes(inputs, cfg)
    phi = phi[::13]
    fp16 = path == "fp16x3"
    with rms.Plan(freq, phi, path, weights=w) as plan:
        op = oracle_mod.plan(freq, "freq", w)
        hi = _bits_to_float(plan.get(rms.RMS_GET_B_HI), fp16)
        lo = _bits_to_float(plan.get(rms.RMS_GET_B_LO), fp16)
        B = hi + lo
        act = op.active
        nact, nphi = len(act), len(phi)
        th = 2.0 * phi[None, :] * (op.lambda2[act, None] - op.lambda0sq)
        wn = (w[act] / w.max())[:, None]
        c, s = (wn * np.cos(th)).T, (wn * np.sin(th)).T          # [nphi][nact]
        tol = 2.0 ** -16 if not fp16 else 2.0 ** -21
        np.testing.assert_allclose(B[0:2 * nphi:2, 0:2 * nact:2], c, rtol=0, atol=tol)
        np.testing.assert_allclose(B[0:2 * nphi:2, 1:2 * nact:2], s, rtol=0, atol=tol)
        np.testing.assert_allclose(B[1:2 * nphi:2, 0:2 * nact:2], -s, rtol=0, atol=tol)
        np.testing.assert_allclose(B[1:2 * nphi:2, 1:2 * nact:2], c, rtol=0, atol=tol)
        assert not B[2 * nphi:, :].any() and not B[:, 2 * nact:].any()   # zero padding


# ------------------------------------------------------------------- synthesis
@pytest.mark.parametrize("layout", ["chan", "los"])
@pytest.mark.parametrize("path", PATHS)
def test_synth_tiny(rms, inputs, oracle_mod, path, layout):
    cfg = inputs.CONFIGS["tiny"]
    freq, w, phi = axes(inputs, cfg)
    Q, U = inputs.make_cube(cfg)
    op = oracle_mod.plan(freq, "freq", w)
    Fo = oracle_mod.synth(Q, U, op, phi)
    with rms.Plan(freq, phi, path, weights=w) as plan:
        F, pidx, pabs, pphi = run(rms, plan, Q, U, layout, cfg.nlos)
        ok, info = gh.gate(path, F[..., 0] + 1j * F[..., 1], Fo)
        print(info)
        assert ok, info
        gh.check_peaks_self(F, pidx, pabs, pphi, phi)
        gh.check_peaks_oracle(pidx, Fo, gh.TOL[path])
        # peak-only mode gives the same peak map
        _, pidx2, pabs2, pphi2 = run(rms, plan, Q, U, layout, cfg.nlos, want_F=False)
        np.testing.assert_array_equal(pidx2, pidx)
        np.testing.assert_array_equal(pabs2, pabs)
        np.testing.assert_array_equal(pphi2, pphi)


@pytest.mark.parametrize("path", PATHS)
def test_edges(rms, inputs, oracle_mod, path):
    """Ragged LOS counts, odd channel counts with flags and NaN there, a NaN
    in an active channel, an all-zero LOS, nphi = 1 and several N tiles."""
    rng = np.random.default_rng(5)
    nchan = 37
    freq = np.linspace(120e6, 168e6, nchan)
    w = rng.uniform(0.5, 1.5, nchan)
    w[[0, 5, 6, 20, 36]] = 0.0
    for nphi, nlos in ((1, 1), (130, 127), (130, 129), (101, 300), (300, 257)):
        phi = np.linspace(-60, 60, nphi) if nphi > 1 else np.array([3.5])
        Q = rng.normal(size=(nlos, nchan)).astype(np.float32)
        U = rng.normal(size=(nlos, nchan)).astype(np.float32)
        Q[:, w == 0] = np.nan
        U[:, w == 0] = np.inf
        if nlos > 3:
            Q[2, 7] = np.nan       # active channel: this LOS becomes all-NaN
            Q[3] = 0.0
            U[3] = 0.0
        op = oracle_mod.plan(freq, "freq", w)
        Fo = oracle_mod.synth(Q, U, op, phi)
        with rms.Plan(freq, phi, path, weights=w) as plan:
            for layout in ("chan", "los"):
                F, pidx, pabs, pphi = run(rms, plan, Q, U, layout, nlos)
                good = np.all(np.isfinite(Fo), axis=1)
                if path == "bf16":
                    # a handful of phi points has no meaningful cube maximum: structure only
                    per, _ = gh.errors(F[good, :, 0] + 1j * F[good, :, 1], Fo[good])
                    ok, info = per.max() <= 1e-2, {"per_los_max": float(per.max())}
                else:
                    ok, info = gh.gate(path, F[good, :, 0] + 1j * F[good, :, 1], Fo[good])
                assert ok, (nphi, nlos, layout, info)
                assert np.all(np.isnan(F[~good]))
                gh.check_peaks_self(F, pidx, pabs, pphi, phi)
                if nlos > 3:
                    assert pidx[2] == -1 and pidx[3] == 0
                gh.check_peaks_oracle(pidx[good], Fo[good], gh.TOL[path])


def test_zero_los_and_bad_args(rms, inputs):
    cfg = inputs.CONFIGS["tiny"]
    freq, w, phi = axes(inputs, cfg)
    with rms.Plan(freq, phi, "bf16x3", weights=w) as plan:
        q = torch.zeros(cfg.nchan * 4, device="cuda")
        F = torch.zeros(4, cfg.nphi, 2, device="cuda")
        plan.synth(q, q, 0, "chan", F)           # nothing to do
        with pytest.raises(rms.RmsError) as e:
            rms.rms_synth(plan.handle, q, q, 4, 7, F)
        assert e.value.status == rms.RMS_ERR_INVALID_ARG
        with pytest.raises(rms.RmsError) as e:
            rms.rms_synth(plan.handle, q, q, -1, "chan", F)
        assert e.value.status == rms.RMS_ERR_INVALID_ARG
        with pytest.raises(rms.RmsError) as e:
            rms.rms_synth(plan.handle, q, q, 4, "chan", F.data_ptr() + 4)    # misaligned F
        assert e.value.status == rms.RMS_ERR_INVALID_ARG
        with pytest.raises(rms.RmsError) as e:
            rms.rms_synth(plan.handle, 0, q, 4, "chan", F)                    # NULL Q
        assert e.value.status == rms.RMS_ERR_INVALID_ARG
        plan.sync()
    for bad in (dict(weights=np.zeros(cfg.nchan)), dict(weights=-w), dict(precision=9)):
        kw = dict(weights=w, precision="bf16x3")
        kw.update(bad)
        with pytest.raises(rms.RmsError) as e:
            rms.rms_plan_create(freq, kw["weights"], phi, kw["precision"])
        assert e.value.status == rms.RMS_ERR_INVALID_ARG
    rms.rms_plan_destroy(None)


# ------------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def lofar(inputs):
    cfg = inputs.CONFIGS["lofar"]
    Q, U = inputs.make_cube(cfg)
    return cfg, Q, U


@pytest.mark.parametrize("layout", ["chan", "los"])
@pytest.mark.parametrize("path", PATHS)
def test_lofar_full(rms, inputs, oracle_mod, lofar, path, layout):
    """LOFAR-HBA-like cube at full size (512^2 LOS x 400 ch x 401 phi), the bench's
    launch; 1024 sampled LOS against the oracle, peaks checked on every LOS."""
    cfg, Q, U = lofar
    freq, w, phi = axes(inputs, cfg)
    rng = np.random.default_rng(77)
    sample = np.unique(np.r_[0, cfg.nlos - 1, rng.choice(cfg.nlos, 1022, replace=False)])
    op = oracle_mod.plan(freq, "freq", w)
    Fo = oracle_mod.synth(Q[sample], U[sample], op, phi)
    with rms.Plan(freq, phi, path, weights=w) as plan:
        F, pidx, pabs, pphi = run(rms, plan, Q, U, layout, cfg.nlos)
        ok, info = gh.gate(path, F[sample, :, 0] + 1j * F[sample, :, 1], Fo)
        print(info)
        assert ok, info
        gh.check_peaks_self(F, pidx, pabs, pphi, phi)
        gh.check_peaks_oracle(pidx[sample], Fo, gh.TOL[path])


# ------------------------------------------------------------------- large cubes
LARGE = [("precision", "bf16x3", 2048), ("precision", "bf16", 512), ("precision", "fp16x3", 512),
         ("precision", "fp32_fly", 512), ("precision", "fp32_table", 512), ("mwa", "bf16x3", 256),
         ("mwa", "fp16x3", 256), ("mwa", "bf16", 256), ("lofar_lr", "bf16x3", 256)]


@pytest.mark.parametrize("cfg_name,path,nsample", LARGE)
def test_large_full(rms, inputs, oracle_mod, cfg_name, path, nsample):
    """Full-size 2048^2 x 800 x 1001, 1024^2 x 1536 x 4001 and 540^2 x 856 x 7000 cubes
    in the launch configuration the benchmark uses.  The device cube repeats a
    host-generated base block of 16384 LOS (row l holds base row l % 16384); sampled
    rows are compared with the oracle on the base rows and their peaks checked."""
    cfg = inputs.CONFIGS[cfg_name]
    freq, w, phi = axes(inputs, cfg)
    nbase = 16384
    Qb, Ub = inputs.make_cube(cfg, 0, nbase)
    reps = (cfg.nlos + nbase - 1) // nbase
    dev = torch.device("cuda")
    q = torch.from_numpy(np.ascontiguousarray(Qb.T)).to(dev).repeat(1, reps)[:, :cfg.nlos].contiguous()
    u = torch.from_numpy(np.ascontiguousarray(Ub.T)).to(dev).repeat(1, reps)[:, :cfg.nlos].contiguous()
    rng = np.random.default_rng(4242)
    sample = np.unique(np.r_[0, cfg.nlos - 1, rng.choice(cfg.nlos, nsample - 2, replace=False)])
    op = oracle_mod.plan(freq, "freq", w)
    Fo = oracle_mod.synth(Qb[sample % nbase], Ub[sample % nbase], op, phi)
    F = torch.empty(cfg.nlos, cfg.nphi, 2, device=dev)
    pidx = torch.empty(cfg.nlos, dtype=torch.int32, device=dev)
    pabs = torch.empty(cfg.nlos, device=dev)
    pphi = torch.empty(cfg.nlos, device=dev)
    with rms.Plan(freq, phi, path, weights=w) as plan:
        plan.synth(q, u, cfg.nlos, "chan", F, pidx, pabs, pphi)
        plan.sync()
        sel = torch.from_numpy(sample).to(dev)
        Fs = F[sel].cpu().numpy()
        ok, info = gh.gate(path, Fs[..., 0] + 1j * Fs[..., 1], Fo)
        info["config"] = cfg_name
        print(info)
        gh.check_peaks_self(Fs, pidx[sel].cpu().numpy(), pabs[sel].cpu().numpy(), pphi[sel].cpu().numpy(), phi)
        near = gh.check_peaks_oracle(pidx[sel].cpu().numpy(), Fo, gh.TOL[path])
        print("near-tie LOS:", near)
        assert ok, info
    del F, q, u
    torch.cuda.empty_cache()


# ------------------------------------------------------------------- kernel timing hook
def test_kernel_timing_hook(rms, inputs):
    cfg = inputs.CONFIGS["tiny"]
    freq, w, phi = axes(inputs, cfg)
    Q, U = inputs.make_cube(cfg)
    dev = torch.device("cuda")
    q = torch.from_numpy(inputs.to_layout(Q, "chan")).to(dev)
    u = torch.from_numpy(inputs.to_layout(U, "chan")).to(dev)
    pidx = torch.empty(cfg.nlos, dtype=torch.int32, device=dev)
    with rms.Plan(freq, phi, "bf16x3", weights=w) as plan:
        plan.synth(q, u, cfg.nlos, "chan", None, pidx)            # timing off: nothing recorded
        rms.rms_plan_set_kernel_timing(plan.handle, True)
        for _ in range(3):
            plan.synth(q, u, cfg.nlos, "chan", None, pidx)
        rms.rms_plan_set_kernel_timing(plan.handle, False)
        plan.synth(q, u, cfg.nlos, "chan", None, pidx)
        a, b, n = rms.rms_plan_kernel_times(plan.handle)
        assert n == 3 and a > 0 and b > 0
        assert rms.rms_plan_kernel_times(plan.handle)[2] == 0     # read once, then forgotten


# ------------------------------------------------------------------- host-buffer entry point
@pytest.mark.parametrize("layout", ["chan", "los"])
def test_synth_host_matches_device(rms, inputs, layout):
    """rms_synth_host pipelines LOS chunks (copy in / synthesis / copy out on three
    streams); every LOS is its own contraction, so its results equal rms_synth's
    bit for bit, across chunk boundaries, slot reuse and a ragged last chunk."""
    from paper_1810_06250_gb300 import learned as L
    cfg = inputs.CONFIGS["lofar"]
    freq, w, phi = axes(inputs, cfg)
    n = 140000                                   # LOS-major: 9 chunks of 16384; channel-major: 3 of 65536
    with rms.Plan(freq, phi, "bf16x3", weights=w) as plan:
        q, u = L.generate(plan.handle, cfg, 0, n, layout)
        F0 = torch.empty(n, cfg.nphi, 2, device="cuda")
        i0 = torch.empty(n, dtype=torch.int32, device="cuda")
        a0 = torch.empty(n, device="cuda")
        p0 = torch.empty(n, device="cuda")
        plan.synth(q, u, n, layout, F0, i0, a0, p0)
        plan.sync()
        qh, uh = q.cpu().pin_memory(), u.cpu().pin_memory()
        F1 = torch.full((n, cfg.nphi, 2), float("nan")).pin_memory()
        i1 = torch.full((n,), -7, dtype=torch.int32).pin_memory()
        a1 = torch.zeros(n).pin_memory()
        p1 = torch.zeros(n).pin_memory()
        for _ in range(2):                       # twice: the slots are reused across calls
            plan.synth_host(qh, uh, n, layout, F1, i1, a1, p1)
        assert torch.equal(F1, F0.cpu())
        assert torch.equal(i1, i0.cpu()) and torch.equal(a1, a0.cpu()) and torch.equal(p1, p0.cpu())
        i2 = torch.full((n,), -7, dtype=torch.int32).pin_memory()
        plan.synth_host(qh, uh, n, layout, None, i2)           # peak map only
        assert torch.equal(i2, i0.cpu())


def test_synth_host_from_registered_buffers(rms, inputs):
    """Host buffers from rms_host_alloc (registered huge-page memory) serve
    rms_synth_host like any pinned memory: results equal rms_synth's bit for bit;
    the buffers are released again."""
    from paper_1810_06250_gb300 import learned as L
    cfg = inputs.CONFIGS["lofar"]
    freq, w, phi = axes(inputs, cfg)
    n = 70000                                    # channel-major: 2 chunks of 65536 (the second ragged)
    with rms.Plan(freq, phi, "bf16x3", weights=w) as plan:
        q, u = L.generate(plan.handle, cfg, 0, n, "chan")
        F0 = torch.empty(n, cfg.nphi, 2, device="cuda")
        i0 = torch.empty(n, dtype=torch.int32, device="cuda")
        plan.synth(q, u, n, "chan", F0, i0)
        plan.sync()
        bufs = [rms.HostBuffer(q.shape), rms.HostBuffer(u.shape), rms.HostBuffer((n, cfg.nphi, 2)),
                rms.HostBuffer(n, "int32")]
        try:
            qh, uh, Fh, ih = (b.tensor for b in bufs)
            assert qh.data_ptr() % 4096 == 0              # page aligned
            qh.copy_(q)
            uh.copy_(u)
            Fh.fill_(float("nan"))
            ih.fill_(-7)
            plan.synth_host(qh, uh, n, "chan", Fh, ih)
            assert torch.equal(Fh, F0.cpu()) and torch.equal(ih, i0.cpu())
        finally:
            for b in bufs:
                b.close()
        assert all(b.ptr == 0 for b in bufs)


# ------------------------------------------------------------------- Q, U and chi0 at the peak
@pytest.mark.parametrize("path", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("layout", ["chan", "los"])
def test_peak_outputs(rms, inputs, oracle_mod, path, layout):
    cfg = inputs.CONFIGS["lofar"]
    freq, w, phi = axes(inputs, cfg)
    n = 3000
    Q, U = inputs.make_cube(cfg, 4242, n)
    dev = torch.device("cuda")
    q = torch.from_numpy(inputs.to_layout(Q, layout)).to(dev)
    u = torch.from_numpy(inputs.to_layout(U, layout)).to(dev)
    with rms.Plan(freq, phi, path, weights=w) as plan:
        F = torch.empty(n, cfg.nphi, 2, device=dev)
        out = [torch.full((n,), -7, dtype=torch.int32, device=dev)] + [torch.full((n,), -7.0, device=dev) for _ in range(5)]
        rms.rms_synth_peaks(plan.handle, q, u, n, layout, F, *out)
        i0 = torch.empty(n, dtype=torch.int32, device=dev)
        a0, p0 = torch.empty(n, device=dev), torch.empty(n, device=dev)
        plan.synth(q, u, n, layout, None, i0, a0, p0)
        plan.sync()
        idx, ab, ph, qp, up, chi = [t.cpu().numpy() for t in out]
        np.testing.assert_array_equal(idx, i0.cpu().numpy())      # same kernel, same peak map
        np.testing.assert_array_equal(ab, a0.cpu().numpy())
        np.testing.assert_array_equal(ph, p0.cpu().numpy())
        Fg = F.cpu().numpy()
        r = np.arange(n)
        np.testing.assert_array_equal(qp, Fg[r, idx, 0])          # F itself at the peak
        np.testing.assert_array_equal(up, Fg[r, idx, 1])
        l0 = plan.rmsf()[0]
        op = oracle_mod.plan(freq, "freq", w)
        Fo = oracle_mod.synth(Q, U, op, phi)
        fo = Fo[r, idx]
        tol = gh.TOL[path] * np.abs(Fo).max(axis=1)
        assert np.all(np.abs(qp - fo.real) <= tol) and np.all(np.abs(up - fo.imag) <= tol)
        co = oracle_mod.chi0(fo, phi[idx], l0)
        d = np.abs(chi.astype(np.float64) - co) % np.pi
        d = np.minimum(d, np.pi - d)
        # the angle's error is about |dF| / (2 |F|) plus FP32 rounding of the stored angle
        assert np.all(d <= tol / np.abs(fo) + 1e-6), float((d / (tol / np.abs(fo) + 1e-6)).max())
        assert np.all((chi >= 0) & (chi < np.pi + 1e-6))


def test_peak_outputs_need_tensor_path(rms, inputs):
    cfg = inputs.CONFIGS["tiny"]
    freq, w, phi = axes(inputs, cfg)
    z = torch.zeros(cfg.nchan * 4, device="cuda")
    with rms.Plan(freq, phi, "fp32_table", weights=w) as plan:
        with pytest.raises(rms.RmsError) as e:
            rms.rms_synth_peaks(plan.handle, z, z, 4, "chan", None, None, None, None, z[:4])
        assert e.value.status == rms.RMS_ERR_UNSUPPORTED


# ------------------------------------------------------------------- sub-grid peak refinement
@pytest.mark.parametrize("path", ["fp32_table", "bf16x3", "fp16x3", "bf16"])
def test_refine_peaks(rms, inputs, oracle_mod, path):
    cfg = inputs.CONFIGS["lofar"]
    freq, w, phi = axes(inputs, cfg)
    n = 2500
    Q, U = inputs.make_cube(cfg, 5151, n)
    dev = torch.device("cuda")
    with rms.Plan(freq, phi, path, weights=w) as plan:
        q = torch.from_numpy(inputs.to_layout(Q, "chan")).to(dev)
        u = torch.from_numpy(inputs.to_layout(U, "chan")).to(dev)
        F = torch.empty(n, cfg.nphi, 2, device=dev)
        pidx = torch.empty(n, dtype=torch.int32, device=dev)
        plan.synth(q, u, n, "chan", F, pidx, None, None)
        phr, abr = torch.full((n,), -7.0, device=dev), torch.full((n,), -7.0, device=dev)
        rms.rms_refine_peaks(plan.handle, F, n, pidx, phr, abr)
        plan.sync()
        Fg, ig, phr, abr = F.cpu().numpy(), pidx.cpu().numpy(), phr.cpu().numpy(), abr.cpu().numpy()
    r = np.arange(n)
    h = phi[1] - phi[0]
    # properties of the GPU's own result: within the neighbours, at least the sampled height
    ag = np.hypot(Fg[r, ig, 0].astype(np.float64), Fg[r, ig, 1].astype(np.float64))
    lo, hi = phi[np.maximum(ig - 1, 0)], phi[np.minimum(ig + 1, cfg.nphi - 1)]
    assert np.all((phr >= lo - 1e-5) & (phr <= hi + 1e-5))
    assert np.all(abr >= ag * (1 - 1e-6))
    # parity with the oracle's refinement of its own FP64 spectra, where the peak samples agree
    op = oracle_mod.plan(freq, "freq", w)
    Fo = oracle_mod.synth(Q, U, op, phi)
    io, _ = oracle_mod.peak(Fo)
    pro, aro = oracle_mod.refine_peak(Fo, phi, io)
    same = ig == io
    assert same.mean() > (0.95 if path == "bf16" else 0.98)
    # per-LOS |F| error bound: the path's tolerance; plain BF16's per-LOS tail reaches 3.5e-3
    eps = (4e-3 if path == "bf16" else gh.TOL[path]) * np.abs(Fo).max(axis=1)
    # curvature a of the oracle's parabola: y0 - 2 y1 + y2 = 2 a h^2 on the uniform grid;
    # |F| errors of eps move the vertex by at most 2.5 eps / (h |a|) and the height by about 4 eps
    yo = np.abs(Fo)
    k = np.clip(io, 1, cfg.nphi - 2)
    a = (yo[r, k - 1] - 2 * yo[r, k] + yo[r, k + 1]) / (2 * h * h)
    inner = same & (io > 0) & (io < cfg.nphi - 1) & (a < 0)
    tol_phi = 2.5 * eps / (h * np.abs(np.where(a < 0, a, -1e-30))) + 4e-6 * np.abs(phi).max()
    tol_abs = 4 * eps + 1e-6 * yo.max(axis=1)
    assert inner.sum() > 0.9 * n
    dphi, dabs = np.abs(phr - pro), np.abs(abr - aro)
    assert np.all(dphi[inner] <= tol_phi[inner]), float((dphi / tol_phi)[inner].max())
    assert np.all(dabs[same] <= tol_abs[same]), float((dabs / tol_abs)[same].max())


def test_refine_peaks_edge_cases(rms, inputs):
    cfg = inputs.CONFIGS["tiny"]
    freq, w, phi = axes(inputs, cfg)
    N = cfg.nphi
    rows = np.full((5, N), 0.25)
    rows[0, 0] = 3.0                                  # peak at the first sample
    rows[1, N - 1] = 3.0                              # peak at the last sample
    rows[2, 10:13] = [1.0, 0.5, 1.0]                  # k = 11 with a convex neighbourhood
    rows[3, 20:23] = [1.0, 2.0, 1.5]                  # interior peak
    F = np.stack([rows, np.zeros_like(rows)], axis=-1).astype(np.float32)
    idx = np.array([0, N - 1, 11, 21, -1], dtype=np.int32)
    dev = torch.device("cuda")
    with rms.Plan(freq, phi, "bf16x3", weights=w) as plan:
        Fd, idd = torch.from_numpy(F).to(dev), torch.from_numpy(idx).to(dev)
        phr, abr = torch.zeros(5, device=dev), torch.zeros(5, device=dev)
        rms.rms_refine_peaks(plan.handle, Fd, 5, idd, phr, abr)
        rms.rms_refine_peaks(plan.handle, Fd, 0, idd, phr, abr)          # empty: no-op
        with pytest.raises(rms.RmsError) as e:
            rms.rms_refine_peaks(plan.handle, Fd, -1, idd, phr, abr)
        assert e.value.status == rms.RMS_ERR_INVALID_ARG
        plan.sync()
        phr, abr = phr.cpu().numpy(), abr.cpu().numpy()
    np.testing.assert_array_equal(phr[:3], phi[idx[:3]].astype(np.float32))
    np.testing.assert_array_equal(abr[:3], F[np.arange(3), idx[:3], 0])
    h = phi[1] - phi[0]
    delta = (1.0 - 1.5) / (2 * (1.0 - 4.0 + 1.5))                       # uniform-grid vertex offset
    assert abs(phr[3] - (phi[21] + delta * h)) < 1e-5
    assert abs(abr[3] - (2.0 - 0.25 * (1.0 - 1.5) * delta)) < 1e-6
    assert np.isnan(phr[4]) and np.isnan(abr[4])


# ------------------------------------------------------------------- failure detection
def test_bounded_wait_gives_up_and_reports(rms, inputs):
    """A wait that cannot complete gives up after its limit, the plan reports
    RMS_ERR_TIMEOUT once, and the context and plan keep working."""
    cfg = inputs.CONFIGS["tiny"]
    freq, w, phi = axes(inputs, cfg)
    with rms.Plan(freq, phi, "bf16x3", weights=w) as plan:
        import time
        t0 = time.perf_counter()
        assert rms.rms_selftest_wait_timeout(plan.handle, 20_000_000) == 2       # 20 ms limit
        assert time.perf_counter() - t0 < 5.0
        with pytest.raises(rms.RmsError) as e:
            plan.sync()
        assert e.value.status == rms.RMS_ERR_TIMEOUT
        plan.sync()                                                               # cleared
        Q, U = inputs.make_cube(cfg)
        F, pidx, pabs, pphi = run(rms, plan, Q, U, "chan", cfg.nlos)              # still synthesises
        assert np.all(pidx >= 0)


# ------------------------------------------------------------------- contraction schedules
@pytest.mark.parametrize("path", ["bf16x3", "fp16x3", "bf16"])
@pytest.mark.parametrize("layout", ["chan", "los"])
def test_schedules_agree(rms, inputs, oracle_mod, path, layout):
    """The contraction's schedules on a 1536-channel x 4001-phi cube (the MWA band),
    16,384 + 77 LOS (a ragged last tile and an odd number of M tiles): single CTAs
    and CTA pairs, each with the whole schedule (every CTA runs all phase tiles of
    its M tile) and the split one (single-tile jobs in several phase-matrix panels,
    peaks merged by atomics).  Within one kernel the two schedules run the same MMAs per
    tile, so F and the peak outputs are bit-identical; the kernels are compared
    with each other and sampled rows with the oracle."""
    cfg = inputs.CONFIGS["mwa"]
    freq, w, phi = axes(inputs, cfg)
    nlos = 16384 + 77
    Q, U = inputs.make_cube(cfg, 0, nlos)
    dev = torch.device("cuda")
    from paper_1810_06250_gb300.inputs import to_layout
    q = torch.from_numpy(to_layout(Q, layout)).to(dev)
    u = torch.from_numpy(to_layout(U, layout)).to(dev)
    rows = np.r_[np.arange(0, nlos, 331), nlos - 1]
    op = oracle_mod.plan(freq, "freq", w)
    Fo = oracle_mod.synth(Q[rows], U[rows], op, phi)
    got = {}
    with rms.Plan(freq, phi, path, weights=w) as plan:
        for kind in (rms.RMS_CONTRACT_SINGLE, rms.RMS_CONTRACT_PAIR):
            for budget in (1 << 40, 16 << 20):
                rms.rms_plan_set_option(plan.handle, rms.RMS_OPT_CONTRACTION, kind)
                rms.rms_plan_set_option(plan.handle, rms.RMS_OPT_SCHEDULE,
                                        rms.RMS_SCHEDULE_WHOLE if budget > (1 << 30) else rms.RMS_SCHEDULE_AUTO)
                rms.rms_plan_set_option(plan.handle, rms.RMS_OPT_L2_BUDGET, budget)
                F = torch.full((nlos, cfg.nphi, 2), float("nan"), device=dev)
                pi = torch.full((nlos,), -7, dtype=torch.int32, device=dev)
                pa, pp, pq, pu, pc = (torch.zeros(nlos, device=dev) for _ in range(5))
                rms.rms_synth_peaks(plan.handle, q, u, nlos, layout, F, pi, pa, pp, pq, pu, pc)
                plan.sync()
                sched = (rms.rms_plan_info(plan.handle, rms.RMS_INFO_LAST_PAIR),
                         rms.rms_plan_info(plan.handle, rms.RMS_INFO_LAST_PANELS))
                assert sched[0] == (kind == rms.RMS_CONTRACT_PAIR)
                assert (sched[1] > 0) == (budget < (1 << 30)), sched
                got[(kind, budget)] = [t.cpu().numpy() for t in (F, pi, pa, pp, pq, pu, pc)]
    for kind in (rms.RMS_CONTRACT_SINGLE, rms.RMS_CONTRACT_PAIR):
        whole, split = got[(kind, 1 << 40)], got[(kind, 16 << 20)]
        for a, b in zip(whole, split):
            np.testing.assert_array_equal(a, b)
    for kind in (rms.RMS_CONTRACT_SINGLE, rms.RMS_CONTRACT_PAIR):
        F, pi, pa, pp, pq, pu, pc = got[(kind, 16 << 20)]
        ok, info = gh.gate(path, F[rows, :, 0] + 1j * F[rows, :, 1], Fo)
        assert ok, info
        gh.check_peaks_self(F, pi, pa, pp, phi)
        gh.check_peaks_oracle(pi[rows], Fo, gh.TOL[path])
        # F at the peak is the stored F there
        k = pi >= 0
        np.testing.assert_array_equal(pq[k], F[np.nonzero(k)[0], pi[k], 0])
        np.testing.assert_array_equal(pu[k], F[np.nonzero(k)[0], pi[k], 1])
    Fs, Fp = got[(rms.RMS_CONTRACT_SINGLE, 1 << 40)][0], got[(rms.RMS_CONTRACT_PAIR, 1 << 40)][0]
    d = np.abs((Fs[..., 0] - Fp[..., 0]) + 1j * (Fs[..., 1] - Fp[..., 1])).max(axis=1)
    m = np.abs(Fs[..., 0] + 1j * Fs[..., 1]).max(axis=1)
    print("single vs pair: max per-LOS difference %.3g, bit-identical %s" % ((d / m).max(), bool((d == 0).all())))
    assert (d / m).max() <= 1e-6


@pytest.mark.parametrize("path", ["bf16x3", "bf16"])
def test_peak_map_only_schedules(rms, inputs, oracle_mod, path):
    """A peak map without F: the automatic choice keeps the whole schedule while one
    panel of the phase matrix fits the L2 budget and splits into panels of single-tile
    jobs (peaks merged by 64-bit atomics) when it does not; both give the same peak
    map, which matches the oracle."""
    cfg = inputs.CONFIGS["lofar"]
    freq, w, phi = axes(inputs, cfg)
    nlos = 20000 + 33
    Q, U = inputs.make_cube(cfg, 99, nlos)
    dev = torch.device("cuda")
    q = torch.from_numpy(inputs.to_layout(Q, "chan")).to(dev)
    u = torch.from_numpy(inputs.to_layout(U, "chan")).to(dev)
    rows = np.r_[np.arange(0, nlos, 97), nlos - 1]
    Fo = oracle_mod.synth(Q[rows], U[rows], oracle_mod.plan(freq, "freq", w), phi)
    got = []
    with rms.Plan(freq, phi, path, weights=w) as plan:
        for budget, split_expected in ((1 << 40, False), (1 << 20, True)):
            rms.rms_plan_set_option(plan.handle, rms.RMS_OPT_L2_BUDGET, budget)
            pi = torch.full((nlos,), -7, dtype=torch.int32, device=dev)
            pa, pp = torch.zeros(nlos, device=dev), torch.zeros(nlos, device=dev)
            plan.synth(q, u, nlos, "chan", None, pi, pa, pp)
            plan.sync()
            assert (rms.rms_plan_info(plan.handle, rms.RMS_INFO_LAST_PANELS) > 0) == split_expected
            got.append([t.cpu().numpy() for t in (pi, pa, pp)])
    for a, b in zip(*got):
        np.testing.assert_array_equal(a, b)
    gh.check_peaks_oracle(got[0][0][rows], Fo, gh.TOL[path])


@pytest.mark.parametrize("nlos", [1, 127, 128, 129, 256, 383])
def test_pair_edges(rms, inputs, oracle_mod, nlos):
    """CTA pairs on small and ragged cubes: 1536 channels (the MWA band) x 801 phi, whose
    phase rows tile as 7 x 240 (> 208, so pairs are chosen), with 1 to 3 M tiles (an
    odd count leaves the last pair's odd CTA a padding tile); both schedules, F and the
    peak outputs against the oracle, and Q, U, chi0 at the peak with and without a
    stored F (without F the whole schedule is kept)."""
    cfg = inputs.CONFIGS["mwa"]
    freq, w = inputs.frequencies(cfg), inputs.weights(cfg)
    phi = np.linspace(-400.0, 400.0, 801)
    Q, U = inputs.make_cube(cfg, 777, nlos)
    op = oracle_mod.plan(freq, "freq", w)
    Fo = oracle_mod.synth(Q, U, op, phi)
    dev = torch.device("cuda")
    q = torch.from_numpy(inputs.to_layout(Q, "chan")).to(dev)
    u = torch.from_numpy(inputs.to_layout(U, "chan")).to(dev)
    with rms.Plan(freq, phi, "bf16x3", weights=w) as plan:
        outs = []
        for budget, with_f in ((1 << 40, True), (1 << 20, True), (1 << 20, False)):
            rms.rms_plan_set_option(plan.handle, rms.RMS_OPT_SCHEDULE,
                                    rms.RMS_SCHEDULE_WHOLE if budget > (1 << 30) else rms.RMS_SCHEDULE_AUTO)
            rms.rms_plan_set_option(plan.handle, rms.RMS_OPT_L2_BUDGET, budget)
            F = torch.full((nlos, len(phi), 2), float("nan"), device=dev) if with_f else None
            pi = torch.full((nlos,), -7, dtype=torch.int32, device=dev)
            pa, pp, pq, pu, pc = (torch.zeros(nlos, device=dev) for _ in range(5))
            rms.rms_synth_peaks(plan.handle, q, u, nlos, "chan", F, pi, pa, pp, pq, pu, pc)
            plan.sync()
            assert rms.rms_plan_info(plan.handle, rms.RMS_INFO_LAST_PAIR) == 1
            outs.append([None if F is None else F.cpu().numpy()] + [t.cpu().numpy() for t in (pi, pa, pp, pq, pu, pc)])
        F = outs[0][0]
        ok, info = gh.gate("bf16x3", F[..., 0] + 1j * F[..., 1], Fo)
        assert ok, info
        gh.check_peaks_self(F, *outs[0][1:4], phi)
        gh.check_peaks_oracle(outs[0][1], Fo, gh.TOL["bf16x3"])
        for o in outs[1:]:                # the other schedules: identical peak outputs
            for a, b in zip(outs[0][1:], o[1:]):
                np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(outs[0][0], outs[1][0])
