"""GPU checks of the learned peak proposal (through the C ABI).

* rms_generate against the host generator (inputs.make_cube), both layouts.
* The network's forward pass against the FP64 network oracle, within a bound
  derived from BF16 rounding of weights, inputs and hidden activations.
* Its gradients against the oracle's (cosine and relative norm), both layouts,
  and one AdamW step against the textbook update.
* Window synthesis against the FP64 synthesis oracle at the window's phi.
* The learned peak map against the standalone entry points it is built from,
  and against the CPU learned-peak oracle where the decisions are not knife-edge.
* Training on the GPU: agreement with full-grid synthesis, fallback rate, and
  what the trained network gains over an untrained one and over a window with
  no proposal.
"""
import numpy as np
import pytest

import gpu_helpers as gh
from oracle import net as onet

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


@pytest.fixture(scope="module")
def L():
    from paper_1810_06250_gb300 import learned
    return learned


@pytest.fixture(scope="module")
def inputs():
    from paper_1810_06250_gb300 import inputs
    return inputs


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def lofar_plan(rms, inputs, precision="bf16x3", cfg="lofar"):
    c = inputs.CONFIGS[cfg]
    return c, rms.Plan(inputs.frequencies(c), inputs.phi_grid(c), precision, weights=inputs.weights(c))


def random_params(rng, nin, hidden, nbins, scale=1.0):
    return {"W1": rng.normal(0, scale / np.sqrt(nin), (hidden, nin)), "b1": rng.normal(0, 0.1, hidden),
            "W2": rng.normal(0, 2.0 * scale / np.sqrt(hidden), (nbins, hidden)), "b2": rng.normal(0, 0.2, nbins)}


def flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"]]).astype(np.float32)


def as64(p):
    return {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}


# --------------------------------------------------------------- generator
@pytest.mark.parametrize("layout", ["chan", "los"])
def test_generate_matches_host_generator(rms, inputs, L, layout):
    cfg, plan = lofar_plan(rms, inputs, cfg="learned")
    with plan:
        n, los0 = 700, 123456
        Q, U = L.generate(plan.handle, cfg, los0, n, layout)
        torch.cuda.synchronize()
        Qh, Uh = inputs.make_cube(cfg, los0, n)
        Qg, Ug = Q.cpu().numpy(), U.cpu().numpy()
        if layout == "chan":
            Qg, Ug = Qg.T, Ug.T
        # same FP64 formula on both sides; the host's and device's libm may differ
        # in the last FP64 bit, which can move an FP32 rounding by one ulp
        for g, h in ((Qg, Qh), (Ug, Uh)):
            ulp = np.spacing(np.abs(h).astype(np.float32))
            assert np.all(np.abs(g - h) <= 2 * ulp)
            assert np.mean(g == h) > 0.99


# --------------------------------------------------------------- forward
def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("layout", ["chan", "los"])
def test_forward_matches_oracle(rms, inputs, L, layout):
    cfg, plan = lofar_plan(rms, inputs)
    with plan:
        H, NB = 64, cfg.nphi
        net = L.Net(plan, hidden=H, max_batch=512, seed=5)
        nin = 2 * plan.nact
        rng = np.random.default_rng(11)
        p = random_params(rng, nin, H, NB)
        net.set_params(flat(p))
        n = 300
        Q, U = inputs.make_cube(cfg, 5000, n)
        q, u = dev(inputs.to_layout(Q, layout)), dev(inputs.to_layout(U, layout))
        z = torch.empty((n, NB), device="cuda")
        b = torch.empty(n, dtype=torch.int32, device="cuda")
        c = torch.empty(n, device="cuda")
        rms.rms_propose(net.handle, q, u, n, layout, 14, z, b, c)
        torch.cuda.synchronize()
        zg, bg, cg = z.cpu().numpy().astype(np.float64), b.cpu().numpy(), c.cpu().numpy()
        act = np.nonzero(inputs.weights(cfg))[0]
        p64 = as64(p)
        x = onet.normalise(Q, U, act)
        zr, _ = onet.forward(p64, x)
        # The oracle fed the operands the kernels multiply: BF16 weights, BF16 raw
        # Q/U (the scale 1/s is applied after the first product), BF16 hidden values.
        s = np.sqrt(np.mean(Q[:, act].astype(np.float64) ** 2 + U[:, act].astype(np.float64) ** 2, axis=1))
        xr = onet.normalise(Q, U, act) * s[:, None]            # un-normalised, interleaved
        a1 = (bf16(xr) @ bf16(p64["W1"]).T) / s[:, None] + p64["b1"]
        hb = bf16(np.maximum(a1, 0.0))
        ze = hb @ bf16(p64["W2"]).T + p64["b2"]
        # what is left is FP32 accumulation, plus an occasional hidden value whose
        # BF16 rounding flips: one BF16 ulp of h times |W2| each
        tol = 2e-3 * (hb @ np.abs(p64["W2"]).T) + 1e-4
        assert np.all(np.abs(zg - ze) <= tol), float(np.max(np.abs(zg - ze) / tol))
        # bin and confidence are functions of the GPU's own logits
        np.testing.assert_array_equal(bg, np.argmax(zg, axis=1))
        pr = np.exp(zg - zg.max(1, keepdims=True))
        pr /= pr.sum(1, keepdims=True)
        cw = np.array([pr[i, max(0, k - 14):k + 15].sum() for i, k in enumerate(bg)])
        np.testing.assert_allclose(cg, cw, atol=2e-5)
        # and the FP64 network's bin wherever its top-2 gap clears the BF16 effect
        err = np.abs(ze - zr).max(axis=1) + tol.max(axis=1)
        srt = np.sort(zr, axis=1)
        clear = (srt[:, -1] - srt[:, -2]) > 2 * err
        assert clear.mean() > 0.5
        np.testing.assert_array_equal(bg[clear], np.argmax(zr, axis=1)[clear])
        net.close()


# --------------------------------------------------------------- gradients
def cosine(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.mark.parametrize("layout", ["chan", "los"])
def test_gradients_match_oracle(rms, inputs, L, layout):
    cfg, plan = lofar_plan(rms, inputs)
    with plan:
        H, NB = 48, cfg.nphi
        net = L.Net(plan, hidden=H, max_batch=256, seed=6)
        nin = 2 * plan.nact
        rng = np.random.default_rng(12)
        p = random_params(rng, nin, H, NB)
        net.set_params(flat(p))
        n = 200
        Q, U = inputs.make_cube(cfg, 9000, n)
        lab = rng.integers(0, NB, n).astype(np.int32)
        loss = torch.zeros(1, device="cuda")
        rms.rms_net_grad(net.handle, dev(inputs.to_layout(Q, layout)), dev(inputs.to_layout(U, layout)), n,
                         layout, dev(lab), loss)
        g = L.unpack(net.grads(), nin, H, NB)
        act = np.nonzero(inputs.weights(cfg))[0]
        p64 = as64(p)
        x = onet.normalise(Q, U, act)
        lr_, gr = onet.loss_and_grads(p64, x, lab)
        assert abs(float(loss.item()) - lr_) <= 1e-2 * abs(lr_)
        # the oracle at the operands the kernels multiply (BF16 weights and raw Q/U):
        # what remains is BF16 rounding of the backward pass's intermediates
        s = np.sqrt(np.mean(Q[:, act].astype(np.float64) ** 2 + U[:, act].astype(np.float64) ** 2, axis=1))
        xq = bf16(x * s[:, None]) / s[:, None]
        pq = dict(p64, W1=bf16(p64["W1"]), W2=bf16(p64["W2"]))
        _, gq = onet.loss_and_grads(pq, xq, lab)
        for k in ("W1", "b1", "W2", "b2"):
            c = cosine(g[k].astype(np.float64), gq[k])
            rel = np.linalg.norm(g[k] - gq[k]) / np.linalg.norm(gq[k])
            assert c >= 0.999 and rel <= 2e-2, (k, c, rel)
            # and close to the unquantised network's gradient (ReLU masks of
            # near-zero pre-activations may differ there)
            assert cosine(g[k].astype(np.float64), gr[k]) >= 0.99, k
        net.close()


def test_adamw_step(rms, inputs, L):
    cfg, plan = lofar_plan(rms, inputs)
    with plan:
        H, NB = 32, cfg.nphi
        net = L.Net(plan, hidden=H, max_batch=256, seed=7)
        nin = 2 * plan.nact
        p0 = flat(random_params(np.random.default_rng(13), nin, H, NB))
        net.set_params(p0)
        n = 128
        Q, U = inputs.make_cube(cfg, 100, n)
        lab = np.random.default_rng(14).integers(0, NB, n).astype(np.int32)
        lr, b1, b2, eps, wd = 1e-3, 0.9, 0.999, 1e-8, 0.01
        rms.rms_train_step(net.handle, dev(Q), dev(U), n, "los", dev(lab), lr, b1, b2, eps, wd)
        g = net.grads().astype(np.float64)
        p1 = net.params().astype(np.float64)
        # AdamW, step 1: m = (1-b1) g, v = (1-b2) g^2, bias-corrected m/(1-b1) = g, v/(1-b2) = g^2
        p = p0.astype(np.float64)
        is_w = np.zeros_like(p, dtype=bool)
        o1 = H * nin
        is_w[:o1] = True
        is_w[o1 + H:o1 + H + NB * H] = True
        exp = p - lr * (g / (np.abs(g) + eps) + np.where(is_w, wd * p, 0.0))
        np.testing.assert_allclose(p1, exp, rtol=2e-6, atol=2e-9)
        assert rms.rms_net_info(net.handle, rms.RMS_NET_STEPS) == 1
        net.close()


# --------------------------------------------------------------- window synthesis
@pytest.mark.parametrize("layout", ["chan", "los"])
@pytest.mark.parametrize("precision", ["bf16x3", "bf16"])
def test_window_synthesis_matches_oracle(rms, inputs, L, oracle_mod, layout, precision):
    cfg, plan = lofar_plan(rms, inputs, precision)
    with plan:
        W = 64
        win = L.Window(plan, W)
        n = 300
        Q, U = inputs.make_cube(cfg, 777, n)
        rng = np.random.default_rng(15)
        centre = rng.integers(32, 770, n).astype(np.int32)
        centre[:4] = [32, 769, 0, 5000]                 # edges, and two clamped out-of-range centres
        F = torch.full((n, W, 2), float("nan"), device="cuda")
        k = torch.empty(n, dtype=torch.int32, device="cuda")
        a = torch.empty(n, device="cuda")
        ph = torch.empty(n, device="cuda")
        rms.rms_synth_window(win.handle, dev(inputs.to_layout(Q, layout)), dev(inputs.to_layout(U, layout)), n,
                             layout, dev(centre), F, k, a, ph)
        torch.cuda.synchronize()
        Fg, kg, ag, pg = F.cpu().numpy(), k.cpu().numpy(), a.cpu().numpy(), ph.cpu().numpy()
        phi = inputs.phi_grid(cfg)
        cc = np.clip(centre, 32, 769)
        op = oracle_mod.plan(inputs.frequencies(cfg), "freq", inputs.weights(cfg))
        Fo = np.empty((n, W), dtype=np.complex128)
        for i in range(n):
            Fo[i] = oracle_mod.synth(Q[i:i + 1], U[i:i + 1], op, onet.fine_phi(phi, cc[i] - 32 + np.arange(W)))[0]
        # A window is a slice of its LOS's F: errors are relative to that LOS's
        # max |F| (on the full grid), or to the cube's max for plain BF16.
        full_max = np.abs(oracle_mod.synth(Q, U, op, phi)).max(axis=1)
        norm = np.full(n, full_max.max()) if precision in gh.CUBE_NORMALISED else full_max
        err = np.abs(Fg[..., 0] + 1j * Fg[..., 1] - Fo).max(axis=1) / norm
        assert err.max() <= gh.TOL[precision], (precision, float(err.max()), float(np.quantile(err, 0.99)))
        kk, best = gh.argmax_fp32(Fg)
        np.testing.assert_array_equal(kg, kk)
        np.testing.assert_array_equal(ag, np.sqrt(best).astype(np.float32))
        np.testing.assert_array_equal(pg, onet.fine_phi(phi, cc - 32 + kg).astype(np.float32))
        # the oracle's window maximum wherever its top-2 gap exceeds 4x the tolerance
        a = np.abs(Fo)
        srt = np.sort(a, axis=1)
        clear = (srt[:, -1] - srt[:, -2]) > 4 * gh.TOL[precision] * norm
        # (plain BF16's tolerance is relative to the cube: few weak windows clear it)
        assert clear.mean() > (0.9 if precision == "bf16x3" else 0.1)
        np.testing.assert_array_equal(kg[clear], np.argmax(a, axis=1)[clear])


def test_window_centres_match_oracle(rms, inputs, L):
    """rms_window_centres (the centres the learned peak map uses; calibration takes
    them from here) equals the oracle's window_centre, including both clamps."""
    cfg, plan = lofar_plan(rms, inputs)
    with plan:
        for W in (8, 64, 128):
            win = L.Window(plan, W)
            bins = np.concatenate([np.arange(cfg.nphi), [0, 1, 3, cfg.nphi - 1, cfg.nphi - 2]]).astype(np.int32)
            c = torch.full((len(bins),), -5, dtype=torch.int32, device="cuda")
            rms.rms_window_centres(win.handle, dev(bins), len(bins), c)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(c.cpu().numpy(), onet.window_centre(bins, cfg.nphi, W))
            win.close()


def test_window_thin_source_on_fine_grid(rms, inputs, L):
    # A thin source half-way between coarse grid points: the window finds it
    # exactly, with |F| = p0 (thin-source identity), which no coarse point can.
    cfg, plan = lofar_plan(rms, inputs)
    with plan:
        win = L.Window(plan, 64)
        lam2 = inputs.lambda2(inputs.frequencies(cfg))
        P = 0.8 * np.exp(2j * (0.4 + 10.25 * lam2))
        Q = np.tile(P.real.astype(np.float32), (3, 1))
        U = np.tile(P.imag.astype(np.float32), (3, 1))
        centre = np.array([440, 420, 460], dtype=np.int32)      # phi 10.0, 5.0, 15.0
        k = torch.empty(3, dtype=torch.int32, device="cuda")
        a = torch.empty(3, device="cuda")
        ph = torch.empty(3, device="cuda")
        rms.rms_synth_window(win.handle, dev(Q), dev(U), 3, "los", dev(centre), None, k, a, ph)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ph.cpu().numpy(), np.float32(10.25))
        np.testing.assert_allclose(a.cpu().numpy(), 0.8, rtol=1e-5)
        win.close()


# --------------------------------------------------------------- learned peak map
@pytest.mark.parametrize("layout", ["chan", "los"])
def test_peakmap_learned_is_its_parts(rms, inputs, L, oracle_mod, layout):
    cfg, plan = lofar_plan(rms, inputs)
    with plan:
        H, W = 64, 64
        net = L.Net(plan, hidden=H, max_batch=512, seed=8)
        nin = 2 * plan.nact
        p = random_params(np.random.default_rng(16), nin, H, cfg.nphi, scale=3.0)
        net.set_params(flat(p))
        win = L.Window(plan, W)
        n = 1000
        Q, U = inputs.make_cube(cfg, 31337, n)
        q, u = dev(inputs.to_layout(Q, layout)), dev(inputs.to_layout(U, layout))
        b = torch.empty(n, dtype=torch.int32, device="cuda")
        c = torch.empty(n, device="cuda")
        rms.rms_propose(net.handle, q, u, n, layout, W // 4 - 2, None, b, c)
        tau = float(np.median(c.cpu().numpy()))
        centre = dev(np.clip(2 * b.cpu().numpy(), 32, 769).astype(np.int32))
        wk = torch.empty(n, dtype=torch.int32, device="cuda")
        wa = torch.empty(n, device="cuda")
        wp = torch.empty(n, device="cuda")
        rms.rms_synth_window(win.handle, q, u, n, layout, centre, None, wk, wa, wp)
        fi = torch.empty(n, dtype=torch.int32, device="cuda")
        fa = torch.empty(n, device="cuda")
        fp = torch.empty(n, device="cuda")
        plan.synth(q, u, n, layout, None, fi, fa, fp)
        php = torch.full((n,), -123.0, device="cuda")
        pka = torch.full((n,), -1.0, device="cuda")
        fb = torch.full((n,), 7, dtype=torch.int32, device="cuda")
        nfb = torch.zeros(1, dtype=torch.int64, device="cuda")
        rms.rms_peakmap_learned(win.handle, net.handle, q, u, n, layout, tau, php, pka, fb, nfb)
        torch.cuda.synchronize()
        cg, wkg = c.cpu().numpy(), wk.cpu().numpy()
        expect_fb = ~(cg >= tau) | (wkg <= 0) | (wkg >= W - 1)
        fbg = fb.cpu().numpy().astype(bool)
        np.testing.assert_array_equal(fbg, expect_fb)
        assert int(nfb.item()) == int(expect_fb.sum())
        assert 0.3 < expect_fb.mean() < 0.99            # both branches exercised
        phg, pag = php.cpu().numpy(), pka.cpu().numpy()
        np.testing.assert_array_equal(phg[~fbg], wp.cpu().numpy()[~fbg])
        np.testing.assert_array_equal(pag[~fbg], wa.cpu().numpy()[~fbg])
        np.testing.assert_array_equal(phg[fbg], fp.cpu().numpy()[fbg])
        np.testing.assert_array_equal(pag[fbg], fa.cpu().numpy()[fbg])
        # against the CPU learned-peak oracle, where its decision is not on a knife edge
        m = 120
        lam2 = inputs.lambda2(inputs.frequencies(cfg))
        oph, _, ofb = onet.learned_peaks(oracle_mod, lam2, inputs.weights(cfg), inputs.phi_grid(cfg), as64(p),
                                         Q[:m].astype(np.float64), U[:m].astype(np.float64), tau, W, W // 4 - 2)
        act = np.nonzero(inputs.weights(cfg))[0]
        ob, oc = onet.propose(as64(p), onet.normalise(Q[:m], U[:m], act), W // 4 - 2)
        firm = (np.abs(oc - tau) > 0.05) & (ob == b.cpu().numpy()[:m])
        assert firm.sum() > 30
        same = (ofb[firm] == fbg[:m][firm]) & (np.abs(oph[firm] - phg[:m][firm]) <= 1e-4)
        assert same.mean() >= 0.97, same.mean()
        net.close()
        win.close()


def test_learned_agreement_and_ablation(rms, inputs, L):
    """Train on the GPU, then: agreement >= 99.5 % with the full grid at a fallback
    rate well below that of an untrained network, which must fall back almost
    everywhere; and a window with no proposal (the grid centre) does not agree."""
    cfg, plan = lofar_plan(rms, inputs, cfg="learned")
    with plan:
        net = L.Net(plan, hidden=256, max_batch=4096, seed=21)
        win = L.Window(plan, 64)
        hist = L.train(plan.handle, net, cfg, n_train=1 << 18, epochs=6, batch=2048)
        assert hist[-1] < 0.75 * hist[0], hist
        tau, st = L.calibrate(plan.handle, net, win, cfg, n_val=1 << 16)
        n = 1 << 17
        Q, U = L.generate(plan.handle, cfg, 0, n, "los", seed=7003)
        _, fphi, _ = L.full_peaks(plan.handle, Q, U, n)
        fphi = fphi.cpu().numpy()

        def run(netw):
            php = torch.empty(n, device="cuda")
            fb = torch.empty(n, dtype=torch.int32, device="cuda")
            rms.rms_peakmap_learned(win.handle, netw.handle, Q, U, n, "los", tau, php, None, fb, None)
            torch.cuda.synchronize()
            agree = np.abs(php.cpu().numpy() - fphi) <= 0.5 * (1 + 1e-6)
            return agree.mean(), fb.cpu().numpy().mean()

        agree, fbr = run(net)
        print("learned: loss %s tau %.4f val-fallback %.4f agreement %.5f fallback %.4f"
              % (["%.3f" % h for h in hist], tau, st["fallback_frac"], agree, fbr))
        assert agree >= 0.995, (agree, fbr, tau)
        assert fbr <= 0.6, (agree, fbr, tau)
        untrained = L.Net(plan, hidden=256, max_batch=4096, seed=22)
        agree_u, fbr_u = run(untrained)
        print("untrained: agreement %.5f fallback %.4f" % (agree_u, fbr_u))
        assert agree_u >= 0.995 and fbr_u >= 0.95, (agree_u, fbr_u)
        # no proposal: every window at the grid centre, nothing falls back
        centre = dev(np.full(n, 400, dtype=np.int32))
        wp = torch.empty(n, device="cuda")
        rms.rms_synth_window(win.handle, Q, U, n, "los", centre, None, None, None, wp)
        torch.cuda.synchronize()
        assert np.mean(np.abs(wp.cpu().numpy() - fphi) <= 0.5 * (1 + 1e-6)) < 0.5
        untrained.close()
        net.close()
        win.close()
