"""Learned peak proposal: training and calibration driver (host logic only).

Every number here is computed by librms.so: rms_generate draws the training
spectra on the device, rms_synth (peak map only) labels them with the full-grid
argmax of |F|, rms_train_step runs the network's forward/backward kernels and
AdamW, rms_propose / rms_synth_window / rms_peakmap_learned run the proposal.
This module only sequences those calls, holds torch tensors as device buffers
and picks the confidence threshold from the results.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B
from .inputs import CubeConfig, frequencies, weights, phi_grid


def source_model(cfg: CubeConfig, seed: int | None = None) -> B.rms_source_model:
    """The C source model for a workload's source distribution (inputs.components)."""
    m = B.rms_source_model()
    m.seed = cfg.seed if seed is None else seed
    m.ncomp_min, m.ncomp_max = cfg.ncomp
    m.phi0_min, m.phi0_max = cfg.phi0
    m.p0_min, m.p0_max = cfg.p0
    m.slab_prob = cfg.slab_prob
    m.slab_w = cfg.slab_w
    m.sigma = cfg.sigma
    m.snr_min, m.snr_max = cfg.snr if cfg.snr is not None else (0.0, 0.0)
    return m


def _handle(plan):
    return plan if isinstance(plan, int) else plan.handle


class Net:
    """Owns one rms_net_t; keeps the plan object it was built on alive."""

    def __init__(self, plan, hidden: int = 256, max_batch: int = 4096, seed: int = 1):
        self.plan = plan
        self.handle = B.rms_net_create(_handle(plan), hidden, max_batch, seed)
        self.nparams = B.rms_net_info(self.handle, B.RMS_NET_NPARAMS)
        self.max_batch = max_batch
        self.hidden = hidden

    def params(self) -> np.ndarray:
        a = np.empty(self.nparams, dtype=np.float32)
        B.rms_net_params(self.handle, B.RMS_NET_PARAMS, a)
        return a

    def grads(self) -> np.ndarray:
        a = np.empty(self.nparams, dtype=np.float32)
        B.rms_net_params(self.handle, B.RMS_NET_GRADS, a)
        return a

    def set_params(self, a):
        B.rms_net_params(self.handle, B.RMS_NET_PARAMS, np.ascontiguousarray(a, dtype=np.float32), set=True)

    def close(self):
        if getattr(self, "handle", None):
            B.rms_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Window:
    """Owns one rms_window_t; keeps the plan object it was built on alive."""

    def __init__(self, plan, width: int = 64):
        self.plan = plan
        self.handle = B.rms_window_create(_handle(plan), width)
        self.width = width

    @property
    def conf_halfwidth(self) -> int:
        return self.width // 4 - 2

    def close(self):
        if getattr(self, "handle", None):
            B.rms_window_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unpack(params: np.ndarray, nin: int, hidden: int, nbins: int) -> dict:
    """Flat parameter array -> {W1, b1, W2, b2} views (include/rms.h order)."""
    o1 = hidden * nin
    o2 = o1 + hidden
    o3 = o2 + nbins * hidden
    return {"W1": params[:o1].reshape(hidden, nin), "b1": params[o1:o2],
            "W2": params[o2:o3].reshape(nbins, hidden), "b2": params[o3:o3 + nbins]}


def generate(plan: int, cfg: CubeConfig, los0: int, nlos: int, layout: str = "los", seed: int | None = None):
    """Device Q, U (torch float32) for lines of sight los0 .. los0 + nlos - 1."""
    import torch
    shape = (nlos, cfg.nchan) if layout == "los" else (cfg.nchan, nlos)
    Q = torch.empty(shape, dtype=torch.float32, device="cuda")
    U = torch.empty(shape, dtype=torch.float32, device="cuda")
    B.rms_generate(plan, source_model(cfg, seed), los0, nlos, layout, Q, U)
    return Q, U


def full_peaks(plan: int, Q, U, nlos: int, layout: str = "los"):
    """Full-grid peak map (index, phi, |F|) from rms_synth, no F written."""
    import torch
    idx = torch.empty(nlos, dtype=torch.int32, device="cuda")
    phi = torch.empty(nlos, dtype=torch.float32, device="cuda")
    ab = torch.empty(nlos, dtype=torch.float32, device="cuda")
    B.rms_synth(plan, Q, U, nlos, layout, None, idx, ab, phi)
    return idx, phi, ab


def train(plan: int, net: Net, cfg: CubeConfig, n_train: int, epochs: int = 8, batch: int = 2048,
          lr: float = 2e-3, lr_decay: float = 0.75, weight_decay: float = 1e-4, seed: int = 7001,
          log_every: int = 0):
    """Train on n_train generated LOS (LOS-major), labels = full-grid argmax bins.

    Returns the per-epoch mean loss (one host sync per epoch).
    """
    import torch
    if batch > net.max_batch:
        raise ValueError("batch exceeds the network's max_batch")
    Q, U = generate(plan, cfg, 0, n_train, "los", seed=seed)
    lab, _, _ = full_peaks(plan, Q, U, n_train, "los")
    # an all-NaN spectrum has no peak (-1): train it towards bin 0
    lab = torch.from_numpy(np.maximum(lab.cpu().numpy(), 0)).cuda()
    nb = n_train // batch
    loss = torch.zeros(nb, dtype=torch.float32, device="cuda")
    hist = []
    rate = lr
    for _ in range(epochs):
        for i in range(nb):
            sl = slice(i * batch, (i + 1) * batch)
            B.rms_train_step(net.handle, Q[sl], U[sl], batch, "los", lab[sl], rate, weight_decay=weight_decay,
                             loss=loss[i:i + 1])
        hist.append(float(loss.cpu().numpy().mean()))
        rate *= lr_decay
    del Q, U, lab
    return hist


def calibrate(plan: int, net: Net, win: Window, cfg: CubeConfig, n_val: int, target: float = 0.997,
              seed: int = 7002, layout: str = "los"):
    """Smallest confidence threshold whose window results agree with the full
    grid (|phi difference| <= one coarse step) on a fraction >= target of a
    validation set, counting fallbacks as agreeing.  Returns (tau, stats)."""
    import torch
    Q, U = generate(plan, cfg, 0, n_val, layout, seed=seed)
    _, fphi, _ = full_peaks(plan, Q, U, n_val, layout)
    bin_ = torch.empty(n_val, dtype=torch.int32, device="cuda")
    conf = torch.empty(n_val, dtype=torch.float32, device="cuda")
    B.rms_propose(net.handle, Q, U, n_val, layout, win.conf_halfwidth, None, bin_, conf)
    centre = torch.empty(n_val, dtype=torch.int32, device="cuda")
    B.rms_window_centres(win.handle, bin_, n_val, centre)      # the centres rms_peakmap_learned uses
    widx = torch.empty(n_val, dtype=torch.int32, device="cuda")
    wphi = torch.empty(n_val, dtype=torch.float32, device="cuda")
    B.rms_synth_window(win.handle, Q, U, n_val, layout, centre, None, widx, None, wphi)
    step = (cfg.phi_max - cfg.phi_min) / (cfg.nphi - 1)
    c = conf.cpu().numpy().astype(np.float64)
    k = widx.cpu().numpy()
    ok = np.abs(wphi.cpu().numpy().astype(np.float64) - fphi.cpu().numpy()) <= step * (1 + 1e-6)
    edge = (k <= 0) | (k >= win.width - 1)
    c = np.where(np.isnan(c), -1.0, c)
    best = (1.0 + 1e-6, 1.0)
    for tau in np.unique(np.concatenate([np.linspace(0, 1, 201), np.quantile(c, np.linspace(0, 1, 401))])):
        fb = edge | (c < tau)
        agree = np.mean(np.where(fb, True, ok))
        if agree >= target:
            best = (float(tau), float(np.mean(fb)))
            break
    return best[0], {"fallback_frac": best[1], "n": n_val}
