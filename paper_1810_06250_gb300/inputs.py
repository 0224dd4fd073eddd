"""Seeded synthetic Stokes Q/U cubes shaped like the paper's workloads.

This module is the one piece shared by the GPU tests, the benchmark and the
oracle-side checks.  It holds none of RM synthesis' arithmetic: it only draws
sources and writes P(lambda^2) = Q + iU for them, so both sides start from the
same numbers.

Source models (Sridhar et al., Sec. 2.1):
  * Faraday-thin component, Eqs. PAdefn and Pdefn:
        P(lambda^2) = p0 exp(2i (chi0 + phi0 lambda^2))
  * Burn slab of width W centred at phi_c: F(phi) = p0 e^{2i chi0} / W on
    [phi_c - W/2, phi_c + W/2]; integrating Eq. Predefn gives
        P(lambda^2) = p0 exp(2i (chi0 + phi_c lambda^2)) sin(W lambda^2) / (W lambda^2)
  * independent Gaussian noise of standard deviation sigma on Q and on U.

Random numbers come from a counter-based generator (a SplitMix64 finaliser
applied to a linear mix of seed, line-of-sight index and draw index), so any
single line of sight can be regenerated without generating the others.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299792458.0  # m/s

_M_SEED = np.uint64(0x9E3779B97F4A7C15)
_M_LOS = np.uint64(0xD1B54A32D192ED03)
_M_DRAW = np.uint64(0x8CB92BA72F3D8DD7)
_NOISE_STREAM = 1 << 32
_FLAG_LOS = 1 << 40


def _mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014), on uint64 arrays."""
    x = x ^ (x >> np.uint64(30))
    x = x * np.uint64(0xBF58476D1CE4E5B9)
    x = x ^ (x >> np.uint64(27))
    x = x * np.uint64(0x94D049BB133111EB)
    x = x ^ (x >> np.uint64(31))
    return x


def uniform(seed: int, los, draw) -> np.ndarray:
    """U(0, 1] doubles for (seed, los, draw); los and draw broadcast."""
    los = np.asarray(los, dtype=np.uint64)
    draw = np.asarray(draw, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = np.uint64(seed) * _M_SEED + los * _M_LOS + draw * _M_DRAW
        h = _mix64(np.asarray(x, dtype=np.uint64))
    return ((h >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed: int, los, draw) -> np.ndarray:
    """N(0, 1) doubles by the Box-Muller cosine branch from two uniforms of a separate stream."""
    draw = np.asarray(draw, dtype=np.uint64)
    u1 = uniform(seed, los, np.uint64(_NOISE_STREAM) + np.uint64(2) * draw)
    u2 = uniform(seed, los, np.uint64(_NOISE_STREAM) + np.uint64(2) * draw + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclass(frozen=True)
class CubeConfig:
    """One synthetic workload: cube shape, band, phi grid and source model."""
    name: str
    nlos: int
    nchan: int
    nu0: float           # Hz, first channel centre
    nu1: float           # Hz, last channel centre
    nphi: int
    phi_min: float       # rad m^-2
    phi_max: float
    seed: int
    flag_frac: float = 0.0
    ncomp: tuple = (1, 3)
    phi0: tuple = (-40.0, 40.0)
    p0: tuple = (0.0, 1.0)
    slab_prob: float = 0.0      # probability that a component is a Burn slab
    slab_w: float = 0.0         # slab width W ~ U(0, slab_w)
    sigma: float = 0.01
    snr: tuple | None = None    # if set, sigma is drawn per LOS so max p0 / sigma_F ~ U(snr)
    extra: dict = field(default_factory=dict)

    @property
    def units(self) -> int:
        return self.nlos * self.nchan * self.nphi


# Workloads shaped like the paper's cubes (WSRT / LOFAR / MWA-like bands);
# names describe what they are.
CONFIGS = {
    # 16x16 LOS, 64 channels 120-168 MHz, 101 phi in +-50, thin sources, sigma 0.01
    "tiny": CubeConfig("tiny", 16 * 16, 64, 120e6, 168e6, 101, -50.0, 50.0, seed=1001),
    # LOFAR-HBA-like: 512^2 LOS, 400 channels 115-178 MHz, 10% flagged, 401 phi in +-100
    "lofar": CubeConfig("lofar", 512 * 512, 400, 115e6, 178e6, 401, -100.0, 100.0, seed=1002,
                        flag_frac=0.10, slab_prob=0.5, slab_w=10.0, sigma=0.005),
    # precision study: 2048^2 LOS, 800 channels 110-190 MHz, 1001 phi in +-500
    "precision": CubeConfig("precision", 2048 * 2048, 800, 110e6, 190e6, 1001, -500.0, 500.0,
                            seed=1003, phi0=(-450.0, 450.0)),
    # MWA-like large phases: 1024^2 LOS, 1536 channels 72-231 MHz, 4001 phi in +-2000
    "mwa": CubeConfig("mwa", 1024 * 1024, 1536, 72e6, 231e6, 4001, -2000.0, 2000.0, seed=1004,
                      phi0=(-1800.0, 1800.0)),
    # the paper's LOFAR benchmark shapes (Sec. 3.3): 856 channels 120.238-166.087 MHz,
    # 7000 phi to about +-350 rad/m^2; low resolution 540^2 LOS, high resolution 4000^2
    "lofar_lr": CubeConfig("lofar_lr", 540 * 540, 856, 120.238e6, 166.087e6, 7000, -350.0, 350.0, seed=1006,
                           phi0=(-300.0, 300.0), slab_prob=0.5, slab_w=10.0, sigma=0.005),
    "lofar_hr": CubeConfig("lofar_hr", 4000 * 4000, 856, 120.238e6, 166.087e6, 7000, -350.0, 350.0, seed=1007,
                           phi0=(-300.0, 300.0), slab_prob=0.5, slab_w=10.0, sigma=0.005),
    # learned-proposal workload: 2048^2 LOS on the LOFAR band and grid, SNR 5-100,
    # thin components and Burn slabs mixed as on the LOFAR cube
    # the LOFAR cube's shape and sources with channels uniform in lambda^2 over the same
    # band (lambda^2 from that of 178 MHz to that of 115 MHz): the case FFT synthesis takes
    "lofar_ul2": CubeConfig("lofar_ul2", 512 * 512, 400, 115e6, 178e6, 401, -100.0, 100.0, seed=1008,
                            flag_frac=0.10, slab_prob=0.5, slab_w=10.0, sigma=0.005,
                            extra={"lambda2_uniform": True}),
    "learned": CubeConfig("learned", 2048 * 2048, 400, 115e6, 178e6, 401, -100.0, 100.0, seed=1005,
                          flag_frac=0.10, slab_prob=0.5, slab_w=10.0, snr=(5.0, 100.0)),
}


def frequencies(cfg: CubeConfig) -> np.ndarray:
    """Channel centres in Hz: inclusive linspace(nu0, nu1, nchan), or, for a config with
    extra["lambda2_uniform"], the frequencies whose lambda^2 = (c / nu)^2 are an inclusive
    linspace from lambda^2(nu0) to lambda^2(nu1)."""
    if cfg.extra.get("lambda2_uniform"):
        l2 = np.linspace((C_LIGHT / cfg.nu0) ** 2, (C_LIGHT / cfg.nu1) ** 2, cfg.nchan)
        return C_LIGHT / np.sqrt(l2)
    return np.linspace(cfg.nu0, cfg.nu1, cfg.nchan)


def weights(cfg: CubeConfig) -> np.ndarray:
    """1 for good channels, 0 for a seeded random flag_frac of the channels."""
    w = np.ones(cfg.nchan)
    nflag = int(round(cfg.flag_frac * cfg.nchan))
    if nflag:
        r = uniform(cfg.seed, _FLAG_LOS, np.arange(cfg.nchan))
        w[np.argsort(r, kind="stable")[:nflag]] = 0.0
    return w


def phi_grid(cfg: CubeConfig) -> np.ndarray:
    """phi_k = phi_min + k (phi_max - phi_min) / (nphi - 1), not accumulated."""
    if cfg.nphi == 1:
        return np.array([cfg.phi_min])
    step = (cfg.phi_max - cfg.phi_min) / (cfg.nphi - 1)
    return cfg.phi_min + step * np.arange(cfg.nphi)


def lambda2(freq: np.ndarray) -> np.ndarray:
    return (C_LIGHT / np.asarray(freq, dtype=np.float64)) ** 2


def components(cfg: CubeConfig, los: np.ndarray) -> dict:
    """The drawn source parameters for the given LOS indices (arrays of shape [n, 3])."""
    los = np.asarray(los, dtype=np.uint64)
    n = los.shape[0]
    s = cfg.seed
    lo, hi = cfg.ncomp
    ncomp = lo + np.minimum((uniform(s, los, 0) * (hi - lo + 1)).astype(np.int64), hi - lo)
    out = {k: np.zeros((n, 3)) for k in ("phi0", "p0", "chi0", "width")}
    out["ncomp"] = ncomp
    for c in range(3):
        d = 1 + 8 * c
        present = c < ncomp
        is_slab = uniform(s, los, d + 0) < cfg.slab_prob
        out["phi0"][:, c] = cfg.phi0[0] + (cfg.phi0[1] - cfg.phi0[0]) * uniform(s, los, d + 1)
        out["p0"][:, c] = np.where(present, cfg.p0[0] + (cfg.p0[1] - cfg.p0[0]) * uniform(s, los, d + 2), 0.0)
        out["chi0"][:, c] = np.pi * uniform(s, los, d + 3)
        out["width"][:, c] = np.where(is_slab, cfg.slab_w * uniform(s, los, d + 4), 0.0)
    if cfg.snr is not None:
        w = weights(cfg)
        snr = cfg.snr[0] + (cfg.snr[1] - cfg.snr[0]) * uniform(s, los, 30)
        noise_gain = np.sqrt(np.sum(w * w)) / np.sum(w)
        out["sigma"] = out["p0"].max(axis=1) / (snr * noise_gain)
        out["snr"] = snr
    else:
        out["sigma"] = np.full(n, cfg.sigma)
    return out


def make_cube(cfg: CubeConfig, start: int = 0, count: int | None = None,
              noise: bool = True, chunk: int = 8192):
    """Q, U as float32 [count][nchan] (LOS-major) for LOS indices start .. start+count-1."""
    if count is None:
        count = cfg.nlos - start
    lam2 = lambda2(frequencies(cfg))
    Q = np.empty((count, cfg.nchan), dtype=np.float32)
    U = np.empty((count, cfg.nchan), dtype=np.float32)
    chan = np.arange(cfg.nchan, dtype=np.uint64)
    for c0 in range(0, count, chunk):
        n = min(chunk, count - c0)
        los = np.arange(start + c0, start + c0 + n, dtype=np.uint64)
        comp = components(cfg, los)
        q = np.zeros((n, cfg.nchan))
        u = np.zeros((n, cfg.nchan))
        for c in range(3):
            p0 = comp["p0"][:, c:c + 1]
            ang = 2.0 * (comp["chi0"][:, c:c + 1] + comp["phi0"][:, c:c + 1] * lam2[None, :])
            wl = comp["width"][:, c:c + 1] * lam2[None, :]
            amp = p0 * np.sinc(wl / np.pi)      # sin(W l^2) / (W l^2), 1 at W = 0
            q += amp * np.cos(ang)
            u += amp * np.sin(ang)
        if noise:
            sig = comp["sigma"][:, None]
            q += sig * normal(cfg.seed, los[:, None], 2 * chan[None, :])
            u += sig * normal(cfg.seed, los[:, None], 2 * chan[None, :] + np.uint64(1))
        Q[c0:c0 + n] = q
        U[c0:c0 + n] = u
    return Q, U


def to_layout(A: np.ndarray, layout: str) -> np.ndarray:
    """LOS-major [nlos][nchan] -> 'los' (unchanged) or 'chan' ([nchan][nlos], FITS plane order)."""
    if layout == "los":
        return np.ascontiguousarray(A)
    if layout == "chan":
        return np.ascontiguousarray(A.T)
    raise ValueError(layout)
