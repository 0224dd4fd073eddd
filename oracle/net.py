"""FP64 CPU oracle of the learned peak proposal -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and the benchmark's CPU-baseline leg use this
module; the library never does.  It is the plain definition the GPU kernels are
checked against.  Nothing here is in the paper: the network proposes which bin
of the full phi grid holds the peak of |F| (Sec. 2.2's peak, Eq. RMSynth), and
exact synthesis then runs on a narrow finer window around the proposal.

Network (a two-layer perceptron on one line of sight's spectrum):
  input   x = [Q_a0, U_a0, Q_a1, U_a1, ...] / s over the active (w > 0) channels
          in ascending channel order, s = sqrt(mean over active channels of
          Q^2 + U^2), s = 1 for an all-zero spectrum
  hidden  h = relu(W1 x + b1)                                       W1: [H][2 Na]
  logits  z = W2 h + b2                                             W2: [NB][H]
  loss    mean over the batch of -log softmax(z)[label]
  proposal  bin = argmax z (lowest index on ties);
            confidence = softmax mass of the bins within `halfwin` of bin
            (halfwin < 0: the largest probability)

Learned peak map (one line of sight), for a uniform phi grid of step D:
  the fine grid is phi_0 + n D / 2, n = 0 .. 2 (NB - 1); the window of width W
  (even) centred on fine point c covers c - W/2 .. c + W/2 - 1, with
  c = 2 bin clamped to [W/2, 2 (NB - 1) - W/2 + 1] so the window stays on the
  fine grid; |F| on the window is exact synthesis (oracle.synth) there; the
  line of sight falls back to the full grid when the confidence is below tau
  (or is NaN), when the window maximum sits on the window's first or last
  point, or when the window holds no finite |F|.

Gradients are the textbook backward pass of the loss above; the finite-
difference test in tests/test_net_oracle.py pins them.
"""
from __future__ import annotations

import numpy as np


def normalise(Q, U, active):
    """[nlos][nchan] LOS-major Q, U -> [nlos][2 Na] network input (float64)."""
    act = np.asarray(active)
    q = np.asarray(Q, dtype=np.float64)[:, act]
    u = np.asarray(U, dtype=np.float64)[:, act]
    s = np.sqrt(np.sum(q * q + u * u, axis=1) / len(act))
    s = np.where(s > 0, s, 1.0)
    x = np.empty((q.shape[0], 2 * len(act)))
    x[:, 0::2] = q
    x[:, 1::2] = u
    return x / s[:, None]


def forward(p, x):
    """Returns (logits, cache)."""
    a1 = x @ p["W1"].T + p["b1"]
    h = np.maximum(a1, 0.0)
    z = h @ p["W2"].T + p["b2"]
    return z, (x, a1, h)


def softmax(z):
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def loss_and_grads(p, x, labels):
    """Mean cross-entropy over the batch and its gradients w.r.t. every parameter."""
    z, (x, a1, h) = forward(p, x)
    n = x.shape[0]
    pr = softmax(z)
    loss = -np.mean(np.log(pr[np.arange(n), labels]))
    dz = pr.copy()
    dz[np.arange(n), labels] -= 1.0
    dz /= n
    g = {"W2": dz.T @ h, "b2": dz.sum(axis=0)}
    dh = dz @ p["W2"]
    da1 = dh * (a1 > 0)
    g["W1"] = da1.T @ x
    g["b1"] = da1.sum(axis=0)
    return loss, g


def propose(p, x, halfwin=-1):
    """(bin, confidence) per row; see the module docstring."""
    z, _ = forward(p, x)
    pr = softmax(z)
    b = np.argmax(z, axis=1)
    if halfwin < 0:
        return b, pr[np.arange(z.shape[0]), b]
    conf = np.array([pr[i, max(0, bi - halfwin):bi + halfwin + 1].sum() for i, bi in enumerate(b)])
    return b, conf


def window_centre(bins, nbins, width):
    """Fine-grid centre index of each window (see the module docstring)."""
    lo, hi = width // 2, 2 * (nbins - 1) - width // 2 + 1
    return np.clip(2 * np.asarray(bins, dtype=np.int64), lo, hi)


def fine_phi(phi, n):
    """phi_0 + n D / 2 for a uniform grid phi."""
    phi = np.asarray(phi, dtype=np.float64)
    d = (phi[-1] - phi[0]) / (len(phi) - 1)
    return phi[0] + np.asarray(n, dtype=np.float64) * (d / 2)


def learned_peaks(oracle_mod, lam2, w, phi, params, Q, U, tau, width, halfwin):
    """The learned peak map on the CPU: (phi_peak, |F|_peak, fell_back) per LOS.

    lam2, w: channel lambda^2 (m^2) and weights; phi: the uniform full grid;
    Q, U LOS-major [nlos][nchan].
    """
    act = np.nonzero(np.asarray(w) > 0)[0]
    nb = len(phi)
    x = normalise(Q, U, act)
    b, conf = propose(params, x, halfwin)
    c = window_centre(b, nb, width)
    plan = oracle_mod.plan(lam2, "lambda2", w)
    full_idx, full_abs = oracle_mod.peak(oracle_mod.synth(Q, U, plan, phi))
    out_phi = np.empty(len(b))
    out_abs = np.empty(len(b))
    fell = np.zeros(len(b), dtype=bool)
    for i in range(len(b)):
        wphi = fine_phi(phi, c[i] - width // 2 + np.arange(width))
        k, a = oracle_mod.peak(oracle_mod.synth(Q[i:i + 1], U[i:i + 1], plan, wphi))
        k, a = int(k[0]), float(a[0])
        if not (conf[i] >= tau) or k <= 0 or k == width - 1:
            fell[i] = True
            kk = int(full_idx[i])
            out_phi[i] = phi[kk] if kk >= 0 else np.nan
            out_abs[i] = full_abs[i] if kk >= 0 else np.nan
        else:
            out_phi[i] = wphi[k]
            out_abs[i] = a
    return out_phi, out_abs, fell
