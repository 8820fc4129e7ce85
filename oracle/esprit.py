"""Damped-mode parameters from a probe time series by ESPRIT -- FP64 numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 5 of the paper extracts the attenuation and phase constants of the
resonator's ring-down with ESPRIT (estimation of signal parameters via
rotational invariance, Roy & Kailath).  Written here from that method's
definition:

* a series s^n = sum_m a_m z_m^n (n = 0 .. N-1) fills an L x M Hankel matrix
  H[i, j] = s^{i+j} (M = N - L + 1); its column space is spanned by the
  Vandermonde vectors (1, z_m, ..., z_m^{L-1}) of the poles;
* the `order` leading left singular vectors U_s span that space; the rows
  1..L-1 of a Vandermonde vector are z_m times rows 0..L-2 (the rotational
  invariance), so Phi = pinv(U_s[:-1]) U_s[1:] has the poles z_m as its
  eigenvalues;
* a pole z = exp((-alpha + i omega) dt) gives f = omega / 2 pi and the
  quality factor Q = omega / (2 alpha).

It serves as an estimator independent of the DFT-window fit in qfit.py: both
must agree on the same ring-down.
"""
from __future__ import annotations

import math

import numpy as np


def poles(s, order, L=None):
    """The `order` poles of the exponentials in series s (complex array)."""
    s = np.asarray(s)
    N = s.size
    if L is None:
        L = N // 2
    if not (order < L <= N - order):
        raise ValueError("series too short for the requested order")
    M = N - L + 1
    idx = np.arange(L)[:, None] + np.arange(M)[None, :]
    H = s[idx]
    U, _, _ = np.linalg.svd(H, full_matrices=False)
    Us = U[:, :order]
    Phi = np.linalg.pinv(Us[:-1]) @ Us[1:]
    return np.linalg.eigvals(Phi)


def modes(s, dt, order, L=None):
    """Damped modes of a real series: list of dicts (f, alpha, Q, |z|), one per
    pole with positive frequency, strongest (least damped first)."""
    z = poles(np.asarray(s, np.float64), order, L)
    out = []
    for p in z:
        w = math.atan2(p.imag, p.real) / dt
        if w <= 0:
            continue
        alpha = -math.log(abs(p)) / dt
        out.append({"f": w / (2 * math.pi), "alpha": alpha, "Q": w / (2 * alpha) if alpha > 0 else math.inf,
                    "z": p})
    out.sort(key=lambda m: m["alpha"])
    return out


def mode_near(s, dt, f_target, order, L=None):
    """The mode whose frequency is closest to f_target."""
    ms = modes(s, dt, order, L)
    if not ms:
        raise ValueError("no oscillating mode found")
    return min(ms, key=lambda m: abs(m["f"] - f_target))
