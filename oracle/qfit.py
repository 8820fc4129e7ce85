"""Q-factor from a windowed probe DFT -- FP64 numpy/scipy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper extracts attenuation and phase constants of the ring-down with
ESPRIT (Sec. 5) and reports Q.  Here the probe keeps a running DFT
    X_k = dt * sum_{n=n0}^{N-1} s^n w_k^n,   w_k = exp(-i 2 pi f_k dt),
and the ring-down is modelled as one damped mode s^n = a z^n + conj(a) conj(z)^n
with z = exp((-alpha + i omega0) dt).  Each term is a geometric series:
    sum_{n=n0}^{N-1} q^n = (q^{n0} - q^N) / (1 - q),
so the model DFT is exact for any window length.  For fixed (alpha, omega0)
the model is linear in (Re a, Im a); those are solved by least squares and
(alpha, omega0) by Levenberg-Marquardt.  Q = omega0 / (2 alpha).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import least_squares


def geometric_window(q, n0, N):
    q = np.asarray(q, np.complex128)
    return (q ** n0 - q ** N) / (1.0 - q)


def model_basis(alpha, omega0, freqs, dt, n0, N):
    """Columns: DFT of Re-part and Im-part unit amplitudes of a z^n + c.c."""
    z = np.exp((-alpha + 1j * omega0) * dt)
    w = np.exp(-2j * np.pi * np.asarray(freqs) * dt)
    g1 = geometric_window(z * w, n0, N) * dt
    g2 = geometric_window(np.conj(z) * w, n0, N) * dt
    # s = a z^n + conj(a) zbar^n with a = ar + i ai
    return np.stack([g1 + g2, 1j * (g1 - g2)], axis=1)


def _solve_amp(A, X):
    M = np.concatenate([A.real, A.imag], axis=0)
    y = np.concatenate([X.real, X.imag])
    coef, *_ = np.linalg.lstsq(M, y, rcond=None)
    return coef, M @ coef - y


def fit(X, freqs, dt, n0, N, f_guess=None, q_guess=100.0):
    """Fit one damped mode to DFT samples X at `freqs`. Returns dict with
    f0 (Hz), alpha (1/s), Q, amplitude and the relative residual."""
    X = np.asarray(X, np.complex128)
    freqs = np.asarray(freqs, np.float64)
    if f_guess is None:
        f_guess = freqs[int(np.argmax(np.abs(X)))]
    w0 = 2 * math.pi * f_guess
    a0 = w0 / (2 * q_guess)
    scale_w = w0

    def res(p):
        alpha, omega = p[0] * scale_w, p[1] * scale_w
        _, r = _solve_amp(model_basis(alpha, omega, freqs, dt, n0, N), X)
        return r / np.linalg.norm(X)

    sol = least_squares(res, x0=[a0 / scale_w, w0 / scale_w], method="lm", xtol=1e-15,
                        ftol=1e-15, gtol=1e-15, max_nfev=2000)
    alpha, omega = sol.x[0] * scale_w, sol.x[1] * scale_w
    coef, r = _solve_amp(model_basis(alpha, omega, freqs, dt, n0, N), X)
    return {"f0": omega / (2 * math.pi), "alpha": alpha, "Q": omega / (2 * alpha),
            "amp": coef[0] + 1j * coef[1], "residual": float(np.linalg.norm(r) / np.linalg.norm(X))}


def dft_of_series(s, freqs, dt, n0):
    """Direct FP64 DFT of a recorded series (window [n0, len(s)))."""
    n = np.arange(n0, len(s), dtype=np.float64)
    ph = np.outer(np.asarray(freqs, np.float64) * dt, n)
    ph -= np.floor(ph)
    return (np.exp(-2j * np.pi * ph) * np.asarray(s[n0:])[None, :]).sum(axis=1) * dt
