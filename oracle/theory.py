"""Closed forms of arXiv 2305.13419, Sec. 4, plus the discrete dispersion
relation of Algorithm 1 -- plain numpy, FP64/complex128.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 8.8541878128e-12


def _inv_lam2(lam):
    lam = np.asarray(lam, np.float64)
    with np.errstate(divide="ignore"):
        return np.where((lam > 0) & np.isfinite(lam), 1.0 / np.where(lam > 0, lam, 1.0) ** 2, 0.0)


def wavenumber(omega, eps_r=1.0, mu_r=1.0, sigma=0.0, lam=0.0):
    """Eq. nk: k = sqrt((mu eps omega^2 - 1/lambda^2) + i mu sigma omega),
    the root with non-negative imaginary part (a wave decaying along +z)."""
    mu, eps = MU0 * mu_r, EPS0 * eps_r
    k2 = (mu * eps * omega ** 2 - _inv_lam2(lam)) + 1j * mu * sigma * omega
    k = np.sqrt(k2 + 0j)
    return np.where(np.imag(k) < 0, -k, k)


def gamma_kappa(omega, eps_r=1.0, mu_r=1.0, sigma=0.0, lam=0.0):
    """Eqs. ngamma and nkappa written out: real and imaginary parts of k."""
    mu, eps = MU0 * mu_r, EPS0 * eps_r
    a = mu * eps * np.asarray(omega, np.float64) ** 2 - _inv_lam2(lam)
    b = mu * sigma * np.asarray(omega, np.float64)
    r = np.sqrt(a * a + b * b)
    return np.sqrt((r + a) / 2.0), np.sqrt((r - a) / 2.0)


def skin_depth(omega, eps_r=1.0, mu_r=1.0, sigma=0.0, lam=0.0):
    """Eq. skin: delta = 1 / kappa (inf for a lossless non-superconductor)."""
    _, kap = gamma_kappa(omega, eps_r, mu_r, sigma, lam)
    with np.errstate(divide="ignore"):
        return np.where(kap > 0, 1.0 / np.where(kap > 0, kap, 1.0), np.inf)


def beta(omega, eps1=1.0, mu1=1.0, eps2=1.0, mu2=1.0, sigma2=0.0, lam2=0.0):
    """Eq. beta: beta = sqrt(mu1/eps1) k2 / (mu2 omega)."""
    k2 = wavenumber(omega, eps2, mu2, sigma2, lam2)
    return np.sqrt((MU0 * mu1) / (EPS0 * eps1)) * k2 / (MU0 * mu2 * omega)


def reflection_amplitude(omega, **kw):
    """E_{0,R}/E_{0,I} = (1 - beta)/(1 + beta)."""
    b = beta(omega, **kw)
    return (1.0 - b) / (1.0 + b)


def reflection(omega, **kw):
    """Eq. Ref: R = |(1 - beta)/(1 + beta)|^2."""
    return np.abs(reflection_amplitude(omega, **kw)) ** 2


def cutoff_frequency(lam, eps_r=1.0, mu_r=1.0):
    """Below f_c = 1/(2 pi lambda sqrt(mu eps)) a sigma = 0 superconductor reflects fully."""
    return 1.0 / (2.0 * math.pi * lam * math.sqrt(MU0 * mu_r * EPS0 * eps_r))


def dt_courant(courant, d):
    """dt = C / (c sqrt(sum 1/d_a^2)), the convention that reproduces the
    paper's quoted dt values."""
    return courant / (C0 * math.sqrt(sum(1.0 / (x * x) for x in d)))


# ---------------------------------------------------------------------------
# discrete relations of Algorithm 1 (derived from the scheme, Sec. 3)
# ---------------------------------------------------------------------------

def discrete_k2(K, d):
    """Symbol of the Yee curl-curl: sum_a (2/d_a sin(K_a d_a / 2))^2."""
    return sum((2.0 / d[a] * math.sin(K[a] * d[a] / 2.0)) ** 2 for a in range(3))


def discrete_omega(K, d, dt, eps_r=1.0, mu_r=1.0, lam=0.0):
    """Lossless modes of the scheme: mu eps Omega^2 = K_d^2 + 1/lambda^2 with
    Omega = (2/dt) sin(omega dt / 2)."""
    mu, eps = MU0 * mu_r, EPS0 * eps_r
    s = (dt / 2.0) * math.sqrt((discrete_k2(K, d) + float(_inv_lam2(lam))) / (mu * eps))
    if s > 1.0:
        raise ValueError("unstable: |sin(omega dt/2)| > 1")
    return 2.0 / dt * math.asin(s)


def discrete_decay(omega, d, dt, eps_r=1.0, mu_r=1.0, lam=0.0):
    """Evanescent decay per metre of the scheme in a sigma = 0 superconductor
    along one axis: (2/d)^2 sinh^2(kd d/2) = 1/lambda^2 - mu eps Omega^2."""
    mu, eps = MU0 * mu_r, EPS0 * eps_r
    Om = 2.0 / dt * math.sin(omega * dt / 2.0)
    rhs = float(_inv_lam2(lam)) - mu * eps * Om * Om
    if rhs <= 0:
        raise ValueError("propagating, not evanescent")
    return 2.0 / d * math.asinh(d / 2.0 * math.sqrt(rhs))


def uniform_recurrence(theta, s, p):
    """A spatially uniform E (no curl) obeys, by steps 2-4 fused,
    (1 + theta s) E^{n+1} - (2 - (1 - 2 theta) s - p) E^n + (1 - (1 - theta) s) E^{n-1} = 0
    with s = sigma dt/eps and p = kappa dt^2/eps. Returns the two roots."""
    a = 1.0 + theta * s
    b = -(2.0 - (1.0 - 2.0 * theta) * s - p)
    c = 1.0 - (1.0 - theta) * s
    return np.roots([a, b, c])
