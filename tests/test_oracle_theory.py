"""Pins of the oracle's closed-form theory (Sec. 4 of arXiv 2305.13419)
against the numbers the paper prints.  CPU only."""
import math

import numpy as np
import pytest

from conftest import read_table
from oracle import theory


def _f(x):
    return math.inf if x == "inf" else float(x)


@pytest.mark.parametrize("row", read_table("table1_skin_depth.txt"))
def test_table1_theory_columns(row):
    """Eqs. nk / nkappa / skin reproduce Table 1's theory columns to the
    printed precision (3 significant figures, +-1 in the last digit)."""
    sigma, f, cond, sc, computed, f_th = map(_f, row)
    w = 2 * math.pi * f_th
    lam = 400e-9
    d_cond = float(theory.skin_depth(w, sigma=sigma, lam=0.0)) * 1e9
    d_sc = float(theory.skin_depth(w, sigma=sigma, lam=lam)) * 1e9
    if math.isinf(cond):
        assert math.isinf(d_cond)
    else:
        assert abs(d_cond - cond) <= max(1.0, 2e-3 * cond), (d_cond, cond)
    assert abs(d_sc - sc) <= max(1.0, 2e-3 * sc), (d_sc, sc)


def test_table1_garbled_row_reading():
    """The sigma = 1e7 "25 GHz" row: the computed 395 nm matches the formula
    at 25 GHz (395.2 nm) while the printed theory 399 nm is the 10 GHz value."""
    d25 = float(theory.skin_depth(2 * math.pi * 25e9, sigma=1e7, lam=400e-9)) * 1e9
    d10 = float(theory.skin_depth(2 * math.pi * 10e9, sigma=1e7, lam=400e-9)) * 1e9
    assert abs(d25 - 395.2) < 0.2
    assert round(d10) == 399


def test_skin_depth_limits():
    """Sec. 4.1: omega -> 0 gives delta -> lambda; 1/lambda^2 = 0 gives the
    conductor skin depth sqrt(2/(mu sigma omega)) in the good-conductor limit."""
    lam = 123e-9
    for s in (0.0, 1e4, 1e7):
        assert abs(float(theory.skin_depth(2 * math.pi * 1e3, sigma=s, lam=lam)) / lam - 1) < 1e-6
    w = 2 * math.pi * 1e9
    good = math.sqrt(2 / (theory.MU0 * 5.8e7 * w))
    assert abs(float(theory.skin_depth(w, sigma=5.8e7)) / good - 1) < 1e-6


def test_gamma_kappa_consistent_with_complex_root():
    w = 2 * math.pi * np.logspace(9, 15, 25)
    for s, lam in ((0.0, 100e-9), (1e4, 400e-9), (1e7, 50e-9), (1e5, 0.0)):
        k = theory.wavenumber(w, sigma=s, lam=lam)
        g, kap = theory.gamma_kappa(w, sigma=s, lam=lam)
        assert np.allclose(k.real, g, rtol=1e-12, atol=1e-12 * np.abs(k).max())
        assert np.allclose(k.imag, kap, rtol=1e-12, atol=1e-12 * np.abs(k).max())


def test_cutoff_frequency():
    """Sec. 4.2: f_c = 1/(2 pi lambda sqrt(eps mu)); the paper quotes 478.75 THz
    for lambda = 100 nm, the formula gives 477.1 THz (0.35 % apart)."""
    fc = theory.cutoff_frequency(100e-9)
    assert abs(fc - 477.1e12) < 0.1e12
    assert abs(fc / 478.75e12 - 1) < 5e-3


def test_reflection_sigma0_total_below_cutoff():
    """Eq. beta_cases: sigma = 0 gives R = 1 below f_c and R < 1 above it."""
    lam = 100e-9
    fc = theory.cutoff_frequency(lam)
    below = 2 * math.pi * np.linspace(0.01, 0.999, 50) * fc
    above = 2 * math.pi * np.linspace(1.01, 3.0, 50) * fc
    assert np.allclose(theory.reflection(below, lam2=lam), 1.0, atol=1e-12)
    assert np.all(theory.reflection(above, lam2=lam) < 1.0)
    # finite sigma: R < 1 everywhere, -> 1 at low frequency
    r = theory.reflection(2 * math.pi * np.logspace(10, 16, 40), sigma2=1e4, lam2=lam)
    assert np.all(r < 1.0) and r[0] > 0.999


def test_reflection_vacuum_and_dielectric():
    """beta = 1 for identical media (R = 0); normal-incidence dielectric
    R = ((1-n)/(1+n))^2."""
    w = 2 * math.pi * 1e12
    assert float(theory.reflection(w)) < 1e-30
    n = math.sqrt(11.7)
    assert abs(float(theory.reflection(w, eps2=11.7)) - ((1 - n) / (1 + n)) ** 2) < 1e-12


@pytest.mark.parametrize("row", read_table("paper_time_steps.txt"))
def test_paper_time_steps(row):
    """The Courant convention dt = C/(c sqrt(sum 1/d^2)) reproduces every dt
    the paper quotes."""
    where, dims, C, dx, dy, dz, dt_q, tol = row
    C, dx, dy, dz, dt_q, tol = map(float, (C, dx, dy, dz, dt_q, tol))
    d = (dz,) if dims == "1d" else (dx, dy, dz)
    assert abs(theory.dt_courant(C, d) / dt_q - 1) < tol, where
