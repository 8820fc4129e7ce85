"""Discrete adjoint of Algorithm 1 in the oracle (oracle/twofluid_oracle.c):
every sub-step's transpose against the sub-step itself (dot-product test),
and the adjoint gradient of a probe-DFT objective against central finite
differences of the forward scheme."""
import numpy as np
import pytest

from oracle import stepper
from paper_2305_13419_gb300 import workloads as W


def _box(theta):
    w = W.random_box(n=(11, 9, 13), bc=("cpml", "cpml", "cpml"), seed=31, cpml_cells=3, theta=theta,
                     mu_range=(1.0, 1.8), sigma_range=(0.0, 4e5))
    return stepper.Grid.from_workload(w)


@pytest.mark.parametrize("theta", [0.5, 1.0])
@pytest.mark.parametrize("op", [1, 2, 3, 4, 5])
def test_substep_transposes(op, theta):
    g = _box(theta)
    for seed in (1, 2):
        l, r = g.adjoint_dot_test(op, seed)
        assert abs(l - r) <= 1e-13 * max(abs(l), abs(r)), (l, r)


def test_periodic_and_pec_transposes():
    for bc in (("periodic", "pec", "periodic"), ("pec", "periodic", "pec")):
        w = W.random_box(n=(7, 8, 6), bc=bc, seed=5, theta=0.5, mu_range=(1.0, 2.0))
        g = stepper.Grid.from_workload(w)
        for op in range(1, 6):
            l, r = g.adjoint_dot_test(op, 9)
            assert abs(l - r) <= 1e-13 * max(abs(l), abs(r)), (bc, op, l, r)


def _cpw_like(eps_sub, lam_film):
    """A scaled CPW-like box: CPML on all faces, random substrate eps_r, a
    superconducting Ohmic film, a soft source above it and a probe."""
    n = (20, 14, 16)
    w = W.random_box(n=n, bc=("cpml", "cpml", "cpml"), seed=77, cpml_cells=3, theta=1.0,
                     sc_fraction=0.0, sigma_range=(0.0, 0.0), eps_range=(1.0, 1.0), mu_range=(1.0, 1.0))
    for name in ("eps_r", "mu_r", "lambda_L", "sigma"):   # FP64 maps: the differences are taken in FP64
        setattr(w, name, np.asarray(getattr(w, name), np.float64).copy())
    w.eps_r[:7] = eps_sub
    w.lambda_L[7:9] = lam_film
    rng = np.random.default_rng(2305_13419 + 4)
    w.sigma[7:9] = rng.uniform(0.0, 1e6, size=w.sigma[7:9].shape)
    f = 6e13
    w.sources = [W.Source(comp=1, lo=(6, 5, 9), hi=(8, 8, 10), amp=1.0e3, kind=W.SRC_GAUSS_SIN, f=f,
                          t0=4 / (2 * f), tw=1 / (2 * f))]
    w.probes = []
    return w, f


def _J(w, nsteps, f):
    g = stepper.Grid.from_workload(w)
    J, ge, gl = g.adjoint_run(nsteps, 1, (12, 7, 8), f, 20)
    return J, ge, gl


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2305_13419 + 40)
    eps_sub = rng.uniform(10.0, 13.0, size=(7, 14, 20))
    lam_film = rng.uniform(2.0, 6.0, size=(2, 14, 20)) * 12e-9
    w, f = _cpw_like(eps_sub, lam_film)
    # cells with lambda well above the stable limit for this grid's dt
    nsteps = 160
    J0, ge, gl = _J(w, nsteps, f)
    assert J0 > 0
    cells = [(int(rng.integers(0, 7)), int(rng.integers(3, 11)), int(rng.integers(3, 17))) for _ in range(8)]
    film = [(int(rng.integers(7, 9)), int(rng.integers(3, 11)), int(rng.integers(3, 17))) for _ in range(8)]
    big_e = np.max(np.abs(ge))
    big_l = np.max(np.abs(gl))
    checked = 0
    for c in cells:
        h = 1e-4 * w.eps_r[c]
        w.eps_r[c] += h
        Jp = _J(w, nsteps, f)[0]
        w.eps_r[c] -= 2 * h
        Jm = _J(w, nsteps, f)[0]
        w.eps_r[c] += h
        fd = (Jp - Jm) / (2 * h)
        if abs(ge[c]) >= 1e-3 * big_e:
            assert abs(fd / ge[c] - 1) < 1e-5, (c, fd, ge[c])
            checked += 1
        else:
            assert abs(fd - ge[c]) < 1e-5 * big_e
    for c in film:
        h = 1e-4 * w.lambda_L[c]
        w.lambda_L[c] += h
        Jp = _J(w, nsteps, f)[0]
        w.lambda_L[c] -= 2 * h
        Jm = _J(w, nsteps, f)[0]
        w.lambda_L[c] += h
        fd = (Jp - Jm) / (2 * h)
        if abs(gl[c]) >= 1e-3 * big_l:
            assert abs(fd / gl[c] - 1) < 1e-5, (c, fd, gl[c])
            checked += 1
        else:
            assert abs(fd - gl[c]) < 1e-5 * big_l
    assert checked >= 8
