"""The Q pipeline of the GPU against two independent references: the exact
pole of a lossy cavity mode of the scheme (closed form), and ESPRIT on the
GPU's own probe time series (the estimator of Sec. 5) against the GPU's FP64
DFT-window fit."""
import math

import numpy as np
import pytest

from oracle import esprit, theory
from paper_2305_13419_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_lossy_cavity_pole_from_gpu_series_and_fit():
    from paper_2305_13419_gb300 import twofluid as tf
    n, d = (6, 5, 7), (10e-9, 11e-9, 9e-9)
    dt = theory.dt_courant(0.9, d)
    theta, sigma, eps_r = 0.5, 3.0e3, 2.0
    g = tf.Grid(n, d, theta=theta, bc=("pec", "pec", "pec"), dt=dt, series_capacity=1200)
    g.set_materials(eps_r, 1.0, 0.0, sigma)
    Nz, Ny, Nx = g.shape
    k_, j_, i_ = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    L = [n[a] * d[a] for a in range(3)]
    g.set_field(1, (np.sin(math.pi * i_ * d[0] / L[0]) * np.sin(math.pi * k_ * d[2] / L[2])).astype(np.float32))
    K = (math.pi / L[0], 0.0, math.pi / L[2])
    eps = theory.EPS0 * eps_r
    roots = theory.uniform_recurrence(theta, sigma * dt / eps, dt * dt * theory.discrete_k2(K, d) / (theory.MU0 * eps))
    z = [r for r in roots if complex(r).imag > 0][0]
    f_exact = math.atan2(z.imag, z.real) / dt / (2 * math.pi)
    al_exact = -math.log(abs(z)) / dt
    q_exact = math.pi * f_exact / al_exact
    N = 1200
    fr = np.linspace(0.8 * f_exact, 1.2 * f_exact, 64)
    g.add_probe(1, (3, 2, 3), fr, 0)
    g.step(N)
    g.sync()
    s = g.probe_series(0, N)
    m = esprit.mode_near(s, dt, f_exact, order=2)
    assert abs(m["f"] / f_exact - 1) < 1e-6
    assert abs(m["Q"] / q_exact - 1) < 1e-3
    r = g.fit_q(0, f_guess=f_exact, q_guess=q_exact)
    assert abs(r["f0"] / f_exact - 1) < 1e-6
    assert abs(r["Q"] / q_exact - 1) < 1e-3


def test_two_cavity_modes_from_the_gpu_series():
    """Two Ey modes, (1, 0, 1) and (1, 0, 2), ring down together in a lossy
    PEC box; ESPRIT on the GPU series separates both exact poles."""
    from paper_2305_13419_gb300 import twofluid as tf
    n, d = (6, 5, 7), (10e-9, 11e-9, 9e-9)
    dt = theory.dt_courant(0.9, d)
    theta, sigma, eps_r = 1.0, 2.0e3, 1.5
    g = tf.Grid(n, d, theta=theta, bc=("pec", "pec", "pec"), dt=dt, series_capacity=1600)
    g.set_materials(eps_r, 1.0, 0.0, sigma)
    Nz, Ny, Nx = g.shape
    k_, j_, i_ = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    L = [n[a] * d[a] for a in range(3)]
    sx = np.sin(math.pi * i_ * d[0] / L[0])
    g.set_field(1, (sx * (np.sin(math.pi * k_ * d[2] / L[2]) + 0.6 * np.sin(2 * math.pi * k_ * d[2] / L[2])))
                .astype(np.float32))
    eps = theory.EPS0 * eps_r
    exact = []
    for mz in (1, 2):
        K = (math.pi / L[0], 0.0, mz * math.pi / L[2])
        roots = theory.uniform_recurrence(theta, sigma * dt / eps,
                                          dt * dt * theory.discrete_k2(K, d) / (theory.MU0 * eps))
        z = [r for r in roots if complex(r).imag > 0][0]
        exact.append((math.atan2(z.imag, z.real) / dt / (2 * math.pi), -math.log(abs(z)) / dt))
    fr = np.linspace(0.5 * exact[0][0], 1.5 * exact[1][0], 64)
    g.add_probe(1, (3, 2, 2), fr, 0)
    g.step(1600)
    g.sync()
    s = g.probe_series(0, 1600)
    for f, al in exact:
        m = esprit.mode_near(s, dt, f, order=4)
        assert abs(m["f"] / f - 1) < 1e-5
        assert abs(m["alpha"] / al - 1) < 2e-3
