"""ESPRIT (oracle/esprit.py), the time-series estimator Sec. 5 uses for the
ring-down, pinned on closed forms and cross-checked against the DFT-window
fit of oracle/qfit.py."""
import math

import numpy as np

from oracle import esprit, qfit, stepper, theory


def _damped(n, dt, modes):
    t = np.arange(n) * dt
    return sum(a * np.exp(-al * t) * np.cos(2 * math.pi * f * t + ph) for a, f, al, ph in modes)


def test_single_mode_recovered_exactly():
    dt, f, al = 1e-15, 3.1e13, 2.2e11
    s = _damped(1500, dt, [(1.7, f, al, 0.4)])
    m = esprit.mode_near(s, dt, f, order=2)
    assert abs(m["f"] / f - 1) < 1e-10
    assert abs(m["alpha"] / al - 1) < 1e-7
    assert abs(m["Q"] / (math.pi * f / al) - 1) < 1e-7


def test_two_modes_separated():
    dt = 1e-15
    modes = [(1.0, 2.0e13, 1e11, 0.0), (0.4, 5.5e13, 6e11, 1.3)]
    s = _damped(2000, dt, modes)
    got = esprit.modes(s, dt, order=4)
    assert len(got) == 2
    for (a, f, al, ph), m in zip(modes, got):    # sorted least damped first
        assert abs(m["f"] / f - 1) < 1e-9 and abs(m["alpha"] / al - 1) < 1e-6


def test_noise_tolerance():
    rng = np.random.default_rng(2305_13419)
    dt, f, al = 1e-15, 4e13, 3e11
    s = _damped(3000, dt, [(1.0, f, al, 0.2)]) + 1e-6 * rng.standard_normal(3000)
    m = esprit.mode_near(s, dt, f, order=2)
    assert abs(m["Q"] / (math.pi * f / al) - 1) < 1e-3


def test_dft_window_fit_and_esprit_agree_on_a_synthetic_ring_down():
    dt, f, al, n0, N = 1e-15, 3e13, 4e11, 300, 2400
    s = _damped(N, dt, [(1.0, f, al, 0.7)])
    fr = np.linspace(0.9 * f, 1.1 * f, 64)
    X = qfit.dft_of_series(s, fr, dt, n0)
    r = qfit.fit(X, fr, dt, n0, N)
    m = esprit.mode_near(s[n0:], dt, f, order=2)
    assert abs(r["Q"] / m["Q"] - 1) < 1e-8 and abs(r["f0"] / m["f"] - 1) < 1e-10


def test_lossy_cavity_mode_of_the_scheme():
    """A PEC box filled with a uniform Ohmic medium: the (1, 0, 1) Ey mode
    obeys the scalar recurrence of Algorithm 1 with p = dt^2 K_d^2 / (mu eps)
    and s = sigma dt / eps, so its pole is a root of
    (1 + theta s) z^2 - (2 - (1 - 2 theta) s - p) z + (1 - (1 - theta) s) = 0.
    ESPRIT on the oracle's probe series recovers that root, and the DFT fit of
    the oracle's own running DFT gives the same Q."""
    n, d = (6, 5, 7), (10e-9, 11e-9, 9e-9)
    dt = theory.dt_courant(0.9, d)
    theta, sigma, eps_r = 0.5, 3.0e3, 2.0
    g = stepper.Grid(n, d, dt, theta=theta, bc=("pec", "pec", "pec"))
    g.set_materials(eps_r, 1.0, 0.0, sigma)
    k_, j_, i_ = np.meshgrid(np.arange(g.N[2]), np.arange(g.N[1]), np.arange(g.N[0]), indexing="ij")
    L = [n[a] * d[a] for a in range(3)]
    g.set_field(1, np.sin(math.pi * i_ * d[0] / L[0]) * np.sin(math.pi * k_ * d[2] / L[2]))
    K = (math.pi / L[0], 0.0, math.pi / L[2])
    eps = theory.EPS0 * eps_r
    s_ = sigma * dt / eps
    p = dt * dt * theory.discrete_k2(K, d) / (theory.MU0 * eps)
    roots = theory.uniform_recurrence(theta, s_, p)
    z = [r for r in roots if complex(r).imag > 0][0]
    f_exact = math.atan2(z.imag, z.real) / dt / (2 * math.pi)
    al_exact = -math.log(abs(z)) / dt
    n0, N = 0, 1200
    fr = np.linspace(0.8 * f_exact, 1.2 * f_exact, 64)
    pid = g.add_probe(1, (3, 2, 3), fr, n0=n0, series=N)
    g.step(N)
    s = g.probe_series(pid, N)
    m = esprit.mode_near(s, dt, f_exact, order=2)
    assert abs(m["f"] / f_exact - 1) < 1e-9
    assert abs(m["alpha"] / al_exact - 1) < 1e-6
    r = qfit.fit(g.probe_dft(pid), fr, dt, n0, N, f_guess=f_exact, q_guess=m["Q"])
    assert abs(r["Q"] / m["Q"] - 1) < 1e-6
