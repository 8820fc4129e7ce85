"""The oracle against the physics the paper validates (arXiv 2305.13419,
Sec. 4): decay inside the superconductor, the two-fluid reflection
coefficient, and the convergence orders of Tables 2-5.  CPU only."""
import itertools
import math

import numpy as np
import pytest

from conftest import read_table
from oracle import qfit, stepper, theory
from paper_2305_13419_gb300 import workloads as W

C0 = stepper.C0
L_PULSE = 80e-9
RATES = {(r[1], r[2], r[3]): float(r[4]) for r in read_table("convergence_rates.txt")}


# ----------------------------------------------------------- helpers (A10)
def _restrict_E(F, c):
    """Coarse E edge = mean of its two collinear fine edges (refined axes only)."""
    def sl(off):
        s = [slice(None)] * 3
        for a in range(3):
            if F.shape[2 - a] > 1:
                s[2 - a] = slice(0, None, 2)
        if F.shape[2 - c] > 1:
            s[2 - c] = slice(off, None, 2)
        return F[tuple(s)]
    return sl(0) if F.shape[2 - c] == 1 else 0.5 * (sl(0) + sl(1))


def _restrict_B(F, c):
    """Coarse B face = mean of the fine faces covering it (refined axes only)."""
    axes = [a for a in range(3) if a != c and F.shape[2 - a] > 1]
    acc, cnt = 0.0, 0
    for offs in itertools.product((0, 1), repeat=len(axes)):
        s = [slice(None)] * 3
        for a in range(3):
            if F.shape[2 - a] > 1:
                s[2 - a] = slice(0, None, 2)
        for a, o in zip(axes, offs):
            s[2 - a] = slice(o, None, 2)
        acc = acc + F[tuple(s)]
        cnt += 1
    return acc / cnt


def _run(n, half, steps, courant, mat_fn, init, one_d=False, edge_rule=0):
    """Periodic cube [-half, half]^3 (or a 1 x 1 x n column), theta = 1/2,
    dt = C d / (c sqrt 3) as in the paper's 3-D convergence runs."""
    shape = (1, 1, n) if one_d else (n, n, n)
    d = 2 * half / n
    g = stepper.Grid(shape, (d, d, d), courant * d / (C0 * math.sqrt(3)), theta=0.5,
                     edge_rule=edge_rule)
    cen = [-half + (np.arange(shape[a]) + 0.5) * d for a in range(3)]
    Z, Y, X = np.meshgrid(cen[2], cen[1], cen[0], indexing="ij")
    lam, sig = mat_fn(X, Y, Z)
    g.set_materials(1.0, 1.0, lam, sig)
    nod = [-half + np.arange(g.N[a]) * d for a in range(3)]
    Z, Y, X = np.meshgrid(nod[2], nod[1], nod[0], indexing="ij")
    for c, f in init(X, Y, Z, 0.5 * d):
        g.set_field(c, f)
    g.step(steps)
    return g


def _gauss(u, u0=0.0):
    return np.exp(-((u - u0) ** 2) / L_PULSE ** 2)


def _three_pulses(X, Y, Z, h):
    """Sec. 4.3.1: Ex = e^{-z^2/L^2}, Ey = e^{-x^2/L^2}, Ez = e^{-y^2/L^2},
    Bx = e^{-y^2/L^2}/c, By = e^{-z^2/L^2}/c, Bz = e^{-x^2/L^2}/c, each at its
    own staggered position."""
    return [(0, _gauss(Z)), (1, _gauss(X)), (2, _gauss(Y)),
            (3, _gauss(Y + h) / C0), (4, _gauss(Z + h) / C0), (5, _gauss(X + h) / C0)]


def _one_pulse(z0):
    """Sec. 4.3.2: Ex = e^{-(z-z0)^2/L^2}, By = Ex/c (integer-level B of a +z wave)."""
    def init(X, Y, Z, h):
        return [(0, _gauss(Z, z0)), (4, 0.5 * (_gauss(Z, z0) + _gauss(Z + 2 * h, z0)) / C0)]
    return init


def _case_d(mask_fn):
    """Case (d): lambda = 40 nm and sigma = 1e4 S/m inside the material."""
    def mat(X, Y, Z):
        m = mask_fn(X, Y, Z)
        return np.where(m, 40e-9, 0.0), np.where(m, 1e4, 0.0)
    return mat


def _space_err(gc, gm, c):
    a, b = gc.field(c), gm.field(c)
    r = _restrict_E(b, c) if c < 3 else _restrict_B(b, c - 3)
    return float(np.mean(np.abs(a - r)))


def _time_err(ga, gb, c):
    return float(np.mean(np.abs(ga.field(c) - gb.field(c))))


# ------------------------------------------------------ convergence (Tables)
@pytest.mark.slow
def test_homogeneous_space_time_second_order():
    """Table 2: case (d) everywhere, three orthogonal pulses; grids 32^3, 64^3,
    128^3 over [-320, 320] nm to the same time (CFL 0.9) -> rate 2."""
    mat = _case_d(lambda X, Y, Z: np.ones_like(X, bool))
    gs = [_run(n, 320e-9, st, 0.9, mat, _three_pulses) for n, st in ((32, 25), (64, 50), (128, 100))]
    for c, fam in ((0, "E"), (1, "E"), (2, "E"), (3, "B"), (4, "B"), (5, "B")):
        rate = math.log2(_space_err(gs[0], gs[1], c) / _space_err(gs[1], gs[2], c))
        assert abs(rate - RATES[("homogeneous", "space+time", fam)]) < 0.1, (c, rate)


STRIP = _case_d(lambda X, Y, Z: np.abs(Z) < 40e-9)


def test_strip_time_second_order():
    """Table 3: strip -40..40 nm, 256 cells, CFL 0.9 / 0.45 / 0.225 to 1.73 fs -> rate 2."""
    gs = [_run(256, 640e-9, st, cfl, STRIP, _one_pulse(-320e-9), one_d=True)
          for cfl, st in ((0.9, 200), (0.45, 400), (0.225, 800))]
    for c, name in ((0, "Ex"), (4, "By")):
        rate = math.log2(_time_err(gs[0], gs[1], c) / _time_err(gs[1], gs[2], c))
        assert abs(rate - RATES[("strip", "time", name)]) < 0.1, (name, rate)


def test_strip_space_first_order():
    """Table 4: sharp sigma and 1/lambda jumps make the scheme first order in
    space (paper: 0.90 / 0.88).  128 / 256 / 512 cells at one dt, 400 steps.
    The interface-edge reading (edges on the interface carry the full
    superconductor value) reproduces the printed rates; the plain four-cell
    mean would give second order instead."""
    gs = [_run(n, 640e-9, 400, cfl, STRIP, _one_pulse(-320e-9), one_d=True)
          for n, cfl in ((128, 0.225), (256, 0.45), (512, 0.9))]
    for c, name in ((0, "Ex"), (4, "By")):
        rate = math.log2(_space_err(gs[0], gs[1], c) / _space_err(gs[1], gs[2], c))
        assert abs(rate - RATES[("strip", "space", name)]) < 0.1, (name, rate)
    gp = [_run(n, 640e-9, 400, cfl, STRIP, _one_pulse(-320e-9), one_d=True, edge_rule=1)
          for n, cfl in ((128, 0.225), (256, 0.45), (512, 0.9))]
    rate_mean = math.log2(_space_err(gp[0], gp[1], 0) / _space_err(gp[1], gp[2], 0))
    assert rate_mean > 1.8


def test_smooth_lambda_second_order():
    """Sec. 4.3.2 (closing remark): sigma = 0 and 1/lambda rising smoothly from
    0 at z = 0 to 1/(40 nm) at the right end keeps second order in space."""
    def mat(X, Y, Z):
        u = np.clip(Z / 640e-9, 0.0, 1.0)
        inv = (3 * u ** 2 - 2 * u ** 3) / 40e-9
        return np.where(inv > 0, 1.0 / np.where(inv > 0, inv, 1.0), 0.0), np.zeros_like(Z)
    gs = [_run(n, 640e-9, 400, cfl, mat, _one_pulse(-320e-9), one_d=True)
          for n, cfl in ((128, 0.225), (256, 0.45), (512, 0.9))]
    for c in (0, 4):
        rate = math.log2(_space_err(gs[0], gs[1], c) / _space_err(gs[1], gs[2], c))
        assert abs(rate - 2.0) < 0.1, (c, rate)


@pytest.mark.slow
def test_cube_time_second_order():
    """Table 5: superconducting cube (case d) -40..40 nm, 64^3 over
    [-640, 640] nm, CFL 0.9 / 0.45 / 0.225 to the same time -> rate 2."""
    cube = _case_d(lambda X, Y, Z: (np.abs(X) < 40e-9) & (np.abs(Y) < 40e-9) & (np.abs(Z) < 40e-9))
    gs = [_run(64, 640e-9, st, cfl, cube, _one_pulse(-320e-9)) for cfl, st in ((0.9, 50), (0.45, 100), (0.225, 200))]
    for c, name in ((0, "Ex"), (4, "By")):
        rate = math.log2(_time_err(gs[0], gs[1], c) / _time_err(gs[1], gs[2], c))
        assert abs(rate - RATES[("cube", "time", name)]) < 0.1, (name, rate)
    for c in (1, 2, 3, 5):   # the field develops every component, all second order in time
        rate = math.log2(_time_err(gs[0], gs[1], c) / _time_err(gs[1], gs[2], c))
        assert abs(rate - 2.0) < 0.1, (c, rate)


# ---------------------------------------------- decay inside the superconductor
def test_slab_decay_matches_discrete_and_continuum():
    """4 x 4 x 2048 slab (lambda = 8 cells, sigma = 0): the ratio of probe DFTs
    8 cells apart inside the superconductor equals exp(-8 kd d), kd from the
    scheme's evanescent dispersion (to 1 %), and tracks the continuum skin
    depth of Eq. skin to O((d/lambda)^2)."""
    w = W.slab(nxy=1, nsteps=6000, probes_z=(1032, 1040, 1048))
    g = stepper.Grid.from_workload(w)
    g.step(w.nsteps)
    X = [g.probe_dft(p) for p in range(3)]
    fr = w.probes[0].freqs
    f0 = w.sources[0].f
    band = (fr > 0.6 * f0) & (fr < 1.4 * f0)
    d = w.d[2]
    lam = 8 * d
    kd = np.array([theory.discrete_decay(2 * math.pi * f, d, w.dt, lam=lam) for f in fr])
    kc = 1.0 / theory.skin_depth(2 * math.pi * fr, lam=lam)
    for a, b in ((0, 1), (1, 2)):
        r = np.abs(X[b] / X[a])[band]
        assert np.max(np.abs(r / np.exp(-8 * d * kd[band]) - 1)) < 1e-2
        assert np.max(np.abs(np.log(r) / (-8 * d * kc[band]) - 1)) < 2e-2


# ------------------------------------------------------------ reflection
def _reflection_runs(sigma, nz=4480, d=20e-9, z_if=350, z_probe=340, steps=15800, tw=0.25e-15):
    """Sec. 4.2 set-up on a 1 x 1 x 4480 column, dz = 20 nm, CFL 0.95 (1-D),
    superconductor (lambda = 100 nm) from 7 um, probe at 6.8 um, Mur walls;
    a short Gaussian soft source (tw = 0.25 fs, t0 = 4 tw) at 100 nm covers
    0 - 1000 THz; the all-vacuum run gives the incident wave."""
    dt = 0.95 * d / C0
    fr = np.linspace(20e12, 1000e12, 64)
    out = []
    for vac in (False, True):
        g = stepper.Grid((1, 1, nz), (d, d, d), dt, theta=1.0, bc=("periodic", "periodic", "mur"))
        lam = np.zeros((nz, 1, 1))
        sig = np.zeros((nz, 1, 1))
        if not vac:
            lam[z_if:] = 100e-9
            sig[z_if:] = sigma
        g.set_materials(1.0, 1.0, lam, sig)
        g.add_source(0, (0, 0, 5), (1, 1, 6), 1.0, W.SRC_GAUSS, 0.0, 4 * tw, tw)
        g.add_probe(0, (0, 0, z_probe), fr, 0, 0)
        g.step(steps)
        out.append(g.probe_dft(0))
    tot, inc = out
    return fr, (tot - inc) / inc


def test_reflection_total_below_cutoff_sigma0():
    """Eq. beta_cases: with sigma = 0 the superconductor reflects everything
    below f_c = 477 THz: |r| = 1 to 1 % across 20 - 400 THz."""
    fr, r = _reflection_runs(0.0)
    band = fr < 400e12
    assert np.max(np.abs(np.abs(r[band]) - 1)) < 1e-2


def test_reflection_sigma_1e4_within_paper_accuracy():
    """Sec. 4.2: simulated R matches Eq. Ref within 10 % where R > 0.4
    (sigma = 1e4 S/m, lambda = 100 nm)."""
    fr, r = _reflection_runs(1e4)
    R = np.abs(r) ** 2
    Rt = theory.reflection(2 * math.pi * fr, sigma2=1e4, lam2=100e-9)
    m = Rt > 0.4
    assert m.sum() > 20
    assert np.max(np.abs(R[m] / Rt[m] - 1)) < 0.10


# ------------------------------------------------------------------ Q-fit
def test_qfit_recovers_synthetic_mode():
    """Exact finite-sum DFT of a z^n + c.c.: the fit returns alpha and omega0 to 1e-9."""
    dt, n0, N = 6e-17, 3000, 20000
    f0, Q = 6.2e12, 350.0
    om = 2 * math.pi * f0
    al = om / (2 * Q)
    fr = np.linspace(0.9, 1.1, 64) * f0
    A = qfit.model_basis(al, om, fr, dt, n0, N)
    X = A @ np.array([0.7, -0.3])
    res = qfit.fit(X, fr, dt, n0, N, f_guess=1.01 * f0, q_guess=200)
    assert abs(res["f0"] / f0 - 1) < 1e-9
    assert abs(res["Q"] / Q - 1) < 1e-9


def test_qfit_matches_series_dft():
    """The closed-form model agrees with a direct DFT of the sampled series."""
    dt, n0, N = 5e-17, 100, 4000
    om, al = 2 * math.pi * 3e12, 2e10
    n = np.arange(N)
    s = 2 * np.real((0.4 - 0.2j) * np.exp((-al + 1j * om) * dt * n))
    fr = np.linspace(2.5e12, 3.5e12, 64)
    X1 = qfit.dft_of_series(s, fr, dt, n0)
    X2 = qfit.model_basis(al, om, fr, dt, n0, N) @ np.array([0.4, -0.2])
    assert np.max(np.abs(X1 - X2)) < 1e-9 * np.max(np.abs(X1))


def test_qfit_on_oracle_damped_oscillation():
    """End to end: a uniform field with sigma and London current rings down as
    E^n = A g^n + c.c., g a root of the scalar recurrence; the fit of the
    oracle's running probe DFT returns Q = arg(g) / (-2 ln|g|)."""
    d = (10e-9,) * 3
    dt = theory.dt_courant(0.9, d)
    lam, sig, th = 60e-9, 2e4, 1.0
    g = stepper.Grid((1, 1, 1), d, dt, theta=th)
    g.set_materials(1.0, 1.0, lam, sig)
    g.set_field(0, 1.0)
    s = sig * dt / stepper.EPS0
    p = dt * dt / (lam * lam * stepper.MU0 * stepper.EPS0)
    root = [r for r in theory.uniform_recurrence(th, s, p) if np.imag(r) > 0][0]
    om = np.angle(root) / dt
    q_exact = np.angle(root) / (-2 * math.log(abs(root)))
    fr = np.linspace(0.9, 1.1, 64) * om / (2 * math.pi)
    n0, N = 200, 3000
    g.add_probe(0, (0, 0, 0), fr, n0, 0)
    g.step(N)
    res = qfit.fit(g.probe_dft(0), fr, dt, n0, N)
    assert abs(res["Q"] / q_exact - 1) < 1e-6
    assert abs(res["f0"] / (om / (2 * math.pi)) - 1) < 1e-9


# ------------------------------------------------ CW skin depth (Table 1)
TABLE1 = [(float(r[0]), float(r[1]), float(r[4]) * 1e-9, float(r[5])) for r in read_table("table1_skin_depth.txt")]


def cw_skin_depth(X, w):
    """Table 1's measure, delta = z0 / ln(E0 / E_z0): E0 the steady-state
    amplitude (|DFT| over whole periods, X[0]) at the interface, E_z0 the one
    at the probe one expected depth inside (X[2])."""
    X = [abs(x) for x in X]
    z0 = (w.probes[2].p[2] - w.probes[0].p[2]) * w.d[2]
    return z0 / math.log(X[0] / X[2])


CW_RUNS = {1e12: (2, 1), 100e12: (40, 2)}   # spin-up and window periods per frequency


@pytest.mark.parametrize("sigma,f", [(s, f) for s in (0.0, 1e4, 1e7) for f in (1e12, 100e12)])
def test_cw_skin_depth_table1(sigma, f):
    """Sec. 4.1, Table 1, by the paper's own method (continuous sine, steady
    state, delta = z0 / ln(E0 / E_z0)) on a 1-D column with dz = 10 nm and
    CFL 0.9, lambda = 400 nm: the oracle reproduces the paper's computed
    column within 1 % where the skin depth spans more than two cells, and
    Eq. skin within 1.2 % (0.8 % of it is the near-cut-off case sigma = 0 at
    100 THz, whose computed value the paper also prints 0.7 % above theory;
    the 1.6-cell case sigma = 1e7 at 100 THz, printed as 13 nm, is
    compared with theory only, within 3 %)."""
    delta_th = float(theory.skin_depth(2 * math.pi * f, sigma=sigma, lam=400e-9))
    sp, wp = CW_RUNS[f]
    w = W.skin_column(sigma, f, delta_th, spinup_periods=sp, window_periods=wp)
    g = stepper.Grid.from_workload(w)
    g.step(w.nsteps)
    delta = cw_skin_depth([g.probe_dft(p, 1)[0] for p in range(len(w.probes))], w)
    row = [r for r in TABLE1 if r[0] == sigma and r[1] == f][0]
    if delta_th > 2 * w.d[2]:
        assert abs(delta / row[2] - 1) < 1e-2, (delta, row)
        assert abs(delta / delta_th - 1) < 1.2e-2, (delta, delta_th)
    else:
        assert abs(delta / delta_th - 1) < 3e-2, (delta, delta_th)
