"""Pins of the FP64 oracle (Algorithm 1 of arXiv 2305.13419) against results
fixed by mathematics rather than by the oracle itself: exact discrete
eigenmodes, scalar recurrences of spatially uniform fields, the discrete
energy identity, exact absorption of first-order Mur at the magic time step,
axis-permutation covariance, and closed-form DFT sums.  CPU only."""
import math

import numpy as np
import pytest

from oracle import stepper, theory
from paper_2305_13419_gb300 import workloads as W

C0, MU0, EPS0 = stepper.C0, stepper.MU0, stepper.EPS0


def _grid_coords(g):
    N = g.N
    return np.meshgrid(np.arange(N[2]), np.arange(N[1]), np.arange(N[0]), indexing="ij")


# -------------------------------------------------------------- uniform fields
@pytest.mark.parametrize("theta", [0.5, 1.0])
@pytest.mark.parametrize("sigma,lam", [(0.0, 50e-9), (3e5, 0.0), (2e5, 70e-9)])
def test_uniform_field_recurrence(theta, sigma, lam):
    """A uniform E has zero curl, so steps 2-4 reduce to the scalar recurrence
    (1 + theta s) E^{n+1} - (2 - (1-2 theta) s - p) E^n + (1 - (1-theta) s) E^{n-1} = 0,
    s = sigma dt/eps, p = kappa dt^2/eps, started from E^0 = 1, B^0 = Js^0 = 0
    (so E^1 = (1 - (1-theta) s - p/2)/(1 + theta s))."""
    d = (10e-9, 10e-9, 10e-9)
    dt = theory.dt_courant(0.9, d)
    eps_r = 2.5
    g = stepper.Grid((1, 1, 1), d, dt, theta=theta)
    g.set_materials(eps_r, 1.0, lam, sigma)
    g.set_field(0, 1.0)
    eps = EPS0 * eps_r
    s = sigma * dt / eps
    kap = 0.0 if lam == 0 else 1.0 / (lam * lam * MU0)
    p = kap * dt * dt / eps
    e_prev, e_cur = 1.0, (1 - (1 - theta) * s - p / 2) / (1 + theta * s)
    exact = [e_prev, e_cur]
    for _ in range(300):
        nxt = ((2 - (1 - 2 * theta) * s - p) * e_cur - (1 - (1 - theta) * s) * e_prev) / (1 + theta * s)
        exact.append(nxt)
        e_prev, e_cur = e_cur, nxt
    got = []
    for n in range(302):
        got.append(g.field(0)[0, 0, 0])
        g.step(1)
    assert np.max(np.abs(np.array(got) - np.array(exact))) < 1e-12


def test_plasma_oscillation_frequency():
    """sigma = 0, uniform field: E^n = cos(omega n dt) with the discrete
    London plasma frequency sin(omega dt/2) = (dt/2) sqrt(kappa/eps)."""
    lam, d = 50e-9, (10e-9,) * 3
    dt = theory.dt_courant(0.9, d)
    g = stepper.Grid((1, 1, 1), d, dt, theta=0.5)
    g.set_materials(1.0, 1.0, lam, 0.0)
    g.set_field(0, 1.0)
    om = theory.discrete_omega((0, 0, 0), d, dt, lam=lam)
    got = []
    for n in range(400):
        got.append(g.field(0)[0, 0, 0])
        g.step(1)
    assert np.max(np.abs(np.array(got) - np.cos(om * dt * np.arange(400)))) < 1e-13


# ------------------------------------------------------------ discrete modes
@pytest.mark.parametrize("mvec", [(1, 0, 0), (0, 2, 0), (0, 0, 1), (1, 2, 1), (2, 1, 3)])
def test_periodic_eigenmode_dispersion(mvec):
    """A transverse Fourier mode of the Yee grid in a homogeneous London medium
    is an exact eigenvector: E^n = E^0 cos(omega n dt) with
    mu eps Omega^2 = sum_a (2/d_a sin(K_a d_a/2))^2 + 1/lambda^2.
    Oblique K exercises every curl component, index and staggering offset."""
    n, d = (8, 6, 10), (10e-9, 12e-9, 9e-9)
    dt = theory.dt_courant(0.9, d)
    eps_r, lam = 2.0, 40e-9
    g = stepper.Grid(n, d, dt, theta=0.5)
    g.set_materials(eps_r, 1.0, lam, 0.0)
    k_, j_, i_ = _grid_coords(g)
    K = tuple(2 * math.pi * mvec[a] / (n[a] * d[a]) for a in range(3))
    Kd = np.array([2 / d[a] * math.sin(K[a] * d[a] / 2) for a in range(3)])
    e = np.cross(Kd, [0.3, 1.0, 0.2])
    e /= np.linalg.norm(e)
    offs = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
    for c in range(3):
        ph = K[0] * (i_ + offs[c][0]) * d[0] + K[1] * (j_ + offs[c][1]) * d[1] + K[2] * (k_ + offs[c][2]) * d[2]
        g.set_field(c, e[c] * np.cos(ph))
    E0 = [g.field(c) for c in range(3)]
    om = theory.discrete_omega(K, d, dt, eps_r=eps_r, lam=lam)
    for nst in (37, 150):
        g.step(nst - g.level)
        for c in range(3):
            assert np.max(np.abs(g.field(c) - E0[c] * math.cos(om * nst * dt))) < 1e-12


@pytest.mark.parametrize("mode", [(1, 0, 1), (2, 0, 1), (1, 1, 0)])
def test_pec_cavity_mode(mode):
    """PEC box, sin-sin cavity modes are exact discrete eigenmodes:
    E^n = E^0 cos(omega n dt), omega from the discrete dispersion with
    K_a = m_a pi / L_a; the other E components stay identically zero."""
    n, d = (6, 5, 7), (10e-9, 11e-9, 9e-9)
    dt = theory.dt_courant(0.9, d)
    g = stepper.Grid(n, d, dt, theta=1.0, bc=("pec", "pec", "pec"))
    k_, j_, i_ = _grid_coords(g)
    L = [n[a] * d[a] for a in range(3)]
    mx, my, mz = mode
    if my == 0:   # Ey(i, j+1/2, k) = sin(mx pi x/Lx) sin(mz pi z/Lz)
        comp = 1
        f = np.sin(mx * math.pi * i_ * d[0] / L[0]) * np.sin(mz * math.pi * k_ * d[2] / L[2])
    else:         # Ez(i, j, k+1/2) = sin(mx pi x/Lx) sin(my pi y/Ly)
        comp = 2
        f = np.sin(mx * math.pi * i_ * d[0] / L[0]) * np.sin(my * math.pi * j_ * d[1] / L[1])
    g.set_field(comp, f)
    E0 = g.field(comp)
    assert np.max(np.abs(E0)) > 0.5
    K = (mx * math.pi / L[0], my * math.pi / L[1], mz * math.pi / L[2])
    om = theory.discrete_omega(K, d, dt)
    g.step(120)
    assert np.max(np.abs(g.field(comp) - E0 * math.cos(om * 120 * dt))) < 1e-12
    for c in range(3):
        if c != comp:
            assert np.max(np.abs(g.field(c))) == 0.0


# ------------------------------------------------------------ energy identity
def _curlE(E, d):
    def D(F, a):
        return (np.roll(F, -1, axis=2 - a) - F) / d[a]
    return [D(E[2], 1) - D(E[1], 2), D(E[0], 2) - D(E[2], 0), D(E[1], 0) - D(E[0], 1)]


def _energy(g):
    """W^n = 1/2 sum eps_e E^2 + 1/2 sum B^{n-1/2} B^{n+1/2} / mu_f
             + 1/2 sum_{kappa>0} Js^{n-1/2} Js^{n+1/2} / kappa_e,
    with the half-level values rebuilt from the integer-level state
    (B^{n+-1/2} = B^n -+ dt/2 curl E^n, Js^{n+-1/2} = Js^n +- dt/2 kappa E^n)."""
    E = [g.field(c) for c in range(3)]
    B = [g.field(c) for c in range(3, 6)]
    J = [g.field(c) for c in range(6, 9)]
    eps = [g.coeff(0, c) for c in range(3)]
    kap = [g.coeff(2, c) for c in range(3)]
    mu = [g.coeff(3, c) for c in range(3)]
    cE = _curlE(E, g.d)
    w = 0.0
    for c in range(3):
        w += 0.5 * np.sum(eps[c] * E[c] ** 2)
        w += 0.5 * np.sum((B[c] + 0.5 * g.dt * cE[c]) * (B[c] - 0.5 * g.dt * cE[c]) / mu[c])
        m = kap[c] > 0
        jm, jp = J[c] - 0.5 * g.dt * kap[c] * E[c], J[c] + 0.5 * g.dt * kap[c] * E[c]
        w += 0.5 * np.sum((jm * jp)[m] / kap[c][m])
    return w


def test_energy_conserved_lossless_heterogeneous():
    """sigma = 0: W^n is exactly conserved by the scheme for any per-edge eps,
    kappa and per-face mu (derivation: the Yee curls are mutual transposes)."""
    w = W.random_box(n=(7, 6, 9), seed=3, theta=0.5, sigma_range=(0, 0), mu_range=(1, 2))
    g = stepper.Grid.from_workload(w)
    st = W.random_state(5, g.N)
    for c in range(9):
        g.set_field(c, st[c])
    w0 = _energy(g)
    for _ in range(4):
        g.step(250)
        assert abs(_energy(g) / w0 - 1) < 1e-12


def test_energy_balance_ohmic_theta_half():
    """theta = 1/2: W^{n+1} - W^n = -dt sum_e sigma_e ((E^n + E^{n+1})/2)^2,
    step by step (the Ohmic dissipation of Alg. 1 step 3)."""
    w = W.random_box(n=(6, 7, 5), seed=4, theta=0.5, sigma_range=(0, 5e5), mu_range=(1, 1.5))
    g = stepper.Grid.from_workload(w)
    st = W.random_state(6, g.N)
    for c in range(9):
        g.set_field(c, st[c])
    sig = [g.coeff(1, c) for c in range(3)]
    for _ in range(20):
        w0, e0 = _energy(g), [g.field(c) for c in range(3)]
        g.step(1)
        w1, e1 = _energy(g), [g.field(c) for c in range(3)]
        diss = g.dt * sum(np.sum(sig[c] * (0.5 * (e0[c] + e1[c])) ** 2) for c in range(3))
        assert diss > 0
        assert abs((w1 - w0) + diss) < 1e-10 * w0


# --------------------------------------------------------- axis permutation
def _perm_workload(w):
    """Relabel axes cyclically: new x = old z, new y = old x, new z = old y."""
    tp = lambda a: np.ascontiguousarray(a.transpose(1, 2, 0))
    return W.Workload(name=w.name + "-perm", n=(w.n[2], w.n[0], w.n[1]), d=(w.d[2], w.d[0], w.d[1]),
                      theta=w.theta, bc=(w.bc[2], w.bc[0], w.bc[1]), eps_r=tp(w.eps_r), mu_r=tp(w.mu_r),
                      lambda_L=tp(w.lambda_L), sigma=tp(w.sigma), courant=w.courant,
                      cpml=(w.cpml[2], w.cpml[0], w.cpml[1]))


@pytest.mark.parametrize("bc", [("periodic", "pec", "cpml"), ("cpml", "periodic", "pec")])
def test_axis_permutation_covariance(bc):
    """Cyclic relabelling of the axes (x->y->z->x) maps the discrete problem
    onto itself: every field must follow exactly (to rounding).  A swapped
    index, a transposed difference or a wrong staggering offset breaks it."""
    w = W.random_box(n=(9, 7, 11), bc=bc, seed=7, theta=1.0, mu_range=(1, 2), cpml_cells=3)
    g = stepper.Grid.from_workload(w)
    wp = _perm_workload(w)
    gp = stepper.Grid.from_workload(wp)
    st = W.random_state(8, g.N)
    tp = lambda a: np.ascontiguousarray(a.transpose(1, 2, 0))
    # component relabelling: new (x,y,z) comps = old (z,x,y)
    newc = {0: 2, 1: 0, 2: 1}
    for fam in (0, 3, 6):
        for c in range(3):
            g.set_field(fam + c, st[fam + c])
            gp.set_field(fam + c, tp(st[fam + newc[c]]))
    g.step(60)
    gp.step(60)
    for fam in (0, 3, 6):
        for c in range(3):
            a = tp(g.field(fam + newc[c]))
            b = gp.field(fam + c)
            scale = max(np.max(np.abs(a)), 1e-300)
            assert np.max(np.abs(a - b)) <= 1e-12 * scale


# ------------------------------------------------------------------ sources
def test_soft_source_first_step():
    """From zero fields, one step leaves E^1 = amp * s(t^1) on the source
    points (the soft source is added after step 3) and zero elsewhere."""
    w = W.random_box(n=(5, 4, 6), bc=("periodic", "pec", "periodic"), seed=9)
    g = stepper.Grid.from_workload(w)
    f, t0, tw, amp = 3e14, 1e-15, 4e-16, -2.5
    g.add_source(1, (1, 1, 2), (4, 3, 4), amp, W.SRC_GAUSS_SIN, f, t0, tw)
    g.step(1)
    t = g.dt
    s = amp * math.exp(-(t - t0) ** 2 / (2 * tw * tw)) * math.sin(2 * math.pi * f * t)
    ey = g.field(1)
    exp_ = np.zeros_like(ey)
    exp_[2:4, 1:3, 1:4] = s
    assert np.max(np.abs(ey - exp_)) < 1e-15 * abs(s) + 1e-300
    assert np.max(np.abs(g.field(0))) == 0 and np.max(np.abs(g.field(2))) == 0


def test_waveform_kinds():
    d = (10e-9,) * 3
    dt = theory.dt_courant(0.5, d)
    for kind, fn in ((W.SRC_GAUSS, lambda t: math.exp(-(t - 3e-16) ** 2 / (2 * 1e-16 ** 2))),
                     (W.SRC_SIN, lambda t: math.sin(2 * math.pi * 2e14 * t))):
        g = stepper.Grid((1, 1, 1), d, dt)
        g.add_source(0, (0, 0, 0), (1, 1, 1), 1.0, kind, 2e14, 3e-16, 1e-16)
        g.step(1)
        assert abs(g.field(0)[0, 0, 0] - fn(dt)) < 1e-15


# ------------------------------------------------------------------- probes
def test_probe_dft_closed_form():
    """Probe on the uniform plasma oscillation E^n = cos(omega n dt): the
    running DFT over n0 <= n < N equals the closed geometric sums
    dt/2 sum (q+^n + q-^n), q+- = exp(i(+-omega - 2 pi f) dt)."""
    lam, d = 60e-9, (10e-9,) * 3
    dt = theory.dt_courant(0.9, d)
    g = stepper.Grid((1, 1, 1), d, dt, theta=0.5)
    g.set_materials(1.0, 1.0, lam, 0.0)
    g.set_field(0, 1.0)
    om = theory.discrete_omega((0, 0, 0), d, dt, lam=lam)
    freqs = np.linspace(0.5, 1.5, 64) * om / (2 * math.pi)
    n0, N = 37, 1500
    g.add_probe(0, (0, 0, 0), freqs, n0, N)
    g.step(N)
    X = g.probe_dft(0)
    w = np.exp(-2j * math.pi * freqs * dt)
    geo = lambda q: (q ** n0 - q ** N) / (1 - q)
    Xe = dt / 2 * (geo(np.exp(1j * om * dt) * w) + geo(np.exp(-1j * om * dt) * w))
    assert np.max(np.abs(X - Xe)) < 1e-10 * np.max(np.abs(Xe))
    s = g.probe_series(0, N)
    assert np.max(np.abs(s - np.cos(om * dt * np.arange(N)))) < 1e-12


# -------------------------------------------------------------- boundaries
def _plane_pulse(g, z0, width):
    """+z travelling Ex/By pulse on a quasi-1-D grid.  At the magic time step
    the discrete wave is Ex^n_k = f(k - n), By^{n+1/2}_{k+1/2} = f(k - n)/c; the
    integer-level By^0 of Alg. 1 is the mean of its two half-level neighbours,
    (f(k) + f(k+1)) / (2c)."""
    z = np.arange(g.N[2], dtype=np.float64)
    f = np.exp(-((z - z0) / width) ** 2)
    g.set_field(0, f[:, None, None])
    g.set_field(4, (0.5 * (f + np.roll(f, -1)) / C0)[:, None, None])


def test_mur_exact_at_magic_time_step():
    """1-D, c dt = dz: Yee is exact and first-order Mur (M = 0) absorbs a
    normally incident pulse completely."""
    d = (10e-9,) * 3
    g = stepper.Grid((1, 1, 400), d, d[2] / C0, theta=1.0, bc=("periodic", "periodic", "mur"))
    _plane_pulse(g, 200, 15.0)
    g.step(500)
    assert np.max(np.abs(g.field(0))) < 1e-12


def test_periodic_translation_at_magic_time_step():
    """1-D, c dt = dz, vacuum: the pulse moves exactly one cell per step."""
    d = (10e-9,) * 3
    g = stepper.Grid((1, 1, 300), d, d[2] / C0)
    _plane_pulse(g, 100, 12.0)
    e0 = g.field(0)
    g.step(77)
    assert np.max(np.abs(g.field(0) - np.roll(e0, 77, axis=0))) < 1e-12


@pytest.mark.parametrize("L,m,bound", [(8, 3, 2e-4), (16, 3, 3e-5), (16, 4, 1e-6)])
def test_cpml_normal_incidence_reflection(L, m, bound):
    """Roden-Gedney CPML (sigma_max = 0.8(m+1)/(eta0 d)): the pulse reflected
    by the layer is below `bound` of the incident one, and shrinks with the
    layer's thickness and grading order (a sign error in b or c grows instead)."""
    d = (10e-9,) * 3
    cp = W.default_cpml(L, d[2], 1e12, order=m)
    g = stepper.Grid((1, 1, 1200), d, 0.5 * d[2] / C0, theta=1.0, bc=("periodic", "periodic", "cpml"),
                     cpml=(None, None, cp))
    _plane_pulse(g, 900, 15.0)
    g.add_probe(0, (0, 0, 1000), [1e12], 0, 2000)
    g.step(2000)
    s = g.probe_series(0, 2000)
    refl = np.max(np.abs(s[600:1800])) / np.max(np.abs(s[:600]))
    assert refl < bound


def test_cpml_3d_absorbs_oblique_waves():
    """A localised, discretely divergence-free 3-D pulse (E = backward curl of
    a Gaussian potential on the Bz faces, so no static part can remain) in a
    CPML box radiates out: the field left after the fronts have crossed the
    layers is < 1e-3 of the initial peak."""
    d = (10e-9,) * 3
    cp = W.default_cpml(8, d[0], 1e12)
    n = (40, 40, 40)
    g = stepper.Grid(n, d, theory.dt_courant(0.9, d), theta=1.0, bc=("cpml",) * 3, cpml=(cp, cp, cp))
    k_, j_, i_ = _grid_coords(g)
    phi = np.exp(-((i_ + 0.5 - 20) ** 2 + (j_ + 0.5 - 20) ** 2 + (k_ - 20) ** 2) / 9.0)
    ex = phi - np.roll(phi, 1, axis=1)
    ey = -(phi - np.roll(phi, 1, axis=2))
    g.set_field(0, ex)
    g.set_field(1, ey)
    e0 = max(np.max(np.abs(g.field(0))), np.max(np.abs(g.field(1))))
    g.step(300)
    assert max(np.max(np.abs(g.field(c))) for c in range(3)) < 1e-3 * e0
