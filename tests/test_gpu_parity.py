"""GPU (FP32 CUDA, through the C ABI) against the FP64 oracle on the same
seeded inputs.  Tolerances: fields rel L2 <= 1e-4, probe spectra and Q
<= 1e-3 relative."""
import math

import numpy as np
import pytest

from oracle import qfit, stepper
from paper_2305_13419_gb300 import workloads as W
from parity_util import (FIELD_TOL, SPEC_TOL, compare_families, compare_fields, crop_workload, family_norms,
                         local_state, rel_l2, run_gpu, run_oracle)

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _state(w, seed):
    return W.random_state(seed, w.storage_dims())


# ----------------------------------------------------------- small boxes
BOXES = [
    dict(n=(9, 7, 11), bc=("periodic", "periodic", "periodic"), theta=0.5),
    dict(n=(33, 1, 65), bc=("periodic", "periodic", "pec"), theta=1.0),
    dict(n=(5, 7, 9), bc=("pec", "pec", "pec"), theta=0.75, mu_range=(1.0, 2.0)),
    dict(n=(40, 19, 23), bc=("cpml", "periodic", "cpml"), theta=1.0, cpml_cells=5),
    dict(n=(17, 30, 37), bc=("cpml", "cpml", "cpml"), theta=0.5, cpml_cells=4, mu_range=(1.0, 1.5)),
    dict(n=(1, 1, 70), bc=("periodic", "periodic", "mur"), theta=1.0),
    dict(n=(6, 5, 2), bc=("periodic", "pec", "mur"), theta=1.0),
    dict(n=(70, 3, 4), bc=("pec", "periodic", "periodic"), theta=1.0, sc_fraction=1.0),
]


@pytest.mark.parametrize("edge_rule", [0, 1])
@pytest.mark.parametrize("kw", BOXES, ids=lambda k: "x".join(map(str, k["n"])) + "-" + "-".join(k["bc"]))
def test_random_box_fields(kw, edge_rule):
    """Odd and ragged sizes, every boundary kind, random heterogeneous
    materials and a random initial state: all nine components after 150 steps."""
    w = W.random_box(seed=sum(kw["n"]), **kw)
    w.edge_rule = edge_rule
    st = _state(w, 11)
    go = run_oracle(w, 150, st)
    gg = run_gpu(w, 150, st, chunks=[1, 49, 100])
    errs, bad = compare_fields(gg, go)
    assert not bad, errs


def test_zero_steps_is_identity_and_readback_of_level0():
    w = W.random_box(n=(8, 9, 10), bc=("cpml", "pec", "periodic"), seed=3)
    st = _state(w, 5)
    go = run_oracle(w, 0, st)
    gg = run_gpu(w, 0, st)
    errs, bad = compare_fields(gg, go, tol=1e-6)
    assert not bad, errs
    assert gg.level == 0


def test_soft_source_and_probe_on_box():
    w = W.random_box(n=(12, 10, 14), bc=("cpml", "cpml", "periodic"), seed=8, cpml_cells=3)
    f = 2e14
    w.sources = [W.Source(comp=2, lo=(5, 4, 6), hi=(8, 6, 9), amp=3.0, kind=W.SRC_GAUSS_SIN, f=f,
                          t0=8e-15, tw=2e-15),
                 W.Source(comp=0, lo=(0, 0, 0), hi=(12, 11, 1), amp=-1.0, kind=W.SRC_GAUSS, t0=5e-15, tw=2e-15)]
    fr = np.linspace(0.5 * f, 1.5 * f, 64)
    w.probes = [W.Probe(comp=2, p=(6, 5, 7), freqs=fr, n0=10), W.Probe(comp=0, p=(1, 3, 0), freqs=fr[:7], n0=0)]
    go = run_oracle(w, 400)
    gg = run_gpu(w, 400)
    errs, bad = compare_fields(gg, go)
    assert not bad, errs
    for p in range(2):
        Xo, Xg = go.probe_dft(p, len(w.probes[p].freqs)), gg.probe_dft(p)
        assert rel_l2(Xg, Xo) < SPEC_TOL


def test_probe_series_and_wall_probe():
    w = W.slab(nxy=1, nz=256, z_sc=128, probes_z=(100, 0, 256), nsteps=300, series=300)
    go = run_oracle(w, 300)
    gg = run_gpu(w, 300)
    for p in range(3):
        so, sg = go.probe_series(p, 300), gg.probe_series(p, 300)
        assert np.max(np.abs(sg - so)) <= 1e-4 * max(np.max(np.abs(so)), 1e-30) + 1e-12


# ----------------------------------------------------------- 4 x 4 x 2048 slab
@pytest.mark.parametrize("boundary", ["mur", "cpml"])
def test_slab_config(boundary):
    """4 x 4 x 2048 slab, 4000 steps: fields, and the probe spectra at the
    interface and inside the superconductor."""
    w = W.slab(boundary=boundary)
    go = run_oracle(w, w.nsteps)
    gg = run_gpu(w, w.nsteps)
    errs, bad = compare_fields(gg, go)
    assert not bad, errs
    for p in range(len(w.probes)):
        Xo, Xg = go.probe_dft(p), gg.probe_dft(p)
        assert rel_l2(Xg, Xo) < SPEC_TOL, p


# ----------------------------------------------------------- CPW resonator (scaled)
def test_cpw_small_fields_spectra_q():
    """Scaled CPW resonator, 3000 steps: fields near their peak (raw relative
    L2), fields at the end of the ring-down (relative to the peak norm of the
    run), both probes' spectra, and the Q factor each side fits to its own
    DFT (the GPU fit runs in FP64 on the GPU)."""
    from oracle import stepper as st_
    from paper_2305_13419_gb300 import twofluid as tf
    w = W.cpw_small(nsteps=3000)
    f0 = w.sources[0].f
    n0 = 1200
    for p in w.probes:
        p.n0 = n0
        p.freqs = np.linspace(0.7 * f0, 1.3 * f0, 64)
    go = st_.Grid.from_workload(w)
    gg = tf.Grid.from_workload(w)
    peak = {"E": 0.0, "B": 0.0, "Js": 0.0}
    done = 0
    for N in (500, 1000, 1500, 2000, 2500, 3000):
        go.step(N - done)
        gg.step(N - done)
        done = N
        for k, v in family_norms(go).items():
            peak[k] = max(peak[k], v)
        if N == 1000:   # near the peak of the transient: plain relative L2
            errs, bad = compare_families(gg, go)
            assert not bad, (N, errs)
    gg.sync()
    errs, bad = compare_families(gg, go, peak)
    assert not bad, errs
    for p in range(2):
        assert rel_l2(gg.probe_dft(p), go.probe_dft(p)) < SPEC_TOL
    fr = w.probes[0].freqs
    ro = qfit.fit(go.probe_dft(0), fr, go.dt, n0, w.nsteps)
    rg = gg.fit_q(0, f_guess=ro["f0"], q_guess=max(ro["Q"], 5.0))
    assert abs(rg["Q"] / ro["Q"] - 1) < SPEC_TOL, (rg, ro)
    assert abs(rg["f0"] / ro["f0"] - 1) < SPEC_TOL


def test_gpu_qfit_matches_oracle_fit_on_same_dft():
    """The FP64 GPU fit and the oracle's fit agree on one and the same DFT."""
    w = W.random_box(n=(1, 1, 1), bc=("periodic",) * 3, seed=2, sc_fraction=1.0,
                     lam_range=(60e-9, 60e-9), sigma_range=(2e4, 2e4), eps_range=(1, 1))
    st = {0: np.ones((1, 1, 1))}
    dt = stepper.dt_from_courant(w.courant, w.d)
    om = 1.0 / math.sqrt(stepper.EPS0 * stepper.MU0) / 60e-9
    fr = np.linspace(0.9, 1.1, 64) * om / (2 * math.pi)
    w.probes = [W.Probe(comp=0, p=(0, 0, 0), freqs=fr, n0=200)]
    gg = run_gpu(w, 3000, st)
    X = gg.probe_dft(0)
    ro = qfit.fit(X, fr, dt, 200, 3000)
    rg = gg.fit_q(0, f_guess=fr[32], q_guess=50.0)
    assert abs(rg["Q"] / ro["Q"] - 1) < 1e-8
    assert abs(rg["f0"] / ro["f0"] - 1) < 1e-10


# ----------------------------------------------------------- failure detection
def test_watchdog_reports_nonfinite():
    from paper_2305_13419_gb300 import twofluid as tf
    w = W.random_box(n=(8, 8, 8), seed=1)
    g = tf.Grid.from_workload(w)
    e = np.zeros(g.shape, np.float32)
    e[3, 3, 3] = np.nan
    g.set_field(0, e)
    g.step(3)
    with pytest.raises(tf.TFError) as ex:
        g.sync()
    assert ex.value.status == tf.TF_ENONFINITE


def test_state_errors():
    from paper_2305_13419_gb300 import twofluid as tf
    w = W.random_box(n=(6, 6, 6), seed=2)
    g = tf.Grid.from_workload(w)
    g.step(1)
    with pytest.raises(tf.TFError) as ex:
        g.set_field(0, np.zeros(g.shape, np.float32))
    assert ex.value.status == tf.TF_ESTATE
    with pytest.raises(tf.TFError) as ex:
        g.set_materials(1.0, 1.0, 0.0, 0.0)
    assert ex.value.status == tf.TF_ESTATE


def test_bad_materials_and_unstable_london_term():
    from paper_2305_13419_gb300 import twofluid as tf
    w = W.random_box(n=(6, 6, 6), seed=2, courant=0.95)
    g = tf.Grid(w.n, w.d, courant=0.95)
    with pytest.raises(tf.TFError) as ex:
        g.set_materials(-1.0, 1.0, 0.0, 0.0)
    assert ex.value.status == tf.TF_EINVAL
    with pytest.raises(tf.TFError) as ex:      # lambda of 0.3 cells breaks C^2 + (c dt/2 lambda)^2 <= 1
        g.set_materials(1.0, 1.0, 0.3 * w.d[0], 0.0)
    assert ex.value.status == tf.TF_EUNSTABLE


def test_deterministic():
    w = W.random_box(n=(16, 12, 20), bc=("cpml", "periodic", "pec"), seed=6, cpml_cells=3)
    st = _state(w, 4)
    a = run_gpu(w, 60, st)
    b = run_gpu(w, 60, st)
    for c in range(9):
        assert np.array_equal(a.field(c), b.field(c))


def test_field_stats_watchdog():
    """Watchdog reduction: sum of squares and max |E| match numpy on the
    read-back field; injected NaN/Inf values are counted."""
    from paper_2305_13419_gb300 import twofluid as tf
    w = W.random_box(n=(20, 13, 17), bc=("cpml", "periodic", "pec"), seed=12, cpml_cells=3)
    g = tf.Grid.from_workload(w)
    st = _state(w, 9)
    for c in range(9):
        g.set_field(c, st[c].astype(np.float32))
    for c in (3, 6):        # before the first step B and Js are stored at level 0 (Js on SC edges only)
        ref = g.field(c).astype(np.float64)
        s, m, n = g.field_stats(c)
        assert abs(s / np.sum(ref * ref) - 1) < 1e-6 and abs(m / np.max(np.abs(ref)) - 1) < 1e-6 and n == 0
    g.step(30)
    g.sync()
    for c in range(3):
        ref = g.field(c).astype(np.float64)
        s, m, n = g.field_stats(c)
        assert abs(s / np.sum(ref * ref) - 1) < 1e-9
        assert m == np.max(np.abs(ref)) and n == 0
    bad = tf.Grid.from_workload(w)
    e = np.zeros(bad.shape, np.float32)
    e[2, 3, 4] = np.nan
    e[5, 6, 7] = np.inf
    e[1, 1, 1] = 2.5
    bad.set_field(0, e)
    s, m, n = bad.field_stats(0)
    assert n == 2 and m == 2.5 and abs(s - 6.25) < 1e-12


@pytest.mark.parametrize("n,bc", [((16, 12, 20), ("cpml", "periodic", "pec")),
                                  ((160, 160, 64), ("cpml", "cpml", "cpml")),
                                  ((4, 4, 300), ("periodic", "periodic", "mur"))],
                         ids=["few-items", "many-items", "slab-like"])
def test_split_calls_are_bit_identical(n, bc):
    """The step hands out its work items through a counter that runs on
    across launches (each CTA's first two items by position, the rest by
    ticket, small grids entirely in pieces).  Stepping in many short calls
    must give the same bits as one long call, on a grid with fewer work items
    than CTA slots, one with more, and a long thin one."""
    w = W.random_box(n=n, bc=bc, seed=21, cpml_cells=4, theta=1.0)
    st = _state(w, 5)
    a = run_gpu(w, 24, st)
    b = run_gpu(w, 24, st, chunks=[1, 1, 1, 5, 1, 15])
    for c in range(9):
        assert np.array_equal(a.field(c), b.field(c)), c
