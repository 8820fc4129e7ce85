"""FP64 GPU stepper against the FP64 oracle: the same discrete scheme, so the
two agree to rounding (<= 1e-12 of the field's scale after 200 steps) on
every boundary kind, with sources and probes."""
import numpy as np
import pytest

from oracle import stepper
from paper_2305_13419_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

BOXES = [
    dict(n=(9, 7, 11), bc=("periodic", "periodic", "periodic"), theta=0.5),
    dict(n=(5, 7, 9), bc=("pec", "pec", "pec"), theta=0.75, mu_range=(1.0, 2.0)),
    dict(n=(17, 30, 37), bc=("cpml", "cpml", "cpml"), theta=0.5, cpml_cells=4, mu_range=(1.0, 1.5)),
    dict(n=(6, 5, 12), bc=("periodic", "pec", "mur"), theta=1.0),
    dict(n=(40, 19, 23), bc=("cpml", "periodic", "cpml"), theta=1.0, cpml_cells=5),
]


def _close(a, b, tol=1e-12):
    scale = max(np.max(np.abs(b)), 1e-300)
    return np.max(np.abs(a - b)) <= tol * scale


@pytest.mark.parametrize("edge_rule", [0, 1])
@pytest.mark.parametrize("kw", BOXES, ids=lambda k: "x".join(map(str, k["n"])) + "-" + "-".join(k["bc"]))
def test_fp64_gpu_matches_oracle(kw, edge_rule):
    from paper_2305_13419_gb300 import twofluid as tf
    w = W.random_box(seed=sum(kw["n"]) + 3, **kw)
    w.edge_rule = edge_rule
    st = W.random_state(13, w.storage_dims())
    o = stepper.Grid.from_workload(w)
    g = tf.Grid64.from_workload(w)
    for c in range(9):
        o.set_field(c, st[c])
        g.set_field(c, np.asarray(o.field(c)))
    o.step(200)
    g.step(200)
    g.sync()
    assert g.level == 200
    for c in range(9):
        assert _close(g.field(c), o.field(c)), c


def test_fp64_gpu_sources_and_probes():
    from paper_2305_13419_gb300 import twofluid as tf
    w = W.slab(nxy=1, nz=512, z_sc=256, probes_z=(100, 256, 264), nsteps=600)
    o = stepper.Grid.from_workload(w)
    g = tf.Grid64.from_workload(w)
    o.step(600)
    g.step(600)
    for c in range(9):
        assert _close(g.field(c), o.field(c)), c
    for p in range(3):
        X, Y = g.probe_dft(p), o.probe_dft(p, len(w.probes[p].freqs))
        assert np.max(np.abs(X - Y)) <= 1e-12 * np.max(np.abs(Y))


def test_fp64_fma_rate_measures_and_rejects_bad_calls():
    """The FP64 FMA-rate probe (the FP64 stepper's arithmetic ceiling)
    returns a finite positive rate and rejects bad arguments."""
    import ctypes as C
    import torch
    from paper_2305_13419_gb300 import twofluid as tf
    r = tf.fp64_fma_rate(iters=2000)
    assert np.isfinite(r) and r > 0
    n = tf.load().tf64_fma_rate_scratch()
    buf = torch.empty(int(n), dtype=torch.uint8, device="cuda")
    g = C.c_double()
    assert tf.load().tf64_fma_rate(C.c_void_p(buf.data_ptr()), int(n) - 8, 10, None, C.byref(g)) == tf.TF_ENOMEM
    assert tf.load().tf64_fma_rate(C.c_void_p(buf.data_ptr()), int(n), 0, None, C.byref(g)) == tf.TF_EINVAL
    assert tf.load().tf64_fma_rate(None, int(n), 10, None, C.byref(g)) == tf.TF_EINVAL
