"""Temporal blocking: the two-step kernel (two steps of Algorithm 1 per pass
on the interior box, the single-step kernel on the shell) gives the same bits
as single steps -- fields, probe DFTs and series -- on grids with CPML, films
with per-point coefficients and Js, sources and probes inside the box,
periodic axes and Mur walls; odd step counts and split calls included.  The
single-step path is the one the oracle parity tests pin."""
import numpy as np
import pytest

from paper_2305_13419_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _cpw_with_inner_source():
    """The scaled CPW with a third source and probes inside the two-step box."""
    w = W.cpw_small(nsteps=60)
    f = w.sources[0].f
    w.sources.append(W.Source(comp=2, lo=(60, 30, 14), hi=(63, 33, 17), amp=0.7, kind=W.SRC_GAUSS_SIN, f=f,
                              t0=w.sources[0].t0, tw=w.sources[0].tw))
    w.probes.append(W.Probe(comp=0, p=(61, 31, 15), freqs=w.probes[0].freqs, n0=0, series=60))
    w.probes.append(W.Probe(comp=2, p=(95, 47, 30), freqs=w.probes[0].freqs[:5], n0=3, series=60))
    return w


CASES = {
    "cpw-small": lambda: W.cpw_small(nsteps=60, series=60),
    "cpw-inner-source": _cpw_with_inner_source,
    "periodic-xy-pec-z": lambda: W.random_box(n=(100, 70, 30), bc=("periodic", "periodic", "pec"), seed=5,
                                              theta=0.5, mu_range=(1.0, 1.0)),
    "periodic-xy-mur-z": lambda: W.random_box(n=(70, 40, 60), bc=("periodic", "periodic", "mur"), seed=9,
                                              theta=1.0, mu_range=(1.0, 1.0)),
    "cpml-xz-periodic-y": lambda: W.random_box(n=(110, 48, 44), bc=("cpml", "periodic", "cpml"), seed=13,
                                               cpml_cells=5, theta=1.0, mu_range=(1.0, 1.0)),
}


def _run(w, two, chunks, state):
    from paper_2305_13419_gb300 import twofluid as tf
    g = tf.Grid.from_workload(w)
    g.set_two_step(two)
    if state is not None:
        for c in range(9):
            g.set_field(c, state[c].astype(np.float32))
    for n in chunks:
        g.step(n)
    g.sync()
    return g


@pytest.mark.parametrize("name", sorted(CASES))
def test_two_step_gives_the_bits_of_single_steps(name):
    w = CASES[name]()
    st = None if name.startswith("cpw") else W.random_state(7, w.storage_dims())
    ref = _run(w, False, [37], st)
    (lo, hi), active = ref.two_step_box()
    assert not active
    for chunks in ([37], [1, 2, 5, 29], [2, 2, 33]):
        g = _run(w, True, chunks, st)
        (lo2, hi2), active = g.two_step_box()
        assert active and all(hi2[a] > lo2[a] for a in range(3)), (lo2, hi2)
        for c in range(9):
            assert np.array_equal(g.field(c), ref.field(c)), (chunks, c)
        for p in range(len(w.probes)):
            assert np.array_equal(g.probe_dft(p), ref.probe_dft(p)), (chunks, p)
            if w.probes[p].series:
                assert np.array_equal(g.probe_series(p, 37), ref.probe_series(p, 37)), (chunks, p)


def test_two_step_timed_reports_both_kernels():
    from paper_2305_13419_gb300 import twofluid as tf
    w = W.cpw_small(nsteps=20)
    g = tf.Grid.from_workload(w)
    kt, total = g.step_timed(21, with_total=True)
    assert kt["step2"][1] == 10 and kt["step"][1] == 2 * 10 + 1
    assert total > 0 and kt["step2"][0] > 0
    h = tf.Grid.from_workload(w)
    h.set_two_step(False)
    h.step(21)
    for c in range(9):
        assert np.array_equal(g.field(c), h.field(c))


def test_non_uniform_mu_keeps_single_steps():
    from paper_2305_13419_gb300 import twofluid as tf
    w = W.random_box(n=(100, 70, 30), bc=("periodic", "periodic", "pec"), seed=5, mu_range=(1.0, 2.0))
    g = tf.Grid.from_workload(w)
    (lo, hi), active = g.two_step_box()
    assert not active and all(hi[a] > lo[a] for a in range(3))
    kt = g.step_timed(4)
    assert "step2" not in kt and kt["step"][1] == 4


@pytest.mark.parametrize("planes", [4, 7, 12, 24])
def test_two_step_item_lengths_give_the_same_bits(planes):
    """The autotuner's knob: every two-step work-item length gives the bits
    of single steps; lengths outside 4 .. 24 are rejected."""
    from paper_2305_13419_gb300 import twofluid as tf
    w = _cpw_with_inner_source()
    ref = _run(w, False, [21], None)
    g = tf.Grid.from_workload(w)
    g.set_two_step(planes)
    g.step(21)
    g.sync()
    assert g.two_step_box()[1]
    for c in range(9):
        assert np.array_equal(g.field(c), ref.field(c)), c
    for bad in (1, 3, 25):
        with pytest.raises(tf.TFError) as ex:
            g.set_two_step(bad)
        assert ex.value.status == tf.TF_EINVAL


@pytest.mark.parametrize("name", ["cpw-small", "cpml-xz-periodic-y", "periodic-xy-mur-z"])
def test_item_length_gives_the_same_bits(name):
    """The single-step kernel's work-item length (tf_set_item_planes: 8 .. 16
    planes per item, in single steps and in the shell of two-step passes)
    changes how the work is cut, not the bits; out-of-range lengths are
    refused."""
    from paper_2305_13419_gb300 import twofluid as tf
    w = CASES[name]()
    st = None if name.startswith("cpw") else W.random_state(7, w.storage_dims())
    for two in (False, True):
        ref = _run(w, two, [23], st)
        for planes in (12, 16):
            g = tf.Grid.from_workload(w)
            g.set_two_step(two)
            g.set_item_planes(planes)
            if st is not None:
                for c in range(9):
                    g.set_field(c, st[c].astype(np.float32))
            g.step(23)
            g.sync()
            for c in range(9):
                assert np.array_equal(g.field(c), ref.field(c)), (name, two, planes, c)
            for p in range(len(w.probes)):
                assert np.array_equal(g.probe_dft(p), ref.probe_dft(p))
    for bad in (7, 17):
        with pytest.raises(tf.TFError) as ex:
            g.set_item_planes(bad)
        assert ex.value.status == tf.TF_EINVAL
