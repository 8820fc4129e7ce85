"""Checkpoint save / load through the C ABI: a run resumed from a checkpoint
continues bit-identically, on a fresh handle (host blob) and by rewinding the
same handle (device blob); a blob from another grid is rejected."""
import numpy as np
import pytest

from paper_2305_13419_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _workload():
    w = W.random_box(n=(37, 21, 29), bc=("cpml", "periodic", "cpml"), seed=41, cpml_cells=4, theta=1.0)
    f = 2e14
    w.sources = [W.Source(comp=2, lo=(10, 8, 12), hi=(13, 11, 15), amp=2.0, kind=W.SRC_GAUSS_SIN, f=f,
                          t0=6e-15, tw=2e-15)]
    w.probes = [W.Probe(comp=2, p=(20, 9, 14), freqs=np.linspace(0.5 * f, 1.5 * f, 64), n0=5, series=200)]
    return w


def _snapshot(g):
    g.sync()
    return [g.field(c) for c in range(9)], g.probe_dft(0), g.probe_series(0, g.level)


def _same(a, b):
    for x, y in zip(a[0], b[0]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("first", [0, 40])
def test_resume_on_a_fresh_handle_is_bit_identical(first):
    from paper_2305_13419_gb300 import twofluid as tf
    w = _workload()
    st = W.random_state(3, w.storage_dims())
    g = tf.Grid.from_workload(w)
    for c in range(9):
        g.set_field(c, st[c].astype(np.float32))
    g.step(first)
    blob = g.save_checkpoint()
    assert blob.nbytes == g.checkpoint_size()
    g.step(30)
    ref = _snapshot(g)
    h = tf.Grid.from_workload(w)
    h.load_checkpoint(blob)
    assert h.level == first
    h.step(30)
    _same(_snapshot(h), ref)


def test_rewind_from_a_device_blob():
    from paper_2305_13419_gb300 import twofluid as tf
    w = _workload()
    g = tf.Grid.from_workload(w)
    g.step(25)
    blob = torch.empty(g.checkpoint_size(), dtype=torch.uint8, device="cuda")
    g.save_checkpoint(blob)
    g.step(35)
    ref = _snapshot(g)
    g.step(11)                      # run on, then rewind
    g.load_checkpoint(blob)
    assert g.level == 25
    g.step(35)
    _same(_snapshot(g), ref)


def test_blob_of_another_grid_is_rejected():
    from paper_2305_13419_gb300 import twofluid as tf
    g = tf.Grid.from_workload(_workload())
    blob = g.save_checkpoint()
    other = tf.Grid.from_workload(W.random_box(n=(36, 21, 29), bc=("cpml", "periodic", "cpml"), seed=41,
                                               cpml_cells=4))
    with pytest.raises(tf.TFError) as ex:
        other.load_checkpoint(blob)
    assert ex.value.status == tf.TF_EINVAL
    with pytest.raises(tf.TFError) as ex:
        g.load_checkpoint(blob[:100])
    assert ex.value.status == tf.TF_EINVAL
