"""Batched stepping of independent grids (tf_batch_step): every grid ends
bit-identical to stepping it alone, whatever streams the grids share."""
import numpy as np
import pytest

from paper_2305_13419_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _variants():
    ws = W.cpw_batch(count=5, seed=11, sizes=(40, 48, 64))
    ws.append(W.random_box(n=(23, 17, 29), bc=("cpml", "periodic", "pec"), seed=4, cpml_cells=3))
    return ws


@pytest.mark.parametrize("nstreams", [1, 3])
def test_batch_matches_single_grids(nstreams):
    from paper_2305_13419_gb300 import twofluid as tf
    ws = _variants()
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    batch = [tf.Grid.from_workload(w, stream=streams[i % nstreams]) for i, w in enumerate(ws)]
    tf.batch_step(batch, 37)
    for g in batch:
        g.sync()
    for w, g in zip(ws, batch):
        ref = tf.Grid.from_workload(w)
        ref.step(37)
        ref.sync()
        assert g.level == 37
        for c in range(9):
            assert np.array_equal(g.field(c), ref.field(c)), (w.name, c)
        for p in range(len(w.probes)):
            assert np.array_equal(g.probe_dft(p), ref.probe_dft(p))


def test_batch_rejects_a_handle_twice():
    from paper_2305_13419_gb300 import twofluid as tf
    g = tf.Grid.from_workload(_variants()[0])
    with pytest.raises(tf.TFError) as ex:
        tf.batch_step([g, g], 1)
    assert ex.value.status == tf.TF_EINVAL
