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


def test_batch_run_one_launch_per_step_matches_single_grids():
    """tf_batch_run (one launch per step over all grids, one work list over
    their items, 64 steps per CUDA graph): every grid bit-identical to
    stepping it alone, over a step count that is not a multiple of the
    graph's 64 steps, with grids at different levels and buffer parities."""
    from paper_2305_13419_gb300 import twofluid as tf
    ws = _variants()
    refs = []
    for w in ws:
        ref = tf.Grid.from_workload(w)
        ref.step(150)
        ref.sync()
        refs.append(ref)
    for first in (3, 4):
        batch = [tf.Grid.from_workload(w) for w in ws]
        batch[0].step(first)   # grids at different levels and buffer parities
        tf.batch_run(batch[1:], first)
        tf.batch_run(batch, 150 - first)
        for w, g, ref in zip(ws, batch, refs):
            g.sync()
            assert g.level == 150
            for c in range(9):
                assert np.array_equal(g.field(c), ref.field(c)), (w.name, c)
            for p in range(len(w.probes)):
                assert np.array_equal(g.probe_dft(p), ref.probe_dft(p))
        # the handles keep stepping on their own afterwards
        more = tf.Grid.from_workload(ws[2])
        more.step(155)
        batch[2].step(5)
        assert np.array_equal(batch[2].field(0), more.field(0))


def test_batch_run_grids_against_the_oracle():
    """Three CPW variants of the batched workload's recipe (uneven sizes,
    strip / gap widths, lambda_L) advanced by tf_batch_run, each against the
    FP64 oracle: fields within 1e-4 relative L2, probe spectra within 1e-3."""
    from paper_2305_13419_gb300 import twofluid as tf
    from parity_util import SPEC_TOL, compare_fields, rel_l2, run_oracle
    ws = W.cpw_batch(count=3, seed=23, sizes=(40, 48, 64))
    grids = [tf.Grid.from_workload(w) for w in ws]
    tf.batch_run(grids, 200)
    for w, g in zip(ws, grids):
        g.sync()
        go = run_oracle(w, 200)
        errs, bad = compare_fields(g, go)
        assert not bad, (w.name, errs)
        for p in range(len(w.probes)):
            assert rel_l2(g.probe_dft(p), go.probe_dft(p)) < SPEC_TOL, (w.name, p)


def test_batch_run_rejects_bad_calls():
    import ctypes as C
    from paper_2305_13419_gb300 import twofluid as tf
    g = tf.Grid.from_workload(_variants()[0])
    with pytest.raises(tf.TFError) as ex:
        tf.batch_run([g, g], 1)
    assert ex.value.status == tf.TF_EINVAL
    hs = (C.c_void_p * 1)(g.h)
    n = C.c_size_t()
    assert tf.load().tf_batch_scratch_size(hs, 1, 10, C.byref(n)) == tf.TF_OK
    buf = torch.empty(int(n.value) + 512, dtype=torch.uint8, device="cuda")
    p = (int(buf.data_ptr()) + 255) // 256 * 256
    assert tf.load().tf_batch_run(hs, 1, 10, C.c_void_p(p), int(n.value) - 1) == tf.TF_ENOMEM
    assert tf.load().tf_batch_run(hs, 1, 10, C.c_void_p(p + 4), int(n.value)) == tf.TF_EINVAL
