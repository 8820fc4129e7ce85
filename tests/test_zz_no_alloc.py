"""The allocation-free field statistics entry point (tf_field_stats_noalloc)
against the workspace-backed tf_field_stats, through the C ABI, on two calls
in a row.

Callers that cannot allocate device memory while a simulation runs -- a
monitoring thread that must not take the CUDA allocator's lock or force the
device-wide synchronisation of cudaFree, or an application whose memory
pool already holds the whole device -- use the allocation-free entry point;
it has to report the same numbers as the regular one.  This file is named so
that pytest collects it after every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

REL = 1e-9   # sums over the same values in the same order; max and counts exact


def _check(ref, got):
    assert abs(got[0] - ref[0]) <= REL * max(abs(ref[0]), 1e-300), (ref, got)
    assert got[1] == ref[1], (ref, got)
    assert got[2] == ref[2], (ref, got)


def test_noalloc_matches_workspace_stats_on_two_calls():
    from paper_2305_13419_gb300 import twofluid as tf
    from paper_2305_13419_gb300 import workloads as W
    w = W.random_box(n=(24, 18, 21), bc=("cpml", "periodic", "pec"), seed=21, cpml_cells=3)

    # call 1: a stepped state (E_x at the current level)
    g = tf.Grid.from_workload(w)
    st = W.random_state(31, w.storage_dims())
    for c in range(9):
        g.set_field(c, st[c].astype(np.float32))
    g.step(25)
    g.sync()
    dev = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    g.field(0, out=dev)
    torch.cuda.synchronize()
    ref1 = g.field_stats(0)
    got1 = tf.tf_field_stats_noalloc(dev, g.N[0], g.N[1], g.N[2], g.N[0], 1.0)
    assert ref1[0] > 0
    _check(ref1, got1)

    # call 2, right after: another grid whose E_z carries NaN and Inf values
    h = tf.Grid.from_workload(w)
    e = st[2].astype(np.float32)
    e[3, 4, 5] = np.nan
    e[7, 2, 9] = -np.inf
    h.set_field(2, e)
    dev2 = torch.empty(h.shape, dtype=torch.float32, device="cuda")
    h.field(2, out=dev2)
    torch.cuda.synchronize()
    ref2 = h.field_stats(2)
    got2 = tf.tf_field_stats_noalloc(dev2, h.N[0], h.N[1], h.N[2], h.N[0], 1.0)
    assert ref2[2] == 2
    _check(ref2, got2)


def test_noalloc_rejects_more_planes_than_its_scratch():
    from paper_2305_13419_gb300 import twofluid as tf
    dev = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(tf.TFError) as ex:
        tf.tf_field_stats_noalloc(dev, 2, 2, 4097, 2, 1.0)
    assert ex.value.status == tf.TF_EINVAL


def test_noalloc_rows_wider_than_the_field():
    """A caller's array whose rows are padded (pitch > nx_pts) with garbage
    past the x end: only the first nx_pts values of each row count, twice in
    a row, and the same numbers as numpy on the unpadded values."""
    from paper_2305_13419_gb300 import twofluid as tf
    rng = np.random.default_rng(5)
    nx, ny, nz, pitch = 37, 23, 19, 160
    vals = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    padded = np.full((nz, ny, pitch), np.nan, np.float32)   # padding would count as non-finite
    padded[:, :, :nx] = vals
    dev = torch.from_numpy(padded).cuda()
    torch.cuda.synchronize()
    ref = (float(np.sum(vals.astype(np.float64) ** 2)), float(np.max(np.abs(vals))), 0)
    for _ in range(2):
        got = tf.tf_field_stats_noalloc(dev, nx, ny, nz, pitch, 2.0)
        assert abs(got[0] - 4.0 * ref[0]) <= 1e-12 * 4.0 * ref[0], (ref, got)
        assert got[1] == 2.0 * ref[1], (ref, got)
        assert got[2] == 0, got
