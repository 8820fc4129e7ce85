"""Bounded device waits: every mbarrier wait of the stepping kernels gives up
after a host-set number of polls (tf_set_wait_limit), latches TF_ETIMEOUT
for tf_sync and returns after its copies in flight have landed.  A limit of
zero polls makes every wait run out at once; the context stays usable and
other grids step on with unchanged bits."""
import numpy as np
import pytest

from paper_2305_13419_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _grid(w, two):
    from paper_2305_13419_gb300 import twofluid as tf
    g = tf.Grid.from_workload(w)
    g.set_two_step(two)
    return g


def _reference(w, nsteps):
    g = _grid(w, False)
    g.step(nsteps)
    g.sync()
    return g


def _expect_timeout(g):
    from paper_2305_13419_gb300 import twofluid as tf
    with pytest.raises(tf.TFError) as ex:
        g.sync()
    assert ex.value.status == tf.TF_ETIMEOUT


@pytest.mark.parametrize("two", [False, True], ids=["single-step", "two-step"])
def test_zero_polls_latch_a_timeout_and_leave_the_context_usable(two):
    w = W.cpw_small(nsteps=12)
    g = _grid(w, two)
    if two:   # the grid has an interior box for the two-step kernel
        (lo, hi), _ = g.two_step_box()
        assert all(hi[a] > lo[a] for a in range(3))
    g.set_wait_limit(0)
    g.step(6)
    _expect_timeout(g)
    # the device and other grids are unaffected: a new grid steps to the same bits
    ref = _reference(w, 6)
    h = _grid(w, two)
    h.step(6)
    h.sync()
    for c in range(9):
        assert np.array_equal(h.field(c), ref.field(c)), c


def test_default_limit_restored_gives_the_same_bits():
    w = W.cpw_small(nsteps=12)
    ref = _reference(w, 9)
    g = _grid(w, True)
    g.set_wait_limit(0)
    g.set_wait_limit(None)
    g.step(9)
    g.sync()
    for c in range(9):
        assert np.array_equal(g.field(c), ref.field(c)), c


def test_a_timeout_in_a_batch_flags_every_grid_of_the_batch():
    """One CTA of a batched launch works on items of several grids; a wait
    that runs out stops it, so every grid of the batch reports the timeout."""
    from paper_2305_13419_gb300 import twofluid as tf
    ws = W.cpw_batch(count=3, seed=5, sizes=(40, 48))
    grids = [tf.Grid.from_workload(x) for x in ws]
    grids[1].set_wait_limit(0)
    tf.batch_run(grids, 4)
    for g in grids:
        _expect_timeout(g)
    # a fresh batch after it runs clean
    fresh = [tf.Grid.from_workload(x) for x in ws]
    tf.batch_run(fresh, 4)
    for x, g in zip(ws, fresh):
        g.sync()
        ref = _reference(x, 4)
        assert np.array_equal(g.field(0), ref.field(0))
