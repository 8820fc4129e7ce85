"""Full-size parity in the launch configuration the benchmark times: the
512 x 256 x 128 and 1024 x 512 x 256 CPW grids stepped through the C ABI,
checked at sampled points against the FP64 oracle run on light-cone crops.

After N steps a value depends only on the initial state within N + 1 cells
(one cell per step in each direction), so each sample point is recomputed by
the oracle on a crop that keeps every real boundary the cone reaches and is
closed by PEC walls N + 4 cells away elsewhere.  The initial state is random
within N + 1 cells of the sample points and zero elsewhere, so the crop and
the full grid start from the same data on the whole cone."""
import numpy as np
import pytest

from oracle import stepper
from paper_2305_13419_gb300 import workloads as W
from parity_util import FIELD_TOL, FAMILIES, crop_workload, local_state

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

NSTEPS = 24
SEED = 77


def _samples(w):
    n = w.n
    s = lambda fx, fy, fz: (int(fx * n[0]), int(fy * n[1]), int(fz * n[2]))
    notes = w.notes
    pts = [s(0.5, 0.5, 0.5), s(0.01, 0.01, 0.02), s(0.99, 0.99, 0.98), s(0.008, 0.5, 0.5),
           s(0.5, 0.985, 0.5), s(0.5, 0.5, 0.95)]
    # metal film edge, source, probes
    z_film = w.sources[0].lo[2]
    pts += [(w.probes[0].p[0], w.probes[0].p[1], z_film), tuple(w.sources[0].lo),
            (w.probes[1].p[0] + 3, w.sources[1].lo[1] - 1, z_film - 2),
            (n[0] // 3, w.sources[0].hi[1] + 2, z_film + 1)]
    return pts


def _full_state(w, centres, radius):
    dims = w.storage_dims()
    shape = (dims[2], dims[1], dims[0])
    st = {}
    for c in range(9):
        a = np.zeros(shape, np.float32)
        for ctr in centres:
            lo = [max(ctr[i] - radius, 0) for i in range(3)]
            hi = [min(ctr[i] + radius + 1, dims[i]) for i in range(3)]
            v = W.counter_uniform(SEED, c, dims, lo, hi) * W.FIELD_SCALE[c]
            a[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = v
        st[c] = a
    return st


@pytest.mark.parametrize("cfg", ["cpw", "cpw_large"])
def test_full_size_light_cone(cfg):
    from paper_2305_13419_gb300 import twofluid as tf
    w = W.cpw() if cfg == "cpw" else W.cpw_large()
    centres = _samples(w)
    dims = w.storage_dims()
    r_rand = NSTEPS + 1
    g = tf.Grid.from_workload(w)
    st = _full_state(w, centres, r_rand)
    for c in range(9):
        g.set_field(c, st[c])
    del st
    g.step(NSTEPS)
    g.sync()
    gpu = [g.field(c) for c in range(9)]
    g.close()
    diff2 = {name: 0.0 for name, _ in FAMILIES}
    ref2 = {name: 0.0 for name, _ in FAMILIES}
    for p in centres:
        crop = crop_workload(w, p, NSTEPS + 4)
        cw = crop.workload
        o = stepper.Grid.from_workload(cw)
        Nl = o.N
        loc = local_state(SEED, dims, centres, r_rand, crop.lo, Nl)
        for c in range(9):
            o.set_field(c, loc[c].astype(np.float32).astype(np.float64))
        o.step(NSTEPS)
        # 3 x 3 x 3 points around p, in crop coordinates
        sl_l = tuple(slice(max(p[a] - crop.lo[a] - 1, 0), p[a] - crop.lo[a] + 2) for a in (2, 1, 0))
        sl_g = tuple(slice(crop.lo[2 - i] + sl_l[i].start, crop.lo[2 - i] + sl_l[i].stop) for i in range(3))
        for name, f in FAMILIES:
            for c in range(f, f + 3):
                a = gpu[c][sl_g].astype(np.float64)
                b = o.field(c)[sl_l]
                diff2[name] += float(np.sum((a - b) ** 2))
                ref2[name] += float(np.sum(b * b))
    for name, _ in FAMILIES:
        assert ref2[name] > 0, name
        err = np.sqrt(diff2[name] / ref2[name])
        assert err <= FIELD_TOL, (name, err)
