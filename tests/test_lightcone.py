"""The light-cone crops used by the full-size GPU parity test reproduce the
full problem exactly: the oracle on the whole grid and the oracle on each
crop agree at the sample points after N steps (CPU only)."""
import numpy as np
import pytest

from oracle import stepper
from paper_2305_13419_gb300 import workloads as W
from parity_util import FAMILIES, crop_workload, local_state

NSTEPS = 10
SEED = 5


@pytest.mark.parametrize("wl", ["cpw_small", "box"])
def test_crops_match_full_oracle(wl):
    if wl == "cpw_small":
        w = W.cpw_small(n=(72, 48, 36), pml=6, margin=2, substrate_cells=6, film_cells=2, strip_w=6, gap_w=3)
        centres = [(36, 24, 18), (2, 2, 2), (70, 46, 35), (w.sources[0].lo[0], w.sources[0].lo[1], 15),
                   (20, 40, 3)]
    else:
        w = W.random_box(n=(40, 9, 44), bc=("pec", "periodic", "cpml"), seed=4, cpml_cells=5)
        centres = [(20, 4, 22), (1, 0, 1), (39, 8, 43), (25, 3, 6)]
    dims = w.storage_dims()
    r_rand = NSTEPS + 1
    full = stepper.Grid.from_workload(w)
    st = local_state(SEED, dims, centres, r_rand, (0, 0, 0), dims)
    for c in range(9):
        full.set_field(c, st[c])
    full.step(NSTEPS)
    ref = [full.field(c) for c in range(9)]
    for p in centres:
        crop = crop_workload(w, p, NSTEPS + 4)
        o = stepper.Grid.from_workload(crop.workload)
        loc = local_state(SEED, dims, centres, r_rand, crop.lo, o.N)
        for c in range(9):
            o.set_field(c, loc[c])
        o.step(NSTEPS)
        sl_l = tuple(slice(max(p[a] - crop.lo[a] - 1, 0), p[a] - crop.lo[a] + 2) for a in (2, 1, 0))
        sl_g = tuple(slice(crop.lo[2 - i] + sl_l[i].start, crop.lo[2 - i] + sl_l[i].stop) for i in range(3))
        for name, f in FAMILIES:
            for c in range(f, f + 3):
                a, b = ref[c][sl_g], o.field(c)[sl_l]
                scale = max(np.max(np.abs(ref[c])), 1e-300)
                assert np.max(np.abs(a - b)) <= 1e-12 * scale, (p, c)
