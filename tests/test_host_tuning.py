"""Host logic of the tuning and measurement layers, with fake grids (no GPU):
the autotuner times every (two-step setting, single-step item length) pair
the grid can use and leaves the fastest set; the bench keys a kernel's ncu
traffic by its launch kind and source hash."""
import json

import pytest

from paper_2305_13419_gb300 import autotune


class FakeGrid:
    """Stands in for twofluid.Grid: records the settings, times a step from a
    table of (two-step planes, item planes) -> ms."""

    def __init__(self, cost, box=((32, 16, 14), (480, 240, 115))):
        self.cost = cost
        self.box = box
        self.two = 24
        self.items = 8
        self.calls = []

    def two_step_box(self):
        return self.box, True

    def set_two_step(self, planes):
        self.two = int(planes)
        self.calls.append(("two", self.two))

    def set_item_planes(self, planes):
        self.items = int(planes)
        self.calls.append(("items", self.items))

    def step(self, n):
        pass

    def sync(self):
        pass

    def step_timed(self, n, with_total=False):
        ms = self.cost[(self.two, self.items)]
        return {"step": (ms, n)}, ms * n


def _cost(best):
    cost = {(p, n): 2.0 + 0.01 * p + 0.001 * n for p in autotune.TWO_STEP_CANDIDATES
            for n in autotune.ITEM_PLANES_CANDIDATES}
    cost[best] = 1.0
    return cost


@pytest.mark.parametrize("best", [(0, 8), (24, 16), (12, 8), (16, 16)])
def test_autotuner_times_every_pair_and_leaves_the_fastest(best):
    g = FakeGrid(_cost(best))
    r = autotune.tune_grid(g, steps=3, warmup=1)
    assert (r["best"], r["item_planes"]) == best
    assert (g.two, g.items) == best                      # the grid is left at the choice
    assert len(r["ms_per_step"]) == len(autotune.TWO_STEP_CANDIDATES) * len(autotune.ITEM_PLANES_CANDIDATES)
    assert r["ms_per_step"][f"{best[0]}/{best[1]}"] == 1.0
    json.dumps(r)                                        # the table is plain JSON


def test_autotuner_skips_two_step_settings_without_a_box():
    g = FakeGrid(_cost((24, 16)), box=((0, 0, 0), (0, 0, 0)))
    r = autotune.tune_grid(g, steps=3, warmup=1)
    assert r["best"] == 0 and r["interior_box"] is None
    assert all(k.startswith("0/") for k in r["ms_per_step"])


def test_class_table_lookup():
    class Wl:
        n = (256, 128, 64)
        bc = ("cpml", "cpml", "cpml")
    table = {autotune.grid_class(Wl): {"best": 16, "item_planes": 16}}
    assert autotune.setting_for(table, Wl) == 16 and autotune.item_planes_for(table, Wl) == 16

    class Other:
        n = (96, 96, 96)
        bc = ("cpml", "cpml", "cpml")
    assert autotune.setting_for(table, Other) == 16 and autotune.item_planes_for(table, Other) == 8


def test_traffic_lookup_keys_and_source_hash(tmp_path, monkeypatch):
    """ncu_traffic answers only for the current step-kernel sources and the
    exact launch kind."""
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "source_hash", lambda: "feedc0de12345678")
    t = {"source_hash": "feedc0de12345678",
         "kernels": {"k_step2": {"w/two-step-24": {"dram_bytes_per_launch": 123}},
                     "k_step": {"w/shell-items-16": {"dram_bytes_per_launch": 45}}}}
    (prof / "traffic.json").write_text(json.dumps(t))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k_step2", "w/two-step-24") == 123
    assert bench.ncu_traffic("k_step2", "w/two-step-16") is None
    assert bench.ncu_traffic("k_step", "w/shell-items-16") == 45
    t["source_hash"] = "0" * 16
    (prof / "traffic.json").write_text(json.dumps(t))
    assert bench.ncu_traffic("k_step2", "w/two-step-24") is None
