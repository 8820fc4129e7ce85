"""The project's autotuner: picks, from measured runs on the GPU, the runtime
settings of libtwofluid per grid and per class of grids.

Every setting gives the same bits (the step's arithmetic does not depend on
how the work is cut), so the tuner only times.  What it chooses:

  * temporal-block depth per grid: single steps (T = 1) or two steps per
    pass over the interior box (T = 2) with two-step work items of 8 to 24
    planes (tf_set_two_step);
  * the single-step kernel's work-item length, 8 or 16 planes
    (tf_set_item_planes): long items on large grids, short ones where a
    grid has few items per CTA.

A batch (tf_batch_run) needs no split to tune: its grids' work items form
one list that the launch's CTAs share through one counter.

The tile shape (32 x 16 columns, 8-plane single-step items) is fixed when the
kernels are compiled; the shapes measured against it are listed in the
design notes.  Results are plain dicts, written to JSON by `save`.
"""
from __future__ import annotations

import json
from typing import Dict, Iterable

TWO_STEP_CANDIDATES = (0, 8, 12, 16, 20, 24)   # 0: single steps; else planes per two-step work item
ITEM_PLANES_CANDIDATES = (8, 16)       # planes per single-step work item


def _time_steps(grid, steps: int) -> float:
    """ms per step of `steps` steps of `grid`, CUDA events on its stream."""
    _, total = grid.step_timed(steps, with_total=True)
    grid.sync()
    return total / steps


def tune_grid(grid, steps: int = 20, warmup: int = 4, candidates: Iterable[int] = TWO_STEP_CANDIDATES,
              item_planes: Iterable[int] = ITEM_PLANES_CANDIDATES) -> Dict:
    """Times each candidate pair (temporal-block setting, single-step item
    length) on `grid` (which advances by (warmup + steps) steps per
    candidate), leaves the fastest set and returns {"best": planes,
    "item_planes": n, "ms_per_step": {"planes/n": ms}} (planes 0 = single
    steps).  Two-step candidates the grid cannot use (no interior box) are
    skipped."""
    (lo, hi), _ = grid.two_step_box()
    usable = all(hi[a] > lo[a] for a in range(3))
    table = {}
    for ip in item_planes:
        grid.set_item_planes(ip)
        for planes in candidates:
            if planes and not usable:
                continue
            grid.set_two_step(planes)
            grid.step(warmup)
            table[(int(planes), int(ip))] = _time_steps(grid, steps)
    best, best_ip = min(table, key=table.get)
    grid.set_two_step(best)
    grid.set_item_planes(best_ip)
    return {"best": best, "item_planes": best_ip, "ms_per_step": {f"{p}/{n}": v for (p, n), v in table.items()},
            "interior_box": [list(lo), list(hi)] if usable else None}


def grid_class(w) -> str:
    """Class of a workload for tuning: its cell counts and boundary kinds."""
    return "x".join(map(str, w.n)) + "-" + "-".join(w.bc)


def tune_classes(workloads, steps: int = 20, device=None) -> Dict:
    """Tunes one grid per class of `workloads` (the first of each class) and
    returns {class: tune_grid result}, ready for `save`."""
    import torch
    from . import twofluid as tf
    table = {}
    for w in workloads:
        key = grid_class(w)
        if key in table:
            continue
        g = tf.Grid.from_workload(w, device=device)
        table[key] = tune_grid(g, steps=steps)
        g.close()
        del g
        torch.cuda.empty_cache()
    return table


def setting_for(table: Dict, w, default: int = 16) -> int:
    """The tuned two-step setting of a workload's class (default if untuned)."""
    r = table.get(grid_class(w))
    return int(r["best"]) if r else default


def item_planes_for(table: Dict, w, default: int = 8) -> int:
    """The tuned single-step item length of a workload's class (default if untuned)."""
    r = table.get(grid_class(w))
    return int(r.get("item_planes", default)) if r else default


def save(table: Dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load_table(path: str) -> Dict:
    with open(path) as f:
        return json.load(f)
