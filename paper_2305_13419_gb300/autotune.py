"""The project's autotuner: picks, from measured runs on the GPU, the runtime
settings of libtwofluid per grid and per class of grids.

Every setting gives the same bits (the step's arithmetic does not depend on
how the work is cut), so the tuner only times.  What it chooses:

  * temporal-block depth per grid: single steps (T = 1) or two steps per
    pass over the interior box (T = 2) with two-step work items of 8, 12 or
    16 planes (tf_set_two_step).

A batch (tf_batch_run) needs no split to tune: its grids' work items form
one list that the launch's CTAs share through one counter.

The tile shape (32 x 16 columns, 8-plane single-step items) is fixed when the
kernels are compiled; the shapes measured against it are listed in the
design notes.  Results are plain dicts, written to JSON by `save`.
"""
from __future__ import annotations

import json
from typing import Dict, Iterable

TWO_STEP_CANDIDATES = (0, 8, 12, 16)   # 0: single steps; else planes per two-step work item


def _time_steps(grid, steps: int) -> float:
    """ms per step of `steps` steps of `grid`, CUDA events on its stream."""
    _, total = grid.step_timed(steps, with_total=True)
    grid.sync()
    return total / steps


def tune_grid(grid, steps: int = 20, warmup: int = 4, candidates: Iterable[int] = TWO_STEP_CANDIDATES) -> Dict:
    """Times each candidate temporal-block setting on `grid` (which advances
    by (warmup + steps) steps per candidate), leaves the fastest set and
    returns {"best": planes, "ms_per_step": {planes: ms}} (planes 0 = single
    steps).  Candidates the grid cannot use (no interior box, non-uniform mu)
    time as single steps and are reported as such."""
    (lo, hi), _ = grid.two_step_box()
    usable = all(hi[a] > lo[a] for a in range(3))
    table = {}
    for planes in candidates:
        if planes and not usable:
            continue
        grid.set_two_step(planes)
        grid.step(warmup)
        table[int(planes)] = _time_steps(grid, steps)
    best = min(table, key=table.get)
    grid.set_two_step(best)
    return {"best": best, "ms_per_step": table, "interior_box": [list(lo), list(hi)] if usable else None}


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


def save(table: Dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load_table(path: str) -> Dict:
    with open(path) as f:
        return json.load(f)
