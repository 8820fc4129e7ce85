"""The project's autotuner: picks, from measured runs on the GPU, the runtime
settings of libtwofluid for a grid and the CTA split of a batch.

Every setting gives the same bits (the step's arithmetic does not depend on
how the work is cut), so the tuner only times.  What it chooses:

  * temporal-block depth per grid: single steps (T = 1) or two steps per
    pass over the interior box (T = 2) with two-step work items of 8, 12 or
    16 planes (tf_set_two_step);
  * for a batch (tf_batch_run): the share of the launch's CTAs each grid
    gets, in proportion to its measured time per step when stepped alone.

The tile shape (32 x 16 columns, 8-plane single-step items) is fixed when the
kernels are compiled; the shapes measured against it are listed in the
design notes.  Results are plain dicts, written to JSON by `save`.
"""
from __future__ import annotations

import json
from typing import Dict, Iterable, List, Sequence

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


def batch_weights(workloads: Sequence, steps: int = 20, warmup: int = 3, device=None) -> List[float]:
    """Measured ms per single step of each workload's grid stepped alone: the
    CTA weights of tf_batch_run."""
    import torch
    from . import twofluid as tf
    out = []
    for w in workloads:
        g = tf.Grid.from_workload(w, device=device)
        g.set_two_step(0)
        g.step(warmup)
        out.append(_time_steps(g, steps))
        g.close()
        del g
        torch.cuda.empty_cache()
    return out


def save(table: Dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load_table(path: str) -> Dict:
    with open(path) as f:
        return json.load(f)
