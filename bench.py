"""Benchmark: Gcell-updates/s of the two-fluid Yee step on the large CPW
resonator (1024 x 512 x 256 cells = 134 M, CPML 16, lambda_L = 4 cells,
London + Ohmic films, soft source, two 64-frequency probe DFTs), plus the
HBM roofline fraction of the dominant kernel, an end-to-end number through
the C ABI with host buffers, the FP64 CPU oracle on a block of the same
workload as the baseline, and the other workloads (512 x 256 x 128 CPW,
4 x 4 x 2048 slab, adjoint, batch) beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as N independent replicas (one resonator variant
per rank, no collective on the data path); `value` is the aggregate.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s & HBM roofline fraction; batched and adjoint vs plain step"
UNIT = "Gcell-updates/s"
L2_BYTES = 129 * 2 ** 20


# ------------------------------------------------------------------ ranks
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist if ws > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_seed(rank: int) -> int:
    """Replica r draws its own sigma map (a different resonator variant)."""
    from paper_2305_13419_gb300 import workloads as W
    return W.BASE_SEED + 5 + 1000 * rank


WORKLOAD = "large"


def headline_workload(rank: int = 0):
    """The 1024 x 512 x 256 CPW (the largest single-GPU configuration); with
    --workload cpw the 512 x 256 x 128 CPW instead (small profiling runs)."""
    from paper_2305_13419_gb300 import workloads as W
    if WORKLOAD == "cpw":
        return W.cpw(seed=W.BASE_SEED + 2 + 1000 * rank)
    return W.cpw_large(seed=replica_seed(rank))


def aggregate(cells_per_rank, steps, max_ms, world):
    """Whole-job throughput: all ranks' cell-updates over the slowest rank's time."""
    return cells_per_rank * steps * world / (max_ms * 1e-3) / 1e9


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline
TILE_SX, TILE_SY = 32, 16   # owned columns per tile of the fused step kernel


def algorithmic_bytes(w, N, box=None):
    """Algorithmic HBM bytes of the fused step kernels, each array element
    moved once per launch (FP32):
      48 B per storage point   E read + write, B read + write;
      12 B per point of a tile-plane whose cells are not all alike
                               (eps, sigma, kappa maps; uniform tile-planes use
                               one precomputed record instead);
       8 B per superconducting edge (Js read + write);
      32 B per CPML slab point and slab axis (two psi_B read old + write new,
                               two psi_E read + write).
    `box` ((lo, hi) in storage points): the two-step kernel's interior box;
    then "box" holds the bytes of one two-step launch (the box's points, two
    steps per pass) and "rest" those of one single-step launch over the
    other points."""
    # points the kernel owns: cells of a walled axis, all points of a periodic
    # one, planes below the top wall along z
    own = [N[a] if w.bc[a] == "periodic" else w.n[a] for a in range(3)]
    inbox = np.zeros((own[2], own[1], own[0]), bool)
    if box is not None:
        (lo, hi) = box
        inbox[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = True
    pts = own[0] * own[1] * own[2]
    pts_box = int(inbox.sum())
    psi = 0
    for a in range(3):
        if w.bc[a] != "cpml":
            continue
        L = w.cpml[a].ncells
        psi += (2 * L) * (pts // own[a])
    # superconducting edges: an E_c edge is SC if any of its four cells is
    sc = w.lambda_L > 0
    sc_edges = sc_box = 0
    for c in range(3):
        m = sc.copy()
        for ax in [2 - b for b in range(3) if b != c]:
            m = m | np.roll(m, 1, axis=ax)
        sc_edges += int(m.sum())
        mm = m[:own[2], :own[1], :own[0]]
        sc_box += int((mm & inbox[:mm.shape[0], :mm.shape[1], :mm.shape[2]]).sum())
    # points in non-uniform tile-planes (cells x0-1..x0+31, y0-1..y0+15, k-1..k)
    per = [w.bc[a] == "periodic" for a in range(3)]
    key = np.stack([w.eps_r, w.sigma, w.lambda_L, w.mu_r], axis=-1)
    kidx = np.arange(own[2])
    kz = [np.clip(kidx - 1, 0, w.n[2] - 1) if not per[2] else (kidx - 1) % w.n[2],
          np.clip(kidx, 0, w.n[2] - 1)]
    nonuni = nonuni_box = 0
    for by in range((N[1] + TILE_SY - 1) // TILE_SY):
        ys = np.arange(by * TILE_SY - 1, by * TILE_SY + TILE_SY)   # y0-1 .. y0+15
        ys = ys % w.n[1] if per[1] else np.clip(ys, 0, w.n[1] - 1)
        own_y = min(TILE_SY, own[1] - by * TILE_SY)
        for bx in range((own[0] + TILE_SX - 1) // TILE_SX):
            xs = np.arange(bx * TILE_SX - 1, bx * TILE_SX + TILE_SX)
            xs = xs % w.n[0] if per[0] else np.clip(xs, 0, w.n[0] - 1)
            own_x = min(TILE_SX, own[0] - bx * TILE_SX)
            blk = key[:, ys][:, :, xs]                       # [nz][ty][tx][4]
            ref = blk[:, :1, :1]
            same_plane = np.all(blk == ref, axis=(1, 2, 3))  # per cell plane
            refk = ref[:, 0, 0]
            uni = same_plane[kz[0]] & same_plane[kz[1]] & np.all(refk[kz[0]] == refk[kz[1]], axis=-1)
            nonuni += int((~uni).sum()) * own_x * own_y
            if box is not None and box[0][0] <= bx * TILE_SX < box[1][0] and box[0][1] <= by * TILE_SY < box[1][1]:
                nonuni_box += int((~uni[box[0][2]:box[1][2]]).sum()) * own_x * own_y
    step = 48 * pts + 12 * nonuni + 8 * sc_edges + 32 * psi
    out = {"step": step, "points": pts, "sc_edges": sc_edges, "psi_points": psi, "nonuniform_points": nonuni,
           "dense_equivalent": 84 * pts + 32 * psi}
    if box is not None:
        out["box"] = 48 * pts_box + 12 * nonuni_box + 8 * sc_box
        out["box_points"] = pts_box
        out["rest"] = step - out["box"]
        out["rest_points"] = pts - pts_box
    return out


def source_hash():
    """Hash of the sources that define the step kernels (single-step and
    two-step kernels, their shared headers)."""
    h = hashlib.sha256()
    for f in ("tf_step.cu", "tf_step2.cu", "tf_internal.cuh", "tf_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2305_13419_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """dram bytes per launch of `kernel` on `workload` from the committed ncu
    summary, if it was taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except ValueError:
        return None
    if d.get("source_hash") != source_hash():
        return None
    k = d.get("kernels", {}).get(kernel, {}).get(workload)
    return None if k is None else k.get("dram_bytes_per_launch")


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["hbm_gbs"]), "measured"
        except (ValueError, KeyError):
            pass
    return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU baseline
def cpu_baseline(w, budget_s=10.0):
    """The FP64 oracle as it stands, on this host's cores, stepping the same
    workload from rest until `budget_s` of stepping has elapsed."""
    from oracle import stepper
    threads = stepper.set_threads(os.cpu_count() or 1)
    g = stepper.Grid.from_workload(w)
    g.step(1)                       # first step outside the clock (psi init, page faults)
    t0 = time.perf_counter()
    n = 0
    while True:
        g.step(1)
        n += 1
        if time.perf_counter() - t0 >= budget_s and n >= 2:
            break
    el = time.perf_counter() - t0
    return {"value": w.ncells * n / el / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{w.name}: {n} FP64 oracle steps after one untimed step ({el:.1f} s)"}


def large_block(nx=256, ny=256, nz=128):
    """A cell block of the 1024 x 512 x 256 CPW cut around the in-port /
    resonator gap at the film plane, closed with PEC walls: the bounded
    sample the FP64 oracle steps on the host cores."""
    from paper_2305_13419_gb300 import workloads as W
    w = headline_workload()
    x0, y0 = 256 - nx // 2 + 128, 256 - ny // 2
    sl = (slice(0, nz), slice(y0, y0 + ny), slice(x0, x0 + nx))
    return W.Workload(name=f"cpw-1024x512x256[{x0}:{x0 + nx},{y0}:{y0 + ny},0:{nz}]", n=(nx, ny, nz), d=w.d,
                      theta=w.theta, bc=("pec", "pec", "pec"), eps_r=np.ascontiguousarray(w.eps_r[sl]),
                      mu_r=np.ascontiguousarray(w.mu_r[sl]), lambda_L=np.ascontiguousarray(w.lambda_L[sl]),
                      sigma=np.ascontiguousarray(w.sigma[sl]), courant=w.courant)


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    from oracle import stepper
    w = large_block(128, 128, 64)
    threads = stepper.set_threads(os.cpu_count() or 1)
    g = stepper.Grid.from_workload(w)
    g.step(args.warmup)
    t0 = time.perf_counter()
    g.step(args.steps)
    el = time.perf_counter() - t0
    v = w.ncells * args.steps / el / 1e9
    sample = f"{w.name}: {args.steps} FP64 oracle steps on a 1/128 block of the workload"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_block(state_bytes=None):
    if WORKLOAD == "cpw":
        c = {"workload": "cpw-512x256x128: CPW resonator, CPML 12, lambda_L = 3 cells, sigma_n ~ U[0,1e6] S/m, "
                         "theta = 1, Courant 0.95, +/- Gaussian-sine port source, 2 probes x 64-frequency DFT",
             "cells": 512 * 256 * 128, "parallelism": "replicas (independent resonator per GPU)"}
    else:
        c = {"workload": "cpw-1024x512x256: CPW resonator, CPML 16, lambda_L = 4 cells, sigma_n ~ U[0,1e6] S/m, "
                         "theta = 1, Courant 0.95, +/- Gaussian-sine port source, 2 probes x 64-frequency DFT",
             "cells": 1024 * 512 * 256, "parallelism": "replicas (independent resonator per GPU)"}
    if state_bytes:
        c["l2"] = f"inputs larger than L2: {state_bytes / 2**20:.0f} MiB of fields and maps per step > 129 MiB"
    return c


def roofline_of(w, g, kt, planes=24, item_planes=8):
    """Roofline of the step kernels from their algorithmic bytes per launch
    over their mean event-timed launch durations, against the measured HBM
    peak.  With two-step passes the two-step kernel (the interior box, two
    steps per launch) and the single-step kernel (the rest of the grid, one
    step per launch) are listed apart; the dominant one (larger share of the
    run's kernel time) heads the object.  `planes`, `item_planes`: the
    two-step and single-step work-item lengths the run used (the ncu
    traffic is keyed by them)."""
    peak, peak_kind = hbm_peak()
    (lo, hi), active = g.two_step_box()
    two = "step2" in kt
    ab = algorithmic_bytes(w, g.N, (lo, hi) if two else None)
    kernels = {}
    if two:
        kernels["k_step2"] = {"algorithmic_bytes": ab["box"], "points": ab["box_points"], "steps_per_launch": 2,
                              "ms": kt["step2"][0], "launches": kt["step2"][1]}
        kernels["k_step"] = {"algorithmic_bytes": ab["rest"], "points": ab["rest_points"], "steps_per_launch": 1,
                             "ms": kt["step"][0], "launches": kt["step"][1]}
    else:
        kernels["k_step"] = {"algorithmic_bytes": ab["step"], "points": ab["points"], "steps_per_launch": 1,
                             "ms": kt["step"][0], "launches": kt["step"][1]}
    # ncu traffic keys: the launch kind on the workload
    keys = {"k_step2": f"{w.name}/two-step-{planes}",
            "k_step": f"{w.name}/shell-items-{item_planes}" if two else f"{w.name}/items-{item_planes}"}
    for k, v in kernels.items():
        v["achieved_GBps"] = v["algorithmic_bytes"] / (v["ms"] * 1e-3) / 1e9
        v["frac"] = v["achieved_GBps"] / peak
        v["share"] = v["ms"] * v["launches"]
        v["traffic"] = ncu_traffic(k, keys[k])
    tot = sum(v["share"] for v in kernels.values())
    for v in kernels.values():
        v["share"] /= tot
    dom = max(kernels, key=lambda k: kernels[k]["share"])
    d = kernels[dom]
    # effective bandwidth: the dense one-pass byte count of every step the run
    # made (a two-step pass launches the single-step kernel twice, so the steps
    # equal the single-step kernel's launches), over the kernels' time
    nsteps = max(1, kernels["k_step"]["launches"])
    ms_per_step = sum(v["ms"] * v["launches"] for v in kernels.values()) / nsteps
    return ab, {"bound": "hbm", "kernel": dom, "achieved": d["achieved_GBps"], "peak": peak, "unit": "GB/s",
                "frac": d["frac"], "traffic": d["traffic"], "algorithmic_bytes": d["algorithmic_bytes"],
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                "kernels": kernels,
                "dense_equivalent_GBps": ab["dense_equivalent"] / (ms_per_step * 1e-3) / 1e9,
                "effective_frac_dense_equivalent": ab["dense_equivalent"] / (ms_per_step * 1e-3) / 1e9 / peak,
                "kernel_ms": {k: v[0] for k, v in kt.items()}}


# ------------------------------------------------------------------ our arm
def run_ours(args, ws, rank, local):
    import torch
    from paper_2305_13419_gb300 import twofluid as tf
    from paper_2305_13419_gb300 import workloads as W

    dist = init_dist(ws, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = headline_workload(rank)
    g = tf.Grid.from_workload(w)
    tuning = None
    if args.two_step == "off":
        g.set_two_step(0)
    elif not args.no_autotune:   # the temporal-block depth and item length, from measured runs
        from paper_2305_13419_gb300 import autotune
        tuning = autotune.tune_grid(g, steps=args.autotune_steps)
    if args.item_planes:   # a fixed single-step item length (reproducible profiling runs)
        g.set_item_planes(args.item_planes)
        if tuning is not None:
            tuning["item_planes"] = args.item_planes
    N = g.N

    # device-timed throughput: inputs resident in HBM, K steps between
    # barriers; CUDA events on the grid's stream around every launch, so the
    # whole run and the kernel's own durations come from the same launches
    g.step(args.warmup)
    g.sync()
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        kt, ms = g.step_timed(args.steps, with_total=True)
        torch.cuda.synchronize()
    barrier(dist)
    g.sync()
    ms_max = max_over_ranks(dist, ms, dev)
    value = aggregate(w.ncells, args.steps, ms_max, ws)
    ab, roof = roofline_of(w, g, kt, planes=tuning["best"] if tuning and tuning["best"] else 24,
                           item_planes=tuning["item_planes"] if tuning else (args.item_planes or 8))
    state_bytes = (9 + 3) * 4 * ab["points"]
    launches = sum(v[1] for v in kt.values())
    g.close()
    del g
    torch.cuda.empty_cache()

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, w, dev, tuning)

    base = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(large_block(), budget_s=args.cpu_budget)
        base["sample"] += " (a 256 x 256 x 128 block of the 1024 x 512 x 256 workload, PEC-closed)"

    adj = batch = extra = None
    w_name = w.name
    del w
    if rank == 0 and not args.no_configs:
        two = args.two_step != "off"
        at = 0 if args.no_autotune else args.autotune_steps
        extra = {"cpw-512x256x128": run_config(W.cpw(), args.cpw_steps, 20, two, at),
                 "slab-4x4x2048": run_config(W.slab(), 4000, 50, two, 0)}
    plain_small = extra["cpw-512x256x128"]["gcell_updates_per_s"] if extra else None
    if rank == 0 and not args.no_adjoint:
        adj = run_adjoint(args)
    if rank == 0 and not args.no_batch:
        batch = run_batch(args, plain_small or value / ws, "cpw-512x256x128" if plain_small else w_name)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_block(state_bytes), "roofline": roof, "cpu_baseline": base, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary(), "autotune": tuning, "adjoint": adj,
                "batched": batch, "other_configs": extra}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_adjoint(args):
    """Gradient of |X(f0)|^2 with respect to every cell's eps_r and lambda_L
    on the 256 x 128 x 64 adjoint CPW by the discrete adjoint (forward with
    checkpoints every --adjoint-segment steps (256), per-segment recompute, transposed steps),
    timed whole, against the plain step on the same grid."""
    import time
    import torch
    from paper_2305_13419_gb300 import twofluid as tf
    from paper_2305_13419_gb300 import workloads as W
    w = W.cpw_adjoint(nsteps=args.adjoint_steps)
    g = tf.Grid.from_workload(w)
    tuning = None
    if not args.no_autotune:   # the plain step at its best setting; the adjoint's forward runs use it too
        from paper_2305_13419_gb300 import autotune
        tuning = autotune.tune_grid(g, steps=args.autotune_steps)
    g.step(20)
    _, tot = g.step_timed(200, with_total=True)
    g.sync()
    plain = tot / 200
    g.close()
    del g
    g = tf.Grid.from_workload(w)
    if tuning is not None:
        g.set_two_step(tuning["best"])
        g.set_item_planes(tuning["item_planes"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, ge, gl = g.adjoint(args.adjoint_steps, 0, 0, segment=args.adjoint_segment)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    per = ms / args.adjoint_steps
    return {"workload": w.name, "steps": args.adjoint_steps, "segment": args.adjoint_segment, "ms": ms,
            "ms_per_step": per,
            "plain_ms_per_step": plain, "vs_plain_step": per / plain, "autotune": tuning,
            "gcell_updates_per_s": w.ncells * args.adjoint_steps / (ms * 1e-3) / 1e9,
            "objective": J, "grad_eps_absmax": float(ge.abs().max()), "grad_lambda_absmax": float(gl.abs().max()),
            "includes": "forward with checkpoints, per-segment recompute, adjoint steps, gradient reduction"}


def run_batch(args, plain_gcells, plain_workload="cpw-512x256x128"):
    """The batched workload: 64 CPW variants with axes from {96, 128, 160}.
    Headline: tf_batch_run, one launch per step over all 64 grids (one work
    list over all grids' items), 64 steps per CUDA graph, timed with CUDA
    events on its stream; beside it tf_batch_step (per-grid launches spread
    over 8 streams)."""
    import time
    import torch
    from paper_2305_13419_gb300 import twofluid as tf
    from paper_2305_13419_gb300 import workloads as W
    ws = W.cpw_batch()
    cells = sum(w.ncells for w in ws)
    out = {"grids": len(ws), "cells": cells, "steps": args.batch_steps, "sizes": [96, 128, 160]}
    grids = [tf.Grid.from_workload(w) for w in ws]
    # algorithmic bytes of one batched launch: every grid's one-pass bytes
    ab = sum(algorithmic_bytes(w, g.N)["step"] for w, g in zip(ws, grids))
    tf.batch_run(grids, 10)
    torch.cuda.synchronize()
    st = grids[0].stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    tf.batch_run(grids, args.batch_steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    for gg in grids:
        gg.sync()
        gg.close()
    del grids
    torch.cuda.empty_cache()
    peak, peak_kind = hbm_peak()
    mps = ms / args.batch_steps
    out["one_launch"] = {"ms_per_step": mps,
                         "gcell_updates_per_s": cells * args.batch_steps / (ms * 1e-3) / 1e9,
                         "timing": "CUDA events on the batch's stream around tf_batch_run (includes its set-up "
                                   "uploads and graph capture)",
                         "roofline": {"bound": "hbm", "kernel": "k_step_t<batch>", "algorithmic_bytes": ab,
                                      "achieved": ab / (mps * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                                      "frac": ab / (mps * 1e-3) / 1e9 / peak,
                                      "traffic": ncu_traffic("k_step_batch", "batch-64-cpw"),
                                      "peak_source": peak_kind}}
    streams = [torch.cuda.Stream() for _ in range(8)]
    grids = [tf.Grid.from_workload(w, stream=streams[i % 8]) for i, w in enumerate(ws)]
    for gg in grids:   # single steps, as in the batched launch (the autotuner's choice on grids this small)
        gg.set_two_step(0)
    tf.batch_step(grids, 10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tf.batch_step(grids, args.batch_steps)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    for gg in grids:
        gg.sync()
        gg.close()
    del grids
    torch.cuda.empty_cache()
    out["streams8"] = {"ms_per_step": ms / args.batch_steps,
                       "gcell_updates_per_s": cells * args.batch_steps / (ms * 1e-3) / 1e9,
                       "timing": "host wall clock around the enqueue of all steps, device synchronised on both sides"}
    out["gcell_updates_per_s"] = out["one_launch"]["gcell_updates_per_s"]
    out["vs_plain_step"] = out["gcell_updates_per_s"] / plain_gcells
    out["plain_step"] = {"workload": plain_workload, "gcell_updates_per_s": plain_gcells}
    return out


def run_batch_singles(args):
    """The batch's grids stepped one at a time (each alone on the GPU, single
    steps): the per-grid rate that the batched stepping is compared with."""
    import time
    import torch
    from paper_2305_13419_gb300 import twofluid as tf
    from paper_2305_13419_gb300 import workloads as W
    rows, cells, secs = [], 0, 0.0
    for w in W.cpw_batch()[:args.batch_singles]:
        g = tf.Grid.from_workload(w)
        g.set_two_step(0)   # single steps, as in the batched launch
        g.step(20)
        g.sync()
        t0 = time.perf_counter()
        g.step(args.batch_steps)
        g.sync()
        dt = (time.perf_counter() - t0) / args.batch_steps
        rows.append({"grid": w.name, "ms_per_step": dt * 1e3, "gcell_updates_per_s": w.ncells / dt / 1e9})
        cells += w.ncells
        secs += dt
        g.close()
        del g
        torch.cuda.empty_cache()
    print(json.dumps({"measure": "batch grids stepped one at a time", "steps": args.batch_steps, "grids": rows,
                      "aggregate_gcell_updates_per_s": cells / secs / 1e9}), flush=True)
    return 0


def run_batch_overhead(args):
    """The batched kernel against the single-grid kernel on the same grid:
    tf_batch_run of a one-grid list and tf_step (single steps), each timed
    with CUDA events on the grid's stream, on the 512 x 256 x 128 and
    1024 x 512 x 256 CPWs.  One JSON line."""
    import torch
    from paper_2305_13419_gb300 import twofluid as tf
    from paper_2305_13419_gb300 import workloads as W
    rows = []
    for w in (W.cpw(), W.cpw_large()):
        g = tf.Grid.from_workload(w)
        g.set_two_step(0)
        g.step(6)
        g.sync()
        st = g.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 256
        e0.record(st)
        g.step(n)
        e1.record(st)
        torch.cuda.synchronize()
        single = e0.elapsed_time(e1) / n
        tf.batch_run([g], 66)
        torch.cuda.synchronize()
        e0.record(st)
        tf.batch_run([g], n)
        e1.record(st)
        torch.cuda.synchronize()
        batched = e0.elapsed_time(e1) / n
        g.sync()
        rows.append({"grid": w.name, "single_grid_kernel_ms_per_step": single, "batched_kernel_ms_per_step": batched,
                     "ratio": batched / single})
        g.close()
        del g
        torch.cuda.empty_cache()
    print(json.dumps({"measure": "batched kernel on one grid vs the single-grid kernel", "steps": 256,
                      "grids": rows}), flush=True)
    return 0


def run_config(w, steps, warmup=5, two_step=True, autotune_steps=0):
    """GPU throughput of the plain step on one workload: the whole run and
    the step kernel's own launches timed with CUDA events on the handle's
    stream over the same launches; the kernel's algorithmic bytes over its
    mean launch time give the roofline fraction."""
    import torch
    from paper_2305_13419_gb300 import twofluid as tf
    g = tf.Grid.from_workload(w)
    tuning = None
    if not two_step:
        g.set_two_step(0)
    elif autotune_steps:
        from paper_2305_13419_gb300 import autotune
        tuning = autotune.tune_grid(g, steps=autotune_steps)
    g.step(warmup)
    g.sync()
    torch.cuda.synchronize()
    kt, ms = g.step_timed(steps, with_total=True)
    g.sync()
    _, roof = roofline_of(w, g, kt, planes=tuning["best"] if tuning and tuning["best"] else 24,
                          item_planes=tuning["item_planes"] if tuning else 8)
    g.close()
    del g
    torch.cuda.empty_cache()
    return {"workload": w.name, "cells": w.ncells, "steps": steps, "ms_per_step": ms / steps,
            "gcell_updates_per_s": w.ncells * steps / (ms * 1e-3) / 1e9, "roofline": roof, "autotune": tuning}


def run_all_configs(args):
    """Every config of the study side by side: GPU throughput (plain step;
    adjoint and batch as in the default line) and the FP64 oracle on this
    host's cores over a bounded sample of the same workload.  One JSON line."""
    from oracle import stepper
    from paper_2305_13419_gb300 import workloads as W
    out = {}
    slab = W.slab()
    out["slab-4x4x2048"] = {"gpu": run_config(slab, 4000, 50), "cpu_oracle": cpu_baseline(slab, budget_s=5.0)}
    cpw = W.cpw()
    out["cpw-512x256x128"] = {"gpu": run_config(cpw, 2000, 20), "cpu_oracle": cpu_baseline(cpw, budget_s=10.0)}
    plain = out["cpw-512x256x128"]["gpu"]["gcell_updates_per_s"]
    out["batch-64-cpw"] = {"gpu": run_batch(args, plain),
                      "cpu_oracle": cpu_baseline(W.cpw_batch(count=1, sizes=(128,))[0], budget_s=10.0)}
    adj_w = W.cpw_adjoint()
    cpu_adj = cpu_baseline(adj_w, budget_s=10.0)
    # the oracle adjoint (serial transposes) over a short window of the same grid
    g = stepper.Grid.from_workload(adj_w, with_probes=False)
    pr = adj_w.probes[0]
    t0 = time.perf_counter()
    g.adjoint_run(16, pr.comp, pr.p, float(pr.freqs[0]), 0)
    el = time.perf_counter() - t0
    cpu_adj["adjoint_forward_plus_backward_gcell_updates_per_s"] = adj_w.ncells * 16 / el / 1e9
    out["adjoint-cpw-256x128x64"] = {"gpu": run_adjoint(args), "cpu_oracle": cpu_adj}
    large = W.cpw_large()
    sl = (slice(0, 128), slice(128, 384), slice(256, 512))
    block = W.Workload(name="cpw-1024x512x256[256:512,128:384,0:128]", n=(256, 256, 128), d=large.d,
                       theta=large.theta, bc=("pec", "pec", "pec"), eps_r=np.ascontiguousarray(large.eps_r[sl]),
                       mu_r=np.ascontiguousarray(large.mu_r[sl]), lambda_L=np.ascontiguousarray(large.lambda_L[sl]),
                       sigma=np.ascontiguousarray(large.sigma[sl]), courant=large.courant)
    out["cpw-1024x512x256"] = {"gpu": run_config(large, args.large_steps, 5), "cpu_oracle": cpu_baseline(block, budget_s=10.0)}
    print(json.dumps({"all_configs": out}), flush=True)
    return 0


def run_precision_study(args):
    """FP32 fused step against the FP64 stepper on the same CPW over a long
    run: relative L2 of each field family (against the family's peak norm
    over the run, as the ring-down decays) at checkpoints, and of both
    probes' spectra at the end.  Prints one JSON line."""
    import numpy as np
    import torch
    from paper_2305_13419_gb300 import twofluid as tf
    from paper_2305_13419_gb300 import workloads as W
    w = W.cpw_large(nsteps=args.fp64_study) if args.study_workload == "cpw_large" else W.cpw(nsteps=args.fp64_study)
    g32 = tf.Grid.from_workload(w)
    g64 = tf.Grid64.from_workload(w)
    fams = (("E", 0), ("B", 3), ("Js", 6))
    peak = {k: 0.0 for k, _ in fams}
    rows = []
    marks = sorted(set(int(round(args.fp64_study * f)) for f in (0.1, 0.25, 0.5, 0.75, 1.0)))
    done = 0
    t32 = t64 = 0.0
    for m in marks:
        for gg, which in ((g32, 32), (g64, 64)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            gg.step(m - done)
            gg.sync()
            dt_ = time.perf_counter() - t0
            if which == 32:
                t32 += dt_
            else:
                t64 += dt_
        done = m
        row = {"step": m}
        for name, f in fams:
            d2 = r2 = 0.0
            for c in range(f, f + 3):
                a = g32.field(c).astype(np.float64)
                b = g64.field(c)
                d2 += float(np.sum((a - b) ** 2))
                r2 += float(np.sum(b * b))
            peak[name] = max(peak[name], r2 ** 0.5)
            row[name] = d2 ** 0.5 / peak[name] if peak[name] > 0 else 0.0
        rows.append(row)
    spec = []
    for p in range(len(w.probes)):
        x, y = g32.probe_dft(p), g64.probe_dft(p)
        spec.append(float(np.linalg.norm(x - y) / np.linalg.norm(y)))
    cells = w.ncells
    line = {"study": "fp32 fused step vs fp64 stepper", "workload": w.name, "steps": args.fp64_study,
            "field_rel_l2_vs_peak": rows, "probe_spectrum_rel_l2": spec,
            "fp32_gcell_updates_per_s": cells * args.fp64_study / t32 / 1e9,
            "fp64_gcell_updates_per_s": cells * args.fp64_study / t64 / 1e9,
            "fp64_fma_gflops": tf.fp64_fma_rate()}
    print(json.dumps(line), flush=True)
    return 0


def run_autotune_table(args):
    """The autotuner over every workload class of the study: temporal-block
    depth and two-step item length per class, from measured runs; writes the
    table to --autotune-table and prints it as one JSON line."""
    from paper_2305_13419_gb300 import autotune
    from paper_2305_13419_gb300 import workloads as W
    ws = [W.slab(), W.cpw(), W.cpw_adjoint(), W.cpw_large(nsteps=10)] + W.cpw_batch()
    table = autotune.tune_classes(ws, steps=args.autotune_steps)
    autotune.save(table, args.autotune_table)
    print(json.dumps({"autotune_table": table}), flush=True)
    return 0


def run_e2e(args, w, dev, tuning=None):
    """Same metric through the public API from host memory: the timed region
    uploads the material maps from pinned host buffers, runs the K steps and
    reads back both probe DFTs and the integer-level Ex field into pinned
    host memory.  The grid takes the settings the autotuner chose for the
    device-timed run (`tuning`), as a user applying its table would."""
    import torch
    from paper_2305_13419_gb300 import twofluid as tf
    g = tf.Grid(w.n, w.d, w.theta, w.bc, w.cpml, courant=w.courant, device=dev)
    cs = (w.n[2], w.n[1], w.n[0])
    maps = []
    for a in (w.eps_r, w.mu_r, w.lambda_L, w.sigma):
        t = torch.empty(cs, dtype=torch.float32, pin_memory=True)
        t.numpy()[...] = a
        maps.append(t)
    out = torch.empty(g.shape, dtype=torch.float32, pin_memory=True)
    for s in w.sources:
        g.add_source(s.comp, s.lo, s.hi, s.amp, s.kind, s.f, s.t0, s.tw)
    for p in w.probes:
        g.add_probe(p.comp, p.p, p.freqs, p.n0)
    if args.two_step == "off":
        g.set_two_step(0)
    elif tuning is not None:
        g.set_two_step(tuning["best"])
    if tuning is not None:
        g.set_item_planes(tuning["item_planes"])
    elif args.item_planes:
        g.set_item_planes(args.item_planes)
    import ctypes as C
    L = tf.load()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = L.tf_set_materials(g.h, *[int(m.data_ptr()) for m in maps], 0)
    assert rc == 0, rc
    g.step(args.steps)
    spectra = [g.probe_dft(p) for p in range(len(w.probes))]
    rc = L.tf_read_field(g.h, 0, int(out.data_ptr()), 0)
    assert rc == 0, rc
    g.sync()
    el = time.perf_counter() - t0
    h2d = 4 * 4 * w.ncells
    d2h = 16 * sum(s.size for s in spectra) + 4 * int(np.prod(g.shape))
    g.close()
    return {"value": w.ncells * args.steps / el / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--cpw-steps", type=int, default=2000, help="steps of the 512 x 256 x 128 CPW line")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default settings")
    ap.add_argument("--autotune-table", default="",
                    help="tune every workload class (slab, CPWs, adjoint grid, the batch's size classes) and "
                         "write the table to this JSON path (one JSON line printed)")
    ap.add_argument("--autotune-steps", type=int, default=20, help="steps timed per autotuner candidate")
    ap.add_argument("--item-planes", type=int, default=0,
                    help="planes per single-step work item of the timed grid (8..16; default: the autotuner's or 8)")
    ap.add_argument("--workload", choices=("large", "cpw"), default="large",
                    help="the timed workload: the 1024 x 512 x 256 CPW (default) or the 512 x 256 x 128 one")
    ap.add_argument("--two-step", choices=("auto", "off"), default="auto",
                    help="two steps per pass on the interior box where the grid has one (auto) or single steps only")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--all-configs", action="store_true", help="per-config GPU and oracle numbers, one JSON line")
    ap.add_argument("--large-steps", type=int, default=200)
    ap.add_argument("--fp64-study", type=int, default=0, help="run only the FP32-vs-FP64 study over this many steps")
    ap.add_argument("--fp64-peak", action="store_true", help="measure only the FP64 FMA rate (one JSON line)")
    ap.add_argument("--batch-singles", type=int, default=0,
                    help="time only the first N grids of the batch one at a time (one JSON line)")
    ap.add_argument("--batch-overhead", action="store_true",
                    help="only the batched kernel against the single-grid kernel on one grid (one JSON line)")
    ap.add_argument("--study-workload", choices=("cpw", "cpw_large"), default="cpw")
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--adjoint-steps", type=int, default=8000)
    ap.add_argument("--adjoint-segment", type=int, default=256, help="steps between the adjoint's checkpoints")
    args = ap.parse_args(argv)
    global WORKLOAD
    WORKLOAD = args.workload
    ws, rank, local = dist_env()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.batch_singles > 0:
        return run_batch_singles(args)
    if args.batch_overhead:
        return run_batch_overhead(args)
    if args.fp64_peak:
        from paper_2305_13419_gb300 import twofluid as tf
        rates = [tf.fp64_fma_rate() for _ in range(3)]
        print(json.dumps({"measure": "FP64 FMA rate (library kernel of independent FMA chains)", "unit": "GFLOP/s",
                          "runs": rates, "best": max(rates)}), flush=True)
        return 0
    if args.fp64_study > 0:
        return run_precision_study(args)
    if args.autotune_table:
        return run_autotune_table(args)
    if args.all_configs:
        return run_all_configs(args)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
