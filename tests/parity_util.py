"""Helpers for GPU-vs-oracle parity: run both sides on one workload and
compare; crop a full-size workload to the light cone of sampled points.

The two sides only share the seeded inputs of paper_2305_13419_gb300.workloads.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from oracle import stepper
from paper_2305_13419_gb300 import workloads as W

FIELD_TOL = 1e-4   # relative L2 on fields after the stated steps
SPEC_TOL = 1e-3    # relative on probe spectra and Q


def rel_l2(a, b, floor=0.0):
    a = np.asarray(a)
    b = np.asarray(b)
    den = max(float(np.linalg.norm(b)), floor)
    if den == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b)) / den


def field_floor(c, ref_fields):
    """Scale below which a component counts as absent: 1e-6 of its family's
    largest norm (E, B or Js), so that an identically-zero component is
    compared absolutely."""
    fam = (c // 3) * 3
    return 1e-6 * max(float(np.linalg.norm(ref_fields[f])) for f in range(fam, fam + 3))


FAMILIES = (("E", 0), ("B", 3), ("Js", 6))


def family_norms(g):
    """L2 norm of each vector field (E, B, Js: three components together)."""
    return {name: float(np.sqrt(sum(np.linalg.norm(g.field(c).astype(np.float64)) ** 2
                                    for c in range(f, f + 3)))) for name, f in FAMILIES}


def compare_families(gg, go, peak=None, tol=FIELD_TOL):
    """Relative L2 of each vector field, ||gpu - oracle|| / max(||oracle||, peak):
    `peak` holds the largest norm each field reached during the run, so a
    transient that has rung down is judged against the scale it had (FP32
    rounding is relative to the largest values the state carried)."""
    errs, bad = {}, {}
    for name, f in FAMILIES:
        d2 = n2 = 0.0
        for c in range(f, f + 3):
            a = gg.field(c).astype(np.float64)
            b = go.field(c)
            d2 += float(np.sum((a - b) ** 2))
            n2 += float(np.sum(b * b))
        den = max(np.sqrt(n2), (peak or {}).get(name, 0.0))
        errs[name] = np.sqrt(d2) / den if den > 0 else np.sqrt(d2)
        if not errs[name] <= tol:
            bad[name] = errs[name]
    return errs, bad


def set_state(grid, state, float32=True):
    for c, v in state.items():
        grid.set_field(c, v.astype(np.float32) if float32 else v)


def run_oracle(w, nsteps, state=None):
    g = stepper.Grid.from_workload(w)
    if state:
        # the oracle takes the very same float32 values the GPU receives
        for c, v in state.items():
            g.set_field(c, v.astype(np.float32).astype(np.float64))
    g.step(nsteps)
    return g


def run_gpu(w, nsteps, state=None, chunks=None):
    from paper_2305_13419_gb300 import twofluid as tf
    g = tf.Grid.from_workload(w)
    if state:
        set_state(g, state)
    if chunks:
        for c in chunks:
            g.step(c)
    else:
        g.step(nsteps)
    g.sync()
    return g


def compare_fields(gg, go, comps=range(9), tol=FIELD_TOL):
    ref = [go.field(c) for c in range(9)]
    errs = {}
    for c in comps:
        a = gg.field(c)
        errs[c] = rel_l2(a, ref[c], field_floor(c, ref))
    bad = {c: e for c, e in errs.items() if not e <= tol}
    return errs, bad


# ---------------------------------------------------------------- light cone
@dataclasses.dataclass
class Crop:
    lo: tuple            # first global cell / storage point of the crop per axis
    workload: W.Workload


def crop_workload(w, p, radius):
    """A standalone problem that reproduces `w` exactly at storage point p for
    as many steps as the cone stays inside it.

    Per axis: if the cone [p - radius, p + radius] reaches neither boundary the
    crop is cut on both sides and closed with PEC walls; if it reaches a
    boundary, the crop keeps that boundary (and its kind) and is cut at
    radius + CPML thickness on the other side; a periodic axis narrower than
    the cone is kept whole.  Sources are intersected with the crop."""
    n = w.n
    lo, hi, bc, cp = [], [], [], []
    for a in range(3):
        kind = w.bc[a]
        L = w.cpml[a].ncells if w.cpml[a] is not None else 0
        if kind == "periodic":
            if 2 * radius + 2 >= n[a]:
                lo.append(0); hi.append(n[a]); bc.append("periodic"); cp.append(None)
                continue
            lo.append(p[a] - radius); hi.append(p[a] + radius + 1); bc.append("pec"); cp.append(None)
            continue
        reach_lo = p[a] - radius <= L + 1
        reach_hi = p[a] + radius >= n[a] - L - 1
        if reach_lo and reach_hi:
            lo.append(0); hi.append(n[a]); bc.append(kind); cp.append(w.cpml[a])
        elif reach_lo:
            lo.append(0); hi.append(min(n[a], p[a] + radius + L + 2)); bc.append(kind); cp.append(w.cpml[a])
        elif reach_hi:
            lo.append(max(0, p[a] - radius - L - 2)); hi.append(n[a]); bc.append(kind); cp.append(w.cpml[a])
        else:
            lo.append(p[a] - radius); hi.append(p[a] + radius + 1); bc.append("pec"); cp.append(None)
    sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
    nn = tuple(hi[a] - lo[a] for a in range(3))
    N = tuple(nn[a] + (0 if bc[a] == "periodic" else 1) for a in range(3))
    srcs = []
    for s in w.sources:
        slo = tuple(max(s.lo[a], lo[a]) - lo[a] for a in range(3))
        shi = tuple(min(s.hi[a], lo[a] + N[a]) - lo[a] for a in range(3))
        if all(shi[a] > slo[a] for a in range(3)):
            srcs.append(dataclasses.replace(s, lo=slo, hi=shi))
    dt = w.dt if w.dt else stepper.dt_from_courant(w.courant, w.d)
    cw = W.Workload(name=w.name + "-crop", n=nn, d=w.d, theta=w.theta, bc=tuple(bc),
                    eps_r=np.ascontiguousarray(w.eps_r[sl]), mu_r=np.ascontiguousarray(w.mu_r[sl]),
                    lambda_L=np.ascontiguousarray(w.lambda_L[sl]), sigma=np.ascontiguousarray(w.sigma[sl]),
                    dt=dt, cpml=tuple(cp), sources=srcs, probes=[], nsteps=w.nsteps,
                    edge_rule=w.edge_rule)
    return Crop(lo=tuple(lo), workload=cw)


def local_state(seed, dims, centres, radius, lo, Nloc):
    """Random fields that are non-zero only within `radius` of the centres
    (global storage coords), restricted to the crop [lo, lo + Nloc)."""
    out = {}
    for c in range(9):
        out[c] = np.zeros((Nloc[2], Nloc[1], Nloc[0]), np.float64)
    for ctr in centres:
        blo = [max(ctr[a] - radius, 0) for a in range(3)]
        bhi = [min(ctr[a] + radius + 1, dims[a]) for a in range(3)]
        # intersect with the crop
        clo = [max(blo[a], lo[a]) for a in range(3)]
        chi = [min(bhi[a], lo[a] + Nloc[a]) for a in range(3)]
        if any(chi[a] <= clo[a] for a in range(3)):
            continue
        st = W.random_state(seed, dims, clo, chi)
        s = (slice(clo[2] - lo[2], chi[2] - lo[2]), slice(clo[1] - lo[1], chi[1] - lo[1]),
             slice(clo[0] - lo[0], chi[0] - lo[0]))
        for c in range(9):
            out[c][s] = st[c]
    return out
