"""Parity at the full step counts of the resonator workloads (arXiv
2305.13419, Sec. 5 runs; Algorithm 1 of Sec. 3):

* the scaled CPW (128 x 64 x 40) for 20000 steps against the FP64 oracle:
  fields, both probe spectra and the Q factor;
* the 512 x 256 x 128 CPW for 20000 steps, FP32 fused step against the FP64
  GPU stepper (itself pinned to the oracle to 1e-12);
* the 256 x 128 x 64 adjoint CPW, 8000 steps with checkpoints every 256:
  the FP32 discrete adjoint's gradients against central differences of the
  FP64 GPU stepper on 16 seeded cells.

Each prints one JSON line with the numbers it checked (run with -s)."""
import json

import numpy as np
import pytest

from oracle import qfit
from oracle import stepper
from paper_2305_13419_gb300 import workloads as W
from parity_util import FAMILIES, FIELD_TOL, SPEC_TOL, compare_families, family_norms, rel_l2

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _plain_family_errors(gg, go):
    """||gpu - ref|| / ||ref|| of each vector field at the current level."""
    return compare_families(gg, go, None, tol=np.inf)[0]


def test_cpw_small_20000_steps_against_oracle():
    """Scaled CPW, 20000 steps (the step count of the 512 x 256 x 128 run):
    fields against the FP64 oracle relative to the largest norm each field
    reached (the transient rings down into the CPML, FP32 rounding stays
    relative to the peak), the plain end-of-run ratio reported beside it;
    both spectra and the Q factor within 1e-3."""
    from paper_2305_13419_gb300 import twofluid as tf
    nsteps = 20000
    w = W.cpw_small(nsteps=nsteps)
    f0 = w.sources[0].f
    n0 = 1200
    for p in w.probes:
        p.n0 = n0
        p.freqs = np.linspace(0.7 * f0, 1.3 * f0, 64)
    go = stepper.Grid.from_workload(w)
    gg = tf.Grid.from_workload(w)
    peak = {k: 0.0 for k, _ in FAMILIES}
    rows, done = [], 0
    for N in (500, 1000, 1500, 2000, 3000, 5000, 8000, 12000, 16000, 20000):
        go.step(N - done)
        gg.step(N - done)
        done = N
        for k, v in family_norms(go).items():
            peak[k] = max(peak[k], v)
        errs, bad = compare_families(gg, go, peak)
        plain = _plain_family_errors(gg, go)
        rows.append({"step": N, "vs_peak": errs, "plain": plain, "norm": family_norms(go)})
        assert not bad, (N, errs)
    gg.sync()
    spec = [rel_l2(gg.probe_dft(p), go.probe_dft(p)) for p in range(2)]
    fr = w.probes[0].freqs
    ro = qfit.fit(go.probe_dft(0), fr, go.dt, n0, nsteps)
    rg = gg.fit_q(0, f_guess=ro["f0"], q_guess=max(ro["Q"], 5.0))
    print(json.dumps({"test": "cpw-small-20000", "rows": rows, "spectra": spec, "Q_oracle": ro["Q"],
                      "Q_gpu": rg["Q"], "f0_oracle": ro["f0"], "f0_gpu": rg["f0"]}))
    assert max(spec) < SPEC_TOL, spec
    assert abs(rg["Q"] / ro["Q"] - 1) < SPEC_TOL, (rg, ro)
    assert abs(rg["f0"] / ro["f0"] - 1) < SPEC_TOL


def test_fp32_against_fp64_gpu_cpw_512x256x128_20000_steps():
    """The 512 x 256 x 128 CPW at its stated 20000 steps: the FP32 fused step
    against the FP64 stepper (Algorithm 1's sub-steps in FP64, pinned to the
    oracle to 1e-12 by test_gpu_fp64): fields relative to their peak norm
    within 1e-4 at every checkpoint (plain ratio reported beside it), both
    probe spectra within 1e-3."""
    from paper_2305_13419_gb300 import twofluid as tf
    nsteps = 20000
    w = W.cpw(nsteps=nsteps)
    g32 = tf.Grid.from_workload(w)
    g64 = tf.Grid64.from_workload(w)
    peak = {k: 0.0 for k, _ in FAMILIES}
    rows, done = [], 0
    for N in (1000, 2500, 5000, 10000, 15000, 20000):
        g32.step(N - done)
        g64.step(N - done)
        done = N
        g32.sync()
        g64.sync()
        for k, v in family_norms(g64).items():
            peak[k] = max(peak[k], v)
        errs, bad = compare_families(g32, g64, peak)
        rows.append({"step": N, "vs_peak": errs, "plain": _plain_family_errors(g32, g64)})
        assert not bad, (N, errs)
    spec = [rel_l2(g32.probe_dft(p), g64.probe_dft(p)) for p in range(len(w.probes))]
    print(json.dumps({"test": "cpw-512x256x128-fp32-vs-fp64-20000", "rows": rows, "spectra": spec}))
    assert max(spec) < SPEC_TOL, spec


def test_adjoint_cpw_256x128x64_against_central_differences():
    """The adjoint workload (256 x 128 x 64 CPW, substrate eps_r ~ U[10, 13],
    8000 steps, checkpoints every 256 steps, J = |X(f0)|^2 of probe 0 with a
    1 V/m source): dJ/d eps_r on 8 seeded substrate cells and dJ/d lambda_L
    on 8 seeded film cells against central differences (h = 1e-4 of the
    value) of the FP64 GPU stepper, within 1e-3.  Cells are drawn among
    those whose gradient is at least 5 % of the largest in their region, so
    that the FP64 difference of J resolves them."""
    from paper_2305_13419_gb300 import twofluid as tf
    nsteps = 8000
    w = W.cpw_adjoint(nsteps=nsteps)
    J, ge, gl = tf.Grid.from_workload(w).adjoint(nsteps, 0, 0, segment=256)
    ge = ge.cpu().numpy().astype(np.float64)
    gl = gl.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(ge)) and np.all(np.isfinite(gl)) and J > 0
    rng = np.random.default_rng(W.BASE_SEED + 44)
    sub = w.eps_r > 5.0            # the substrate (eps_r from U[10, 13]; vacuum elsewhere)
    metal = w.lambda_L > 0

    def pick(g, region, k):
        cand = np.argwhere(region & (np.abs(g) >= 0.05 * np.max(np.abs(g[region]))))
        return [tuple(c) for c in cand[rng.choice(len(cand), size=k, replace=False)]]

    def J64(eps, lam):
        g = tf.Grid64(w.n, w.d, w.theta, w.bc, w.cpml, courant=w.courant, edge_rule=w.edge_rule)
        g.set_materials(eps, w.mu_r, lam, w.sigma)
        for s in w.sources:
            g.add_source(s.comp, s.lo, s.hi, s.amp, s.kind, s.f, s.t0, s.tw)
        p = w.probes[0]
        g.add_probe(p.comp, p.p, p.freqs, p.n0)
        g.step(nsteps)
        g.sync()
        x = g.probe_dft(0)[0]
        g.close()
        return float(abs(x) ** 2)

    eps0 = w.eps_r.astype(np.float64)
    lam0 = w.lambda_L.astype(np.float64)
    J0 = J64(eps0, lam0)
    rows, worst = [], 0.0
    for name, g, region, base in (("eps", ge, sub, eps0), ("lambda", gl, metal, lam0)):
        for c in pick(g, region, 8):
            h = 1e-4 * base[c]
            vals = []
            for sgn in (1.0, -1.0):
                m = base.copy()
                m[c] += sgn * h
                vals.append(J64(m, lam0) if name == "eps" else J64(eps0, m))
            fd = (vals[0] - vals[1]) / (2.0 * h)
            rel = abs(g[c] / fd - 1.0)
            worst = max(worst, rel)
            rows.append({"map": name, "cell": [int(x) for x in c], "adjoint": g[c], "central_difference": fd,
                         "rel": rel})
    print(json.dumps({"test": "adjoint-cpw-256x128x64-8000", "J_fp32": J, "J_fp64": J0, "cells": rows,
                      "worst_rel": worst}))
    assert abs(J / J0 - 1) < SPEC_TOL, (J, J0)
    assert worst < SPEC_TOL, rows
