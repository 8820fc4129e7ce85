"""ctypes wrapper of the C oracle (twofluid_oracle.c): Algorithm 1 of
arXiv 2305.13419 in FP64, SI units, state at integer time levels.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Optional

import numpy as np

from . import build as _build

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 8.8541878128e-12

BC = {"periodic": 0, "pec": 1, "mur": 2, "cpml": 3}

_lib = None


class _Desc(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("d", C.c_double * 3), ("dt", C.c_double), ("theta", C.c_double),
                ("bc", C.c_int * 3), ("pml_n", C.c_int * 3), ("pml_m", C.c_double * 3),
                ("pml_sigma_max", C.c_double * 3), ("pml_alpha_max", C.c_double * 3),
                ("edge_rule", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
        L.or_create.restype = vp
        L.or_create.argtypes = [C.POINTER(_Desc)]
        L.or_destroy.argtypes = [vp]
        L.or_storage_dims.argtypes = [vp, ip]
        L.or_set_materials.argtypes = [vp, dp, dp, dp, dp]
        L.or_set_field.argtypes = [vp, C.c_int, dp]
        L.or_get_field.argtypes = [vp, C.c_int, dp]
        L.or_get_coeff.argtypes = [vp, C.c_int, C.c_int, dp]
        L.or_add_source.argtypes = [vp, C.c_int, ip, ip, C.c_double, C.c_int, C.c_double,
                                    C.c_double, C.c_double]
        L.or_add_probe.argtypes = [vp, C.c_int, ip, dp, C.c_int, C.c_int64, C.c_int64]
        L.or_step.argtypes = [vp, C.c_int64]
        L.or_level.restype = C.c_int64
        L.or_level.argtypes = [vp]
        L.or_probe_dft.argtypes = [vp, C.c_int, dp, dp]
        L.or_probe_series.argtypes = [vp, C.c_int, dp, C.c_int64]
        L.or_set_threads.argtypes = [C.c_int]
        L.or_adjoint_dot_test.argtypes = [vp, C.c_int, C.c_uint64, dp, dp]
        L.or_adjoint_run.argtypes = [vp, C.c_int64, C.c_int, ip, C.c_double, C.c_int64, dp, dp, dp]
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    return lib().or_set_threads(int(n))


def dt_from_courant(courant: float, d) -> float:
    """Courant convention pinned by the paper's quoted time steps (Secs. 4-5):
    dt = C / (c sqrt(sum_a 1/d_a^2)) over the three axes."""
    return courant / (C0 * math.sqrt(sum(1.0 / (x * x) for x in d)))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Grid:
    """One FP64 oracle grid. Arrays in and out are [k][j][i] (x fastest)."""

    def __init__(self, n, d, dt, theta=1.0, bc=("periodic",) * 3, cpml=(None, None, None),
                 edge_rule=0):
        L = lib()
        desc = _Desc()
        for a in range(3):
            desc.n[a] = int(n[a])
            desc.d[a] = float(d[a])
            desc.bc[a] = BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
            cp = cpml[a]
            if cp is not None:
                desc.pml_n[a] = int(cp.ncells)
                desc.pml_m[a] = float(cp.order)
                desc.pml_sigma_max[a] = float(cp.sigma_max)
                desc.pml_alpha_max[a] = float(cp.alpha_max)
        desc.dt = float(dt)
        desc.theta = float(theta)
        desc.edge_rule = int(edge_rule)
        h = L.or_create(C.byref(desc))
        if not h:
            raise ValueError("oracle rejected the grid description")
        self._h = C.c_void_p(h)
        self.n = tuple(int(x) for x in n)
        self.d = tuple(float(x) for x in d)
        self.dt = float(dt)
        self.theta = float(theta)
        self.bc = tuple(bc)
        self.edge_rule = int(edge_rule)
        N = (C.c_int * 3)()
        L.or_storage_dims(self._h, N)
        self.N = (N[0], N[1], N[2])
        self.shape = (self.N[2], self.N[1], self.N[0])
        self.nprobes = 0

    @classmethod
    def from_workload(cls, w, with_sources=True, with_probes=True):
        dt = w.dt if w.dt else dt_from_courant(w.courant, w.d)
        g = cls(w.n, w.d, dt, w.theta, w.bc, w.cpml, getattr(w, "edge_rule", 0))
        g.set_materials(w.eps_r, w.mu_r, w.lambda_L, w.sigma)
        if with_sources:
            for s in w.sources:
                g.add_source(s.comp, s.lo, s.hi, s.amp, s.kind, s.f, s.t0, s.tw)
        if with_probes:
            for p in w.probes:
                g.add_probe(p.comp, p.p, p.freqs, p.n0, p.series)
        return g

    def __del__(self):
        try:
            if self._h:
                lib().or_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def set_materials(self, eps_r, mu_r, lambda_L, sigma):
        cs = (self.n[2], self.n[1], self.n[0])
        arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), cs)) for x in
                (eps_r, mu_r, lambda_L, sigma)]
        rc = lib().or_set_materials(self._h, *[_dp(a) for a in arrs])
        if rc:
            raise ValueError(f"or_set_materials rc={rc}")

    def set_field(self, comp: int, arr):
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(arr, np.float64), self.shape))
        rc = lib().or_set_field(self._h, int(comp), _dp(a))
        if rc:
            raise ValueError(f"or_set_field rc={rc}")

    def field(self, comp: int) -> np.ndarray:
        out = np.empty(self.shape, np.float64)
        lib().or_get_field(self._h, int(comp), _dp(out))
        return out

    def coeff(self, kind: int, comp: int) -> np.ndarray:
        out = np.empty(self.shape, np.float64)
        rc = lib().or_get_coeff(self._h, int(kind), int(comp), _dp(out))
        if rc:
            raise ValueError("bad coefficient request")
        return out

    def add_source(self, comp, lo, hi, amp, kind, f=0.0, t0=0.0, tw=1.0):
        lo_ = (C.c_int * 3)(*[int(x) for x in lo])
        hi_ = (C.c_int * 3)(*[int(x) for x in hi])
        rc = lib().or_add_source(self._h, int(comp), lo_, hi_, float(amp), int(kind), float(f),
                                 float(t0), float(tw))
        if rc:
            raise ValueError("or_add_source failed")

    def add_probe(self, comp, p, freqs, n0=0, series=0) -> int:
        fr = np.ascontiguousarray(np.asarray(freqs, np.float64))
        p_ = (C.c_int * 3)(*[int(x) for x in p])
        rc = lib().or_add_probe(self._h, int(comp), p_, _dp(fr), int(fr.size), int(n0), int(series))
        if rc:
            raise ValueError("or_add_probe failed")
        self.nprobes += 1
        return self.nprobes - 1

    def step(self, nsteps: int):
        rc = lib().or_step(self._h, int(nsteps))
        if rc:
            raise ValueError("or_step failed")

    @property
    def level(self) -> int:
        return int(lib().or_level(self._h))

    def probe_dft(self, pid: int, nfreq: int = 64) -> np.ndarray:
        re = np.zeros(64, np.float64)
        im = np.zeros(64, np.float64)
        lib().or_probe_dft(self._h, int(pid), _dp(re), _dp(im))
        return (re + 1j * im)[:nfreq]

    def probe_series(self, pid: int, n: int) -> np.ndarray:
        out = np.empty(int(n), np.float64)
        rc = lib().or_probe_series(self._h, int(pid), _dp(out), int(n))
        if rc:
            raise ValueError("series request beyond capacity")
        return out

    def adjoint_dot_test(self, op: int, seed: int):
        """(<M v, w>, <v, M^T w>) for Algorithm 1 sub-step `op` (1 B half step,
        2 Js half step, 3 psi_E update, 4 theta step for E, 5 psi_B update)."""
        l, r = C.c_double(), C.c_double()
        if lib().or_adjoint_dot_test(self._h, int(op), int(seed), C.byref(l), C.byref(r)):
            raise ValueError("or_adjoint_dot_test failed")
        return l.value, r.value

    def adjoint_run(self, nsteps: int, comp: int, p, freq: float, n0: int):
        """J = |X(freq)|^2 of the probe DFT of E_comp at p over [n0, nsteps),
        and dJ/d eps_r, dJ/d lambda_L per cell ([nz][ny][nx]), by the
        discrete adjoint (runs the forward from level 0 first)."""
        cs = (self.n[2], self.n[1], self.n[0])
        ge, gl = np.zeros(cs), np.zeros(cs)
        J = C.c_double()
        p_ = (C.c_int * 3)(*[int(x) for x in p])
        if lib().or_adjoint_run(self._h, int(nsteps), int(comp), p_, float(freq), int(n0), C.byref(J), _dp(ge),
                                _dp(gl)):
            raise ValueError("or_adjoint_run failed")
        return J.value, ge, gl

    def fields(self):
        return [self.field(c) for c in range(9)]
