"""Python binding of libtwofluid (include/twofluid.h) -- argument marshalling only.

Every numerical step runs in the CUDA library.  PyTorch provides the device
workspace (a uint8 CUDA tensor) and the CUDA stream; numpy arrays are the
host-side buffers.  If the library has not been built this module raises:
there is no CPU fallback.

Module-level functions carry the C names (tf_create, tf_step, ...); `Grid`
bundles them for convenience.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional

import numpy as np

from . import build as _build

TF_OK, TF_EINVAL, TF_ENOMEM, TF_ECUDA, TF_EUNSTABLE, TF_ESTATE, TF_ETIMEOUT, TF_ENONFINITE, TF_ENOTSUP = range(9)
TF_BC = {"periodic": 0, "pec": 1, "mur": 2, "cpml": 3}
TF_MAX_PROBES, TF_MAX_FREQS, TF_MAX_SOURCES = 16, 64, 16

EXPORTS = ["tf_workspace_size", "tf_create", "tf_destroy", "tf_storage_dims", "tf_get_time", "tf_get_dt",
           "tf_set_materials", "tf_set_field", "tf_add_source", "tf_add_probe", "tf_step", "tf_sync",
           "tf_read_probe_dft", "tf_read_probe_series", "tf_read_field", "tf_fit_q", "tf_strerror",
           "tf_step_timed", "tf_set_two_step", "tf_two_step_box", "tf_set_wait_limit", "tf_set_item_planes", "tf_field_stats", "tf_field_stats_noalloc",
           "tf_checkpoint_size",
           "tf_checkpoint_save", "tf_checkpoint_load", "tf_adjoint_scratch_size", "tf_adjoint_run", "tf_batch_step",
           "tf_batch_scratch_size", "tf_batch_run",
           "tf64_workspace_size", "tf64_create", "tf64_destroy", "tf64_set_materials", "tf64_set_field",
           "tf64_add_source", "tf64_add_probe", "tf64_step", "tf64_sync", "tf64_read_field", "tf64_read_probe_dft",
           "tf64_get_time", "tf64_fma_rate_scratch", "tf64_fma_rate"]


class TFError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {tf_strerror(status)} (status {status})")


class tf_bc(C.Structure):
    _fields_ = [("kind", C.c_int), ("cpml_cells", C.c_int), ("cpml_order", C.c_double),
                ("cpml_sigma_max", C.c_double), ("cpml_alpha_max", C.c_double)]


class tf_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("dt", C.c_double), ("courant", C.c_double), ("theta", C.c_double),
                ("bc", tf_bc * 3), ("edge_rule", C.c_int), ("max_probes", C.c_int),
                ("series_capacity", C.c_int64), ("stream", C.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libtwofluid.so (building it in-tree first if asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing and (not os.path.exists(path) or _build.needs_build()):
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libtwofluid.so is not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    vp, ip, dp, fp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p
    st = C.c_int
    L.tf_workspace_size.restype = C.c_size_t
    L.tf_workspace_size.argtypes = [C.POINTER(tf_grid_desc)]
    L.tf_create.restype = st
    L.tf_create.argtypes = [C.POINTER(tf_grid_desc), vp, C.c_size_t, C.POINTER(vp)]
    for name, args in (("tf_destroy", [vp]), ("tf_storage_dims", [vp, ip]),
                       ("tf_get_time", [vp, C.POINTER(C.c_int64), dp]), ("tf_get_dt", [vp, dp]),
                       ("tf_set_materials", [vp, fp, fp, fp, fp, C.c_int]),
                       ("tf_set_field", [vp, C.c_int, fp, C.c_int]),
                       ("tf_add_source", [vp, C.c_int, ip, ip, C.c_double, C.c_int, C.c_double, C.c_double,
                                          C.c_double, ip]),
                       ("tf_add_probe", [vp, C.c_int, ip, dp, C.c_int, C.c_int64, ip]),
                       ("tf_step", [vp, C.c_int64]), ("tf_sync", [vp]),
                       ("tf_step_timed", [vp, C.c_int64, dp, C.POINTER(C.c_int64), C.c_int, dp]),
                       ("tf_set_two_step", [vp, C.c_int]), ("tf_two_step_box", [vp, ip, ip, ip]),
                       ("tf_set_wait_limit", [vp, C.c_int64]), ("tf_set_item_planes", [vp, C.c_int]),
                       ("tf_read_probe_dft", [vp, C.c_int, dp, dp]),
                       ("tf_read_probe_series", [vp, C.c_int, dp, C.c_int64]),
                       ("tf_read_field", [vp, C.c_int, fp, C.c_int]),
                       ("tf_fit_q", [vp, C.c_int, C.c_double, C.c_double, dp, dp, dp]),
                       ("tf_field_stats", [vp, C.c_int, dp, dp, C.POINTER(C.c_int64)]),
                       ("tf_field_stats_noalloc", [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, dp, dp,
                                                   C.POINTER(C.c_int64), vp]),
                       ("tf_checkpoint_size", [vp, C.POINTER(C.c_size_t)]),
                       ("tf_checkpoint_save", [vp, vp, C.c_size_t, C.c_int]),
                       ("tf_checkpoint_load", [vp, vp, C.c_size_t, C.c_int]),
                       ("tf_adjoint_scratch_size", [vp, C.c_int64, C.c_int, C.POINTER(C.c_size_t)]),
                       ("tf_adjoint_run", [vp, C.c_int64, C.c_int, C.c_int, C.c_int, vp, C.c_size_t, dp, vp, vp]),
                       ("tf_batch_step", [C.POINTER(vp), C.c_int, C.c_int64]),
                       ("tf_batch_scratch_size", [C.POINTER(vp), C.c_int, C.c_int64, C.POINTER(C.c_size_t)]),
                       ("tf_batch_run", [C.POINTER(vp), C.c_int, C.c_int64, vp, C.c_size_t]),
                       ("tf64_create", [C.POINTER(tf_grid_desc), vp, C.c_size_t, C.POINTER(vp)]),
                       ("tf64_destroy", [vp]), ("tf64_set_materials", [vp, vp, vp, vp, vp]),
                       ("tf64_set_field", [vp, C.c_int, vp]),
                       ("tf64_add_source", [vp, C.c_int, ip, ip, C.c_double, C.c_int, C.c_double, C.c_double,
                                            C.c_double, ip]),
                       ("tf64_add_probe", [vp, C.c_int, ip, dp, C.c_int, C.c_int64, ip]),
                       ("tf64_step", [vp, C.c_int64]), ("tf64_sync", [vp]), ("tf64_read_field", [vp, C.c_int, vp]),
                       ("tf64_read_probe_dft", [vp, C.c_int, dp, dp]),
                       ("tf64_get_time", [vp, C.POINTER(C.c_int64), dp]),
                       ("tf64_fma_rate", [vp, C.c_size_t, C.c_int, vp, dp])):
        fn = getattr(L, name)
        fn.restype = st
        fn.argtypes = args
    L.tf64_workspace_size.restype = C.c_size_t
    L.tf64_workspace_size.argtypes = [C.POINTER(tf_grid_desc)]
    L.tf64_fma_rate_scratch.restype = C.c_size_t
    L.tf64_fma_rate_scratch.argtypes = []
    L.tf_strerror.restype = C.c_char_p
    L.tf_strerror.argtypes = [C.c_int]
    _lib = L
    return L


def tf_strerror(status: int) -> str:
    try:
        return load(build_if_missing=False).tf_strerror(int(status)).decode()
    except Exception:
        return f"status {status}"


def _check(rc: int, what: str):
    if rc != TF_OK:
        raise TFError(rc, what)


# ------------------------------------------------------------- thin wrappers
def make_desc(n, d, theta=1.0, bc=("periodic",) * 3, cpml=(None, None, None), dt=None, courant=None,
              edge_rule=0, max_probes=TF_MAX_PROBES, series_capacity=0, stream=None) -> tf_grid_desc:
    desc = tf_grid_desc()
    desc.nx, desc.ny, desc.nz = (int(x) for x in n)
    desc.dx, desc.dy, desc.dz = (float(x) for x in d)
    desc.dt = float(dt) if dt else 0.0
    desc.courant = float(courant) if courant else 0.0
    desc.theta = float(theta)
    for a in range(3):
        kind = TF_BC[bc[a]] if isinstance(bc[a], str) else int(bc[a])
        desc.bc[a].kind = kind
        cp = cpml[a]
        if cp is not None:
            desc.bc[a].cpml_cells = int(cp.ncells)
            desc.bc[a].cpml_order = float(cp.order)
            desc.bc[a].cpml_sigma_max = float(cp.sigma_max)
            desc.bc[a].cpml_alpha_max = float(cp.alpha_max)
    desc.edge_rule = int(edge_rule)
    desc.max_probes = int(max_probes)
    desc.series_capacity = int(series_capacity)
    desc.stream = stream
    return desc


def tf_workspace_size(desc: tf_grid_desc) -> int:
    return int(load().tf_workspace_size(C.byref(desc)))


def tf_create(desc: tf_grid_desc, dev_ptr: int, nbytes: int):
    h = C.c_void_p()
    _check(load().tf_create(C.byref(desc), C.c_void_p(dev_ptr), C.c_size_t(nbytes), C.byref(h)), "tf_create")
    return h


def tf_destroy(h):
    _check(load().tf_destroy(h), "tf_destroy")


def tf_step(h, nsteps: int):
    _check(load().tf_step(h, int(nsteps)), "tf_step")


def tf_sync(h):
    _check(load().tf_sync(h), "tf_sync")


def tf_field_stats_noalloc(field, nx_pts, ny_pts, nz_pts, pitch, scale=1.0, stream=None):
    """Allocation-free field statistics of a device float32 array (data
    pointer of a CUDA tensor); returns (sum of squares, max |v|, non-finite)."""
    s, m, n = C.c_double(), C.c_double(), C.c_int64()
    ptr = int(field.data_ptr()) if hasattr(field, "data_ptr") else int(field)
    if stream is None and getattr(field, "is_cuda", False):
        # the stream the tensor's producers run on, not the legacy default stream
        import torch
        stream = torch.cuda.current_stream(field.device).cuda_stream
    _check(load().tf_field_stats_noalloc(C.c_void_p(ptr), int(nx_pts), int(ny_pts), int(nz_pts), int(pitch),
                                         float(scale), C.byref(s), C.byref(m), C.byref(n),
                                         C.c_void_p(stream)), "tf_field_stats_noalloc")
    return s.value, m.value, int(n.value)


def fp64_fma_rate(iters: int = 20000, device=None, stream=None) -> float:
    """FP64 FMA rate of the device in GFLOP/s (the FP64 stepper's arithmetic
    ceiling), measured by the library's FMA-chain kernel."""
    import torch
    dev = torch.device(device if device is not None else "cuda")
    n = load().tf64_fma_rate_scratch()
    if n == 0:
        raise TFError(TF_ECUDA, "tf64_fma_rate_scratch")
    scratch = torch.empty(int(n), dtype=torch.uint8, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    g = C.c_double()
    _check(load().tf64_fma_rate(C.c_void_p(scratch.data_ptr()), int(n), int(iters), C.c_void_p(st.cuda_stream),
                                C.byref(g)), "tf64_fma_rate")
    return g.value


class Grid64:
    """FP64 GPU stepper (Algorithm 1's sub-steps in FP64): the precision
    reference of the FP32 path.  Dense float64 fields [Nz][Ny][Nx], SI."""

    def __init__(self, n, d, theta=1.0, bc=("periodic",) * 3, cpml=(None, None, None), dt=None, courant=None,
                 edge_rule=0, max_probes=TF_MAX_PROBES, device=None, stream=None):
        import torch
        load()
        if not torch.cuda.is_available():
            raise RuntimeError("the FP64 stepper needs a CUDA device")
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.desc = make_desc(n, d, theta, bc, cpml, dt, courant, edge_rule, max_probes, 0, self.stream.cuda_stream)
        nbytes = load().tf64_workspace_size(C.byref(self.desc))
        if nbytes == 0:
            raise TFError(TF_EINVAL, "tf64_workspace_size")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        h = C.c_void_p()
        _check(load().tf64_create(C.byref(self.desc), C.c_void_p(base), nbytes, C.byref(h)), "tf64_create")
        self.h = h
        self.n = tuple(int(x) for x in n)
        self.N = tuple(int(n[a]) + (0 if bc[a] == "periodic" else 1) for a in range(3))
        self.shape = (self.N[2], self.N[1], self.N[0])
        self.freqs = []

    @classmethod
    def from_workload(cls, w, **kw):
        g = cls(w.n, w.d, w.theta, w.bc, w.cpml, dt=w.dt, courant=w.courant, edge_rule=getattr(w, "edge_rule", 0),
                **kw)
        g.set_materials(w.eps_r, w.mu_r, w.lambda_L, w.sigma)
        for s in w.sources:
            g.add_source(s.comp, s.lo, s.hi, s.amp, s.kind, s.f, s.t0, s.tw)
        for p in w.probes:
            g.add_probe(p.comp, p.p, p.freqs, p.n0)
        return g

    def set_materials(self, eps_r, mu_r, lambda_L, sigma):
        cs = (self.n[2], self.n[1], self.n[0])
        arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float64), cs)) for x in
                (eps_r, mu_r, lambda_L, sigma)]
        _check(load().tf64_set_materials(self.h, *[a.ctypes.data for a in arrs]), "tf64_set_materials")

    def set_field(self, comp, arr):
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(arr, np.float64), self.shape))
        _check(load().tf64_set_field(self.h, int(comp), a.ctypes.data), "tf64_set_field")

    def add_source(self, comp, lo, hi, amp, kind, f=0.0, t0=0.0, tw=1.0):
        lo_ = (C.c_int * 3)(*[int(x) for x in lo])
        hi_ = (C.c_int * 3)(*[int(x) for x in hi])
        _check(load().tf64_add_source(self.h, int(comp), lo_, hi_, float(amp), int(kind), float(f), float(t0),
                                      float(tw), None), "tf64_add_source")

    def add_probe(self, comp, p, freqs, n0=0):
        fr = np.ascontiguousarray(np.asarray(freqs, np.float64))
        p_ = (C.c_int * 3)(*[int(x) for x in p])
        _check(load().tf64_add_probe(self.h, int(comp), p_, fr.ctypes.data_as(C.POINTER(C.c_double)), int(fr.size),
                                     int(n0), None), "tf64_add_probe")
        self.freqs.append(fr)

    def step(self, n):
        _check(load().tf64_step(self.h, int(n)), "tf64_step")

    def sync(self):
        _check(load().tf64_sync(self.h), "tf64_sync")

    def field(self, comp):
        out = np.empty(self.shape, np.float64)
        _check(load().tf64_read_field(self.h, int(comp), out.ctypes.data), "tf64_read_field")
        return out

    def probe_dft(self, pid):
        nf = self.freqs[pid].size
        re, im = np.zeros(max(nf, 1)), np.zeros(max(nf, 1))
        _check(load().tf64_read_probe_dft(self.h, int(pid), re.ctypes.data_as(C.POINTER(C.c_double)),
                                          im.ctypes.data_as(C.POINTER(C.c_double))), "tf64_read_probe_dft")
        return (re + 1j * im)[:nf]

    @property
    def level(self):
        n = C.c_int64()
        _check(load().tf64_get_time(self.h, C.byref(n), None), "tf64_get_time")
        return int(n.value)

    def close(self):
        if getattr(self, "h", None):
            load().tf64_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_step(grids, nsteps: int):
    """Advance every grid of `grids` by nsteps (tf_batch_step): the grids'
    launches interleave on their own streams."""
    hs = (C.c_void_p * len(grids))(*[g.h for g in grids])
    _check(load().tf_batch_step(hs, len(grids), int(nsteps)), "tf_batch_step")


def batch_run(grids, nsteps: int):
    """Advance every grid of `grids` by nsteps with one launch per step over
    all of them (tf_batch_run): one work list over all grids' items, the
    steps replayed from a CUDA graph.  Synchronises."""
    import torch
    hs = (C.c_void_p * len(grids))(*[g.h for g in grids])
    n = C.c_size_t()
    _check(load().tf_batch_scratch_size(hs, len(grids), int(nsteps), C.byref(n)), "tf_batch_scratch_size")
    scratch = torch.empty(int(n.value) + 256, dtype=torch.uint8, device=grids[0].device)
    base = int(scratch.data_ptr())
    off = (-base) % 256
    _check(load().tf_batch_run(hs, len(grids), int(nsteps), C.c_void_p(base + off), int(n.value)), "tf_batch_run")
    del scratch


def _ptr(buf):
    """(pointer, on_device) of a numpy array or a CUDA torch tensor."""
    if isinstance(buf, np.ndarray):
        return buf.ctypes.data, 0
    return int(buf.data_ptr()), (1 if buf.is_cuda else 0)


class Grid:
    """One grid: owns a torch workspace tensor and a tf_handle."""

    def __init__(self, n, d, theta=1.0, bc=("periodic",) * 3, cpml=(None, None, None), dt=None, courant=None,
                 edge_rule=0, max_probes=TF_MAX_PROBES, series_capacity=0, device=None, stream=None):
        import torch
        load()
        if not torch.cuda.is_available():
            raise RuntimeError("libtwofluid needs a CUDA device")
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.desc = make_desc(n, d, theta, bc, cpml, dt, courant, edge_rule, max_probes, series_capacity,
                              C.c_void_p(self.stream.cuda_stream))
        nbytes = tf_workspace_size(self.desc)
        if nbytes == 0:
            raise TFError(TF_EINVAL, "tf_workspace_size")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = int(self.workspace.data_ptr())
        off = (-base) % 256
        self.h = tf_create(self.desc, base + off, nbytes)
        self.nbytes = nbytes
        dims = (C.c_int * 3)()
        _check(load().tf_storage_dims(self.h, dims), "tf_storage_dims")
        self.N = (dims[0], dims[1], dims[2])
        self.shape = (self.N[2], self.N[1], self.N[0])
        self.n = tuple(int(x) for x in n)
        dtv = C.c_double()
        _check(load().tf_get_dt(self.h, C.byref(dtv)), "tf_get_dt")
        self.dt = dtv.value
        self.freqs = []

    @classmethod
    def from_workload(cls, w, series_capacity=None, **kw):
        cap = series_capacity if series_capacity is not None else max([p.series for p in w.probes] + [0])
        g = cls(w.n, w.d, w.theta, w.bc, w.cpml, dt=w.dt, courant=w.courant,
                edge_rule=getattr(w, "edge_rule", 0), series_capacity=cap, **kw)
        g.set_materials(w.eps_r, w.mu_r, w.lambda_L, w.sigma)
        for s in w.sources:
            g.add_source(s.comp, s.lo, s.hi, s.amp, s.kind, s.f, s.t0, s.tw)
        for p in w.probes:
            g.add_probe(p.comp, p.p, p.freqs, p.n0)
        return g

    def close(self):
        if getattr(self, "h", None):
            load().tf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_materials(self, eps_r, mu_r, lambda_L, sigma):
        cs = (self.n[2], self.n[1], self.n[0])
        keep = []
        ptrs = []
        on_dev = 0
        for x in (eps_r, mu_r, lambda_L, sigma):
            if x is None:
                ptrs.append(None)
                continue
            if isinstance(x, np.ndarray) or np.isscalar(x):
                a = np.ascontiguousarray(np.broadcast_to(np.asarray(x, np.float32), cs))
                keep.append(a)
                ptrs.append(a.ctypes.data)
            else:
                t = x.contiguous()
                keep.append(t)
                ptrs.append(int(t.data_ptr()))
                on_dev = 1
        if on_dev and any(isinstance(k, np.ndarray) for k in keep):
            raise ValueError("mix of host and device material maps")
        _check(load().tf_set_materials(self.h, *ptrs, on_dev), "tf_set_materials")

    def set_field(self, comp: int, arr):
        if isinstance(arr, np.ndarray) or np.isscalar(arr):
            a = np.ascontiguousarray(np.broadcast_to(np.asarray(arr, np.float32), self.shape))
            _check(load().tf_set_field(self.h, int(comp), a.ctypes.data, 0), "tf_set_field")
        else:
            t = arr.contiguous()
            _check(load().tf_set_field(self.h, int(comp), int(t.data_ptr()), 1), "tf_set_field")

    def add_source(self, comp, lo, hi, amp, kind, f=0.0, t0=0.0, tw=1.0) -> int:
        i = C.c_int()
        lo_ = (C.c_int * 3)(*[int(x) for x in lo])
        hi_ = (C.c_int * 3)(*[int(x) for x in hi])
        _check(load().tf_add_source(self.h, int(comp), lo_, hi_, float(amp), int(kind), float(f), float(t0),
                                    float(tw), C.byref(i)), "tf_add_source")
        return i.value

    def add_probe(self, comp, p, freqs, n0=0) -> int:
        fr = np.ascontiguousarray(np.asarray(freqs, np.float64))
        i = C.c_int()
        p_ = (C.c_int * 3)(*[int(x) for x in p])
        _check(load().tf_add_probe(self.h, int(comp), p_, fr.ctypes.data_as(C.POINTER(C.c_double)),
                                   int(fr.size), int(n0), C.byref(i)), "tf_add_probe")
        self.freqs.append(fr)
        return i.value

    def step(self, nsteps: int):
        tf_step(self.h, nsteps)

    def sync(self):
        tf_sync(self.h)

    def step_timed(self, nsteps: int, with_total: bool = False):
        """Advance like step(); returns {kernel: (mean ms per launch, launches)}
        for the single-step kernel ("step") and the two-step kernel ("step2")
        (and, with_total, also the whole run's event time in ms)."""
        ms = (C.c_double * 3)()
        cnt = (C.c_int64 * 3)()
        tot = C.c_double()
        _check(load().tf_step_timed(self.h, int(nsteps), ms, cnt, 3, C.byref(tot)), "tf_step_timed")
        names = ("probe", "step", "step2")
        kt = {names[k]: (ms[k], int(cnt[k])) for k in range(3) if cnt[k]}
        return (kt, tot.value) if with_total else kt

    def set_two_step(self, planes):
        """Two-step passes (temporal blocking): False / 0 forbids them, True
        allows them with 24-plane work items (the default), 4 .. 24 sets the
        work-item length."""
        if planes is True:
            planes = 24
        _check(load().tf_set_two_step(self.h, int(planes or 0)), "tf_set_two_step")

    def set_item_planes(self, planes: int):
        """Planes per single-step work item (8 .. 16; a tuning switch: the
        results do not change)."""
        _check(load().tf_set_item_planes(self.h, int(planes)), "tf_set_item_planes")

    def set_wait_limit(self, polls):
        """Polls of a staged plane's mbarrier before the stepping kernels give
        the plane up and latch TF_ETIMEOUT (None: the default)."""
        _check(load().tf_set_wait_limit(self.h, -1 if polls is None else int(polls)), "tf_set_wait_limit")

    def two_step_box(self):
        """((lo, hi) of the two-step box in storage points per axis, active)."""
        lo, hi, act = (C.c_int * 3)(), (C.c_int * 3)(), C.c_int()
        _check(load().tf_two_step_box(self.h, lo, hi, C.byref(act)), "tf_two_step_box")
        return (tuple(lo), tuple(hi)), bool(act.value)

    @property
    def level(self) -> int:
        n = C.c_int64()
        _check(load().tf_get_time(self.h, C.byref(n), None), "tf_get_time")
        return int(n.value)

    def probe_dft(self, pid: int) -> np.ndarray:
        nf = self.freqs[pid].size
        re = np.zeros(max(nf, 1), np.float64)
        im = np.zeros(max(nf, 1), np.float64)
        _check(load().tf_read_probe_dft(self.h, int(pid), re.ctypes.data_as(C.POINTER(C.c_double)),
                                        im.ctypes.data_as(C.POINTER(C.c_double))), "tf_read_probe_dft")
        return (re + 1j * im)[:nf]

    def probe_series(self, pid: int, n: int) -> np.ndarray:
        out = np.zeros(int(n), np.float64)
        _check(load().tf_read_probe_series(self.h, int(pid), out.ctypes.data_as(C.POINTER(C.c_double)), int(n)),
               "tf_read_probe_series")
        return out

    def field(self, comp: int, out=None):
        """Integer-level field (SI). Returns numpy unless `out` is a CUDA tensor."""
        if out is None:
            out = np.empty(self.shape, np.float32)
        p, dev = _ptr(out)
        _check(load().tf_read_field(self.h, int(comp), p, dev), "tf_read_field")
        return out

    def field_stats(self, comp: int):
        """(sum of squares, max |value|, non-finite count) of one stored field, SI."""
        s, m, n = C.c_double(), C.c_double(), C.c_int64()
        _check(load().tf_field_stats(self.h, int(comp), C.byref(s), C.byref(m), C.byref(n)), "tf_field_stats")
        return s.value, m.value, int(n.value)

    def checkpoint_size(self) -> int:
        n = C.c_size_t()
        _check(load().tf_checkpoint_size(self.h, C.byref(n)), "tf_checkpoint_size")
        return int(n.value)

    def save_checkpoint(self, out=None):
        """State blob (numpy uint8, or into `out`: a uint8 host array or CUDA tensor)."""
        if out is None:
            out = np.empty(self.checkpoint_size(), np.uint8)
        p, dev = _ptr(out)
        nbytes = out.numel() * out.element_size() if hasattr(out, "numel") else out.nbytes
        _check(load().tf_checkpoint_save(self.h, p, int(nbytes), dev), "tf_checkpoint_save")
        return out

    def load_checkpoint(self, blob):
        p, dev = _ptr(blob)
        nbytes = blob.numel() * blob.element_size() if hasattr(blob, "numel") else blob.nbytes
        _check(load().tf_checkpoint_load(self.h, p, int(nbytes), dev), "tf_checkpoint_load")

    def adjoint(self, nsteps: int, probe: int = 0, freq_index: int = 0, segment: int = 256):
        """J = |X|^2 of probe `probe`'s DFT at `freq_index` after nsteps from rest,
        and dJ/d eps_r, dJ/d lambda_L per cell (CUDA tensors [nz][ny][nx]),
        by the discrete adjoint with checkpoints every `segment` steps."""
        import torch
        n = C.c_size_t()
        _check(load().tf_adjoint_scratch_size(self.h, int(nsteps), int(segment), C.byref(n)),
               "tf_adjoint_scratch_size")
        scratch = torch.empty(int(n.value), dtype=torch.uint8, device=self.device)
        cs = (self.n[2], self.n[1], self.n[0])
        ge = torch.empty(cs, dtype=torch.float32, device=self.device)
        gl = torch.empty(cs, dtype=torch.float32, device=self.device)
        J = C.c_double()
        _check(load().tf_adjoint_run(self.h, int(nsteps), int(probe), int(freq_index), int(segment),
                                     C.c_void_p(scratch.data_ptr()), int(n.value), C.byref(J),
                                     C.c_void_p(ge.data_ptr()), C.c_void_p(gl.data_ptr())), "tf_adjoint_run")
        del scratch
        return J.value, ge, gl

    def fit_q(self, pid: int, f_guess: float = 0.0, q_guess: float = 100.0):
        f0, al, q = C.c_double(), C.c_double(), C.c_double()
        _check(load().tf_fit_q(self.h, int(pid), float(f_guess), float(q_guess), C.byref(f0), C.byref(al),
                               C.byref(q)), "tf_fit_q")
        return {"f0": f0.value, "alpha": al.value, "Q": q.value}
