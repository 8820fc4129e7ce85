"""Seeded synthetic workloads for the two-fluid (Maxwell + London) Yee solver.

This module only *describes* problems: grid sizes, cell spacings, boundary
kinds, per-cell material maps, soft sources, probes and seeded random numbers.
It holds none of the scheme's arithmetic (no curls, no coefficients, no time
step rule), so both the CUDA library and the FP64 oracle can be fed from it
without sharing any of the method.

Geometry follows the paper's problem statement:
  * quasi-1-D slab: vacuum half-space against a superconducting half-space
    (reflection / skin-depth study, Sec. 4.1-4.2);
  * coplanar-waveguide (CPW) resonator: silicon substrate, thin metal films
    forming in-port / gap / resonator / gap / out-port along the line with
    ground planes beside it, absorbing boundaries on every face (Sec. 5).
The paper's own input decks are not available; the recipes below are the
cell-based stand-ins, with every constant written next to its meaning.

Conventions shared by every consumer:
  * material maps are float32 arrays indexed [k][j][i] (x fastest) over cells;
  * lambda_L is in metres, 0 marks a non-superconducting cell;
  * sigma is the normal-fluid conductivity in S/m;
  * boundary kinds per axis: "periodic", "pec", "mur" (z only), "cpml";
  * field component ids: 0..2 = Ex,Ey,Ez; 3..5 = Bx,By,Bz; 6..8 = Jsx,Jsy,Jsz.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# SI constants (CODATA 2018); used here only to state problem parameters
# (source frequency from a wavelength in cells, CPML strength, dt of the
# 1-D slab) -- never to advance fields.
C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 8.8541878128e-12
ETA0 = MU0 * C0

COMP = {"Ex": 0, "Ey": 1, "Ez": 2, "Bx": 3, "By": 4, "Bz": 5, "Jsx": 6, "Jsy": 7, "Jsz": 8}

SRC_GAUSS, SRC_SIN, SRC_GAUSS_SIN = 0, 1, 2
BC_KIND = {"periodic": 0, "pec": 1, "mur": 2, "cpml": 3}

BASE_SEED = 2305_13419


@dataclasses.dataclass
class CPML:
    ncells: int
    order: float
    sigma_max: float  # S/m at the outer face
    alpha_max: float  # S/m at the inner face (complex-frequency shift)


@dataclasses.dataclass
class Source:
    comp: int
    lo: Tuple[int, int, int]  # storage-point box [lo, hi)
    hi: Tuple[int, int, int]
    amp: float
    kind: int
    f: float = 0.0
    t0: float = 0.0
    tw: float = 1.0


@dataclasses.dataclass
class Probe:
    comp: int
    p: Tuple[int, int, int]
    freqs: np.ndarray  # float64, <= 64 entries, Hz
    n0: int = 0
    series: int = 0  # number of time levels to record (0: none)


@dataclasses.dataclass
class Workload:
    name: str
    n: Tuple[int, int, int]
    d: Tuple[float, float, float]
    theta: float
    bc: Tuple[str, str, str]
    eps_r: np.ndarray
    mu_r: np.ndarray
    lambda_L: np.ndarray
    sigma: np.ndarray
    courant: Optional[float] = None  # 3-D Courant number, when dt is not given
    dt: Optional[float] = None
    cpml: Tuple[Optional[CPML], Optional[CPML], Optional[CPML]] = (None, None, None)
    sources: List[Source] = dataclasses.field(default_factory=list)
    probes: List[Probe] = dataclasses.field(default_factory=list)
    nsteps: int = 0
    edge_rule: int = 0  # 0: conductor-mean at edges (interface edges fully SC), 1: plain mean
    notes: str = ""

    @property
    def ncells(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    def storage_dims(self) -> Tuple[int, int, int]:
        """Points per axis: n on a periodic axis, n + 1 (both walls) otherwise."""
        return tuple(self.n[a] + (0 if self.bc[a] == "periodic" else 1) for a in range(3))


def default_cpml(ncells: int, d: float, f_min: float, order: float = 3.0) -> CPML:
    """Roden-Gedney CPML strength: sigma_max = 0.8 (m+1) / (eta0 d), kappa = 1,
    alpha_max = 2 pi eps0 f_min (graded to zero at the outer face)."""
    return CPML(ncells=ncells, order=order,
                sigma_max=0.8 * (order + 1.0) / (ETA0 * d),
                alpha_max=2.0 * math.pi * EPS0 * f_min)


# ---------------------------------------------------------------------------
# counter-based random numbers (SplitMix64) so that any sub-box of a large
# random field can be generated without materialising the whole array
# ---------------------------------------------------------------------------
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def counter_uniform(seed: int, comp: int, dims: Sequence[int], lo: Sequence[int] = (0, 0, 0),
                    hi: Optional[Sequence[int]] = None) -> np.ndarray:
    """Uniform(-1, 1) float64 values for points [lo, hi) of a (Nx, Ny, Nz) grid,
    returned as [k][j][i]. Value = f(seed, comp, linear index) only."""
    if hi is None:
        hi = dims
    i = np.arange(lo[0], hi[0], dtype=np.uint64)
    j = np.arange(lo[1], hi[1], dtype=np.uint64)
    k = np.arange(lo[2], hi[2], dtype=np.uint64)
    lin = (k[:, None, None] * np.uint64(dims[1]) + j[None, :, None]) * np.uint64(dims[0]) + i[None, None, :]
    key = np.uint64((seed * 0x100000001B3 + comp * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        r = _splitmix64(lin ^ key)
    return (r >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


FIELD_SCALE = (1.0, 1.0, 1.0, 1.0 / C0, 1.0 / C0, 1.0 / C0, 1.0e5, 1.0e5, 1.0e5)
"""Typical magnitudes (SI) of E [V/m], B [T], Js [A/m^2] for random states."""


def random_state(seed: int, dims: Sequence[int], lo=(0, 0, 0), hi=None, comps=range(9)):
    """Random initial fields (SI units) on storage points [lo, hi)."""
    return {c: counter_uniform(seed, c, dims, lo, hi) * FIELD_SCALE[c] for c in comps}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def slab(boundary: str = "mur", vacuum: bool = False, nsteps: int = 4000, nxy: int = 4,
         nz: int = 2048, z_sc: int = 1024, lam_cells: float = 8.0, sigma_sc: float = 0.0,
         d: float = 12.5e-9, probes_z: Sequence[int] = (700, 1024, 1032, 1040, 1048, 1056),
         z_src: int = 200, wavelength_cells: float = 400.0, series: int = 0) -> Workload:
    """Quasi-1-D slab: 4 x 4 x 2048 cells, periodic in x and y, vacuum for
    z < 1024 and a superconductor (lambda_L = 8 cells, sigma = 0) above.
    Cell size 12.5 nm puts lambda_L at 100 nm (the reflection study of Sec. 4.2).
    An x-polarised soft source on the whole z = 200 plane emits a Gaussian-
    modulated sine with a vacuum wavelength of 400 cells; dt = 0.5 dz / c.
    `vacuum=True` gives the all-vacuum companion run used to separate the
    incident and reflected waves."""
    n = (nxy, nxy, nz)
    eps = np.ones((nz, nxy, nxy), np.float32)
    mu = np.ones_like(eps)
    lam = np.zeros_like(eps)
    sig = np.zeros_like(eps)
    if not vacuum:
        lam[z_sc:] = lam_cells * d
        sig[z_sc:] = sigma_sc
    f = C0 / (wavelength_cells * d)
    tw = 1.0 / (2.0 * f)
    dt = 0.5 * d / C0
    freqs = np.linspace(0.25 * f, 2.0 * f, 64)
    cp = None
    if boundary == "cpml":
        cp = default_cpml(16, d, freqs[0])
    src = Source(comp=0, lo=(0, 0, z_src), hi=(nxy, nxy, z_src + 1), amp=1.0,
                 kind=SRC_GAUSS_SIN, f=f, t0=4.0 * tw, tw=tw)
    prb = [Probe(comp=0, p=(0, 0, z), freqs=freqs, n0=0, series=series) for z in probes_z]
    return Workload(name=f"slab-{nxy}x{nxy}x{nz}-{boundary}{'-vacuum' if vacuum else ''}",
                    n=n, d=(d, d, d), theta=1.0, bc=("periodic", "periodic", boundary),
                    eps_r=eps, mu_r=mu, lambda_L=lam, sigma=sig, dt=dt,
                    cpml=(None, None, cp), sources=[src], probes=prb, nsteps=nsteps,
                    notes="f = c/(400 dz), tw = 1/(2f), t0 = 4 tw, dt = 0.5 dz/c")


def _segments(total: int, weights: Sequence[float]) -> List[int]:
    """Split `total` cells into integer segments proportional to `weights`."""
    acc, out, s = 0.0, [], sum(weights)
    prev = 0
    for w in weights:
        acc += w
        cur = int(round(total * acc / s))
        out.append(cur - prev)
        prev = cur
    return out


def cpw(n: Tuple[int, int, int] = (512, 256, 128), pml: int = 12, margin: int = 4,
        substrate_cells: int = 32, film_cells: int = 4, strip_w: int = 16, gap_w: int = 8,
        lam_cells: float = 3.0, sigma_max: float = 1.0e6, eps_sub: float = 11.7,
        d: float = 100e-9 / 3.0, courant: float = 0.95, theta: float = 1.0,
        nsteps: int = 20000, seed: int = BASE_SEED + 2, sigma_override: Optional[float] = None,
        series: int = 0, n0: Optional[int] = None) -> Workload:
    """3-D coplanar-waveguide resonator (Sec. 5 geometry, cell-based):

    * CPML of `pml` cells on all six faces, `margin` cells of vacuum/dielectric
      between any metal and the CPML (the paper keeps the PML off the London
      region);
    * silicon substrate (eps_r = 11.7) for z < pml + substrate_cells;
    * metal films `film_cells` thick on top of it: eps_r = 1, lambda_L =
      `lam_cells` cells, sigma drawn per metal cell from U[0, sigma_max] S/m;
    * the line runs along x: in-port / gap / resonator / gap / out-port in the
      paper's 100 : 100 : 600 : 100 : 100 length ratio between the margins;
      centre strip `strip_w` cells wide, `gap_w`-cell gaps, ground planes
      filling the rest of y up to the margin;
    * +/- soft source on Ey in the two gaps at the start of the in-port with a
      Gaussian-modulated sine at the estimated half-wave resonance
      f0 = c / (2 L_res sqrt((1 + eps_sub)/2)), tw = 1/(2 f0), t0 = 4 tw;
    * probes on Ey in the gap at the resonator's front edge and half way down
      the in-port, 64 frequencies uniform in [0.5 f0, 1.5 f0].
    """
    nx, ny, nz = n
    rng = np.random.Generator(np.random.PCG64(seed))
    x0, x1 = pml + margin, nx - pml - margin
    seg = _segments(x1 - x0, (100, 100, 600, 100, 100))
    xs = np.cumsum([x0] + seg)  # boundaries: inport, gap, res, gap, outport
    y0, y1 = pml + margin, ny - pml - margin
    g = (y1 - y0 - strip_w - 2 * gap_w) // 2
    y_gnd_lo = (y0, y0 + g)
    y_gap_lo = (y0 + g, y0 + g + gap_w)
    y_strip = (y0 + g + gap_w, y0 + g + gap_w + strip_w)
    y_gap_hi = (y_strip[1], y_strip[1] + gap_w)
    y_gnd_hi = (y_gap_hi[1], y1)
    z_sub = pml + substrate_cells
    z_film = (z_sub, z_sub + film_cells)

    eps = np.ones((nz, ny, nx), np.float32)
    eps[:z_sub] = eps_sub
    metal = np.zeros((nz, ny, nx), bool)
    zf = slice(*z_film)
    metal[zf, slice(*y_gnd_lo), x0:x1] = True
    metal[zf, slice(*y_gnd_hi), x0:x1] = True
    for a, b in ((xs[0], xs[1]), (xs[2], xs[3]), (xs[4], xs[5])):  # in-port, resonator, out-port
        metal[zf, slice(*y_strip), a:b] = True
    lam = np.where(metal, np.float32(lam_cells * d), np.float32(0.0)).astype(np.float32)
    if sigma_override is not None:
        sig = np.where(metal, np.float32(sigma_override), np.float32(0.0)).astype(np.float32)
    else:
        draw = rng.uniform(0.0, sigma_max, size=metal.shape).astype(np.float32)
        sig = np.where(metal, draw, np.float32(0.0)).astype(np.float32)
    mu = np.ones_like(eps)

    l_res = (xs[3] - xs[2]) * d
    f0 = C0 / (2.0 * l_res * math.sqrt((1.0 + eps_sub) / 2.0))
    tw = 1.0 / (2.0 * f0)
    freqs = np.linspace(0.5 * f0, 1.5 * f0, 64)
    cp = default_cpml(pml, d, freqs[0])
    src_x = (xs[0], xs[0] + max(1, (xs[1] - xs[0]) // 12))
    kz = (z_film[0] + 1, z_film[1])
    sources = [
        Source(comp=1, lo=(src_x[0], y_gap_lo[0], kz[0]), hi=(src_x[1], y_gap_lo[1], kz[1]),
               amp=+1.0, kind=SRC_GAUSS_SIN, f=f0, t0=4.0 * tw, tw=tw),
        Source(comp=1, lo=(src_x[0], y_gap_hi[0], kz[0]), hi=(src_x[1], y_gap_hi[1], kz[1]),
               amp=-1.0, kind=SRC_GAUSS_SIN, f=f0, t0=4.0 * tw, tw=tw),
    ]
    yprobe = (y_gap_lo[0] + y_gap_lo[1]) // 2
    zprobe = (z_film[0] + z_film[1]) // 2
    n0v = 0 if n0 is None else n0
    probes = [Probe(comp=1, p=(int(xs[2]), yprobe, zprobe), freqs=freqs, n0=n0v, series=series),
              Probe(comp=1, p=(int((xs[0] + xs[1]) // 2), yprobe, zprobe), freqs=freqs, n0=n0v,
                    series=series)]
    return Workload(name=f"cpw-{nx}x{ny}x{nz}", n=n, d=(d, d, d), theta=theta,
                    bc=("cpml", "cpml", "cpml"), eps_r=eps, mu_r=mu, lambda_L=lam, sigma=sig,
                    courant=courant, cpml=(cp, cp, cp), sources=sources, probes=probes,
                    nsteps=nsteps,
                    notes=(f"x segments {list(map(int, xs))}, y gnd/gap/strip/gap/gnd "
                           f"{y_gnd_lo}/{y_gap_lo}/{y_strip}/{y_gap_hi}/{y_gnd_hi}, "
                           f"film z {z_film}, f0 = {f0:.4e} Hz"))


def cpw_small(seed: int = BASE_SEED + 12, nsteps: int = 1200, **kw) -> Workload:
    """A scaled CPW the FP64 oracle finishes in seconds: 128 x 64 x 40 cells,
    CPML 8, 2-cell margins, 8-cell substrate, 2-cell films, 8-wide strip."""
    args = dict(n=(128, 64, 40), pml=8, margin=2, substrate_cells=8, film_cells=2,
                strip_w=8, gap_w=4, lam_cells=3.0, nsteps=nsteps, seed=seed)
    args.update(kw)
    w = cpw(**args)
    w.name = "cpw-small-" + "x".join(map(str, w.n))
    return w


def cpw_large(nsteps: int = 50000, **kw) -> Workload:
    """1024 x 512 x 256 CPW (134 M cells), lambda_L = 4 cells, CPML 16; the
    512 x 256 x 128 CPW template with every transverse feature doubled."""
    args = dict(n=(1024, 512, 256), pml=16, margin=4, substrate_cells=64, film_cells=8,
                strip_w=32, gap_w=16, lam_cells=4.0, nsteps=nsteps, seed=BASE_SEED + 5)
    args.update(kw)
    return cpw(**args)


def cpw_adjoint(nsteps: int = 8000, seed: int = BASE_SEED + 4, **kw) -> Workload:
    """The adjoint workload: a 256 x 128 x 64 CPW (the 512 x 256 x 128 template at
    half size: CPML 12, 16-cell substrate, 2-cell films, 8-wide strip) whose
    substrate eps_r is drawn per cell from U[10, 13]; the objective is |X|^2
    of probe 0's DFT at the template's resonance estimate f0 (frequency
    index 0 of a one-frequency probe)."""
    args = dict(n=(256, 128, 64), pml=12, margin=4, substrate_cells=16, film_cells=2, strip_w=8, gap_w=4,
                lam_cells=3.0, nsteps=nsteps, seed=seed)
    args.update(kw)
    w = cpw(**args)
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    z_sub = args["pml"] + args["substrate_cells"]
    w.eps_r = np.asarray(w.eps_r, np.float32).copy()
    w.eps_r[:z_sub] = rng.uniform(10.0, 13.0, size=w.eps_r[:z_sub].shape).astype(np.float32)
    f0 = w.sources[0].f
    for p in w.probes:
        p.freqs = np.array([f0])
    w.name = "cpw-adjoint-" + "x".join(map(str, w.n))
    return w


def cpw_batch(count: int = 64, seed: int = BASE_SEED + 3, nsteps: int = 8000, sizes=(96, 128, 160)):
    """The batched workload: `count` CPW resonator variants, each axis drawn
    independently from `sizes`; the 512 x 256 x 128 CPW template scaled to each grid
    (CPML, margin, substrate and film thickness in proportion to the axis),
    strip and gap widths drawn from U{4..16}, lambda_L from U[2, 6] cells and
    sigma_n per metal cell from U[0, 1e6] S/m."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        nx, ny, nz = (int(rng.choice(sizes)) for _ in range(3))
        pml = max(6, round(12 * min(nx, ny, nz) / 128))
        margin = max(2, round(4 * min(nx, ny, nz) / 128))
        sub = max(8, round(32 * nz / 128))
        film = max(2, round(4 * nz / 128))
        free_y = ny - 2 * (pml + margin)
        strip = int(rng.integers(4, 17))
        gap = int(rng.integers(4, 17))
        while strip + 2 * gap > free_y - 4:   # keep ground planes on both sides
            strip, gap = max(4, strip - 2), max(4, gap - 2)
        lam = float(rng.uniform(2.0, 6.0))
        w = cpw(n=(nx, ny, nz), pml=pml, margin=margin, substrate_cells=sub, film_cells=film, strip_w=strip,
                gap_w=gap, lam_cells=lam, nsteps=nsteps, seed=seed * 1000 + i)
        w.name = f"cpw-batch-{i}-{nx}x{ny}x{nz}"
        out.append(w)
    return out


# A 1-D column is a 1 x 1 x nz grid, periodic in x and y: a uniform plane
# wave has no x or y differences, so the transverse spacing does not enter
# the fields.  It is set to 1 mm so that the 3-D Courant number of the
# column is its 1-D one along z (the paper's 1-D runs quote the 1-D number).
COLUMN_DXY = 1.0e-3


def skin_column(sigma: float, f: float, depth: float, lam: float = 400e-9, d: float = 10e-9,
                courant_1d: float = 0.9, n_vac: int = 100, z_src: int = 50, spinup_periods: int = 4,
                window_periods: int = 2) -> Workload:
    """Skin-depth run of Sec. 4.1 / Table 1 as a 1-D column: vacuum for
    z < n_vac, a superconductor (London depth `lam`, conductivity `sigma`)
    above, dz = 10 nm, dt = 0.9 dz / c.  An x-polarised soft source at z_src
    emits a continuous sine of frequency f; after `spinup_periods` periods the
    probes' DFTs at f run over `window_periods` whole periods (the steady
    state's amplitude).  `depth` (metres, the caller's expected skin depth)
    sets the probe spacing and the column length: probes on Ex at the
    interface and at depths of 1/2, 1 and 2 `depth` inside; the
    superconductor is 25 depths thick (at least 40 cells) and ends on a wall
    of the Mur kind, as does the vacuum end."""
    m = max(1, int(round(depth / d)))
    nz = n_vac + max(25 * m, 40) + 1
    dt = courant_1d * d / C0
    per = 1.0 / (f * dt)                        # steps per period
    n0 = int(round(spinup_periods * per))
    nsteps = n0 + int(round(window_periods * per))
    eps = np.ones((nz, 1, 1), np.float32)
    mu = np.ones_like(eps)
    lam_map = np.zeros_like(eps)
    sig = np.zeros_like(eps)
    lam_map[n_vac:] = lam
    sig[n_vac:] = sigma
    src = Source(comp=0, lo=(0, 0, z_src), hi=(1, 1, z_src + 1), amp=1.0, kind=SRC_SIN, f=f)
    prb = [Probe(comp=0, p=(0, 0, n_vac + z), freqs=np.array([f]), n0=n0) for z in (0, m // 2, m, 2 * m)]
    return Workload(name=f"skin-column-sigma{sigma:g}-f{f:g}", n=(1, 1, nz), d=(COLUMN_DXY, COLUMN_DXY, d),
                    theta=1.0, bc=("periodic", "periodic", "mur"), eps_r=eps, mu_r=mu, lambda_L=lam_map, sigma=sig,
                    dt=dt, sources=[src], probes=prb, nsteps=nsteps,
                    notes=f"probe depths 0, {m // 2}, {m}, {2 * m} cells; window [{n0}, {nsteps})")


def reflection_column(sigma: float, vacuum: bool = False, nz: int = 4480, d: float = 20e-9, z_if: int = 350,
                      z_probe: int = 340, nsteps: int = 15800, tw: float = 0.25e-15) -> Workload:
    """Reflection run of Sec. 4.2 as a 1-D column: 4480 cells of dz = 20 nm,
    dt = 0.95 dz / c, a superconductor (lambda_L = 100 nm, conductivity
    `sigma`) from 7 um, Mur walls; a short Gaussian soft source (tw = 0.25 fs,
    t0 = 4 tw) on Ex at 100 nm covers 0 - 1000 THz; probe at 6.8 um with 64
    frequencies over 20 - 1000 THz.  `vacuum=True` is the companion run
    without the superconductor (the incident wave)."""
    eps = np.ones((nz, 1, 1), np.float32)
    mu = np.ones_like(eps)
    lam = np.zeros_like(eps)
    sig = np.zeros_like(eps)
    if not vacuum:
        lam[z_if:] = 100e-9
        sig[z_if:] = sigma
    src = Source(comp=0, lo=(0, 0, 5), hi=(1, 1, 6), amp=1.0, kind=SRC_GAUSS, t0=4 * tw, tw=tw)
    prb = [Probe(comp=0, p=(0, 0, z_probe), freqs=np.linspace(20e12, 1000e12, 64), n0=0)]
    return Workload(name=f"reflection-column-sigma{sigma:g}{'-vacuum' if vacuum else ''}", n=(1, 1, nz),
                    d=(COLUMN_DXY, COLUMN_DXY, d), theta=1.0, bc=("periodic", "periodic", "mur"), eps_r=eps,
                    mu_r=mu, lambda_L=lam, sigma=sig, dt=0.95 * d / C0, sources=[src], probes=prb, nsteps=nsteps)


def random_box(n=(9, 7, 11), bc=("periodic", "periodic", "periodic"), seed: int = 1,
               d=(10e-9, 12e-9, 8e-9), courant: float = 0.9, theta: float = 0.5,
               sc_fraction: float = 0.5, lam_range=(30e-9, 60e-9), sigma_range=(0.0, 1e6),
               eps_range=(1.0, 4.0), mu_range=(1.0, 1.0), cpml_cells: int = 4) -> Workload:
    """Small heterogeneous box with random per-cell materials, for exactness and
    parity checks on odd sizes and every boundary kind."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 1000 + seed))
    shape = (n[2], n[1], n[0])
    eps = rng.uniform(*eps_range, size=shape).astype(np.float32)
    mu = rng.uniform(*mu_range, size=shape).astype(np.float32)
    sc = rng.uniform(size=shape) < sc_fraction
    lam = np.where(sc, rng.uniform(*lam_range, size=shape), 0.0).astype(np.float32)
    sig = rng.uniform(*sigma_range, size=shape).astype(np.float32)
    cp = tuple(default_cpml(cpml_cells, d[a], 1e12) if bc[a] == "cpml" else None for a in range(3))
    return Workload(name=f"box-{'x'.join(map(str, n))}-{'-'.join(bc)}", n=tuple(n), d=tuple(d),
                    theta=theta, bc=tuple(bc), eps_r=eps, mu_r=mu, lambda_L=lam, sigma=sig,
                    courant=courant, cpml=cp)


def all_configs():
    """Named workloads: the 4 x 4 x 2048 slab, the 512 x 256 x 128 CPW and the 1024 x 512 x 256 CPW."""
    return {"slab": slab, "cpw": cpw, "cpw_small": cpw_small, "cpw_large": cpw_large}
