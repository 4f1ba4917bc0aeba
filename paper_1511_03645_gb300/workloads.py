"""Seeded synthetic inputs for the adjoint-guided AMR wave solver.

This module is shared by the CUDA library's tests/benchmarks and by the CPU
oracle.  It holds NO arithmetic of the numerical method (no Riemann solver,
limiter, interpolation, flagging or clustering): only the problem data of the
workloads -- domains, media, initial conditions, targets, tolerances -- and
the seeded random draws that define them.  Every transcendental (exp, tanh)
is evaluated here, once, and the same numbers go to both implementations.

Workloads (Davis & LeVeque, "Adjoint methods for guiding adaptive mesh
refinement in wave propagation problems"):

* ``config1``: 1D variable-coefficient acoustics (Sec. 5.1 setting), 2 levels.
* ``config2``: 2D layered acoustics (Sec. 5.2 setting), 3 levels.
* ``config3``: 2D linearised shallow water over synthetic bathymetry
  (Sec. 5.3 setting, synthetic stand-in for the Pacific/Crescent City case).
* ``config4``: 4096 independent patches of uneven sizes (batching stress).
* ``config5``: a seeded Poisson stream of 2D acoustics requests (serving).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

# Equation / boundary / mode codes.  Both implementations use these values.
EQ_ACOUSTICS = 0       # forward variable-coefficient acoustics (wave form)
EQ_ACOUSTICS_ADJ = 1   # time-reversed adjoint acoustics (f-wave form)
EQ_SW = 2              # forward linearised shallow water (f-wave form)
EQ_SW_ADJ = 3          # time-reversed adjoint linearised shallow water (f-wave)

BC_EXTRAP = 0
BC_WALL = 1
BC_PERIODIC = 2

FLAG_BRACKET_MAX = 0
FLAG_LINEAR = 1
FLAG_DIFFERENCE = 2   # standard flagging: undivided differences of every component
FLAG_SURFACE = 3      # standard flagging: |first component| (surface elevation)
FLAG_ERROR = 4        # adjoint-weighted Richardson error estimate (Sec. 7)
FLAG_RICHARDSON = 5   # standard flagging: the Richardson error estimate itself (Sec. 1)

GRAV = 9.81

# q_out layout is field-major: q_out[f*n + k] for field f of point k.
QINIT_CFUNC = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.c_int,
                               ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double),
                               ctypes.c_void_p)


def make_qinit_callback(fn: Callable[[np.ndarray, np.ndarray], np.ndarray], m: int):
    """Wrap ``fn(xc, yc) -> q[m, n]`` as a C callback.

    The C side calls ``cb(level, n, xc, yc, q_out, user)``; ``xc``/``yc`` are
    cell centres computed by the caller, ``q_out`` receives ``m*n`` doubles.
    The returned object must be kept alive while either library may call it.
    """

    def _cb(level, n, xc, yc, q_out, user):
        if n <= 0:
            return
        x = np.ctypeslib.as_array(xc, shape=(n,)).copy()
        y = np.ctypeslib.as_array(yc, shape=(n,)).copy()
        q = np.asarray(fn(x, y), dtype=np.float64).reshape(m, n)
        out = np.ctypeslib.as_array(q_out, shape=(m * n,))
        out[:] = q.reshape(-1)

    return QINIT_CFUNC(_cb)


@dataclass
class Target:
    """phi = weight * indicator(box) on field 0 (pressure or surface)."""
    x0: float
    x1: float
    y0: float = 0.0
    y1: float = 1.0
    weight: float = 1.0


@dataclass
class Medium:
    """Primary medium data.

    kind == "layered": piecewise-constant layers along ``axis`` (0 = x,
      1 = y); layer k holds cells whose centre coordinate c satisfies
      iface[k-1] <= c < iface[k]; acoustics only (rho, K per layer).
    kind == "dense": one array per level covering that level's whole index
      space, ``fields[level]`` of shape (nmed, M_l, N_l); acoustics: (rho, K),
      shallow water: (hbar,).
    """
    kind: str
    axis: int = 0
    iface: Optional[np.ndarray] = None
    rho: Optional[np.ndarray] = None
    K: Optional[np.ndarray] = None
    fields: Optional[list] = None
    cmax: float = 0.0


@dataclass
class Workload:
    name: str
    dim: int
    eqn: int
    lo: tuple
    hi: tuple
    n0: tuple
    ratios: tuple
    bc: tuple
    cfl: float
    cfl_max: float
    t0: float
    tf: float
    ts: float
    tol: float
    medium: Medium
    qinit: Callable[[np.ndarray, np.ndarray], np.ndarray]
    target: Target
    adj_n: tuple
    nsnap: int
    regrid_interval: int = 2
    buffer: int = 2
    cluster_eff: float = 0.7
    min_patch: int = 8
    max_patch: int = 64
    max_patch0: int = 64
    flag_mode: int = FLAG_BRACKET_MAX
    reflux: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def nlevels(self) -> int:
        return len(self.ratios) + 1

    @property
    def m(self) -> int:
        return 2 if self.dim == 1 else 3

    @property
    def adj_eqn(self) -> int:
        return EQ_ACOUSTICS_ADJ if self.eqn == EQ_ACOUSTICS else EQ_SW_ADJ

    def level_shape(self, level: int):
        """(N_l, M_l): index extents of level ``level``."""
        r = 1
        for k in range(level):
            r *= self.ratios[k]
        nx = self.n0[0] * r
        ny = self.n0[1] * r if self.dim == 2 else 1
        return nx, ny

    def level_dx(self, level: int):
        nx, ny = self.level_shape(level)
        dx = (self.hi[0] - self.lo[0]) / nx
        dy = (self.hi[1] - self.lo[1]) / ny if self.dim == 2 else 1.0
        return dx, dy

    def adjoint_phi(self) -> np.ndarray:
        """Adjoint data at t_f on the adjoint grid: phi = weight * (fraction
        of the cell inside the target box) on field 0, zero elsewhere.
        Shape (m, ny, nx) (ny = 1 in 1D)."""
        nx = self.adj_n[0]
        ny = self.adj_n[1] if self.dim == 2 else 1
        dx = (self.hi[0] - self.lo[0]) / nx
        xl = self.lo[0] + np.arange(nx) * dx
        fx = np.clip(np.minimum(xl + dx, self.target.x1) - np.maximum(xl, self.target.x0), 0.0, None) / dx
        if self.dim == 2:
            dy = (self.hi[1] - self.lo[1]) / ny
            yl = self.lo[1] + np.arange(ny) * dy
            fy = np.clip(np.minimum(yl + dy, self.target.y1) - np.maximum(yl, self.target.y0), 0.0, None) / dy
        else:
            fy = np.ones(1)
        phi = np.zeros((self.m, ny, nx))
        phi[0] = self.target.weight * fy[:, None] * fx[None, :]
        return phi

    def qinit_callback(self):
        return make_qinit_callback(self.qinit, self.m)


def _layered_cmax(rho, K):
    return float(np.max(np.sqrt(np.asarray(K, dtype=np.float64) / np.asarray(rho, dtype=np.float64))))


# --------------------------------------------------------------------------
# config 1: 1D variable-coefficient acoustics, 2 levels
# --------------------------------------------------------------------------
def config1(n0: int = 200, ratio: int = 4, tf: float = 20.0, adj_n: int = 800, nsnap: int = 100,
            tol: float = 1e-3, bc=(BC_EXTRAP, BC_EXTRAP), ts: float = 0.0) -> Workload:
    """1D acoustics on [-4,4]: rho=1,K=4 (x<0) | rho=1,K=1 (x>=0); Gaussian
    pressure exp(-20(x+2)^2), u=0; target: pressure on [0.5,1.5] over the
    time range [t_s, t_f] (default t_s = 0: with extrapolation boundaries all
    waves leave the domain long before t_f = 20, so a single time point of
    interest would flag nothing)."""
    rho = np.array([1.0, 1.0])
    K = np.array([4.0, 1.0])
    med = Medium(kind="layered", axis=0, iface=np.array([0.0]), rho=rho, K=K, cmax=_layered_cmax(rho, K))

    def qinit(x, y):
        p = np.exp(-20.0 * (x + 2.0) ** 2)
        return np.stack([p, np.zeros_like(p)])

    return Workload(name="acoustics1d", dim=1, eqn=EQ_ACOUSTICS, lo=(-4.0, 0.0), hi=(4.0, 1.0),
                    n0=(n0, 1), ratios=(ratio,), bc=(bc[0], bc[1], BC_EXTRAP, BC_EXTRAP),
                    cfl=0.9, cfl_max=1.0, t0=0.0, tf=tf, ts=ts, tol=tol, medium=med, qinit=qinit,
                    target=Target(0.5, 1.5), adj_n=(adj_n, 1), nsnap=nsnap,
                    min_patch=4, max_patch=256, max_patch0=256)


# --------------------------------------------------------------------------
# config 2: 2D layered acoustics, 3 levels (ratios 2, 4)
# --------------------------------------------------------------------------
def config2(seed: int = 0, n0: int = 100, ratios=(2, 4), tf: float = 8.0, adj_n: int = 400,
            nsnap: int = 200, tol: float = 0.01, ts: Optional[float] = None,
            bc=(BC_EXTRAP,) * 4, lo=-4.0, hi=4.0, target=(2.0, 2.5, 2.0, 2.5),
            min_patch: int = 8, max_patch: int = 64) -> Workload:
    """2D acoustics on [-4,4]^2 with 4 horizontal layers (interfaces y=-2,0,2;
    rho ~ U[1,3], c ~ U[1,4] per layer, K = rho c^2); pressure Gaussian
    exp(-r^2/0.2^2) at a seeded centre in [-3,3]^2 at least 0.5 away from the
    target box; target: pressure on [2,2.5]^2."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(1.0, 3.0, size=4)
    c = rng.uniform(1.0, 4.0, size=4)
    K = rho * c * c
    med = Medium(kind="layered", axis=1, iface=np.array([-2.0, 0.0, 2.0]) * (hi - lo) / 8.0,
                 rho=rho, K=K, cmax=_layered_cmax(rho, K))
    tx0, tx1, ty0, ty1 = target
    span = 3.0 * (hi - lo) / 8.0
    while True:
        xc, yc = rng.uniform(-span, span, size=2)
        dxb = max(tx0 - xc, 0.0, xc - tx1)
        dyb = max(ty0 - yc, 0.0, yc - ty1)
        if math.hypot(dxb, dyb) >= 0.5:
            break
    w = 0.2

    def qinit(x, y):
        p = np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (w * w))
        z = np.zeros_like(p)
        return np.stack([p, z, z])

    return Workload(name="acoustics2d", dim=2, eqn=EQ_ACOUSTICS, lo=(lo, lo), hi=(hi, hi),
                    n0=(n0, n0), ratios=tuple(ratios), bc=tuple(bc), cfl=0.9, cfl_max=1.0,
                    t0=0.0, tf=tf, ts=tf if ts is None else ts, tol=tol, medium=med, qinit=qinit,
                    target=Target(tx0, tx1, ty0, ty1), adj_n=(adj_n, adj_n), nsnap=nsnap,
                    min_patch=min_patch, max_patch=max_patch, max_patch0=64,
                    extra={"source": (float(xc), float(yc))})


# --------------------------------------------------------------------------
# config 3: 2D linearised shallow water over synthetic bathymetry
# --------------------------------------------------------------------------
def bathymetry(x: np.ndarray, y: np.ndarray, mounts: np.ndarray, L: float = 2.0e6) -> np.ndarray:
    """Depth below sea level (m) at points (x, y) in metres.

    Abyssal plain of 4000 m rising through a tanh ramp centred at 0.75 L to a
    200 m shelf in the east, minus seeded Gaussian seamounts
    (height, width, cx, cy), floored at 50 m so that every cell is wet."""
    s = L / 2.0e6
    h0 = 200.0 + 3800.0 * 0.5 * (1.0 - np.tanh((x - 1.5e6 * s) / (5.0e4 * s)))
    bump = np.zeros_like(x)
    for hgt, wid, cx, cy in mounts:
        bump += hgt * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (wid * wid))
    return np.maximum(h0 - bump, 50.0)


def config3(seed: int = 0, n0: int = 200, ratios=(4, 4, 2), tf: float = 4.0 * 3600.0,
            adj_n: int = 1000, nsnap: int = 300, tol: float = 4e-3, L: float = 2.0e6,
            nmounts: int = 20, min_patch: int = 8, max_patch: int = 64,
            dense_levels: Optional[int] = None) -> Workload:
    """Linearised shallow water on [0,L]^2 (L = 2000 km), all cells wet.

    Medium per cell of every level = bathymetry at the cell centre (dense
    per-level arrays).  Initial condition: 1 m Gaussian surface hump of width
    50 km at a seeded point with x < 0.5 L; zero momentum.  Target: a
    20 km x 20 km box on the shelf, [1900,1920] x [990,1010] km (scaled with
    L).  Time range of interest [t_f/2, t_f]."""
    rng = np.random.default_rng(seed)
    s = L / 2.0e6
    mounts = np.stack([rng.uniform(500.0, 2500.0, nmounts),
                       rng.uniform(2.0e4, 8.0e4, nmounts) * s,
                       rng.uniform(0.0, 1.3e6 * s, nmounts),
                       rng.uniform(0.0, L, nmounts)], axis=1)
    src = (float(rng.uniform(0.1 * L, 0.5 * L)), float(rng.uniform(0.2 * L, 0.8 * L)))
    wl = Workload(name="shallow_water2d", dim=2, eqn=EQ_SW, lo=(0.0, 0.0), hi=(L, L),
                  n0=(n0, n0), ratios=tuple(ratios), bc=(BC_EXTRAP,) * 4, cfl=0.9, cfl_max=1.0,
                  t0=0.0, tf=tf, ts=0.5 * tf, tol=tol, medium=Medium(kind="dense"),
                  qinit=None, target=Target(1.9e6 * s, 1.92e6 * s, 0.99e6 * s, 1.01e6 * s),
                  adj_n=(adj_n, adj_n), nsnap=nsnap, min_patch=min_patch, max_patch=max_patch,
                  max_patch0=64, extra={"mounts": mounts, "source": src})
    wsrc = 5.0e4 * s

    def qinit(x, y):
        eta = np.exp(-((x - src[0]) ** 2 + (y - src[1]) ** 2) / (wsrc * wsrc))
        z = np.zeros_like(eta)
        return np.stack([eta, z, z])

    wl.qinit = qinit
    nlev = wl.nlevels if dense_levels is None else dense_levels
    fields = []
    for lev in range(nlev):
        nx, ny = wl.level_shape(lev)
        dx, dy = wl.level_dx(lev)
        xc = wl.lo[0] + (np.arange(nx) + 0.5) * dx
        yc = wl.lo[1] + (np.arange(ny) + 0.5) * dy
        X, Y = np.meshgrid(xc, yc)
        fields.append(bathymetry(X, Y, mounts, L)[None, :, :].copy())
    hmax = max(float(f.max()) for f in fields)
    wl.medium = Medium(kind="dense", fields=fields, cmax=float(np.sqrt(GRAV * hmax)))
    return wl


def config3_adjoint_medium(wl: Workload, ratios=None):
    """Bathymetry of a config-3 workload at the cell centres of its adjoint
    grid, shape (1, ay, ax) (the adjoint solve's dense medium); with ratios,
    the list of those arrays for every level of an adjoint hierarchy whose
    level 0 is the adjoint grid."""
    out = []
    nx, ny = wl.adj_n
    for r in [1] + list(ratios or []):
        nx, ny = nx * r, ny * r
        xa = wl.lo[0] + (np.arange(nx) + 0.5) * (wl.hi[0] - wl.lo[0]) / nx
        ya = wl.lo[1] + (np.arange(ny) + 0.5) * (wl.hi[1] - wl.lo[1]) / ny
        X, Y = np.meshgrid(xa, ya)
        out.append(bathymetry(X, Y, wl.extra["mounts"], wl.hi[0])[None])
    return out if ratios is not None else out[0]


# --------------------------------------------------------------------------
# the paper's two-dimensional acoustics examples (Sec. 5.2)
# --------------------------------------------------------------------------
PAPER_5_2_VARIANTS = ("timepoint_walls", "range_walls", "range_mixed")


def paper_5_2(variant: str = "range_walls", n0: int = 50, nsnap: Optional[int] = None,
              tol: float = 0.02) -> Workload:
    """Sec. 5.2: homogeneous acoustics (K = 4, rho = 1) on [-4,8] x [-1,11],
    a radially symmetric pressure hump at (0.5, 1), the pressure over
    [3.32,3.8] x [0.32,0.8] with weight 2 (Eq. eq:phi_2d) as the quantity of
    interest, 3 levels with ratio 2, coarse and adjoint grids 50 x 50,
    tolerance 0.02.

    Variants: "timepoint_walls" (Sec. 5.2.1: walls, t_s = t_f = 1.5),
    "range_walls" (Sec. 5.2.2: walls, t_f = 6, t_s = 1), "range_mixed"
    (Sec. 5.2.3: walls at x = 8 and y = -1, outflow at x = -4 and y = 11).
    The hump is read as p = 1 + cos(pi (r - 0.3)/w) for |r - 0.3| <= w,
    w = 0.15 (the printed formula is garbled: its centre differs between the
    two expressions and "3 + cos" does not vanish at the edge).  Snapshots:
    one every 0.05 in time (the paper does not say how many)."""
    if variant not in PAPER_5_2_VARIANTS:
        raise ValueError(variant)
    tf, ts = (1.5, 1.5) if variant == "timepoint_walls" else (6.0, 1.0)
    if variant == "range_mixed":
        bc = (BC_EXTRAP, BC_WALL, BC_WALL, BC_EXTRAP)   # x = a outflow, x = b wall, y = alpha wall, y = beta outflow
    else:
        bc = (BC_WALL,) * 4
    rho = np.array([1.0])
    K = np.array([4.0])
    med = Medium(kind="layered", axis=0, iface=np.zeros(0), rho=rho, K=K, cmax=_layered_cmax(rho, K))
    w = 0.15

    def qinit(x, y):
        r = np.sqrt((x - 0.5) ** 2 + (y - 1.0) ** 2)
        p = np.where(np.abs(r - 0.3) <= w, 1.0 + np.cos(np.pi * (r - 0.3) / w), 0.0)
        z = np.zeros_like(p)
        return np.stack([p, z, z])

    if nsnap is None:
        nsnap = int(round(tf / 0.05)) + 1
    return Workload(name="acoustics2d-sec5.2-" + variant, dim=2, eqn=EQ_ACOUSTICS, lo=(-4.0, -1.0),
                    hi=(8.0, 11.0), n0=(n0, n0), ratios=(2, 2), bc=bc, cfl=0.9, cfl_max=1.0, t0=0.0, tf=tf,
                    ts=ts, tol=tol, medium=med, qinit=qinit, target=Target(3.32, 3.8, 0.32, 0.8, weight=2.0),
                    adj_n=(n0, n0), nsnap=nsnap, min_patch=8, max_patch=64, max_patch0=64,
                    extra={"gauge": (3.5, 0.5)})


# --------------------------------------------------------------------------
# config 4: batching stress test, 4096 independent patches
# --------------------------------------------------------------------------
@dataclass
class PatchBatch:
    """Independent 2D acoustics patches; each patch is its own domain with
    extrapolation boundaries.  Arrays have one entry per patch."""
    nx: np.ndarray
    ny: np.ndarray
    level: np.ndarray
    dx: np.ndarray
    dt: np.ndarray
    x0: np.ndarray          # lower-left corner of the patch
    y0: np.ndarray
    medium_id: np.ndarray   # index into media
    media: list             # list of Medium (layered along y)
    src: np.ndarray         # Gaussian centre per patch (x, y)
    order: np.ndarray       # shuffled submission order

    @property
    def npatch(self) -> int:
        return int(self.nx.shape[0])

    def cells(self) -> int:
        return int(np.sum(self.nx.astype(np.int64) * self.ny.astype(np.int64)))

    def qinit_patch(self, k: int) -> np.ndarray:
        """Initial (p, u, v) on patch k's interior, shape (3, ny, nx)."""
        nx, ny, dx = int(self.nx[k]), int(self.ny[k]), float(self.dx[k])
        xc = self.x0[k] + (np.arange(nx) + 0.5) * dx
        yc = self.y0[k] + (np.arange(ny) + 0.5) * dx
        X, Y = np.meshgrid(xc, yc)
        w = 0.2
        p = np.exp(-((X - self.src[k, 0]) ** 2 + (Y - self.src[k, 1]) ** 2) / (w * w))
        z = np.zeros_like(p)
        return np.stack([p, z, z])


def config4(seed: int = 0, npatch: int = 4096, emin: int = 8, emax: int = 128, nmedia: int = 4) -> PatchBatch:
    """4096 patches: nx ~ U{emin..emax}, ny ~ U{max(emin, ceil(nx/4)) ..
    min(emax, 4 nx)}; level ~ U{0,1,2} with dx = 0.08/(1,2,8); dt from
    CFL 0.9 on each patch's own medium maximum speed; 4-layer seeded media."""
    rng = np.random.default_rng(seed)
    nx = rng.integers(emin, emax + 1, size=npatch)
    ny = np.array([rng.integers(max(emin, -(-int(a) // 4)), min(emax, 4 * int(a)) + 1) for a in nx])
    level = rng.integers(0, 3, size=npatch)
    dxs = np.array([0.08, 0.04, 0.01])
    dx = dxs[level]
    media = []
    for _ in range(nmedia):
        rho = rng.uniform(1.0, 3.0, size=4)
        c = rng.uniform(1.0, 4.0, size=4)
        K = rho * c * c
        media.append(Medium(kind="layered", axis=1, iface=np.array([-2.0, 0.0, 2.0]),
                            rho=rho, K=K, cmax=_layered_cmax(rho, K)))
    medium_id = rng.integers(0, nmedia, size=npatch)
    x0 = np.array([rng.uniform(-4.0, 4.0 - n * d) if n * d < 8.0 else -4.0 for n, d in zip(nx, dx)])
    y0 = np.array([rng.uniform(-4.0, 4.0 - n * d) if n * d < 8.0 else -4.0 for n, d in zip(ny, dx)])
    cm = np.array([media[i].cmax for i in medium_id])
    dt = 0.9 * dx / cm
    src = np.stack([x0 + 0.5 * nx * dx, y0 + 0.5 * ny * dx], axis=1)
    order = rng.permutation(npatch)
    return PatchBatch(nx=nx.astype(np.int32), ny=ny.astype(np.int32), level=level.astype(np.int32),
                      dx=dx, dt=dt, x0=x0, y0=y0, medium_id=medium_id.astype(np.int32), media=media,
                      src=src, order=order.astype(np.int32))


# --------------------------------------------------------------------------
# config 5: serving, Poisson arrivals of 2D acoustics requests
# --------------------------------------------------------------------------
@dataclass
class Request:
    rid: int
    arrival: float        # seconds after the start of the stream
    n0: int
    ratios: tuple
    medium_id: int
    source: tuple


def config5(seed: int = 0, nreq: int = 512, rate: float = 1.0, nmedia: int = 8,
            nmin: int = 64, nmax: int = 512):
    """Requests with coarse grids n0 log-uniform in [nmin, nmax] (rounded to a
    multiple of 8), 2 or 3 levels (ratios (2,) or (2,4)), a medium drawn from
    ``nmedia`` shared layered media and a seeded Gaussian source; arrival
    times from a Poisson process of the given rate (requests/second)."""
    rng = np.random.default_rng(seed)
    media = []
    for _ in range(nmedia):
        rho = rng.uniform(1.0, 3.0, size=4)
        c = rng.uniform(1.0, 4.0, size=4)
        K = rho * c * c
        media.append(Medium(kind="layered", axis=1, iface=np.array([-2.0, 0.0, 2.0]),
                            rho=rho, K=K, cmax=_layered_cmax(rho, K)))
    gaps = rng.exponential(1.0 / rate, size=nreq)
    arrivals = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(nreq):
        n0 = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax))) / 8.0)) * 8
        ratios = (2,) if rng.integers(0, 2) == 0 else (2, 4)
        mid = int(rng.integers(0, nmedia))
        while True:
            xc, yc = rng.uniform(-3.0, 3.0, size=2)
            if math.hypot(max(2.0 - xc, 0.0, xc - 2.5), max(2.0 - yc, 0.0, yc - 2.5)) >= 0.5:
                break
        reqs.append(Request(rid=i, arrival=float(arrivals[i]), n0=n0, ratios=ratios,
                            medium_id=mid, source=(float(xc), float(yc))))
    return media, reqs


def request_workload(req: Request, media, tf: float = 8.0, tol: float = 0.01,
                     adj_n: int = 400, nsnap: int = 200) -> Workload:
    """The 2D acoustics workload of one serving request (domain and t_f as
    config 2; the adjoint grid is the shared one of its medium)."""
    med = media[req.medium_id]
    xc, yc = req.source
    w = 0.2

    def qinit(x, y):
        p = np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (w * w))
        z = np.zeros_like(p)
        return np.stack([p, z, z])

    return Workload(name=f"request{req.rid}", dim=2, eqn=EQ_ACOUSTICS, lo=(-4.0, -4.0), hi=(4.0, 4.0),
                    n0=(req.n0, req.n0), ratios=req.ratios, bc=(BC_EXTRAP,) * 4, cfl=0.9,
                    cfl_max=1.0, t0=0.0, tf=tf, ts=tf, tol=tol, medium=med, qinit=qinit,
                    target=Target(2.0, 2.5, 2.0, 2.5), adj_n=(adj_n, adj_n), nsnap=nsnap)
