"""ctypes front end of the plain CPU FP64 oracle (``adjamr_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by ``bench.py``'s CPU-baseline leg, never by the library.  The oracle is
compiled here with ``gcc -O2 -ffp-contract=off`` (no fused multiply-add, every
operation rounded as written).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adjamr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXLEV = 8


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("eqn", ctypes.c_int),
        ("lo", ctypes.c_double * 2), ("hi", ctypes.c_double * 2),
        ("n0", ctypes.c_int * 2), ("nlevels", ctypes.c_int),
        ("ratio", ctypes.c_int * MAXLEV), ("bc", ctypes.c_int * 4),
        ("cfl", ctypes.c_double), ("cfl_max", ctypes.c_double), ("cmax", ctypes.c_double),
        ("dt0", ctypes.c_double),
        ("t0", ctypes.c_double), ("tf", ctypes.c_double), ("ts", ctypes.c_double), ("tol", ctypes.c_double),
        ("regrid_interval", ctypes.c_int), ("buffer", ctypes.c_int),
        ("cluster_eff", ctypes.c_double),
        ("min_patch", ctypes.c_int), ("max_patch", ctypes.c_int), ("max_patch0", ctypes.c_int),
        ("flag_mode", ctypes.c_int),
        ("qinit", ctypes.c_void_p), ("qinit_user", ctypes.c_void_p),
        ("reflux", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            dp = P(ctypes.c_double)
            L.orc_create.restype = vp
            L.orc_create.argtypes = [P(OrcParams)]
            L.orc_destroy.argtypes = [vp]
            L.orc_set_medium_layered.argtypes = [vp, i, i, dp, dp, dp]
            L.orc_set_medium_dense.argtypes = [vp, i, dp]
            L.orc_set_adjoint.argtypes = [vp, i, i, i, dp, P(ctypes.c_ubyte)]
            L.orc_regrid.argtypes = [vp, i, i]
            L.orc_advance.argtypes = [vp, i, dp]
            L.orc_flag.argtypes = [vp, i, d, P(ctypes.c_ubyte), P(ctypes.c_long)]
            L.orc_error_estimate.argtypes = [vp, i, dp, ctypes.c_long]
            L.orc_set_nstep.argtypes = [vp, i, ctypes.c_long]
            L.orc_npatches.argtypes = [vp, i]
            L.orc_get_patches.argtypes = [vp, i, P(ctypes.c_int)]
            L.orc_level_dt.restype = d
            L.orc_level_dt.argtypes = [vp, i]
            L.orc_cell_updates.restype = ctypes.c_longlong
            L.orc_cell_updates.argtypes = [vp]
            L.orc_level_nstep.restype = ctypes.c_long
            L.orc_level_nstep.argtypes = [vp, i]
            L.orc_error.restype = ctypes.c_char_p
            L.orc_error.argtypes = [vp]
            L.orc_read_level.restype = ctypes.c_long
            L.orc_read_level.argtypes = [vp, i, dp]
            L.orc_write_level.restype = ctypes.c_long
            L.orc_write_level.argtypes = [vp, i, dp]
            L.orc_read_patch_ghosted.restype = ctypes.c_long
            L.orc_read_patch_ghosted.argtypes = [vp, i, i, dp, dp]
            L.orc_fill_ghosts.argtypes = [vp, i]
            L.orc_functional.restype = d
            L.orc_functional.argtypes = [vp, d, d, d, d, d]
            L.orc_step_patch.argtypes = [i, i, i, i, dp, dp, d, d, d, dp, dp]
            L.orc_adjoint_solve.argtypes = [P(OrcParams), i, i, dp, dp, dp, dp, dp, i, dp]
            L.orc_cluster.argtypes = [P(ctypes.c_ubyte), P(ctypes.c_ubyte), i, i, i, i, d, P(ctypes.c_int), i]
            L.orc_set_gauges.argtypes = [vp, i, dp, dp]
            L.orc_set_layout.argtypes = [vp, i, i, P(ctypes.c_int)]
            L.orc_adjoint_solve_amr.argtypes = [P(OrcParams), i, i, dp, dp, dp, dp, dp, i, dp]
            L.orc_read_gauges.restype = ctypes.c_long
            L.orc_read_gauges.argtypes = [vp, dp, ctypes.c_long]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def params_from_workload(wl, eqn=None, nlevels=None, n0=None, tol=None, dt0=0.0, qinit=None, tf=None):
    P = OrcParams()
    P.dim = wl.dim
    P.eqn = wl.eqn if eqn is None else eqn
    P.lo[0], P.lo[1] = wl.lo
    P.hi[0], P.hi[1] = wl.hi
    nn = wl.n0 if n0 is None else n0
    P.n0[0], P.n0[1] = nn[0], (nn[1] if wl.dim == 2 else 1)
    P.nlevels = wl.nlevels if nlevels is None else nlevels
    for k, r in enumerate(wl.ratios):
        P.ratio[k] = r
    for k in range(4):
        P.bc[k] = wl.bc[k]
    P.cfl, P.cfl_max, P.cmax, P.dt0 = wl.cfl, wl.cfl_max, wl.medium.cmax, dt0
    P.t0, P.tf, P.ts = wl.t0, (wl.tf if tf is None else tf), wl.ts
    P.tol = wl.tol if tol is None else tol
    P.regrid_interval, P.buffer, P.cluster_eff = wl.regrid_interval, wl.buffer, wl.cluster_eff
    P.min_patch, P.max_patch, P.max_patch0 = wl.min_patch, wl.max_patch, wl.max_patch0
    P.flag_mode = wl.flag_mode
    P.reflux = int(getattr(wl, "reflux", 0))
    if qinit is not None:
        P.qinit = ctypes.cast(qinit, ctypes.c_void_p)
    return P


class OracleHierarchy:
    """The oracle's AMR hierarchy for one workload."""

    def __init__(self, wl, *, nlevels=None, tol=None, dt0=0.0, with_qinit=True, tf=None):
        self.wl = wl
        self.m = wl.m
        self._cb = wl.qinit_callback() if (with_qinit and wl.qinit is not None) else None
        self.P = params_from_workload(wl, nlevels=nlevels, tol=tol, dt0=dt0, qinit=self._cb, tf=tf)
        self.nlevels = self.P.nlevels
        self.h = lib().orc_create(ctypes.byref(self.P))
        if not self.h:
            raise RuntimeError("orc_create failed")
        self._keep = []
        med = wl.medium
        if med.kind == "layered":
            iface = np.ascontiguousarray(med.iface, dtype=np.float64)
            if iface.size == 0:
                iface = np.zeros(1)
            f0 = np.ascontiguousarray(med.rho, dtype=np.float64)
            f1 = np.ascontiguousarray(med.K, dtype=np.float64)
            self._keep += [iface, f0, f1]
            rc = lib().orc_set_medium_layered(self.h, med.axis, f0.size, _dp(iface), _dp(f0), _dp(f1))
            if rc:
                raise RuntimeError("orc_set_medium_layered failed")
        else:
            for lev in range(self.nlevels):
                arr = np.ascontiguousarray(med.fields[lev], dtype=np.float64)
                rc = lib().orc_set_medium_dense(self.h, lev, _dp(arr))
                if rc:
                    raise RuntimeError("orc_set_medium_dense failed")

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def error(self) -> str:
        return lib().orc_error(self.h).decode()

    def set_adjoint(self, snaps: np.ndarray, wet: np.ndarray | None = None):
        snaps = np.ascontiguousarray(snaps, dtype=np.float64)
        S = snaps.shape[0]
        ax = snaps.shape[-1]
        ay = snaps.shape[-2] if self.wl.dim == 2 else 1
        wp = None
        if wet is not None:
            wet = np.ascontiguousarray(wet, dtype=np.uint8)
            wp = wet.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        rc = lib().orc_set_adjoint(self.h, S, ax, ay, _dp(snaps), wp)
        if rc:
            raise RuntimeError("orc_set_adjoint failed")

    def regrid(self, level=0, init=False):
        rc = lib().orc_regrid(self.h, level, 1 if init else 0)
        if rc:
            raise RuntimeError("orc_regrid failed: " + self.error())

    def advance(self, nsteps: int) -> float:
        cfl = ctypes.c_double(0.0)
        rc = lib().orc_advance(self.h, nsteps, ctypes.byref(cfl))
        if rc == 1:
            raise RuntimeError("orc_advance failed: " + self.error())
        return cfl.value

    def nsteps_total(self) -> int:
        dt = lib().orc_level_dt(self.h, 0)
        return int(round((self.P.tf - self.P.t0) / dt))

    def cell_updates(self) -> int:
        return int(lib().orc_cell_updates(self.h))

    def level_dt(self, level: int) -> float:
        return lib().orc_level_dt(self.h, level)

    def patches(self, level: int) -> np.ndarray:
        n = lib().orc_npatches(self.h, level)
        b = np.zeros((max(n, 1), 4), dtype=np.int32)
        lib().orc_get_patches(self.h, level, b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return b[:n].copy()

    def flag(self, level: int, tol: float):
        b = self.patches(level)
        n = int(np.sum(b[:, 2].astype(np.int64) * b[:, 3])) if len(b) else 0
        out = np.zeros(max(n, 1), dtype=np.uint8)
        cnt = ctypes.c_long(0)
        lib().orc_flag(self.h, level, tol, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), ctypes.byref(cnt))
        return out[:n], cnt.value

    def error_estimate(self, level: int) -> np.ndarray:
        """Richardson estimate tau of one step's local error on level
        `level` at its current time, laid out as read_level (per patch
        [m][ny][nx])."""
        b = self.patches(level)
        n = int(np.sum(b[:, 2].astype(np.int64) * b[:, 3])) * self.m if len(b) else 0
        out = np.zeros(max(n, 1))
        if lib().orc_error_estimate(self.h, level, _dp(out), out.size):
            raise RuntimeError("orc_error_estimate failed: " + self.error())
        return out[:n]

    def set_gauges(self, xs, ys=None):
        """Points recorded after every level-0 step."""
        xs = np.ascontiguousarray(xs, dtype=np.float64)
        ys = np.ascontiguousarray(np.zeros_like(xs) if ys is None else ys, dtype=np.float64)
        self._keep += [xs, ys]
        if lib().orc_set_gauges(self.h, xs.size, _dp(xs), _dp(ys)):
            raise RuntimeError("orc_set_gauges failed")
        self._ng = xs.size

    def gauges(self) -> np.ndarray:
        """Records [nrec, ngauge, 1 + m]: time and the values of the cell holding
        each point on the finest level covering it."""
        ng = getattr(self, "_ng", 0)
        n = lib().orc_read_gauges(self.h, None, 0)
        out = np.zeros((max(n, 1), max(ng, 1), 1 + self.m))
        lib().orc_read_gauges(self.h, _dp(out), n)
        return out[:n, :ng]

    def read_level(self, level: int) -> np.ndarray:
        b = self.patches(level)
        n = int(np.sum(b[:, 2].astype(np.int64) * b[:, 3])) * self.m if len(b) else 0
        out = np.zeros(max(n, 1))
        lib().orc_read_level(self.h, level, _dp(out))
        return out[:n]

    def write_level(self, level: int, data: np.ndarray):
        data = np.ascontiguousarray(data, dtype=np.float64)
        lib().orc_write_level(self.h, level, _dp(data))

    def level_patch_arrays(self, level: int):
        """List of (box, q[m, ny, nx]) for the interior of every patch."""
        flat = self.read_level(level)
        out, o = [], 0
        for b in self.patches(level):
            nx, ny = int(b[2]), int(b[3])
            sz = self.m * nx * ny
            out.append((tuple(int(v) for v in b), flat[o:o + sz].reshape(self.m, ny, nx)))
            o += sz
        return out

    def level_dense(self, level: int, fill=np.nan) -> np.ndarray:
        """Level data scattered onto the level's full index space."""
        N = self.wl.level_shape(level)
        arr = np.full((self.m, N[1], N[0]), fill)
        for (ilo, jlo, nx, ny), q in self.level_patch_arrays(level):
            arr[:, jlo:jlo + ny, ilo:ilo + nx] = q
        return arr

    def set_layout(self, level: int, boxes):
        """Replace the patches of a level by boxes [n, 4] = (ilo, jlo, nx, ny);
        state zero, medium filled."""
        b = np.ascontiguousarray(np.asarray(boxes, dtype=np.int32).reshape(-1, 4))
        if lib().orc_set_layout(self.h, level, b.shape[0], b.ctypes.data_as(ctypes.POINTER(ctypes.c_int))):
            raise RuntimeError("orc_set_layout failed")

    def set_level_time(self, level: int, nstep: int):
        """Set the step counter of a level (its time is t0 + nstep * dt)."""
        if lib().orc_set_nstep(self.h, level, int(nstep)):
            raise RuntimeError("orc_set_nstep failed")

    def fill_ghosts(self, level: int):
        rc = lib().orc_fill_ghosts(self.h, level)
        if rc:
            raise RuntimeError("orc_fill_ghosts failed: " + self.error())

    def patch_ghosted(self, level: int, k: int):
        b = self.patches(level)[k]
        gy = 2 if self.wl.dim == 2 else 0
        sx, sy = int(b[2]) + 4, int(b[3]) + 2 * gy
        nmed = 1 if self.wl.eqn in (2, 3) else 2
        q = np.zeros(self.m * sx * sy)
        med = np.zeros(nmed * sx * sy)
        lib().orc_read_patch_ghosted(self.h, level, k, _dp(q), _dp(med))
        return q.reshape(self.m, sy, sx), med.reshape(nmed, sy, sx)

    def functional(self, target=None) -> float:
        t = self.wl.target if target is None else target
        return lib().orc_functional(self.h, t.x0, t.x1, t.y0, t.y1, t.weight)


def step_patch(dim, eqn, q, med, dt, dx, dy=1.0):
    """One step of a standalone ghosted patch; q: [m, sy, sx], med: [nmed, sy, sx]."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    med = np.ascontiguousarray(med, dtype=np.float64)
    m = q.shape[0]
    sy, sx = q.shape[-2], q.shape[-1]
    nx = sx - 4
    ny = sy - 4 if dim == 2 else 1
    out = np.zeros(m * nx * ny)
    cfl = ctypes.c_double(0.0)
    lib().orc_step_patch(dim, eqn, nx, ny, _dp(q), _dp(med), dt, dx, dy, _dp(out), ctypes.byref(cfl))
    return out.reshape(m, ny, nx), cfl.value


def adjoint_solve(wl, nsnap=None, n=None, medium_dense=None, tf=None, phi=None):
    """Adjoint snapshots [nsnap, m, ny, nx] in forward-time order."""
    nn = wl.adj_n if n is None else n
    S = wl.nsnap if nsnap is None else nsnap
    P = params_from_workload(wl, eqn=wl.adj_eqn, nlevels=1, n0=nn, tf=tf)
    if phi is None:
        phi = wl.adjoint_phi() if n is None else _phi_for(wl, nn)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    nx = nn[0]
    ny = nn[1] if wl.dim == 2 else 1
    out = np.zeros((S, wl.m, ny, nx))
    med = wl.medium
    if medium_dense is not None or med.kind == "dense":
        dense = np.ascontiguousarray(medium_dense, dtype=np.float64)
        z = np.zeros(1)
        rc = lib().orc_adjoint_solve(ctypes.byref(P), 0, 1, _dp(z), _dp(z), _dp(z), _dp(dense), _dp(phi), S, _dp(out))
    else:
        iface = np.ascontiguousarray(med.iface if med.iface.size else np.zeros(1), dtype=np.float64)
        f0 = np.ascontiguousarray(med.rho, dtype=np.float64)
        f1 = np.ascontiguousarray(med.K, dtype=np.float64)
        rc = lib().orc_adjoint_solve(ctypes.byref(P), med.axis, f0.size, _dp(iface), _dp(f0), _dp(f1),
                                     None, _dp(phi), S, _dp(out))
    if rc:
        raise RuntimeError("orc_adjoint_solve failed")
    return out


def adjoint_solve_amr(wl, ratios, flag_mode, tol, nsnap=None, n=None, phi=None, medium_dense_levels=None,
                      reflux=0):
    """Adjoint snapshots [nsnap, m, ny, nx] (forward-time order) from an AMR
    solve of the adjoint whose level 0 is the snapshot grid (n, default
    wl.adj_n), refined by `ratios` under a standard flagger (flag_mode,
    tol); medium_dense_levels: dense media [nmed][M_l][N_l] per level (dense
    workloads)."""
    import copy
    nn = tuple(wl.adj_n if n is None else n)
    S = wl.nsnap if nsnap is None else nsnap
    w2 = copy.copy(wl)
    w2.n0, w2.ratios, w2.flag_mode, w2.tol, w2.reflux = nn, tuple(ratios), flag_mode, tol, reflux
    P = params_from_workload(w2, eqn=wl.adj_eqn, nlevels=len(ratios) + 1, n0=nn)
    if phi is None:
        phi = _phi_for(wl, nn)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    nx = nn[0]
    ny = nn[1] if wl.dim == 2 else 1
    out = np.zeros((S, wl.m, ny, nx))
    med = wl.medium
    z = np.zeros(1)
    if medium_dense_levels is not None or med.kind == "dense":
        dense = np.concatenate([np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in medium_dense_levels])
        rc = lib().orc_adjoint_solve_amr(ctypes.byref(P), 0, 1, _dp(z), _dp(z), _dp(z), _dp(dense), _dp(phi), S,
                                         _dp(out))
    else:
        iface = np.ascontiguousarray(med.iface if med.iface.size else np.zeros(1), dtype=np.float64)
        f0 = np.ascontiguousarray(med.rho, dtype=np.float64)
        f1 = np.ascontiguousarray(med.K, dtype=np.float64)
        rc = lib().orc_adjoint_solve_amr(ctypes.byref(P), med.axis, f0.size, _dp(iface), _dp(f0), _dp(f1),
                                         None, _dp(phi), S, _dp(out))
    if rc:
        raise RuntimeError("orc_adjoint_solve_amr failed")
    return out


def _phi_for(wl, nn):
    import copy
    w2 = copy.copy(wl)
    w2.adj_n = tuple(nn)
    return w2.adjoint_phi()


def cluster(flags: np.ndarray, mc: int = 1, eff: float = 0.7, nest: np.ndarray | None = None) -> np.ndarray:
    """Berger-Rigoutsos boxes (i0, i1, j0, j1) of a flag field [M, N]."""
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    M, N = flags.shape
    dim = 2 if M > 1 else 1
    cap = N * M + 1
    out = np.zeros((cap, 4), dtype=np.int32)
    npt = None
    if nest is not None:
        nest = np.ascontiguousarray(nest, dtype=np.uint8)
        npt = nest.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    n = lib().orc_cluster(flags.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), npt, N, M, dim, mc, eff,
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), cap)
    return out[:n].copy()
