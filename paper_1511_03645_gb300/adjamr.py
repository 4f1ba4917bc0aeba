"""Thin ctypes binding of libadjamr (include/adjamr.h): argument marshalling
only.  Every step of the hot path runs in the library's CUDA kernels; there
is no CPU fallback -- loading fails loudly when the library or a GPU is
missing."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads as W

MAXLEV = 8
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, EBUDGET, ECFL, ETIMEOUT, ECUDA, ESTATE, ENEST = range(9)
LAUNCH_WORKLIST, LAUNCH_PERSISTENT, LAUNCH_PER_PATCH, LAUNCH_DYNAMIC, LAUNCH_SUBSTEPS = 0, 1, 2, 3, 4
MEDIUM_LAYERED, MEDIUM_DENSE = 1, 2
_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "EBUDGET", 4: "ECFL", 5: "ETIMEOUT", 6: "ECUDA", 7: "ESTATE",
          8: "ENEST"}


class AdjamrError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"adjamr {_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
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
        ("stream", ctypes.c_void_p),
        ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
        ("launch_mode", ctypes.c_int),
        ("reflux", ctypes.c_int),
    ]


class Medium(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("axis", ctypes.c_int), ("nlayers", ctypes.c_int),
                ("iface", ctypes.POINTER(ctypes.c_double)), ("f0", ctypes.POINTER(ctypes.c_double)),
                ("f1", ctypes.POINTER(ctypes.c_double)),
                ("dense", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))), ("ndense", ctypes.c_int)]


class Target(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
                ("y1", ctypes.c_double), ("weight", ctypes.c_double)]


class Patch(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("ilo", ctypes.c_int), ("jlo", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("params", Params), ("medium", Medium), ("adjoint", ctypes.c_void_p), ("target", Target)]


class Result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("J", ctypes.c_double),
                ("cell_updates", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_finish", ctypes.c_double),
                ("bytes_reserved", ctypes.c_size_t), ("error", ctypes.c_char * 128)]


class Stats(ctypes.Structure):
    _fields_ = [("cell_updates", ctypes.c_longlong), ("adjoint_cell_updates", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("regrids", ctypes.c_longlong),
                ("cfl_max_seen", ctypes.c_double), ("step_kernel_ms", ctypes.c_double),
                ("step_kernel_launches", ctypes.c_longlong), ("regrid_host_ms", ctypes.c_double),
                ("cluster_host_ms", ctypes.c_double), ("level_rebuilds", ctypes.c_longlong),
                ("regrid_phase_ms", ctypes.c_double * 6),
                ("level_step_ms", ctypes.c_double * MAXLEV),
                ("level_step_launches", ctypes.c_longlong * MAXLEV),
                ("level_cell_updates", ctypes.c_longlong * MAXLEV),
                ("cluster_phase_ms", ctypes.c_double * 4),
                ("level_ghost_ms", ctypes.c_double * MAXLEV),
                ("level_rebuilds_skipped", ctypes.c_longlong)]


# every entry point declared in include/adjamr.h
SYMBOLS = [
    "adjamr_init_grid_hierarchy", "adjamr_set_medium", "adjamr_load_adjoint_snapshots", "adjamr_solve_adjoint",
    "adjamr_set_adjoint", "adjamr_adjoint_read", "adjamr_adjoint_release", "adjamr_regrid",
    "adjamr_advance_level", "adjamr_flag_cells", "adjamr_integrate_functional", "adjamr_get_patches",
    "adjamr_read_level", "adjamr_write_level", "adjamr_error_estimate", "adjamr_reset", "adjamr_fill_ghosts",
    "adjamr_read_patch_ghosted",
    "adjamr_step_level_only", "adjamr_get_stats", "adjamr_set_timing", "adjamr_set_level_kernel",
    "adjamr_substep_wait_selftest", "adjamr_set_gauges",
    "adjamr_read_gauges", "adjamr_cluster_boxes", "adjamr_time_info",
    "adjamr_last_error",
    "adjamr_destroy", "adjamr_batch_create", "adjamr_batch_set_order", "adjamr_batch_set_ghost_fusion",
    "adjamr_batch_step",
    "adjamr_batch_step_graph", "adjamr_batch_read", "adjamr_batch_cells", "adjamr_batch_destroy",
    "adjamr_fp64_peak", "adjamr_estimate_bytes", "adjamr_server_create", "adjamr_server_submit",
    "adjamr_server_poll", "adjamr_server_wait", "adjamr_server_info", "adjamr_server_now", "adjamr_server_destroy",
    "adjamr_weighted_sum_noalloc",
]


def lib_path() -> str:
    from .build import LIB
    return LIB


def load(build_if_missing: bool = True):
    """Load libadjamr.so (building it first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if build_if_missing:
            from .build import build
            build()
        if not os.path.exists(path):
            raise RuntimeError(f"libadjamr not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        i, d, vp, ll, sz = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_size_t
        dp, ip, ucp = P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_ubyte)
        sig = {
            "adjamr_init_grid_hierarchy": [P(Params), P(vp)],
            "adjamr_set_medium": [vp, P(Medium)],
            "adjamr_load_adjoint_snapshots": [vp, vp, i, i, i, ucp, i, P(vp)],
            "adjamr_solve_adjoint": [vp, P(Params), P(Medium), dp, i, P(vp)],
            "adjamr_set_adjoint": [vp, vp],
            "adjamr_adjoint_read": [vp, dp, sz],
            "adjamr_regrid": [vp, i, i],
            "adjamr_advance_level": [vp, i, i],
            "adjamr_flag_cells": [vp, i, d, d, ucp, P(ll)],
            "adjamr_integrate_functional": [vp, P(Target), dp],
            "adjamr_get_patches": [vp, i, P(Patch), i, ip],
            "adjamr_read_level": [vp, i, dp, sz],
            "adjamr_error_estimate": [vp, i, dp, sz],
            "adjamr_reset": [vp],
            "adjamr_write_level": [vp, i, dp, sz],
            "adjamr_fill_ghosts": [vp, i],
            "adjamr_read_patch_ghosted": [vp, i, i, dp, dp],
            "adjamr_step_level_only": [vp, i],
            "adjamr_get_stats": [vp, P(Stats)],
            "adjamr_set_timing": [vp, i],
            "adjamr_set_level_kernel": [vp, i, i, i, i, i],
            "adjamr_substep_wait_selftest": [vp, dp],
            "adjamr_set_gauges": [vp, i, dp, dp],
            "adjamr_cluster_boxes": [ucp, ucp, i, i, i, i, d, ip, i, ip],
            "adjamr_read_gauges": [vp, dp, ll, ctypes.POINTER(ll)],
            "adjamr_time_info": [vp, dp, ip],
            "adjamr_batch_create": [i, ip, ip, dp, dp, dp, dp, dp, ip, P(Medium), i, dp, vp, P(vp)],
            "adjamr_batch_set_order": [vp, ip],
            "adjamr_batch_set_ghost_fusion": [vp, i],
            "adjamr_batch_step": [vp, i, i, i, i],
            "adjamr_batch_step_graph": [vp, i, i, i, i],
            "adjamr_batch_read": [vp, dp, sz],
            "adjamr_batch_cells": [vp, P(ll)],
            "adjamr_fp64_peak": [i, i, dp, dp],
            "adjamr_server_create": [sz, i, P(vp)],
            "adjamr_server_submit": [vp, P(Request), P(ll)],
            "adjamr_server_poll": [vp, ll, P(Result)],
            "adjamr_server_wait": [vp, ll, P(Result)],
            "adjamr_server_info": [vp, P(sz), ip, ip],
            "adjamr_weighted_sum_noalloc": [vp, vp, ll, d, vp, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.adjamr_last_error.argtypes = [vp]
        L.adjamr_last_error.restype = ctypes.c_char_p
        L.adjamr_destroy.argtypes = [vp]
        L.adjamr_destroy.restype = None
        L.adjamr_adjoint_release.argtypes = [vp]
        L.adjamr_adjoint_release.restype = None
        L.adjamr_batch_destroy.argtypes = [vp]
        L.adjamr_batch_destroy.restype = None
        L.adjamr_server_destroy.argtypes = [vp]
        L.adjamr_server_destroy.restype = None
        L.adjamr_server_now.argtypes = [vp]
        L.adjamr_server_now.restype = ctypes.c_double
        L.adjamr_estimate_bytes.argtypes = [P(Params)]
        L.adjamr_estimate_bytes.restype = ctypes.c_size_t
        _lib = L
        return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def make_params(wl, *, eqn=None, nlevels=None, n0=None, tol=None, dt0=0.0, qinit=None, tf=None, stream=None,
                tile=(0, 0), launch_mode=LAUNCH_WORKLIST):
    p = Params()
    p.dim = wl.dim
    p.eqn = wl.eqn if eqn is None else eqn
    p.lo[0], p.lo[1] = wl.lo
    p.hi[0], p.hi[1] = wl.hi
    nn = wl.n0 if n0 is None else n0
    p.n0[0], p.n0[1] = nn[0], (nn[1] if wl.dim == 2 else 1)
    p.nlevels = wl.nlevels if nlevels is None else nlevels
    for k, r in enumerate(wl.ratios):
        p.ratio[k] = r
    for k in range(4):
        p.bc[k] = wl.bc[k]
    p.cfl, p.cfl_max, p.cmax, p.dt0 = wl.cfl, wl.cfl_max, wl.medium.cmax, dt0
    p.t0, p.tf, p.ts = wl.t0, (wl.tf if tf is None else tf), wl.ts
    p.tol = wl.tol if tol is None else tol
    p.regrid_interval, p.buffer, p.cluster_eff = wl.regrid_interval, wl.buffer, wl.cluster_eff
    p.min_patch, p.max_patch, p.max_patch0 = wl.min_patch, wl.max_patch, wl.max_patch0
    p.flag_mode = wl.flag_mode
    if qinit is not None:
        p.qinit = ctypes.cast(qinit, ctypes.c_void_p)
    p.stream = stream
    p.tile_x, p.tile_y = tile
    p.launch_mode = launch_mode
    p.reflux = int(getattr(wl, "reflux", 0))
    return p


class _MediumHolder:
    """A Medium struct plus the arrays it points to (kept alive)."""

    def __init__(self, med, nlevels=None, dense_fields=None):
        self.keep = []
        self.m = Medium()
        if med.kind == "layered" and dense_fields is None:
            iface = np.ascontiguousarray(med.iface if med.iface is not None and med.iface.size else np.zeros(1),
                                         dtype=np.float64)
            f0 = np.ascontiguousarray(med.rho, dtype=np.float64)
            f1 = np.ascontiguousarray(med.K, dtype=np.float64)
            self.keep += [iface, f0, f1]
            self.m.kind = MEDIUM_LAYERED
            self.m.axis = med.axis
            self.m.nlayers = f0.size
            self.m.iface, self.m.f0, self.m.f1 = _dp(iface), _dp(f0), _dp(f1)
        else:
            fields = dense_fields if dense_fields is not None else med.fields
            arrs = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
            self.keep += arrs
            ptrs = (ctypes.POINTER(ctypes.c_double) * len(arrs))(*[_dp(a) for a in arrs])
            self.keep.append(ptrs)
            self.m.kind = MEDIUM_DENSE
            self.m.dense = ctypes.cast(ptrs, ctypes.POINTER(ctypes.POINTER(ctypes.c_double)))
            self.m.ndense = len(arrs)


def _check(rc, h=None, what=""):
    if rc != OK:
        msg = what
        if h:
            msg += ": " + load().adjamr_last_error(h).decode()
        raise AdjamrError(rc, msg)


class Adjoint:
    """A device-resident snapshot set (reference-counted)."""

    def __init__(self, handle, shape):
        self.h = handle
        self.shape = shape

    def read(self) -> np.ndarray:
        out = np.zeros(self.shape)
        _check(load().adjamr_adjoint_read(self.h, _dp(out), out.size), None, "adjoint_read")
        return out

    def release(self):
        if self.h:
            load().adjamr_adjoint_release(self.h)
            self.h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Hierarchy:
    """One forward (or adjoint) solve: an AMR hierarchy on the GPU."""

    def __init__(self, wl, *, nlevels=None, tol=None, dt0=0.0, with_qinit=True, tf=None, stream=None,
                 tile=(0, 0), launch_mode=LAUNCH_WORKLIST, eqn=None, n0=None):
        L = load()
        self.wl = wl
        self.m = wl.m
        self._cb = wl.qinit_callback() if (with_qinit and wl.qinit is not None) else None
        self.P = make_params(wl, eqn=eqn, nlevels=nlevels, n0=n0, tol=tol, dt0=dt0, qinit=self._cb, tf=tf,
                             stream=stream, tile=tile, launch_mode=launch_mode)
        self.nlevels = self.P.nlevels
        h = ctypes.c_void_p()
        _check(L.adjamr_init_grid_hierarchy(ctypes.byref(self.P), ctypes.byref(h)), None, "init_grid_hierarchy")
        self.h = h
        self._med = _MediumHolder(wl.medium)
        _check(L.adjamr_set_medium(self.h, ctypes.byref(self._med.m)), self.h, "set_medium")

    def close(self):
        if getattr(self, "h", None):
            load().adjamr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- adjoint ----
    def load_adjoint(self, snaps: np.ndarray, wet=None, on_device_ptr=None) -> Adjoint:
        L = load()
        out = ctypes.c_void_p()
        S = snaps.shape[0] if snaps is not None else on_device_ptr[1][0]
        if on_device_ptr is not None:
            ptr, shape = on_device_ptr
            ax, ay = shape[-1], (shape[-2] if self.wl.dim == 2 else 1)
            rc = L.adjamr_load_adjoint_snapshots(self.h, ctypes.c_void_p(ptr), shape[0], ax, ay, None, 1,
                                                 ctypes.byref(out))
            shp = tuple(shape)
        else:
            snaps = np.ascontiguousarray(snaps, dtype=np.float64)
            ax, ay = snaps.shape[-1], (snaps.shape[-2] if self.wl.dim == 2 else 1)
            wp = None
            if wet is not None:
                wet = np.ascontiguousarray(wet, dtype=np.uint8)
                wp = wet.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
            rc = L.adjamr_load_adjoint_snapshots(self.h, snaps.ctypes.data_as(ctypes.c_void_p), S, ax, ay, wp, 0,
                                                 ctypes.byref(out))
            shp = snaps.shape
        _check(rc, self.h, "load_adjoint_snapshots")
        return Adjoint(out, shp)

    def set_adjoint(self, adj: Adjoint):
        _check(load().adjamr_set_adjoint(self.h, adj.h), self.h, "set_adjoint")

    # ---- stepping ----
    def regrid(self, level=0, init=False):
        _check(load().adjamr_regrid(self.h, level, 1 if init else 0), self.h, "regrid")

    def advance(self, nsteps: int):
        _check(load().adjamr_advance_level(self.h, 0, nsteps), self.h, "advance_level")

    def time_info(self):
        dt = ctypes.c_double()
        n = ctypes.c_int()
        _check(load().adjamr_time_info(self.h, ctypes.byref(dt), ctypes.byref(n)), self.h, "time_info")
        return dt.value, n.value

    def nsteps_total(self) -> int:
        return self.time_info()[1]

    def fill_ghosts(self, level):
        _check(load().adjamr_fill_ghosts(self.h, level), self.h, "fill_ghosts")

    def step_level_only(self, level):
        _check(load().adjamr_step_level_only(self.h, level), self.h, "step_level_only")

    def set_timing(self, on=True):
        _check(load().adjamr_set_timing(self.h, 1 if on else 0), self.h, "set_timing")

    def stats(self) -> dict:
        s = Stats()
        _check(load().adjamr_get_stats(self.h, ctypes.byref(s)), self.h, "get_stats")
        d = {k: getattr(s, k) for k, _ in Stats._fields_}
        for k in ("regrid_phase_ms", "level_step_ms", "level_step_launches", "level_cell_updates", "cluster_phase_ms",
                  "level_ghost_ms"):
            d[k] = list(getattr(s, k))
        return d

    def set_gauges(self, xs, ys=None) -> None:
        """Points recorded on the device after every level-0 step."""
        xs = np.ascontiguousarray(xs, dtype=np.float64)
        ys = np.ascontiguousarray(np.zeros_like(xs) if ys is None else ys, dtype=np.float64)
        _check(load().adjamr_set_gauges(self.h, xs.size, _dp(xs), _dp(ys)), self.h, "set_gauges")
        self._ng = xs.size

    def gauges(self) -> np.ndarray:
        """Records [nrec, ngauge, 1 + m]: time and the values of the cell holding
        each point on the finest level covering it."""
        ng = getattr(self, "_ng", 0)
        n = ctypes.c_longlong(0)
        _check(load().adjamr_read_gauges(self.h, None, 0, ctypes.byref(n)), self.h, "read_gauges")
        out = np.zeros((max(n.value, 1), max(ng, 1), 1 + self.m))
        _check(load().adjamr_read_gauges(self.h, _dp(out), n.value, ctypes.byref(n)), self.h, "read_gauges")
        return out[:n.value, :ng]

    def set_level_kernel(self, level: int, tile, fuse_ghosts: bool = True, mode: int = -1) -> None:
        """Step-kernel tile (tx, ty), ghost fusion and launch mode (-1: keep)
        of one level (-1: all levels); results do not depend on them."""
        _check(load().adjamr_set_level_kernel(self.h, level, int(tile[0]), int(tile[1]) if len(tile) > 1 else 1,
                                              1 if fuse_ghosts else 0, int(mode)), self.h, "set_level_kernel")

    def substep_wait_selftest(self):
        """(status, ms): a substep launch of the finest level whose waits
        can never be satisfied; expected status ETIMEOUT after about 1 s."""
        ms = ctypes.c_double()
        rc = load().adjamr_substep_wait_selftest(self.h, ctypes.byref(ms))
        return rc, ms.value

    # ---- queries ----
    def patches(self, level: int) -> np.ndarray:
        L = load()
        n = ctypes.c_int()
        _check(L.adjamr_get_patches(self.h, level, None, 0, ctypes.byref(n)), self.h, "get_patches")
        arr = (Patch * max(n.value, 1))()
        _check(L.adjamr_get_patches(self.h, level, arr, max(n.value, 1), ctypes.byref(n)), self.h, "get_patches")
        return np.array([[p.ilo, p.jlo, p.nx, p.ny] for p in arr[:n.value]], dtype=np.int32).reshape(-1, 4)

    def read_level(self, level: int) -> np.ndarray:
        b = self.patches(level)
        n = int(np.sum(b[:, 2].astype(np.int64) * b[:, 3])) * self.m if len(b) else 0
        out = np.zeros(max(n, 1))
        _check(load().adjamr_read_level(self.h, level, _dp(out), out.size), self.h, "read_level")
        return out[:n]

    def reset(self) -> None:
        """Start a new solve in this context (level 0 from qinit at t0, finer
        levels dropped, statistics cleared; adjoint, medium and kernels kept)."""
        _check(load().adjamr_reset(self.h), self.h, "reset")

    def error_estimate(self, level: int) -> np.ndarray:
        """Richardson estimate of one step's local error on the level at its
        current time, laid out as read_level."""
        b = self.patches(level)
        n = int(np.sum(b[:, 2].astype(np.int64) * b[:, 3])) * self.m if len(b) else 0
        out = np.zeros(max(n, 1))
        _check(load().adjamr_error_estimate(self.h, level, _dp(out), out.size), self.h, "error_estimate")
        return out[:n]

    def write_level(self, level: int, data):
        data = np.ascontiguousarray(data, dtype=np.float64)
        _check(load().adjamr_write_level(self.h, level, _dp(data), data.size), self.h, "write_level")

    def level_dense(self, level: int, fill=np.nan) -> np.ndarray:
        N = self.wl.level_shape(level)
        arr = np.full((self.m, N[1], N[0]), fill)
        flat = self.read_level(level)
        o = 0
        for ilo, jlo, nx, ny in self.patches(level):
            sz = self.m * nx * ny
            arr[:, jlo:jlo + ny, ilo:ilo + nx] = flat[o:o + sz].reshape(self.m, ny, nx)
            o += sz
        return arr

    def flag(self, level: int, tol: float, ts: float | None = None):
        """Flags of the level's interior cells for the range of interest
        [ts, tf] (default: the workload's ts)."""
        b = self.patches(level)
        n = int(np.sum(b[:, 2].astype(np.int64) * b[:, 3])) if len(b) else 0
        out = np.zeros(max(n, 1), dtype=np.uint8)
        cnt = ctypes.c_longlong()
        t_s = self.wl.ts if ts is None else ts
        _check(load().adjamr_flag_cells(self.h, level, tol, t_s, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                        ctypes.byref(cnt)), self.h, "flag_cells")
        return out[:n], cnt.value

    def functional(self, target=None) -> float:
        t = self.wl.target if target is None else target
        tg = Target(t.x0, t.x1, t.y0, t.y1, t.weight)
        J = ctypes.c_double()
        _check(load().adjamr_integrate_functional(self.h, ctypes.byref(tg), ctypes.byref(J)), self.h,
               "integrate_functional")
        return J.value

    def patch_ghosted(self, level: int, k: int):
        b = self.patches(level)[k]
        gy = 2 if self.wl.dim == 2 else 0
        sx, sy = int(b[2]) + 4, int(b[3]) + 2 * gy
        nmed = 1 if self.P.eqn in (2, 3) else 2
        q = np.zeros(self.m * sx * sy)
        med = np.zeros(nmed * sx * sy)
        _check(load().adjamr_read_patch_ghosted(self.h, level, k, _dp(q), _dp(med)), self.h, "read_patch_ghosted")
        return q.reshape(self.m, sy, sx), med.reshape(nmed, sy, sx)


def solve_adjoint(wl, *, nsnap=None, n=None, phi=None, medium_dense=None, stream=None, ctx: Hierarchy = None,
                  tf=None, tile=(0, 0), amr=None) -> Adjoint:
    """Adjoint snapshots computed on the GPU (device-resident handle);
    tile: the step-kernel tile of the adjoint grid (0: default).
    amr = (ratios, flag_mode, tol[, reflux]): the adjoint solved with AMR on a
    hierarchy whose level 0 is the snapshot grid; medium_dense is then the
    list of the levels' dense media (dense workloads)."""
    import copy
    L = load()
    nn = wl.adj_n if n is None else n
    S = wl.nsnap if nsnap is None else nsnap
    wa = wl
    nlev = 1
    if amr is not None:
        wa = copy.copy(wl)
        wa.ratios, wa.flag_mode, wa.tol = tuple(amr[0]), amr[1], amr[2]
        wa.reflux = amr[3] if len(amr) > 3 else 0
        nlev = len(wa.ratios) + 1
    p = make_params(wa, eqn=wl.adj_eqn, nlevels=nlev, n0=nn, stream=stream, tf=tf, tile=tile)
    if phi is None:
        import copy
        w2 = copy.copy(wl)
        w2.adj_n = tuple(nn)
        phi = w2.adjoint_phi()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    dense = None
    if medium_dense is not None:
        dense = list(medium_dense) if amr is not None else [medium_dense]
    mh = _MediumHolder(wl.medium, dense_fields=dense)
    out = ctypes.c_void_p()
    rc = L.adjamr_solve_adjoint(ctx.h if ctx is not None else None, ctypes.byref(p), ctypes.byref(mh.m), _dp(phi), S,
                                ctypes.byref(out))
    _check(rc, ctx.h if ctx is not None else None, "solve_adjoint")
    nx = nn[0]
    ny = nn[1] if wl.dim == 2 else 1
    return Adjoint(out, (S, wl.m, ny, nx))


class Batch:
    """Independent 2D acoustics patches advanced together (config-4 shape)."""

    def __init__(self, pb: "W.PatchBatch", stream=None):
        L = load()
        self.pb = pb
        n = pb.npatch
        self.nx = np.ascontiguousarray(pb.nx, dtype=np.int32)
        self.ny = np.ascontiguousarray(pb.ny, dtype=np.int32)
        self.x0 = np.ascontiguousarray(pb.x0, dtype=np.float64)
        self.y0 = np.ascontiguousarray(pb.y0, dtype=np.float64)
        self.x1 = np.ascontiguousarray(pb.x0 + pb.nx * pb.dx, dtype=np.float64)
        self.y1 = np.ascontiguousarray(pb.y0 + pb.ny * pb.dx, dtype=np.float64)
        self.dt = np.ascontiguousarray(pb.dt, dtype=np.float64)
        self.mid = np.ascontiguousarray(pb.medium_id, dtype=np.int32)
        self._meds = [_MediumHolder(m) for m in pb.media]
        marr = (Medium * len(self._meds))(*[h.m for h in self._meds])
        self._marr = marr
        q0 = np.concatenate([pb.qinit_patch(k).reshape(-1) for k in range(n)])
        self.q0 = q0
        h = ctypes.c_void_p()
        rc = L.adjamr_batch_create(n, _ip(self.nx), _ip(self.ny), _dp(self.x0), _dp(self.y0), _dp(self.x1),
                                   _dp(self.y1), _dp(self.dt), _ip(self.mid), marr, len(self._meds), _dp(q0),
                                   ctypes.c_void_p(stream) if stream else None, ctypes.byref(h))
        _check(rc, None, "batch_create")
        self.h = h

    def set_order(self, order):
        o = np.ascontiguousarray(order, dtype=np.int32)
        _check(load().adjamr_batch_set_order(self.h, _ip(o)), None, "batch_set_order")

    def set_ghost_fusion(self, on: bool):
        _check(load().adjamr_batch_set_ghost_fusion(self.h, 1 if on else 0), None, "batch_set_ghost_fusion")

    def step(self, nsteps=1, mode=LAUNCH_WORKLIST, tile=(32, 8), graph=False):
        f = load().adjamr_batch_step_graph if graph else load().adjamr_batch_step
        _check(f(self.h, nsteps, mode, tile[0], tile[1]), None, "batch_step")

    def read(self) -> np.ndarray:
        n = 3 * int(np.sum(self.nx.astype(np.int64) * self.ny))
        out = np.zeros(n)
        _check(load().adjamr_batch_read(self.h, _dp(out), n), None, "batch_read")
        return out

    def cells(self) -> int:
        c = ctypes.c_longlong()
        _check(load().adjamr_batch_cells(self.h, ctypes.byref(c)), None, "batch_cells")
        return c.value

    def close(self):
        if getattr(self, "h", None):
            load().adjamr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp64_peak(kind=0, iters=4096):
    """(flop/s, ms) of the FP64 throughput micro-benchmark (0 DFMA, 1 DADD, 2 DMUL)."""
    f = ctypes.c_double()
    ms = ctypes.c_double()
    _check(load().adjamr_fp64_peak(kind, iters, ctypes.byref(f), ctypes.byref(ms)), None, "fp64_peak")
    return f.value, ms.value


class Server:
    """Serving loop: continuous admission of forward solves by memory budget,
    one CUDA stream per slot (include/adjamr.h, adjamr_server_*)."""

    def __init__(self, budget_bytes: int, max_slots: int):
        L = load()
        h = ctypes.c_void_p()
        _check(L.adjamr_server_create(int(budget_bytes), int(max_slots), ctypes.byref(h)), None, "server_create")
        self.h = h
        self._keep = {}

    def submit(self, wl, adj: Adjoint) -> int:
        L = load()
        cb = wl.qinit_callback() if wl.qinit is not None else None
        rq = Request()
        rq.params = make_params(wl, qinit=cb)
        mh = _MediumHolder(wl.medium)
        rq.medium = mh.m
        rq.adjoint = adj.h
        t = wl.target
        rq.target = Target(t.x0, t.x1, t.y0, t.y1, t.weight)
        tk = ctypes.c_longlong()
        _check(L.adjamr_server_submit(self.h, ctypes.byref(rq), ctypes.byref(tk)), None, "server_submit")
        self._keep[tk.value] = (cb, mh, rq)
        return tk.value

    @staticmethod
    def _res(r: Result) -> dict:
        d = {k: getattr(r, k) for k, _ in Result._fields_ if k != "error"}
        d["error"] = r.error.decode(errors="replace")
        return d

    def poll(self, ticket: int) -> dict:
        r = Result()
        _check(load().adjamr_server_poll(self.h, ticket, ctypes.byref(r)), None, "server_poll")
        return self._res(r)

    def wait(self, ticket: int) -> dict:
        r = Result()
        _check(load().adjamr_server_wait(self.h, ticket, ctypes.byref(r)), None, "server_wait")
        self._keep.pop(ticket, None)
        return self._res(r)

    def info(self):
        used = ctypes.c_size_t()
        a = ctypes.c_int()
        q = ctypes.c_int()
        _check(load().adjamr_server_info(self.h, ctypes.byref(used), ctypes.byref(a), ctypes.byref(q)), None,
               "server_info")
        return used.value, a.value, q.value

    def now(self) -> float:
        return load().adjamr_server_now(self.h)

    def close(self):
        if getattr(self, "h", None):
            load().adjamr_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def estimate_bytes(wl) -> int:
    p = make_params(wl)
    return int(load().adjamr_estimate_bytes(ctypes.byref(p)))


NOALLOC_MAX_TERMS = 1 << 20


def weighted_sum_noalloc(q_ptr: int, w_ptr: int, n: int, weight: float, out_ptr: int, stream=None):
    """adjamr_weighted_sum_noalloc on caller-owned device buffers (raw device
    pointers, e.g. tensor.data_ptr()); the library allocates nothing."""
    rc = load().adjamr_weighted_sum_noalloc(ctypes.c_void_p(q_ptr), ctypes.c_void_p(w_ptr), int(n), float(weight),
                                            ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream) if stream else None)
    _check(rc, None, "weighted_sum_noalloc")


def cluster_boxes(flags: np.ndarray, mc: int = 1, eff: float = 0.7, nest: np.ndarray | None = None) -> np.ndarray:
    """Boxes (i0, i1, j0, j1) of the library's Berger-Rigoutsos clustering of a
    flag field [M, N] (host code, no GPU)."""
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    M, N = flags.shape
    dim = 2 if M > 1 else 1
    cap = N * M + 1
    out = np.zeros((cap, 4), dtype=np.int32)
    n = ctypes.c_int(0)
    npt = None
    if nest is not None:
        nest = np.ascontiguousarray(nest, dtype=np.uint8)
        npt = nest.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    _check(load().adjamr_cluster_boxes(flags.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), npt, N, M, dim, mc, eff,
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), cap, ctypes.byref(n)),
           None, "cluster_boxes")
    return out[:n.value].copy()
