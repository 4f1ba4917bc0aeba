"""Pins of the oracle's standard flaggers and gauges (no GPU).

The paper compares adjoint flagging against the flagging AMRClaw and GeoClaw
use by default (Sec. 5.2.4: a spatial difference of every component in each
direction above a tolerance; Sec. 5.3: the surface elevation above a
tolerance) and judges accuracy by gauges, time series at points.  These
tests pin the oracle's versions by closed forms on hand-built states and by
the AMR limits (tol < 0 is the uniform fine run, tol = +inf the uniform
coarse run)."""
import math

import numpy as np

from oracle import oracle as O
from paper_1511_03645_gb300 import workloads as W


def _uniform(n=12, flag_mode=W.FLAG_DIFFERENCE, dim=2):
    if dim == 1:
        wl = W.config1(n0=n, tf=0.5)
    else:
        wl = W.config2(seed=1, n0=n, ratios=(2,), tf=0.5, adj_n=2 * n, nsnap=4)
    wl.flag_mode = flag_mode
    wl.max_patch0 = 5  # several patches: neighbours across patch edges come from same-level ghosts
    return wl


def _write(h, wl, field):
    """Write q[f][J][I] (level-0 index space) into the hierarchy's patch order."""
    out = []
    for ilo, jlo, nx, ny in h.patches(0):
        out.append(field[:, jlo:jlo + ny, ilo:ilo + nx].reshape(-1))
    h.write_level(0, np.concatenate(out))


def _dense_flags(h, wl, tol):
    fl, cnt = h.flag(0, tol)
    N, M = wl.n0 if wl.dim == 2 else (wl.n0[0], 1)
    dense = np.zeros((M, N), dtype=np.uint8)
    o = 0
    for ilo, jlo, nx, ny in h.patches(0):
        dense[jlo:jlo + ny, ilo:ilo + nx] = fl[o:o + nx * ny].reshape(ny, nx)
        o += nx * ny
    assert cnt == int(dense.sum())
    return dense


def test_difference_flags_are_centred_undivided_differences():
    """A ramp of 1/8 per cell in one component: the centred difference is
    exactly 1/4 inside, and 1/8 in the first and last columns, where the
    extrapolation ghost repeats the boundary cell.  The test is strict (> tol)
    and covers every component and both directions."""
    wl = _uniform()
    N = wl.n0[0]
    ramp = 0.125 * np.arange(N, dtype=np.float64)
    for comp, axis in ((0, "x"), (1, "x"), (2, "y")):
        h = O.OracleHierarchy(wl, nlevels=1, with_qinit=False)
        q = np.zeros((3, N, N))
        q[comp] = ramp[None, :] if axis == "x" else ramp[:, None]
        _write(h, wl, q)
        inside = np.zeros((N, N), dtype=np.uint8)
        if axis == "x":
            inside[:, 1:-1] = 1
        else:
            inside[1:-1, :] = 1
        assert np.array_equal(_dense_flags(h, wl, 0.2), inside)
        assert _dense_flags(h, wl, 0.25).sum() == 0          # 1/4 is not above 1/4
        assert _dense_flags(h, wl, 0.1).sum() == N * N       # 1/8 is above 1/10 everywhere
        h.close()


def test_difference_flags_mark_both_neighbours_of_a_jump():
    """A unit jump in pressure between columns s-1 and s: exactly the cells in
    columns s-1 and s see it (their centred differences straddle the jump)."""
    wl = _uniform(n=16)
    N = 16
    for s in (3, 5, 11):  # across and inside patches of at most 5 cells
        h = O.OracleHierarchy(wl, nlevels=1, with_qinit=False)
        q = np.zeros((3, N, N))
        q[0, :, s:] = 1.0
        _write(h, wl, q)
        want = np.zeros((N, N), dtype=np.uint8)
        want[:, s - 1:s + 1] = 1
        assert np.array_equal(_dense_flags(h, wl, 0.5), want)
        h.close()


def test_difference_flags_in_one_dimension():
    wl = _uniform(n=20, dim=1)
    h = O.OracleHierarchy(wl, nlevels=1, with_qinit=False)
    q = np.zeros((2, 1, 20))
    q[1, 0, 7:] = -2.0
    _write(h, wl, q)
    want = np.zeros((1, 20), dtype=np.uint8)
    want[0, 6:8] = 1
    assert np.array_equal(_dense_flags(h, wl, 1.0), want)


def test_surface_flags_look_at_the_first_component_only():
    wl = _uniform(flag_mode=W.FLAG_SURFACE)
    N = wl.n0[0]
    sign = np.where((np.arange(N)[None, :] + np.arange(N)[:, None]) % 2 == 0, 1.0, -1.0)
    h = O.OracleHierarchy(wl, nlevels=1, with_qinit=False)
    q = np.zeros((3, N, N))
    q[0] = 0.5 * sign
    q[1] = 7.0 * sign    # large momentum does not count
    _write(h, wl, q)
    assert _dense_flags(h, wl, 0.4).sum() == N * N
    assert _dense_flags(h, wl, 0.5).sum() == 0
    q[0, 2:4, 5:9] = 0.0
    _write(h, wl, q)
    assert _dense_flags(h, wl, 0.4).sum() == N * N - 8


def test_gauge_records_are_cell_values_of_the_containing_cell():
    """On one level a gauge records, after every step, the level-0 time and
    the values of the cell whose closed-open box holds the point."""
    wl = W.config2(seed=2, n0=20, ratios=(2,), tf=0.4, adj_n=40, nsnap=4)
    h = O.OracleHierarchy(wl, nlevels=1)
    dx = (wl.hi[0] - wl.lo[0]) / 20
    pts = [(wl.lo[0] + 3.5 * dx, wl.lo[1] + 7.25 * dx), (wl.lo[0] + 12.0 * dx, wl.lo[1] + 0.5 * dx),
           (wl.hi[0] + 1.0, wl.lo[1] - 1.0)]
    cells = [(3, 7), (12, 0), (19, 0)]  # the last point lies outside: clamped to the corner cell
    h.set_gauges([p[0] for p in pts], [p[1] for p in pts])
    dt = h.level_dt(0)
    for k in range(1, 4):
        h.advance(1)
        rec = h.gauges()
        assert rec.shape == (k, 3, 4)
        field = np.zeros((3, 20, 20))
        for (ilo, jlo, nx, ny), q in h.level_patch_arrays(0):
            field[:, jlo:jlo + ny, ilo:ilo + nx] = q
        for g, (I, J) in enumerate(cells):
            assert rec[-1, g, 0] == wl.t0 + k * dt
            assert np.array_equal(rec[-1, g, 1:], field[:, J, I])


def test_gauges_follow_the_finest_level_in_the_amr_limits():
    """tol < 0 refines everything: the gauge series is that of the uniform run
    on the finest grid, bit for bit; tol = +inf refines nothing: it is that of
    the uniform coarse run."""
    wl = W.config2(seed=4, n0=12, ratios=(2,), tf=0.5, adj_n=24, nsnap=6)
    xs, ys = [0.3, -2.9, 1.7], [0.1, 2.2, -3.3]
    n_coarse = None
    series = {}
    for tol in (-1.0, math.inf):
        amr = O.OracleHierarchy(wl, tol=tol)
        amr.set_adjoint(O.adjoint_solve(wl))
        amr.regrid(0, init=True)
        amr.set_gauges(xs, ys)
        n_coarse = amr.nsteps_total()
        amr.advance(n_coarse)
        series[tol] = amr.gauges()
    coarse = O.OracleHierarchy(wl, nlevels=1)
    coarse.set_gauges(xs, ys)
    coarse.advance(n_coarse)
    assert np.array_equal(series[math.inf], coarse.gauges())
    fine_wl = W.config2(seed=4, n0=24, ratios=(), tf=0.5, adj_n=24, nsnap=6)
    fine_wl.medium = wl.medium
    fine = O.OracleHierarchy(fine_wl, nlevels=1, dt0=O.OracleHierarchy(wl, tol=-1.0).level_dt(1))
    fine.set_gauges(xs, ys)
    fine.advance(2 * n_coarse)
    g_fine = fine.gauges()[1::2]   # one record per coarse step
    assert np.array_equal(series[-1.0][:, :, 1:], g_fine[:, :, 1:])
