"""Pins of the CPU oracle's AMR machinery (no GPU): hierarchy limits that
reduce to uniform runs, space-time interpolation, adjoint flagging against
brute force, Berger-Rigoutsos invariants (exhaustive on small fields), the
functional, and the forward-adjoint time invariance the method rests on
(Sec. 2, Eq. eq:q_equality / eq:J)."""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_03645_gb300 import workloads as W


def _small2d(n0=16, ratios=(2,), tf=0.6, **kw):
    return W.config2(seed=1, n0=n0, ratios=ratios, tf=tf, adj_n=2 * n0, nsnap=12, **kw)


def _all_levels_equal(a, b, nlev):
    for lev in range(nlev):
        assert np.array_equal(a.patches(lev), b.patches(lev))
        assert np.array_equal(a.read_level(lev), b.read_level(lev))


# ------------------------------------------------------ limits of the AMR
@pytest.mark.parametrize("which", ["1d", "2d"])
def test_infinite_tolerance_equals_uniform_coarse_bitwise(which):
    """tol = +inf flags nothing: no finer level exists and the run is the
    uniform coarse run, bit for bit."""
    wl = W.config1(n0=50, tf=3.0) if which == "1d" else _small2d()
    amr = O.OracleHierarchy(wl, tol=math.inf)
    amr.set_adjoint(O.adjoint_solve(wl))
    amr.regrid(0, init=True)
    uni = O.OracleHierarchy(wl, nlevels=1)
    n = uni.nsteps_total()
    amr.advance(n)
    uni.advance(n)
    assert len(amr.patches(1)) == 0
    assert np.array_equal(amr.read_level(0), uni.read_level(0))


@pytest.mark.parametrize("which", ["1d", "2d", "2d3"])
def test_full_refinement_equals_uniform_fine_bitwise(which):
    """tol < 0 flags every cell: the finest level covers the domain, never
    needs coarse interpolation, and evolves exactly like a uniform run on the
    finest grid with dt = dt_0 / prod(r)."""
    if which == "1d":
        wl = W.config1(n0=40, tf=2.0)
    elif which == "2d":
        wl = _small2d(n0=12, ratios=(2,), tf=0.5)
    else:
        wl = _small2d(n0=8, ratios=(2, 2), tf=0.4)
    amr = O.OracleHierarchy(wl, tol=-1.0)
    amr.regrid(0, init=True)
    L = wl.nlevels - 1
    dtf = amr.level_dt(L)
    fine_wl = W.config1(n0=wl.level_shape(L)[0], tf=wl.tf) if which == "1d" else \
        _small2d(n0=wl.level_shape(L)[0], ratios=(), tf=wl.tf)
    fine_wl.medium = wl.medium
    uni = O.OracleHierarchy(fine_wl, nlevels=1, dt0=dtf)
    n0 = amr.nsteps_total()
    amr.advance(n0)
    r = 1
    for k in range(L):
        r *= wl.ratios[k]
    uni.advance(n0 * r)
    a = amr.level_dense(L)
    b = uni.level_dense(0)
    assert not np.isnan(a).any()
    assert np.array_equal(a, b)


def test_amr_against_brute_force_uniform_fine():
    """Adjoint-guided AMR vs a uniform run on the finest grid (tiny 2D
    domain): inside the target the AMR solution must track the uniform fine
    one closely, and J must agree to a few percent."""
    wl = W.config2(seed=3, n0=24, ratios=(2,), tf=2.0, adj_n=48, nsnap=12, ts=0.0, tol=1e-4)
    amr = O.OracleHierarchy(wl)
    amr.set_adjoint(O.adjoint_solve(wl))
    amr.regrid(0, init=True)
    n0 = amr.nsteps_total()
    amr.advance(n0)
    fine_wl = W.config2(seed=3, n0=48, ratios=(), tf=wl.tf)
    fine_wl.medium = wl.medium
    fine_wl.qinit = wl.qinit
    uni = O.OracleHierarchy(fine_wl, nlevels=1, dt0=amr.level_dt(1))
    uni.advance(2 * n0)
    Ja, Ju = amr.functional(), uni.functional()
    Jc = O.OracleHierarchy(wl, nlevels=1)
    Jc.advance(n0)
    Jcoarse = Jc.functional()
    assert abs(Ja - Ju) <= 0.05 * abs(Ju) + 1e-12
    # AMR must be closer to the fine answer than the coarse grid is
    assert abs(Ja - Ju) <= abs(Jcoarse - Ju) + 1e-15


# ------------------------------------------------------ interpolation
def _boxed_adjoint(wl, box, S=4):
    """Snapshots with qhat = (1, 0, 0) inside box (adjoint-grid cells), 0 outside."""
    nx, ny = wl.adj_n
    s = np.zeros((S, wl.m, ny, nx))
    i0, i1, j0, j1 = box
    s[:, 0, j0:j1, i0:i1] = 1.0
    return s


def test_coarse_fine_interpolation_reproduces_linear_data():
    """Minmod-limited piecewise-linear interpolation is exact (to round-off)
    for data linear in x and y: every ghost cell of a fine patch equals the
    linear function at its centre (Sec. 3, space interpolation)."""
    a, b, c = 0.3, 0.7, -0.4
    wl = _small2d(n0=24, ratios=(2,), tf=1.0, tol=0.5)
    wl.qinit = lambda x, y: np.stack([5.0 + a * x + b * y, 1.0 + c * x, 2.0 + b * y])
    h = O.OracleHierarchy(wl)
    h.set_adjoint(_boxed_adjoint(wl, (20, 28, 20, 28)))
    h.regrid(0, init=True)
    P = h.patches(1)
    assert len(P) >= 1
    h.fill_ghosts(1)
    dx, dy = wl.level_dx(1)
    checked = 0
    for k, (ilo, jlo, nx, ny) in enumerate(P):
        q, _ = h.patch_ghosted(1, k)
        xs = wl.lo[0] + (ilo - 2 + np.arange(nx + 4) + 0.5) * dx
        ys = wl.lo[1] + (jlo - 2 + np.arange(ny + 4) + 0.5) * dy
        X, Y = np.meshgrid(xs, ys)
        ex = np.stack([5.0 + a * X + b * Y, 1.0 + c * X, 2.0 + b * Y])
        ring = np.ones((ny + 4, nx + 4), bool)
        ring[2:-2, 2:-2] = False
        inside = (X > wl.lo[0]) & (X < wl.hi[0]) & (Y > wl.lo[1]) & (Y < wl.hi[1])
        sel = ring & inside
        assert np.allclose(q[:, sel], ex[:, sel], rtol=0, atol=1e-13)
        checked += int(sel.sum())
    assert checked > 0


def test_average_down_of_constant_is_constant():
    """Averaging r^d equal children returns the value (to one rounding)."""
    wl = _small2d(n0=16, ratios=(2,), tf=0.2, tol=0.1)
    wl.qinit = lambda x, y: np.stack([np.full_like(x, 0.37), np.full_like(x, -1.25), np.full_like(x, 2.0)])
    h = O.OracleHierarchy(wl)
    h.set_adjoint(_boxed_adjoint(wl, (8, 20, 8, 20)))
    h.regrid(0, init=True)
    assert len(h.patches(1)) >= 1
    h.advance(1)   # constant state is steady; average-down writes level 0 under level 1
    q0 = h.level_dense(0)
    assert np.allclose(q0[0], 0.37, rtol=1e-15, atol=0)
    assert np.allclose(q0[1], -1.25, rtol=1e-15, atol=0)
    assert np.allclose(q0[2], 2.0, rtol=1e-15, atol=0)


# ------------------------------------------------------ adjoint flagging
def _flag_setup(mode, t_s, snaps_time_values, qcell=(0.8, -0.3, 0.5)):
    """One level-0 grid whose cells all hold qcell; adjoint snapshots are
    spatially constant with snapshot n equal to snaps_time_values[n]."""
    wl = W.config2(seed=1, n0=8, ratios=(2,), tf=1.0, adj_n=8, nsnap=len(snaps_time_values), ts=t_s)
    wl.flag_mode = mode
    wl.qinit = lambda x, y: np.stack([np.full_like(x, qcell[0]), np.full_like(x, qcell[1]),
                                      np.full_like(x, qcell[2])])
    h = O.OracleHierarchy(wl)
    S = len(snaps_time_values)
    snaps = np.zeros((S, 3, 8, 8))
    for n, v in enumerate(snaps_time_values):
        snaps[n] = np.asarray(v)[:, None, None]
    h.set_adjoint(snaps)
    return wl, h, np.asarray(snaps_time_values, float)


def _threshold_flag(h, val):
    """(flag at tol just below val, flag at tol just above val) of cell 0."""
    lo, _ = h.flag(0, val * (1 - 1e-12) if val > 0 else -1e-300)
    hi, _ = h.flag(0, val * (1 + 1e-12))
    return int(lo[0]), int(hi[0])


@pytest.mark.parametrize("t_s", [1.0, 0.55, 0.0])
def test_flag_linear_mode_equals_dense_time_sampling(t_s):
    """LINEAR mode: qhat is piecewise linear in time, so the window maximum
    of |qhat . q| sits at a breakpoint.  Brute force: 10^4 sample times in
    [t, T] plus the breakpoints; the oracle's value is their maximum."""
    rng = np.random.default_rng(5)
    S = 9
    vals = rng.normal(size=(S, 3))
    wl, h, V = _flag_setup(W.FLAG_LINEAR, t_s, vals)
    q = np.array([0.8, -0.3, 0.5])
    t = 0.0
    T = min(t + wl.tf - t_s, wl.tf)
    tn = wl.t0 + np.arange(S) * (wl.tf - wl.t0) / (S - 1)
    taus = np.concatenate([np.linspace(t, T, 10001), tn[(tn >= t) & (tn <= T)]])
    best = 0.0
    for tau in taus:
        n = min(int(np.searchsorted(tn, tau, side="right") - 1), S - 2)
        w = (tau - tn[n]) / (tn[1] - tn[0])
        qh = (1 - w) * V[n] + w * V[n + 1]
        best = max(best, abs(qh @ q))
    lo, hi = _threshold_flag(h, best)
    assert (lo, hi) == (1, 0)


@pytest.mark.parametrize("t_s", [1.0, 0.55, 0.0])
def test_flag_bracket_mode_is_max_over_bracketing_snapshots(t_s):
    """BRACKET-MAX (default; Sec. 4, both bracketing snapshots count): the maximum
    of |qhat_n . q| over the snapshots from the last one at or before t to
    the first one at or after T = min(t + t_f - t_s, t_f)."""
    rng = np.random.default_rng(6)
    S = 9
    vals = rng.normal(size=(S, 3))
    wl, h, V = _flag_setup(W.FLAG_BRACKET_MAX, t_s, vals)
    q = np.array([0.8, -0.3, 0.5])
    t = 0.0
    T = min(t + wl.tf - t_s, wl.tf)
    tn = wl.t0 + np.arange(S) * (wl.tf - wl.t0) / (S - 1)
    nlo = max(n for n in range(S) if tn[n] <= t)
    nhi = min(n for n in range(S) if tn[n] >= T)
    best = max(abs(V[n] @ q) for n in range(nlo, nhi + 1))
    assert _threshold_flag(h, best) == (1, 0)
    # bracket-max is never below the linear-in-time value
    wl2, h2, _ = _flag_setup(W.FLAG_LINEAR, t_s, vals)
    assert h2.flag(0, best * (1 + 1e-12))[0][0] == 0


def test_flag_bilinear_exact_for_linear_adjoint_and_dry_mask():
    """Bilinear interpolation reproduces an adjoint linear in space, so the
    flag threshold of every cell is |qhat(x_c, y_c) . q| with qhat evaluated
    analytically; cells over a dry adjoint cell are never flagged
    (Sec. 5.3: inner product set to zero where the adjoint is dry)."""
    wl = W.config2(seed=2, n0=10, ratios=(2,), tf=1.0, adj_n=20, nsnap=3)
    wl.qinit = lambda x, y: np.stack([np.ones_like(x), np.full_like(x, 0.5), np.zeros_like(x)])
    h = O.OracleHierarchy(wl)
    dxa = 8.0 / 20
    xa = -4 + (np.arange(20) + 0.5) * dxa
    XA, YA = np.meshgrid(xa, xa)
    lin = 0.1 + 0.05 * XA - 0.02 * YA
    snaps = np.zeros((3, 3, 20, 20))
    snaps[:, 0] = lin
    snaps[:, 1] = 2 * lin
    h.set_adjoint(snaps)
    dx = 0.8
    xc = -4 + (np.arange(10) + 0.5) * dx
    X, Y = np.meshgrid(xc, xc)
    ex = np.abs((0.1 + 0.05 * X - 0.02 * Y) * (1.0 + 0.5 * 2.0))
    flags_lo, _ = h.flag(0, 0.0)
    assert flags_lo.all()
    patches = h.patches(0)
    for tol_scale, expect in ((1 - 1e-9, 1), (1 + 1e-9, 0)):
        # evaluate cell by cell so each threshold is exact for that cell
        for (ilo, jlo, nx, ny) in patches[:1]:
            for (j, i) in [(0, 0), (3, 5), (ny - 1, nx - 1)]:
                tol = ex[jlo + j, ilo + i] * tol_scale
                f, _ = h.flag(0, tol)
                assert f[j * nx + i] == expect
    wet = np.ones((20, 20), np.uint8)
    wet[:10, :] = 0
    h.set_adjoint(snaps, wet=wet)
    f, _ = h.flag(0, 0.0)
    o = 0
    for (ilo, jlo, nx, ny) in patches:
        ff = f[o:o + nx * ny].reshape(ny, nx)
        o += nx * ny
        ycen = -4 + (jlo + np.arange(ny) + 0.5) * dx
        assert not ff[ycen < 0].any()
        assert ff[ycen > 0].all()


# ------------------------------------------------------ clustering
def _check_boxes(flags, boxes, eff, mc=1, nest=None):
    M, N = flags.shape
    cover = np.zeros_like(flags, dtype=int)
    for i0, i1, j0, j1 in boxes:
        assert 0 <= i0 <= i1 < N and 0 <= j0 <= j1 < M
        cover[j0:j1 + 1, i0:i1 + 1] += 1
        sub = flags[j0:j1 + 1, i0:i1 + 1]
        # tight: the box is the bounding box of its flags
        assert sub[:, 0].any() and sub[:, -1].any() and sub[0, :].any() and sub[-1, :].any()
        if nest is not None:
            assert nest[j0:j1 + 1, i0:i1 + 1].all()
        if mc == 1:
            assert sub.mean() >= eff - 1e-12
    assert cover.max(initial=0) <= 1
    assert np.all(cover[flags.astype(bool)] == 1)


def test_berger_rigoutsos_exhaustive_4x4():
    """Every one of the 2^16 flag fields on a 4x4 grid: boxes are disjoint,
    tight, cover every flag, and meet the efficiency cut-off."""
    for bits in range(1 << 16):
        f = np.array([(bits >> k) & 1 for k in range(16)], np.uint8).reshape(4, 4)
        b = O.cluster(f, mc=1, eff=0.7)
        _check_boxes(f, b, 0.7)


def test_berger_rigoutsos_random_fields_and_determinism():
    rng = np.random.default_rng(0)
    for trial in range(300):
        M, N = rng.integers(1, 9), rng.integers(1, 9)
        if trial % 3 == 0:
            M = 1  # 1D
        f = (rng.random((M, N)) < rng.uniform(0.05, 0.8)).astype(np.uint8)
        nest = None
        if trial % 4 == 1:
            nest = (rng.random((M, N)) < 0.9).astype(np.uint8)
            f &= nest
        b1 = O.cluster(f, mc=1, eff=0.7, nest=nest)
        b2 = O.cluster(f, mc=1, eff=0.7, nest=nest)
        assert np.array_equal(b1, b2)
        _check_boxes(f, b1, 0.7, nest=nest)
        # with a minimum box length, boxes still cover and stay disjoint
        b3 = O.cluster(f, mc=2, eff=0.7, nest=nest)
        _check_boxes(f, b3, 0.7, mc=2, nest=nest)


def test_regrid_invariants_in_hierarchy():
    """After a regrid: level-1 patches are disjoint, at most max_patch per
    side, properly nested (every cell within 2 coarse cells of a fine patch
    is a level-0 cell or outside the domain) and cover every buffered flag."""
    wl = _small2d(n0=32, ratios=(2, 2), tf=1.0, ts=0.0, tol=1e-3, max_patch=16)
    h = O.OracleHierarchy(wl)
    h.set_adjoint(O.adjoint_solve(wl))
    h.regrid(0, init=True)
    h.advance(3)
    h.regrid(0)
    for lev in (0, 1):
        C = wl.level_shape(lev)
        r = wl.ratios[lev]
        cov = np.zeros((C[1], C[0]), bool)
        for ilo, jlo, nx, ny in h.patches(lev):
            cov[jlo:jlo + ny, ilo:ilo + nx] = True
        fine = h.patches(lev + 1)
        if lev == 0:
            f, _ = h.flag(0, wl.tol)
            F = np.zeros_like(cov)
            o = 0
            for ilo, jlo, nx, ny in h.patches(0):
                F[jlo:jlo + ny, ilo:ilo + nx] = f[o:o + nx * ny].reshape(ny, nx).astype(bool)
                o += nx * ny
            B = np.zeros_like(F)
            for dj, di in itertools.product(range(-2, 3), repeat=2):
                B |= np.roll(np.roll(np.pad(F, 2), dj, 0), di, 1)[2:-2, 2:-2]
            fc = np.zeros_like(cov)
            for ilo, jlo, nx, ny in fine:
                fc[jlo // r:(jlo + ny) // r, ilo // r:(ilo + nx) // r] = True
            assert np.all(fc[B])
        fc = np.zeros((C[1], C[0]), int)
        pc = np.pad(cov, 2, constant_values=True)
        for ilo, jlo, nx, ny in fine:
            assert nx <= wl.max_patch and ny <= wl.max_patch
            assert ilo % r == 0 and jlo % r == 0 and nx % r == 0 and ny % r == 0
            fc[jlo // r:(jlo + ny) // r, ilo // r:(ilo + nx) // r] += 1
            i0, i1, j0, j1 = ilo // r, (ilo + nx) // r, jlo // r, (jlo + ny) // r
            assert pc[j0:j1 + 4, i0:i1 + 4].all()
        assert fc.max(initial=0) <= 1


@pytest.mark.parametrize("reflux", [0, 1])
def test_a_second_regrid_at_one_state_changes_nothing(reflux):
    """Regridding twice at the same state: the second regrid finds the boxes
    the first made, and the new-patch initialisation (Sec. 3: a new fine cell
    takes the old fine value where one exists) puts every value back where it
    was, so every level's layout and state are unchanged bit for bit, and the
    run continues exactly as without the second regrid."""
    wl = W.config2(seed=3, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=1e-4, min_patch=8,
                   max_patch=32)
    wl.reflux = reflux
    snaps = O.adjoint_solve(wl)
    runs = []
    for twice in (False, True):
        h = O.OracleHierarchy(wl)
        h.set_adjoint(snaps)
        h.regrid(0, init=True)
        h.advance(h.nsteps_total() // 3)
        h.regrid(0)
        before = [(h.patches(lev), h.read_level(lev)) for lev in range(wl.nlevels)]
        assert len(before[1][0]) > 0 and len(before[2][0]) > 0
        if twice:
            h.regrid(0)
            for lev, (p, q) in enumerate(before):
                assert np.array_equal(h.patches(lev), p) and np.array_equal(h.read_level(lev), q), lev
        h.advance(4)
        runs.append(h)
    _all_levels_equal(runs[0], runs[1], wl.nlevels)
    assert runs[0].functional() == runs[1].functional()


# ------------------------------------------------------ functional
def test_functional_of_constant_field_on_composite_grid():
    """J of q0 = const over the composite grid is const * weight * |box|,
    whatever the patch layout (each point counted once, at its finest
    level)."""
    wl = _small2d(n0=20, ratios=(2, 2), tf=1.0, tol=0.5)
    wl.qinit = lambda x, y: np.stack([np.full_like(x, 1.5), np.zeros_like(x), np.zeros_like(x)])
    wl.target = W.Target(-0.33, 1.71, -1.1, 0.47, weight=2.0)
    h = O.OracleHierarchy(wl)
    h.set_adjoint(_boxed_adjoint(wl, (16, 28, 14, 26)))
    h.regrid(0, init=True)
    assert len(h.patches(2)) > 0
    area = (1.71 + 0.33) * (0.47 + 1.1)
    assert h.functional() == pytest.approx(1.5 * 2.0 * area, rel=1e-14)


# ------------------------------------------------------ time invariance
@pytest.mark.parametrize("dim", [1, 2])
def test_forward_adjoint_inner_product_time_invariance(dim):
    """Eq. eq:q_equality / eq:J: with wall boundaries, int qhat^T q dx is the
    same at every t in [t_0, t_f] and equals J = int phi^T q(t_f) dx.  The
    adjoint is discretised independently of the forward problem, so the
    identity holds to discretisation error: the maximum deviation over the
    snapshot times shrinks under grid refinement."""
    devs = []
    Ns = (100, 200, 400) if dim == 1 else (24, 48)
    for N in Ns:
        if dim == 1:
            wl = W.config1(n0=N, adj_n=N, tf=6.0, nsnap=7, bc=(W.BC_WALL, W.BC_WALL))
            L = 8.0
            x = -4 + (np.arange(N) + 0.5) * L / N
            phi = np.zeros((2, 1, N))
            phi[0, 0] = np.exp(-((x - 1.0) / 0.3) ** 2)
            dA = L / N
        else:
            wl = W.config2(seed=3, n0=N, adj_n=N, tf=2.0, nsnap=5, bc=(W.BC_WALL,) * 4)
            xc = -4 + (np.arange(N) + 0.5) * 8.0 / N
            X, Y = np.meshgrid(xc, xc)
            phi = np.zeros((3, N, N))
            phi[0] = np.exp(-((X - 2.25) ** 2 + (Y - 2.25) ** 2) / 0.5 ** 2)
            dA = (8.0 / N) ** 2
        snaps = O.adjoint_solve(wl, phi=phi)
        S = snaps.shape[0]
        dts = (wl.tf - wl.t0) / (S - 1)
        dmin = 8.0 / N
        nsub = int(math.ceil(dts / (wl.cfl * dmin / wl.medium.cmax)))
        h = O.OracleHierarchy(wl, nlevels=1, dt0=dts / nsub)
        Js = []
        for n in range(S):
            if n:
                h.advance(nsub)
            q = h.level_dense(0)
            Js.append(float(np.sum(snaps[n] * q.reshape(snaps[n].shape)) * dA))
        Jf = float(np.sum(phi[0] * q[0].reshape(phi[0].shape)) * dA)
        assert abs(Js[-1] - Jf) <= 1e-12 * abs(Jf)   # at t_f the adjoint is phi itself
        devs.append(max(abs(j - Jf) for j in Js) / abs(Jf))
    for a, b in zip(devs, devs[1:]):
        assert b < 0.75 * a, devs
    assert devs[-1] < 0.05, devs


# ------------------------------------------------------ refluxing
def _composite_sum(h, wl, f=0):
    """Sum over the composite grid (each point on the finest level that
    covers it) of field f times the cell area."""
    tot = 0.0
    for lev in range(wl.nlevels):
        if len(h.patches(lev)) == 0:
            break
        q = h.level_dense(lev, fill=0.0)[f]
        dx, dy = wl.level_dx(lev)
        if lev + 1 < wl.nlevels and len(h.patches(lev + 1)):
            r = wl.ratios[lev]
            cov = np.zeros(q.shape, dtype=bool)
            for ilo, jlo, nx, ny in h.patches(lev + 1):
                cov[jlo // r:(jlo + ny) // r, ilo // r:(ilo + nx) // r] = True
            q = np.where(cov, 0.0, q)
        tot += float(q.sum()) * dx * dy
    return tot


def _reflux_workload(case, reflux):
    if case in ("acoustics_homog", "acoustics_adj_layered"):
        wl = W.config2(seed=2, n0=24, ratios=(2, 2), tf=3.0, bc=(W.BC_WALL,) * 4, tol=0.05)
        if case == "acoustics_homog":
            wl.medium = W.Medium(kind="layered", axis=1, iface=np.array([0.0]), rho=np.ones(2),
                                 K=np.full(2, 4.0), cmax=2.0)
        else:
            wl.eqn = W.EQ_ACOUSTICS_ADJ
    else:
        wl = W.config3(seed=4, n0=24, ratios=(2, 2), L=4.0e5, nmounts=6)
        wl.bc = (W.BC_WALL,) * 4
        wl.tf = 3.0 * 4.0e5 / wl.medium.cmax
        wl.tol = 0.05
        if case == "sw_adj":
            wl.eqn = W.EQ_SW_ADJ
    wl.flag_mode = W.FLAG_SURFACE
    wl.reflux = reflux
    return wl


@pytest.mark.parametrize("case", ["acoustics_homog", "acoustics_adj_layered", "sw", "sw_adj"])
def test_reflux_makes_amr_conserve_with_walls(case):
    """Conservation fix-up at coarse-fine interfaces (Sec. 3, AMR after
    Berger and LeVeque).  With walls nothing crosses the boundary, and on one
    grid the first field of these systems is conserved to round-off
    (homogeneous acoustics: sum p; adjoint acoustics in a layered medium and
    shallow water over bathymetry, forward and adjoint, all in f-wave form:
    sum of the first field).  On three levels whose patches follow the wave
    (surface flagging, regrid every 2 steps) the composite sum keeps that
    value to 1e-13 with the fix-up, and drifts measurably without it."""
    drift = {}
    for reflux in (1, 0):
        wl = _reflux_workload(case, reflux)
        h = O.OracleHierarchy(wl)
        h.regrid(0, init=True)
        assert len(h.patches(2)) > 0
        s0, scale = _composite_sum(h, wl), None
        q = h.level_dense(0)[0]
        scale = float(np.abs(q).sum()) * np.prod(wl.level_dx(0))
        h.advance(1)
        s1 = _composite_sum(h, wl)
        moved = 0
        before = [h.patches(lev).copy() for lev in range(3)]
        h.advance(h.nsteps_total() - 1)
        for lev in (1, 2):
            moved += not np.array_equal(before[lev], h.patches(lev))
        assert moved > 0, "patches never moved"
        drift[reflux] = abs(_composite_sum(h, wl) - s1) / scale
        del s0
    assert drift[1] <= 1e-13, drift
    assert drift[0] >= 1e-6, drift


def test_reflux_is_a_no_op_on_one_level_and_under_full_refinement():
    """Without a finer level, or with the finest level covering the domain,
    no cell has a coarse-fine side: the runs are bit for bit those without
    the fix-up."""
    for tol in (math.inf, -1.0):
        runs = []
        for reflux in (0, 1):
            wl = _small2d(n0=12, ratios=(2,), tf=0.5)
            wl.reflux = reflux
            h = O.OracleHierarchy(wl, tol=tol)
            h.set_adjoint(O.adjoint_solve(wl))
            h.regrid(0, init=True)
            h.advance(h.nsteps_total())
            runs.append(h)
        _all_levels_equal(runs[0], runs[1], 2)


# ------------------------------------------------------ AMR accuracy
@pytest.mark.parametrize("reflux", [0, 1])
def test_pulse_through_a_fixed_fine_box_reflects_less_under_refinement(reflux):
    """A y-independent pressure pulse (homogeneous medium, c = Z = 1) runs
    through a fine box held fixed by a constant adjoint that is 1 on the box
    (the state sits on a background p = 1, so |qhat . q| > 1/2 exactly on
    the box).  Any wave the box sends back is an artefact of the
    coarse-fine coupling (ghost interpolation in space and time, average
    down, and the fix-up when it is on); measured against the uniform coarse
    run behind the box after the pulse has passed, it falls at least 2.5x
    per halving of the mesh (second order, Sec. 3)."""
    amps = []
    for n0 in (32, 64, 128):
        wl = W.config2(n0=n0, ratios=(2,), tf=3.0, adj_n=n0, nsnap=2, tol=0.5, ts=0.0)
        wl.medium = W.Medium(kind="layered", axis=1, iface=np.array([0.0]), rho=np.ones(2), K=np.ones(2), cmax=1.0)
        wl.reflux = reflux

        def qinit(x, y):
            f = 0.4 * np.exp(-((x + 2.5) ** 2) / 0.25) + 0.0 * y
            return np.stack([1.0 + f, f, 0.0 * f])

        wl.qinit = qinit
        xa = -4 + (np.arange(n0) + 0.5) * 8.0 / n0
        X, Y = np.meshgrid(xa, xa)
        box = (np.abs(X) < 1) & (np.abs(Y) < 1)
        s = np.zeros((2, 3, n0, n0))
        s[:, 0, box] = 1.0
        h = O.OracleHierarchy(wl)
        h.set_adjoint(s)
        h.regrid(0, init=True)
        fine0 = h.patches(1).copy()
        h.advance(h.nsteps_total())
        assert np.array_equal(fine0, h.patches(1))           # the box never moved
        u = O.OracleHierarchy(wl, nlevels=1)
        u.advance(u.nsteps_total())
        behind = X < -1.5
        amps.append(float(np.abs(h.level_dense(0)[0][behind] - u.level_dense(0)[0][behind]).max()))
    assert amps[0] > 1e-5
    for a, b in zip(amps, amps[1:]):
        assert b * 2.5 <= a, amps


def test_adjoint_flagged_functional_converges_to_the_uniform_fine_one():
    """Sec. 5.2.1 at the paper's sizes (walls, time point t_f = 1.5, coarse
    and adjoint grids 50 x 50, ratios 2, 2) with the conservation fix-up:
    J of the adjoint-flagged run is within 5 % of the uniform finest-grid J at
    the paper's tolerance 0.02, and the error shrinks as the tolerance does,
    to below 0.5 % at 3e-4 (Sec. 4: cells whose inner product with the
    adjoint stays below the tolerance contribute little to J)."""
    wl = W.paper_5_2("timepoint_walls")
    wl.reflux = 1
    snaps = O.adjoint_solve(wl)

    def J(tol):
        h = O.OracleHierarchy(wl, tol=tol)
        h.set_adjoint(snaps)
        h.regrid(0, init=True)
        h.advance(h.nsteps_total())
        return h.functional()

    Jf = J(-1.0)
    errs = [abs(J(t) - Jf) / abs(Jf) for t in (0.02, 1.25e-3, 3e-4)]
    assert errs[0] < 0.05, errs
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 5e-3, errs


def test_set_layout_reproduces_a_hierarchy():
    """The oracle's layout entry (used to check another implementation's ghost
    cells on that implementation's own layout): a hierarchy copied level by
    level (patches, then interior states) fills its ghost cells and medium
    exactly like the original."""
    wl = _reflux_workload("acoustics_adj_layered", 0)   # layered medium, surface flags, walls
    a = O.OracleHierarchy(wl)
    a.regrid(0, init=True)
    a.advance(7)
    b = O.OracleHierarchy(wl, with_qinit=False)
    for lev in range(wl.nlevels):
        b.set_layout(lev, a.patches(lev))
        b.write_level(lev, a.read_level(lev))
    assert len(a.patches(2)) > 0
    for lev in range(1, wl.nlevels):
        a.fill_ghosts(lev)
        b.fill_ghosts(lev)
        for k in range(len(a.patches(lev))):
            qa, ma = a.patch_ghosted(lev, k)
            qb, mb = b.patch_ghosted(lev, k)
            assert np.array_equal(qa, qb) and np.array_equal(ma, mb)


# ------------------------------------------------------ adjoint with AMR
def _two_stage_average(q, rs):
    """Average a fine field [m, M, N] down level by level (ratios rs from
    the finest), each cell the sum of its children row by row times 1/r^2,
    as the hierarchy's average-down does."""
    for r in rs:
        m, M, N = q.shape
        out = np.zeros((m, M // r, N // r))
        inv = 1.0 / (r * r)
        for f in range(m):
            for b in range(M // r):
                for a in range(N // r):
                    s = 0.0
                    for jj in range(r):
                        for ii in range(r):
                            s = s + q[f, b * r + jj, a * r + ii]
                    out[f, b, a] = s * inv
        q = out
    return q


def _adjoint_fine_reference(wl, N, ratios, S):
    """Uniform adjoint on the finest grid with the hierarchy's finest step,
    averaged onto the snapshot grid in the hierarchy's order."""
    import copy
    rf = int(np.prod(ratios))
    dts = (wl.tf - wl.t0) / (S - 1)
    nsub = int(math.ceil(dts / (wl.cfl * (8.0 / N) / wl.medium.cmax)))
    wf = copy.copy(wl)
    wf.eqn, wf.n0, wf.ratios = wl.adj_eqn, (N * rf, N * rf), ()
    hf = O.OracleHierarchy(wf, nlevels=1, with_qinit=False, dt0=dts / nsub / rf)
    phif = O._phi_for(wl, (N * rf, N * rf))
    hf.write_level(0, np.concatenate([phif[:, jlo:jlo + ny, ilo:ilo + nx].reshape(-1)
                                      for ilo, jlo, nx, ny in hf.patches(0)]))
    out = []
    for s in range(S):
        if s:
            hf.advance(nsub * rf)
        out.append(_two_stage_average(hf.level_dense(0), list(reversed(ratios))))
    return np.array(out[::-1])


def test_adjoint_with_amr_limits_and_accuracy():
    """The adjoint solved with AMR (Sec. 7 proposes it for a more accurate
    inner product), snapshots from its level 0 after each Berger-Oliger step.
    Limits: tol = +inf refines nothing and gives the fixed-grid adjoint bit
    for bit; tol < 0 refines everything and gives the uniform finest-grid
    adjoint averaged onto the snapshot grid, bit for bit (target box on
    level-0 cell edges, so the interpolated initial data is the finest
    grid's).  Between them the snapshots approach that finest-grid adjoint as
    the tolerance falls, far closer than the fixed grid of the same size."""
    N, S, ratios = 16, 5, (2, 2)
    wl = W.config2(seed=3, n0=N, adj_n=N, tf=2.0, nsnap=S, bc=(W.BC_WALL,) * 4)
    uni = O.adjoint_solve(wl)
    assert np.array_equal(O.adjoint_solve_amr(wl, ratios, W.FLAG_DIFFERENCE, math.inf), uni)
    ref = _adjoint_fine_reference(wl, N, ratios, S)
    assert np.array_equal(O.adjoint_solve_amr(wl, ratios, W.FLAG_DIFFERENCE, -1.0), ref)
    e_uni = float(np.abs(uni - ref).max())
    errs = [float(np.abs(O.adjoint_solve_amr(wl, ratios, W.FLAG_DIFFERENCE, tol) - ref).max())
            for tol in (0.1, 0.03, 0.01)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-3 * e_uni, (errs, e_uni)
    # the same with the standard Richardson flagger (Sec. 1) on the adjoint's
    # own error estimate: exact limits, and the error falls with the tolerance
    assert np.array_equal(O.adjoint_solve_amr(wl, ratios, W.FLAG_RICHARDSON, math.inf), uni)
    assert np.array_equal(O.adjoint_solve_amr(wl, ratios, W.FLAG_RICHARDSON, -1.0), ref)
    errs = [float(np.abs(O.adjoint_solve_amr(wl, ratios, W.FLAG_RICHARDSON, tol) - ref).max())
            for tol in (3e-3, 1e-3, 3e-4)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-3 * e_uni, (errs, e_uni)
