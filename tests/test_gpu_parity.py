"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  States, adjoint snapshots and J must agree within 1e-12
relative (both follow the same operation order, so they agree exactly);
flags and patch layouts must agree bit for bit."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1511_03645_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_03645_gb300 import adjamr
    adjamr.load()
    return adjamr


def close(a, b, rtol=RTOL):
    a = np.asarray(a)
    b = np.asarray(b)
    assert a.shape == b.shape, (a.shape, b.shape)
    if a.size == 0:
        return
    scale = max(float(np.max(np.abs(b))), 1e-300)
    err = float(np.max(np.abs(a - b)))
    assert err <= rtol * scale, f"max abs diff {err:.3e} vs scale {scale:.3e}"


def scatter_write(h, level, dense):
    parts = [dense[:, jlo:jlo + ny, ilo:ilo + nx].reshape(-1) for ilo, jlo, nx, ny in h.patches(level)]
    h.write_level(level, np.concatenate(parts))


def dense_wl(dim, eqn, N, fields, bc, L=8.0, tf=1.0):
    if dim == 2:
        wl = W.config2(n0=N, lo=-L / 2, hi=L / 2, bc=bc, max_patch=64)
    else:
        wl = W.config1(n0=N, bc=bc[:2])
        wl.lo, wl.hi = (-L / 2, 0.0), (L / 2, 1.0)
    wl.eqn = eqn
    wl.tf = tf
    if eqn in (W.EQ_SW, W.EQ_SW_ADJ):
        cmax = float(np.sqrt(W.GRAV * fields.max()))
    else:
        cmax = float(np.sqrt(fields[1] / fields[0]).max())
    wl.medium = W.Medium(kind="dense", fields=[fields], cmax=cmax)
    return wl


# ---------------------------------------------------------- single level
CASES = [
    (1, W.EQ_ACOUSTICS, (W.BC_EXTRAP, W.BC_WALL, 0, 0)),
    (1, W.EQ_ACOUSTICS_ADJ, (W.BC_PERIODIC, W.BC_PERIODIC, 0, 0)),
    (2, W.EQ_ACOUSTICS, (W.BC_EXTRAP, W.BC_WALL, W.BC_PERIODIC, W.BC_PERIODIC)),
    (2, W.EQ_ACOUSTICS_ADJ, (W.BC_WALL, W.BC_EXTRAP, W.BC_WALL, W.BC_EXTRAP)),
    (2, W.EQ_SW, (W.BC_WALL, W.BC_WALL, W.BC_EXTRAP, W.BC_EXTRAP)),
    (2, W.EQ_SW_ADJ, (W.BC_PERIODIC, W.BC_PERIODIC, W.BC_WALL, W.BC_WALL)),
]


@pytest.mark.parametrize("dim,eqn,bc", CASES)
def test_uniform_grid_steps_match_oracle_bitwise(A, dim, eqn, bc):
    """Random medium and state on a multi-patch uniform grid with ragged
    tiles; 7 steps; every interior value identical."""
    rng = np.random.default_rng(100 + 10 * dim + eqn)
    N = 83 if dim == 2 else 301
    M = N if dim == 2 else 1
    if eqn in (W.EQ_SW, W.EQ_SW_ADJ):
        fields = rng.uniform(100, 4000, (1, M, N))
        L = 8e5
    else:
        fields = np.stack([rng.uniform(1, 3, (M, N)), rng.uniform(1, 30, (M, N))])
        L = 8.0
    wl = dense_wl(dim, eqn, N, fields, bc, L=L, tf=1.0)
    wl.max_patch0 = 40 if dim == 2 else 120
    q0 = rng.normal(size=(wl.m, M, N))
    o = O.OracleHierarchy(wl, nlevels=1, with_qinit=False)
    g = A.Hierarchy(wl, nlevels=1, with_qinit=False)
    assert np.array_equal(g.patches(0), o.patches(0))
    scatter_write(o, 0, q0)
    scatter_write(g, 0, q0)
    o.advance(7)
    g.advance(7)
    a, b = g.read_level(0), o.read_level(0)
    close(a, b)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("dim,eqn,bc", CASES)
def test_error_estimate_matches_oracle_bitwise(A, dim, eqn, bc):
    """The Richardson error estimate (Sec. 7) of a uniform grid of ragged,
    odd-sized patches (random medium and state, every boundary kind, after
    two steps): identical to the oracle's."""
    rng = np.random.default_rng(200 + 10 * dim + eqn)
    N = 83 if dim == 2 else 301
    M = N if dim == 2 else 1
    if eqn in (W.EQ_SW, W.EQ_SW_ADJ):
        fields = rng.uniform(100, 4000, (1, M, N))
        L = 8e5
    else:
        fields = np.stack([rng.uniform(1, 3, (M, N)), rng.uniform(1, 30, (M, N))])
        L = 8.0
    wl = dense_wl(dim, eqn, N, fields, bc, L=L, tf=1.0)
    wl.max_patch0 = 41 if dim == 2 else 121
    q0 = rng.normal(size=(wl.m, M, N))
    o = O.OracleHierarchy(wl, nlevels=1, with_qinit=False)
    g = A.Hierarchy(wl, nlevels=1, with_qinit=False)
    assert np.array_equal(g.patches(0), o.patches(0))
    scatter_write(o, 0, q0)
    scatter_write(g, 0, q0)
    o.advance(2)
    g.advance(2)
    cu = g.stats()["cell_updates"]
    a, b = g.error_estimate(0), o.error_estimate(0)
    assert np.any(b != 0.0)
    close(a, b)
    assert np.array_equal(a, b)
    # the estimate's steps are not forward steps
    assert g.stats()["cell_updates"] == cu
    assert np.array_equal(g.read_level(0), o.read_level(0))


@pytest.mark.parametrize("tile", [(16, 8), (16, 16), (32, 16), (64, 8), (8, 8), (12, 8), (24, 12), (5, 3)])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_tile_shapes_and_launch_modes_agree_bitwise(A, tile, mode):
    """Every tile size (compiled shapes and smaller cuts run by the smallest
    compiled shape holding them) and launch mode (work-list, persistent, per
    patch, dynamic) computes the same bits as the default configuration."""
    rng = np.random.default_rng(7)
    N = 70
    fields = np.stack([rng.uniform(1, 3, (N, N)), rng.uniform(1, 30, (N, N))])
    wl = dense_wl(2, W.EQ_ACOUSTICS, N, fields, (W.BC_EXTRAP,) * 4)
    wl.max_patch0 = 33
    q0 = rng.normal(size=(3, N, N))
    ref = A.Hierarchy(wl, nlevels=1, with_qinit=False)
    g = A.Hierarchy(wl, nlevels=1, with_qinit=False, tile=tile, launch_mode=mode)
    scatter_write(ref, 0, q0)
    scatter_write(g, 0, q0)
    ref.advance(5)
    g.advance(5)
    assert np.array_equal(ref.read_level(0), g.read_level(0))


# ---------------------------------------------------------- adjoint solve
@pytest.mark.parametrize("which", ["1d", "2d", "sw"])
def test_adjoint_snapshots_match_oracle(A, which):
    if which == "1d":
        wl = W.config1(adj_n=300, nsnap=25, tf=6.0, bc=(W.BC_WALL, W.BC_EXTRAP))
        med = None
    elif which == "2d":
        wl = W.config2(seed=4, n0=40, adj_n=90, nsnap=14, tf=2.0)
        med = None
    else:
        wl = W.config3(seed=1, n0=20, ratios=(2,), adj_n=50, nsnap=8, tf=3600.0, dense_levels=2)
        xa = (np.arange(50) + 0.5) * (2e6 / 50)
        X, Y = np.meshgrid(xa, xa)
        med = W.bathymetry(X, Y, wl.extra["mounts"])[None]
    ref = O.adjoint_solve(wl, medium_dense=med)
    adj = A.solve_adjoint(wl, medium_dense=med)
    got = adj.read()
    close(got, ref)
    assert np.array_equal(got, ref)
    assert np.abs(ref[0]).max() > 0


# ---------------------------------------------------------- AMR runs
def _amr_pair(A, wl, snaps=None, stream=None, **kw):
    if snaps is None:
        snaps = O.adjoint_solve(wl)
    o = O.OracleHierarchy(wl, **kw)
    o.set_adjoint(snaps)
    o.regrid(0, init=True)
    g = A.Hierarchy(wl, stream=stream, **kw)
    g.load_adjoint(snaps)
    g.regrid(0, init=True)
    return o, g


def _compare_all(o, g, nlev):
    for lev in range(nlev):
        assert np.array_equal(g.patches(lev), o.patches(lev)), f"layout of level {lev}"
        a, b = g.read_level(lev), o.read_level(lev)
        close(a, b)


@pytest.mark.parametrize("which", ["c1", "c2", "c2_linear", "c2_walls", "c3", "c1_diff", "c2_diff", "c3_surface",
                                   "p521", "p522", "p523", "p523_diff", "c2_sub", "c2_walls_sub",
                                   "c3_sub", "p523_sub",
                                   "c1_rx", "c2_rx", "c2_walls_rx", "c3_rx", "c3_surface_rx", "p521_rx",
                                   "p523_diff_rx", "c2_rx_sub", "c3_rx_sub",
                                   "c1_err", "c2_err", "c2_walls_err", "c3_err", "p521_err", "p523_err",
                                   "c2_err_rx", "p523_err_rx", "c2_err_sub",
                                   "c1_rich", "c2_rich", "c3_rich", "p523_rich", "c2_rich_rx"])
def test_amr_run_matches_oracle(A, which):
    """Adjoint-guided AMR runs (reduced sizes of the workloads): layouts of
    every level bit-exact after every regrid, states within 1e-12, flags
    bit-exact, J within 1e-12.  The _sub variants run the finest level's
    substeps as single substep launches; the _rx variants add the
    conservation fix-up at coarse-fine interfaces; the _err variants flag by
    the adjoint-weighted error estimate (Sec. 7) and the _rich variants by
    the estimate alone (the standard Richardson flagger, Sec. 1), whose
    values are compared on every flagged level too (their rings interpolate
    from coarser levels)."""
    sub = which.endswith("_sub")
    which = which[:-4] if sub else which
    rx = which.endswith("_rx")
    which = which[:-3] if rx else which
    err = which.endswith("_err")
    which = which[:-4] if err else which
    rich = which.endswith("_rich")
    which = which[:-5] if rich else which
    if which.startswith("p52"):
        # the paper's Sec. 5.2 examples at their own sizes
        wl = W.paper_5_2({"p521": "timepoint_walls", "p522": "range_walls"}.get(which[:4], "range_mixed"))
        if which.endswith("_diff"):
            wl.flag_mode, wl.tol = W.FLAG_DIFFERENCE, 0.1
        chunks = 4
    elif which.startswith("c1"):
        wl = W.config1(n0=100, tf=6.0, adj_n=400, nsnap=30)
        if which == "c1_diff":
            wl.flag_mode, wl.tol = W.FLAG_DIFFERENCE, 0.02
        chunks = 6
    elif which.startswith("c2"):
        bc = (W.BC_WALL,) * 4 if which == "c2_walls" else (W.BC_EXTRAP,) * 4
        wl = W.config2(seed=3, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=1e-4, bc=bc,
                       min_patch=8, max_patch=32)
        if which == "c2_linear":
            wl.flag_mode = W.FLAG_LINEAR
        if which == "c2_diff":
            wl.flag_mode, wl.tol = W.FLAG_DIFFERENCE, 0.05
        chunks = 4
    else:
        wl = W.config3(seed=2, n0=24, ratios=(2, 2), tf=4 * 3600.0, adj_n=48, nsnap=20, tol=1e-5, L=2.0e6,
                       dense_levels=3)
        if which == "c3_surface":
            wl.flag_mode, wl.tol = W.FLAG_SURFACE, 0.02
        chunks = 4
    wl.reflux = 1 if rx else 0
    if err:
        wl.flag_mode = W.FLAG_ERROR
        wl.tol = {"p": 1e-4, "c1": 1e-7, "c2": 1e-5, "c3": 1e-7}[which[:2] if which[0] == "c" else "p"]
    if rich:
        wl.flag_mode = W.FLAG_RICHARDSON
        wl.tol = {"p": 1e-3, "c1": 1e-3, "c2": 1e-3, "c3": 1e-2}[which[:2] if which[0] == "c" else "p"]
    snaps = O.adjoint_solve(wl, medium_dense=None if wl.medium.kind != "dense" else _adj_medium(wl))
    o, g = _amr_pair(A, wl, snaps=snaps)
    if sub:
        g.set_level_kernel(-1, (16, 12), True, A.LAUNCH_SUBSTEPS)
    _compare_all(o, g, wl.nlevels)
    n = o.nsteps_total()
    assert g.nsteps_total() == n
    refined = 0
    for c in range(chunks):
        k = n // chunks if c < chunks - 1 else n - (chunks - 1) * (n // chunks)
        o.advance(k)
        g.advance(k)
        _compare_all(o, g, wl.nlevels)
        refined += sum(len(o.patches(lev)) for lev in range(1, wl.nlevels))
        for lev in range(wl.nlevels - 1):
            fo, co = o.flag(lev, wl.tol)
            fg, cg = g.flag(lev, wl.tol)
            assert co == cg and np.array_equal(fo, fg)
            if (err or rich) and len(o.patches(lev)):
                assert np.array_equal(g.error_estimate(lev), o.error_estimate(lev)), f"estimate of level {lev}"
    assert refined > 0, "the case never refined"
    if sub:
        st = g.stats()
        fine = wl.nlevels - 1
        assert st["level_cell_updates"][fine] > 0
        # one launch per coarser step (r substeps each would exceed it)
        assert st["level_step_launches"][fine] <= st["level_step_launches"][fine - 1]
    Jo, Jg = o.functional(), g.functional()
    assert abs(Jg - Jo) <= RTOL * max(abs(Jo), 1e-300)


@pytest.mark.parametrize("reflux", [0, 1])
def test_per_level_kernels_compute_the_same_bits(A, reflux):
    """A different step-kernel tile on each level, with the ghost ring computed
    inside the step kernel or by the separate fill kernel, and with strided,
    per-patch or dynamically fetched tiles, changes nothing in the results
    (with and without the conservation fix-up); the per-level statistics add
    up to the totals."""
    wl = W.config2(seed=3, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=1e-4,
                   min_patch=8, max_patch=32)
    wl.reflux = reflux
    adj = A.solve_adjoint(wl)
    runs = []
    for cfg in (None, [((8, 8), False, 3), ((16, 16), True, 0), ((64, 8), False, 3)],
                [((32, 16), True, 3), ((16, 8), False, 1), ((8, 8), True, 3)],
                [((12, 8), True, 0), ((24, 12), False, 0), ((12, 8), False, 0)],
                # substep launches on the finest level; on the others mode 4 acts as mode 3
                [((12, 8), True, 4), ((8, 8), False, 4), ((16, 12), False, 4)],
                [((16, 8), False, 0), ((12, 8), True, 0), ((5, 3), True, 4)],
                [((32, 8), True, 0), ((16, 16), True, 1), ((16, 8), True, 4)]):
        h = A.Hierarchy(wl)
        h.set_adjoint(adj)
        h.set_timing(True)
        if cfg:
            for lev, (t, fuse, mode) in enumerate(cfg):
                h.set_level_kernel(lev, t, fuse, mode)
        h.regrid(0, init=True)
        h.advance(h.nsteps_total())
        st = h.stats()
        assert sum(st["level_cell_updates"]) == st["cell_updates"]
        assert sum(st["level_step_launches"]) == st["step_kernel_launches"]
        assert abs(sum(st["level_step_ms"]) - st["step_kernel_ms"]) <= 1e-6 * max(st["step_kernel_ms"], 1.0)
        assert sum(st["level_cell_updates"][1:]) > 0, "the case never refined"
        runs.append((h.functional(), [h.read_level(lev) for lev in range(wl.nlevels)],
                     [h.patches(lev) for lev in range(wl.nlevels)]))
        h.close()
    for J, lv, pt in runs[1:]:
        assert J == runs[0][0]
        assert all(np.array_equal(a, b) for a, b in zip(lv, runs[0][1]))
        assert all(np.array_equal(a, b) for a, b in zip(pt, runs[0][2]))
    h = A.Hierarchy(wl)
    with pytest.raises(A.AdjamrError):
        h.set_level_kernel(0, (40, 16))   # no compiled tile holds 40 x 16
    with pytest.raises(A.AdjamrError):
        h.set_level_kernel(0, (0, 8))
    with pytest.raises(A.AdjamrError):
        h.set_level_kernel(wl.nlevels, (32, 8))
    with pytest.raises(A.AdjamrError):
        h.set_level_kernel(0, (32, 8), True, 5)
    h.close()


@pytest.mark.parametrize("case", ["acoustics", "shallow_water", "acoustics_error_flags"])
def test_dry_adjoint_cells_match_oracle(A, case):
    """Adjoint cells marked dry (Sec. 5.3: no flag where the adjoint grid is
    dry) over part of the grid where this run flags: flags, layouts and
    states of the AMR run agree with the oracle's, no flag lies in a dry
    adjoint cell, and without the mask some would.  Acoustics (config 2
    reduced, x >= 1.5 dry), shallow water over bathymetry (config 3 reduced,
    x >= 250 km dry) and acoustics flagged by the adjoint-weighted error
    estimate, whose weight the mask zeroes as well."""
    if case == "shallow_water":
        wl = W.config3(seed=2, n0=24, ratios=(2, 2), tf=4 * 3600.0, adj_n=48, nsnap=20, tol=1e-5, L=2.0e6,
                       dense_levels=3)
        snaps = O.adjoint_solve(wl, medium_dense=_adj_medium(wl))
        wet = np.ones((48, 48), np.uint8)
        wet[:, 6:] = 0    # adjoint columns with x >= 250 km
        x_dry = 250000.0
    else:
        wl = W.config2(seed=3, n0=32, ratios=(2, 4), tf=1.5, adj_n=64, nsnap=20, ts=0.0, tol=1e-6,
                       min_patch=8, max_patch=32)
        if case == "acoustics_error_flags":
            wl.flag_mode = W.FLAG_ERROR
        snaps = O.adjoint_solve(wl)
        wet = np.ones((64, 64), np.uint8)
        wet[:, 44:] = 0   # adjoint columns with x >= 1.5
        x_dry = 1.5

    def flagged_x(h, lev, fl):
        dx = (wl.hi[0] - wl.lo[0]) / (wl.n0[0] * int(np.prod(wl.ratios[:lev])))
        xs, off = [], 0
        for ilo, jlo, nx, ny in h.patches(lev):
            ff = fl[off:off + nx * ny].reshape(ny, nx)
            off += nx * ny
            xs.extend((wl.lo[0] + (ilo + np.nonzero(ff)[1] + 0.5) * dx).tolist())
        return np.array(xs)

    plain = O.OracleHierarchy(wl)
    plain.set_adjoint(snaps)
    plain.regrid(0, init=True)
    assert (flagged_x(plain, 0, plain.flag(0, wl.tol)[0]) >= x_dry).any()
    o = O.OracleHierarchy(wl)
    o.set_adjoint(snaps, wet=wet)
    o.regrid(0, init=True)
    g = A.Hierarchy(wl)
    g.load_adjoint(snaps, wet=wet)
    g.regrid(0, init=True)
    _compare_all(o, g, wl.nlevels)
    n = o.nsteps_total()
    for c in range(3):
        k = n // 3 if c < 2 else n - 2 * (n // 3)
        o.advance(k)
        g.advance(k)
        _compare_all(o, g, wl.nlevels)
        for lev in range(wl.nlevels - 1):
            fo, co = o.flag(lev, wl.tol)
            fg, cg = g.flag(lev, wl.tol)
            assert co == cg and np.array_equal(fo, fg)
            assert not (flagged_x(g, lev, fg) >= x_dry).any()
    assert abs(g.functional() - o.functional()) <= RTOL * max(abs(o.functional()), 1e-300)


def test_substep_waits_give_up_and_the_context_stays_usable(A):
    """A substep launch whose tiles wait on a counter nothing advances: the
    bounded waits give up after about a second, the call reports ETIMEOUT,
    and the run then goes on to the oracle's results."""
    wl = W.config2(seed=3, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=1e-4,
                   min_patch=8, max_patch=32)
    o, g = _amr_pair(A, wl)
    g.set_level_kernel(-1, (16, 12), True, A.LAUNCH_SUBSTEPS)
    n = o.nsteps_total()
    k = n // 2
    o.advance(k)
    g.advance(k)
    assert len(g.patches(wl.nlevels - 1)) > 0
    rc, ms = g.substep_wait_selftest()
    assert rc == A.ETIMEOUT
    assert 500.0 <= ms <= 10000.0
    _compare_all(o, g, wl.nlevels)
    o.advance(n - k)
    g.advance(n - k)
    _compare_all(o, g, wl.nlevels)
    assert abs(g.functional() - o.functional()) <= RTOL * max(abs(o.functional()), 1e-300)


def test_gauges_match_oracle_bitwise(A):
    """Gauge series (finest level covering each point, after every coarse
    step) of an adjoint-flagged run and of a difference-flagged run equal the
    oracle's bit for bit."""
    for mode, tol in ((W.FLAG_BRACKET_MAX, 1e-4), (W.FLAG_DIFFERENCE, 0.05)):
        wl = W.config2(seed=3, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=tol,
                       min_patch=8, max_patch=32)
        wl.flag_mode = mode
        o, g = _amr_pair(A, wl)
        xs, ys = [2.25, 0.0, -3.9, 1.3], [2.25, 0.0, 3.9, -0.7]
        o.set_gauges(xs, ys)
        g.set_gauges(xs, ys)
        n = o.nsteps_total()
        o.advance(n // 2)
        g.advance(n // 2)
        o.advance(n - n // 2)
        g.advance(n - n // 2)
        go, gg = o.gauges(), g.gauges()
        assert go.shape == gg.shape == (n, 4, 4)
        assert np.array_equal(go, gg)
        assert np.any(go[:, 0, 1] != 0.0)


def _adj_medium(wl):
    nx = wl.adj_n[0]
    xa = wl.lo[0] + (np.arange(nx) + 0.5) * (wl.hi[0] - wl.lo[0]) / nx
    X, Y = np.meshgrid(xa, xa)
    return W.bathymetry(X, Y, wl.extra["mounts"], wl.hi[0])[None]


def test_edge_cases_no_refinement_and_full_refinement(A):
    """tol = +inf: no finer level; tol < 0: the finest level covers the
    domain; both agree with the oracle bit for bit."""
    wl = W.config2(seed=5, n0=20, ratios=(2,), tf=0.5, adj_n=40, nsnap=6)
    for tol in (math.inf, -1.0):
        snaps = O.adjoint_solve(wl)
        o, g = _amr_pair(A, wl, snaps=snaps, tol=tol)
        n = o.nsteps_total()
        o.advance(n)
        g.advance(n)
        _compare_all(o, g, wl.nlevels)
        if tol > 0:
            assert len(g.patches(1)) == 0
        else:
            cov = sum(int(nx) * int(ny) for _, _, nx, ny in g.patches(1))
            assert cov == 40 * 40


@pytest.mark.parametrize("case", ["ratio16", "odd_ratio3_1d", "two_snapshots", "ragged_n0_37", "ratios_3_5"])
def test_degenerate_parameters_match_oracle(A, case):
    """Limits the method admits, each against the oracle bit for bit: the
    largest refinement ratio (16: the time-fraction table is full), odd
    ratios (fine cells straddle no coarse centre symmetrically: offsets
    (2m + 1 - r)/(2r) with r odd), the fewest adjoint snapshots (2: every
    window brackets the whole run), a coarse grid whose size no tile divides,
    and an advance by zero steps (a no-op)."""
    if case == "ratio16":
        wl = W.config2(seed=4, n0=12, ratios=(16,), tf=0.4, adj_n=48, nsnap=8, ts=0.0, tol=1e-3,
                       min_patch=16, max_patch=64)
    elif case == "odd_ratio3_1d":
        wl = W.config1(n0=60, ratio=3, tf=3.0, adj_n=180, nsnap=12)
    elif case == "two_snapshots":
        wl = W.config2(seed=6, n0=20, ratios=(2,), tf=0.6, adj_n=40, nsnap=2, ts=0.0, tol=1e-6)
    elif case == "ragged_n0_37":
        wl = W.config2(seed=7, n0=37, ratios=(2, 2), tf=0.5, adj_n=74, nsnap=10, ts=0.0, tol=0.02)
    else:
        wl = W.config2(seed=8, n0=18, ratios=(3, 5), tf=0.4, adj_n=54, nsnap=10, ts=0.0, tol=0.02,
                       min_patch=15, max_patch=60)
    if case in ("ragged_n0_37", "ratios_3_5"):
        wl.flag_mode = W.FLAG_DIFFERENCE   # layouts from the undivided differences of the state
    snaps = O.adjoint_solve(wl)
    o, g = _amr_pair(A, wl, snaps=snaps)
    g.advance(0)
    _compare_all(o, g, wl.nlevels)
    n = o.nsteps_total()
    refined = 0
    for c in range(3):
        k = n // 3 if c < 2 else n - 2 * (n // 3)
        o.advance(k)
        g.advance(k)
        _compare_all(o, g, wl.nlevels)
        refined += sum(len(o.patches(lev)) for lev in range(1, wl.nlevels))
    assert refined > 0, "the case never refined"
    assert abs(g.functional() - o.functional()) <= RTOL * max(abs(o.functional()), 1e-300)


@pytest.mark.parametrize("case", ["c2", "c2_rx", "c1"])
def test_unchanged_layout_is_kept(A, case):
    """A regrid that finds a level's current boxes again, over a coarser level
    it left as it was, keeps the level (a rebuild would reproduce it bit for
    bit): a second regrid at the same state keeps every finer level, an empty
    level stays empty without a rebuild, and the runs then go on to the
    oracle's results, whose regrids always rebuild."""
    if case == "c1":
        wl = W.config1(n0=100, tf=6.0, adj_n=400, nsnap=30)
    else:
        wl = W.config2(seed=3, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=1e-4,
                       min_patch=8, max_patch=32)
    wl.reflux = 1 if case.endswith("_rx") else 0
    snaps = O.adjoint_solve(wl)
    o, g = _amr_pair(A, wl, snaps=snaps)
    n = o.nsteps_total()
    k = n // 3
    o.advance(k)
    g.advance(k)
    # the first regrid at this state may change the layout (the last one ran
    # at an earlier step); the second finds the same boxes on every level
    o.regrid(0)
    g.regrid(0)
    _compare_all(o, g, wl.nlevels)
    nfine = [len(g.patches(lev)) for lev in range(1, wl.nlevels)]
    kept0, built0 = g.stats()["level_rebuilds_skipped"], g.stats()["level_rebuilds"]
    o.regrid(0)
    g.regrid(0)
    _compare_all(o, g, wl.nlevels)
    st = g.stats()
    # every finer level up to the first empty one is kept, none rebuilt
    want = next((i + 1 for i, c in enumerate(nfine) if c == 0), len(nfine))
    assert st["level_rebuilds_skipped"] - kept0 == want
    assert st["level_rebuilds"] == built0
    o.advance(n - k)
    g.advance(n - k)
    _compare_all(o, g, wl.nlevels)
    assert abs(g.functional() - o.functional()) <= RTOL * max(abs(o.functional()), 1e-300)


def test_cfl_violation_is_reported(A):
    """Courant number above cfl_max returns ADJAMR_ECFL, not a crash."""
    wl = W.config2(seed=5, n0=16, ratios=(2,), tf=0.5)
    wl.cfl_max = 0.5
    g = A.Hierarchy(wl, nlevels=1)
    with pytest.raises(A.AdjamrError) as ei:
        g.advance(2)
    assert ei.value.code == A.ECFL


def test_torch_stream_interop(A):
    """Work issued on a PyTorch stream; results identical to the default stream."""
    import torch
    wl = W.config2(seed=6, n0=24, ratios=(2,), tf=0.6, adj_n=48, nsnap=8, ts=0.0, tol=1e-4)
    snaps = O.adjoint_solve(wl)
    s = torch.cuda.Stream()
    o, g = _amr_pair(A, wl, snaps=snaps, stream=s.cuda_stream)
    n = o.nsteps_total()
    o.advance(n)
    g.advance(n)
    _compare_all(o, g, wl.nlevels)


# ---------------------------------------------------------- batched patches
def test_batched_patches_modes_agree_and_match_oracle(A):
    """4096 uneven patches (the batching stress configuration): the fused
    work-list launch, the persistent grid, one launch per patch, and the
    CUDA-graph replay, each with the ghost ring filled by its own kernel or
    inside the step kernel, all produce the same bits; sampled patches (smallest,
    largest, and random) match the oracle run of that patch alone."""
    pb = W.config4(seed=0)
    results = []
    for mode, graph, fuse in ((0, False, False), (1, False, False), (2, False, False), (0, True, False),
                              (1, True, False), (0, False, True), (1, True, True), (2, False, True),
                              (3, False, False), (3, True, True)):
        import torch
        s = torch.cuda.Stream()
        b = A.Batch(pb, stream=s.cuda_stream)
        b.set_ghost_fusion(fuse)
        b.step(4, mode=mode, tile=(32, 8), graph=graph)
        results.append(b.read())
        b.close()
    for r in results[1:]:
        assert np.array_equal(r, results[0])
    cells = pb.nx.astype(np.int64) * pb.ny
    offs = np.concatenate([[0], np.cumsum(3 * cells)])
    rng = np.random.default_rng(1)
    sample = sorted({int(np.argmin(cells)), int(np.argmax(cells))} | set(rng.choice(pb.npatch, 6, replace=False).tolist()))
    for k in sample:
        nx, ny = int(pb.nx[k]), int(pb.ny[k])
        x0, y0 = float(pb.x0[k]), float(pb.y0[k])
        x1, y1 = x0 + nx * float(pb.dx[k]), y0 + ny * float(pb.dx[k])
        wl = W.config2(n0=nx, lo=x0, hi=x1, bc=(W.BC_EXTRAP,) * 4)
        wl.n0 = (nx, ny)
        wl.lo, wl.hi = (x0, y0), (x1, y1)
        wl.medium = pb.media[int(pb.medium_id[k])]
        wl.max_patch0 = 1024
        o = O.OracleHierarchy(wl, nlevels=1, with_qinit=False, dt0=float(pb.dt[k]))
        o.write_level(0, pb.qinit_patch(k).reshape(-1))
        o.advance(4)
        got = results[0][offs[k]:offs[k + 1]]
        assert np.array_equal(got, o.read_level(0)), f"patch {k}"


# ---------------------------------------------------------- full size, sampled
def _ghosts_match_oracle_on_gpu_layout(g, wl, picks):
    """The ghost rings and medium of sampled patches, checked independently
    of the GPU's ghost fill: the oracle takes the GPU's patch layouts and
    interior states of every level, fills the ghost cells itself (same-level
    copies, boundary maps, coarse space interpolation, Sec. 3) and computes
    the medium of every storage cell; both must equal the GPU's bit for bit.
    picks: {level: [patch indices]}."""
    o = O.OracleHierarchy(wl, with_qinit=False)
    for lev in range(wl.nlevels):
        P = g.patches(lev)
        if len(P) == 0:
            break
        o.set_layout(lev, P)
        o.write_level(lev, g.read_level(lev))
    n = 0
    for lev, ks in picks.items():
        g.fill_ghosts(lev)
        o.fill_ghosts(lev)
        for k in ks:
            qg, mg = g.patch_ghosted(lev, k)
            qo, mo = o.patch_ghosted(lev, k)
            assert np.array_equal(qg, qo), f"ghost ring, level {lev} patch {k}"
            assert np.array_equal(mg, mo), f"medium, level {lev} patch {k}"
            n += 1
    o.close()
    return n


def test_full_size_config2_sampled_step_parity(A):
    """Config 2 at full size (100^2 coarse, ratios 2 and 4, adjoint 400^2 x
    200 snapshots) in the benchmark's launch configuration: after an adjoint-
    guided run of 40 coarse steps, the ghost rings and medium of sampled
    patches of every refined level equal the oracle's own fill from the GPU's
    interior states, and one step of sampled finest-level patches is
    recomputed by the oracle from that ghosted input and must match bit for
    bit; layouts satisfy the size invariants."""
    wl = W.config2(seed=0, ts=0.0, tol=1e-3)
    adj = A.solve_adjoint(wl)
    g = A.Hierarchy(wl)
    g.set_adjoint(adj)
    for lev, (t, fuse) in enumerate((((16, 8), True), ((8, 8), True), ((16, 12), False))):
        g.set_level_kernel(lev, t, fuse, A.LAUNCH_WORKLIST)   # the benchmark's usual per-level choice
    g.regrid(0, init=True)
    g.advance(40)
    L = wl.nlevels - 1
    P = g.patches(L)
    assert len(P) > 0
    rng = np.random.default_rng(0)
    picks = {lev: sorted(set(rng.choice(len(g.patches(lev)), min(12, len(g.patches(lev))), replace=False).tolist()))
             for lev in range(1, wl.nlevels) if len(g.patches(lev))}
    assert _ghosts_match_oracle_on_gpu_layout(g, wl, picks) >= 12
    g.fill_ghosts(L)
    ks = sorted(set(rng.choice(len(P), min(12, len(P)), replace=False).tolist()))
    inputs = [g.patch_ghosted(L, k) for k in ks]
    dt = g.time_info()[0] / (wl.ratios[0] * wl.ratios[1])
    dx, dy = wl.level_dx(L)
    g.step_level_only(L)
    flat = g.read_level(L)
    offs = np.concatenate([[0], np.cumsum([3 * int(nx) * int(ny) for _, _, nx, ny in P])])
    for k, (q, med) in zip(ks, inputs):
        ref, _ = O.step_patch(2, W.EQ_ACOUSTICS, q, med, dt, dx, dy)
        assert np.array_equal(flat[offs[k]:offs[k + 1]], ref.reshape(-1)), f"patch {k}"
    for lev in range(1, wl.nlevels):
        for ilo, jlo, nx, ny in g.patches(lev):
            assert nx <= wl.max_patch and ny <= wl.max_patch
    # the adjoint snapshot at t_f is phi itself
    snaps = adj.read()
    close(snaps[-1], wl.adjoint_phi())


def test_full_size_config2_error_estimate_matches_oracle(A):
    """Config 2 at full size flagged by the adjoint-weighted error estimate
    (tol 1e-6), in the benchmark's per-level launch configuration: after 24
    coarse steps (every level at the same time), the estimate of each flagged
    level equals, bit for bit, the one the oracle computes on the GPU's layout
    from the GPU's interior states of that level and the coarser ones."""
    wl = W.config2(seed=0, ts=0.0, tol=1e-6)
    wl.flag_mode = W.FLAG_ERROR
    adj = A.solve_adjoint(wl)
    g = A.Hierarchy(wl)
    g.set_adjoint(adj)
    for lev, (t, fuse) in enumerate((((16, 8), True), ((8, 8), True), ((16, 12), False))):
        g.set_level_kernel(lev, t, fuse, A.LAUNCH_WORKLIST)
    g.regrid(0, init=True)
    g.advance(24)
    assert len(g.patches(2)) > 0
    n0 = 24
    for lev in range(wl.nlevels - 1):
        o = O.OracleHierarchy(wl, with_qinit=False)
        r = 1
        for k in range(lev + 1):
            o.set_layout(k, g.patches(k))
            o.write_level(k, g.read_level(k))
            o.set_level_time(k, n0 * r)
            if k < lev:
                r *= wl.ratios[k]
        a, b = g.error_estimate(lev), o.error_estimate(lev)
        assert np.any(b != 0.0)
        assert np.array_equal(a, b), f"level {lev}"


@pytest.mark.parametrize("case", ["bracket", "error_reflux"])
def test_reset_gives_the_bits_of_a_new_context(A, case):
    """adjamr_reset: a second solve in the same context (after a first one
    that refined and recorded gauges) gives the layouts, states, J, gauge
    records and cell-update count of the first, bit for bit."""
    wl = W.config2(seed=3, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=1e-4, min_patch=8,
                   max_patch=32)
    if case == "error_reflux":
        wl.flag_mode, wl.tol, wl.reflux = W.FLAG_ERROR, 1e-5, 1
    snaps = O.adjoint_solve(wl)
    g = A.Hierarchy(wl)
    g.load_adjoint(snaps)
    g.set_gauges([0.3, -1.1], [0.2, 0.7])

    def solve():
        g.regrid(0, init=True)
        g.advance(g.nsteps_total())
        levels = [(g.patches(lev), g.read_level(lev)) for lev in range(wl.nlevels)]
        return levels, g.functional(), g.gauges(), g.stats()["cell_updates"]

    first = solve()
    assert sum(len(p) for p, _ in first[0][1:]) > 0
    g.reset()
    assert g.stats()["cell_updates"] == 0 and len(g.patches(1)) == 0
    second = solve()
    for (pa, qa), (pb, qb) in zip(first[0], second[0]):
        assert np.array_equal(pa, pb) and np.array_equal(qa, qb)
    assert first[1] == second[1]
    assert np.array_equal(first[2], second[2])
    assert first[3] == second[3]
    g.close()


@pytest.mark.parametrize("keep_first", [False, True])
def test_second_adjoint_set_in_the_same_context(A, keep_first):
    """A second snapshot set of the same shape loaded into a context (after a
    solve with the first): the solve then follows the second set to the
    oracle's bits.  With no other holder the first set's device buffers take
    the second (refilled in place); a first set still held elsewhere keeps
    its values and the second gets buffers of its own."""
    wl = W.config2(seed=3, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=1e-4, min_patch=8,
                   max_patch=32)
    snaps_a = O.adjoint_solve(wl)
    wl_b = W.config2(seed=5, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=1e-4, min_patch=8,
                     max_patch=32)
    snaps_b = O.adjoint_solve(wl_b)
    assert snaps_a.shape == snaps_b.shape and not np.array_equal(snaps_a, snaps_b)
    g = A.Hierarchy(wl)
    first = g.load_adjoint(snaps_a)
    if not keep_first:
        first.release()
    g.regrid(0, init=True)
    g.advance(g.nsteps_total() // 2)
    g.reset()
    second = g.load_adjoint(snaps_b)
    assert np.array_equal(second.read(), snaps_b)
    if keep_first:
        assert np.array_equal(first.read(), snaps_a)
        first.release()
    g.regrid(0, init=True)
    o = O.OracleHierarchy(wl)
    o.set_adjoint(snaps_b)
    o.regrid(0, init=True)
    _compare_all(o, g, wl.nlevels)
    n = o.nsteps_total()
    o.advance(n)
    g.advance(n)
    _compare_all(o, g, wl.nlevels)
    assert abs(g.functional() - o.functional()) <= RTOL * max(abs(o.functional()), 1e-300)
    second.release()
    g.close()


def test_error_estimate_of_a_shallowly_nested_level_is_refused_and_the_run_goes_on(A):
    """A hierarchy flagged by the bracket rule nests its finest level only 2
    coarse cells deep; with ratio 2 the estimate's ring of 4 fine cells then
    needs coarse cells outside the coarser level, and both sides refuse the
    estimate (ENEST on the GPU).  The refusal leaves the context usable: the
    run goes on to the oracle's bits."""
    wl = W.config2(seed=1, n0=32, ratios=(2, 2), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=1e-4, min_patch=8,
                   max_patch=32)
    o, g = _amr_pair(A, wl)
    o.advance(1)
    g.advance(1)
    _compare_all(o, g, wl.nlevels)
    assert len(g.patches(2)) > 0
    with pytest.raises(RuntimeError):
        o.error_estimate(2)
    with pytest.raises(A.AdjamrError) as ei:
        g.error_estimate(2)
    assert ei.value.code == A.ENEST
    assert np.array_equal(g.error_estimate(0), o.error_estimate(0))
    o.advance(4)
    g.advance(4)
    _compare_all(o, g, wl.nlevels)
    assert abs(g.functional() - o.functional()) <= RTOL * max(abs(o.functional()), 1e-300)


def test_full_size_config1_matches_oracle_everywhere(A):
    """Config 1 at full size (200 coarse cells, ratio 4, adjoint 800 cells x
    100 snapshots, t_f = 20): the whole run, element by element, with the
    layout and the flags compared at every tenth of the run."""
    wl = W.config1()
    snaps = O.adjoint_solve(wl)
    adj = A.solve_adjoint(wl)
    assert np.array_equal(adj.read(), snaps)
    o = O.OracleHierarchy(wl)
    o.set_adjoint(snaps)
    o.regrid(0, init=True)
    g = A.Hierarchy(wl)
    g.set_adjoint(adj)
    g.regrid(0, init=True)
    n = o.nsteps_total()
    refined = 0
    for c in range(10):
        k = n // 10 if c < 9 else n - 9 * (n // 10)
        o.advance(k)
        g.advance(k)
        _compare_all(o, g, wl.nlevels)
        refined += len(o.patches(1))
        fo, co = o.flag(0, wl.tol)
        fg, cg = g.flag(0, wl.tol)
        assert co == cg and np.array_equal(fo, fg)
    assert refined > 0
    assert abs(g.functional() - o.functional()) <= RTOL * max(abs(o.functional()), 1e-300)


def test_full_size_config3_sampled_step_parity(A):
    """Config 3 at full size (coarse 200^2 over 2000 km, ratios 4, 4, 2 --
    finest 6400^2 index space -- adjoint 1000^2 x 300 snapshots solved on the
    GPU): after an adjoint-guided run until the finest level is refined (at
    least 8 coarse steps, regrids every 2 steps of each level), the ghost rings and
    medium of sampled patches of every refined level equal the oracle's own
    fill from the GPU's interior states and its own bathymetry, and one step
    of sampled patches of every refined level is recomputed by the oracle
    from that ghosted input (f-wave shallow water over the bathymetry) and
    must match bit for bit."""
    wl = W.config3(seed=0)
    nx = wl.adj_n[0]
    xa = wl.lo[0] + (np.arange(nx) + 0.5) * (wl.hi[0] - wl.lo[0]) / nx
    X, Y = np.meshgrid(xa, xa)
    adj_med = W.bathymetry(X, Y, wl.extra["mounts"], wl.hi[0])[None]
    adj = A.solve_adjoint(wl, medium_dense=adj_med)
    snaps_last = adj.read()[-1]
    close(snaps_last, wl.adjoint_phi())
    g = A.Hierarchy(wl)
    g.set_adjoint(adj)
    g.regrid(0, init=True)
    # advance (regrids every 2 steps of each level) until the finest level
    # holds patches, at most 200 of the 320 coarse steps
    steps = 0
    while steps < 200 and (steps < 8 or len(g.patches(wl.nlevels - 1)) == 0):
        g.advance(8)
        steps += 8
    dt0 = g.time_info()[0]
    rng = np.random.default_rng(3)
    picks = {lev: sorted(set(rng.choice(len(g.patches(lev)), min(6, len(g.patches(lev))), replace=False).tolist()))
             for lev in range(1, wl.nlevels) if len(g.patches(lev))}
    assert len(picks) >= 2, f"only levels {sorted(picks)} refined after {steps} coarse steps"
    assert _ghosts_match_oracle_on_gpu_layout(g, wl, picks) >= 6
    checked = 0
    for L in range(1, wl.nlevels):
        P = g.patches(L)
        if len(P) == 0:
            continue
        g.fill_ghosts(L)
        ks = sorted(set(rng.choice(len(P), min(3, len(P)), replace=False).tolist()))
        inputs = [g.patch_ghosted(L, k) for k in ks]
        flat_before = g.read_level(L)
        g.step_level_only(L)
        flat = g.read_level(L)
        dt = dt0
        for k in range(L):
            dt = dt / wl.ratios[k]
        dx, dy = wl.level_dx(L)
        offs = np.concatenate([[0], np.cumsum([3 * int(a) * int(b) for _, _, a, b in P])])
        for k, (q, med) in zip(ks, inputs):
            ref, _ = O.step_patch(2, W.EQ_SW, q, med, dt, dx, dy)
            assert np.array_equal(flat[offs[k]:offs[k + 1]], ref.reshape(-1)), f"level {L} patch {k}"
            checked += 1
        assert flat_before.shape == flat.shape
    assert checked > 0


def test_reflux_conserves_on_the_gpu_with_walls(A):
    """The conservation fix-up on the GPU: homogeneous acoustics with walls on
    three levels whose patches follow the wave keeps the composite sum of p
    constant to 1e-13 (as the oracle's pin shows for the same run), and the
    run without the fix-up does not."""
    import test_oracle_amr as T
    drift = {}
    for reflux in (1, 0):
        wl = T._reflux_workload("acoustics_homog", reflux)
        g = A.Hierarchy(wl)
        g.regrid(0, init=True)
        g.advance(1)
        s1 = T._composite_sum(g, wl)
        q = g.level_dense(0)[0]
        scale = float(np.abs(q).sum()) * np.prod(wl.level_dx(0))
        g.advance(g.nsteps_total() - 1)
        drift[reflux] = abs(T._composite_sum(g, wl) - s1) / scale
        g.close()
    assert drift[1] <= 1e-13 and drift[0] >= 1e-6, drift


def test_flag_time_range_per_call_and_level0_only_advance(A):
    """adjamr_flag_cells takes the start t_s of the range of interest per call
    (Sec. 5.1.2): flags for a t_s other than the run's equal the oracle's
    flags for a run with that t_s, bit for bit.  adjamr_advance_level starts
    every advance at level 0 (finer levels advance only inside a coarser
    step), so any other level is refused with EINVAL, and so is a t_s outside
    [t0, tf]; neither changes the hierarchy."""
    import ctypes
    wl = W.config2(seed=3, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=0.0, tol=1e-4,
                   min_patch=8, max_patch=32)
    snaps = O.adjoint_solve(wl)
    o, g = _amr_pair(A, wl, snaps=snaps)
    n = o.nsteps_total()
    o.advance(n // 3)
    g.advance(n // 3)
    for ts in (0.0, 0.7, 1.3, wl.tf):
        wt = W.config2(seed=3, n0=32, ratios=(2, 4), tf=2.0, adj_n=64, nsnap=20, ts=ts, tol=1e-4,
                       min_patch=8, max_patch=32)
        ot = O.OracleHierarchy(wt)
        ot.set_adjoint(snaps)
        ot.regrid(0, init=True)
        ot.advance(n // 3)
        for lev in range(wl.nlevels - 1):
            fo, co = ot.flag(lev, wl.tol)
            fg, cg = g.flag(lev, wl.tol, ts=ts)
            assert np.array_equal(ot.patches(lev), g.patches(lev))
            assert co == cg and np.array_equal(fo, fg), (ts, lev)
    L = A.load()
    before = [g.read_level(lev) for lev in range(wl.nlevels)]
    assert L.adjamr_advance_level(g.h, 1, 1) == A.EINVAL
    cnt = ctypes.c_longlong()
    assert L.adjamr_flag_cells(g.h, 0, wl.tol, -0.5, None, ctypes.byref(cnt)) == A.EINVAL
    assert L.adjamr_flag_cells(g.h, 0, wl.tol, wl.tf + 1.0, None, ctypes.byref(cnt)) == A.EINVAL
    for lev in range(wl.nlevels):
        assert np.array_equal(before[lev], g.read_level(lev))
    g.close()


@pytest.mark.parametrize("case", ["acoustics2d", "acoustics2d_reflux", "acoustics1d", "shallow_water2d",
                                  "acoustics2d_richardson", "shallow_water2d_richardson"])
def test_adjoint_with_amr_matches_oracle(A, case):
    """The adjoint solved with AMR (finer levels flagged by the undivided
    differences of the adjoint solution -- or, the _richardson cases, by its
    Richardson error estimate --, snapshots from level 0 after every
    Berger-Oliger step): every snapshot equal to the oracle's bit for bit, in
    1D and 2D acoustics (with and without the conservation fix-up) and the
    shallow-water adjoint over bathymetry; the fixed-grid adjoint differs."""
    flag = W.FLAG_RICHARDSON if case.endswith("_richardson") else W.FLAG_DIFFERENCE
    case = case.replace("_richardson", "")
    med = None
    if case.startswith("acoustics2d"):
        wl = W.config2(seed=3, n0=32, adj_n=32, tf=2.0, nsnap=6, bc=(W.BC_WALL,) * 4)
        ratios, tol = (2, 2), 0.02
    elif case == "acoustics1d":
        wl = W.config1(n0=100, adj_n=100, tf=6.0, nsnap=8)
        ratios, tol = (4,), 0.01
    else:
        wl = W.config3(seed=2, n0=24, ratios=(2,), adj_n=24, nsnap=6, L=2.0e6, dense_levels=1)
        ratios, tol = (2, 2), 0.02
        med = W.config3_adjoint_medium(wl, ratios=ratios)
    reflux = 1 if case.endswith("reflux") else 0
    if flag == W.FLAG_RICHARDSON:
        tol = 1e-3 if case.startswith("acoustics") else 1e-4
    ref = O.adjoint_solve_amr(wl, ratios, flag, tol, medium_dense_levels=med, reflux=reflux)
    adj = A.solve_adjoint(wl, amr=(ratios, flag, tol, reflux), medium_dense=med)
    got = adj.read()
    adj.release()
    assert np.array_equal(got, ref)
    fixed = O.adjoint_solve(wl, medium_dense=None if med is None else med[0])
    assert not np.array_equal(fixed, ref), "the AMR adjoint never refined"
