"""Pins of the CPU oracle's wave-propagation step against facts the paper and
the mathematics fix (no GPU).  Each test names what it pins.

The oracle is the plain FP64 restatement of the method; these tests tie it
to closed forms (impedance reflection/transmission, d'Alembert), invariants
(conservation, well-balance, symmetries) and the structure of the 2D scheme
(a y-independent 2D run is the 1D run)."""
import math
import os

import numpy as np
import pytest
from scipy.special import erf

from oracle import oracle as O
from paper_1511_03645_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _ghosted_1d(p, u, rho, K):
    q = np.stack([p, u])[:, None, :]
    med = np.stack([rho, K])[:, None, :]
    return q, med


# ---------------------------------------------------------------- Riemann
def test_interface_reflection_transmission_one_step():
    """A right-going wave (p, u) = (1, 1/Z_l) meets the interface of the
    Sec. 5.1-type medium; after one step the cells beside the interface change
    by exactly dt/dx * c * {T, R} (first-order update: the limiter is 0 at an
    isolated jump).  Golden: R = -1/3, T = 2/3 for Z_l = 2, Z_r = 1."""
    g = _golden("interface_rt.txt")
    nx, k = 8, 4            # interface between local cells k-1 and k
    sx = nx + 4
    x = np.arange(sx) - 2
    left = x < k
    rho = np.ones(sx)
    K = np.where(left, g["c_l"] ** 2, g["c_r"] ** 2)
    p0 = 1.0
    p = np.where(left, p0, 0.0)
    u = np.where(left, p0 / g["Z_l"], 0.0)
    q, med = _ghosted_1d(p, u, rho, K)
    dt, dx = 0.01, 0.1
    out, cfl = O.step_patch(1, W.EQ_ACOUSTICS, q, med, dt, dx)
    dtdx = dt / dx
    dp = out[0, 0] - p[2:-2]
    T = dp[k] / (dtdx * g["c_r"] * p0)
    R = dp[k - 1] / (dtdx * g["c_l"] * p0)
    assert abs(T - g["T"]) <= 1e-14
    assert abs(R - g["R"]) <= 1e-14
    others = [i for i in range(nx) if i not in (k - 1, k)]
    assert np.all(dp[others] == 0.0)
    assert cfl == pytest.approx(dtdx * 2.0, rel=1e-15)


@pytest.mark.parametrize("dim", [1, 2])
def test_constant_state_is_steady_bitwise(dim):
    """Constant (p, u, v) in an arbitrary medium: every jump is zero, so every
    wave and fluctuation is zero and the step returns the input bitwise."""
    rng = np.random.default_rng(1)
    nx, ny = 12, (9 if dim == 2 else 1)
    gy = 2 if dim == 2 else 0
    sx, sy = nx + 4, ny + 2 * gy
    m = 3 if dim == 2 else 2
    qc = rng.normal(size=m)
    q = np.broadcast_to(qc[:, None, None], (m, sy, sx)).copy()
    med = np.stack([rng.uniform(1, 3, (sy, sx)), rng.uniform(1, 30, (sy, sx))])
    out, _ = O.step_patch(dim, W.EQ_ACOUSTICS, q, med, 0.001, 0.05, 0.05)
    assert np.array_equal(out, q[:, gy:gy + ny, 2:2 + nx])


# ------------------------------------------------------------- d'Alembert
def _gauss_avg(a, b, beta):
    s = math.sqrt(beta)
    return math.sqrt(math.pi / beta) / (2.0 * (b - a)) * (erf(s * b) - erf(s * a))


def _scatter_write(h, level, dense):
    """Write a dense [m, M, N] array into the hierarchy's patches (patch order)."""
    parts = []
    for ilo, jlo, nx, ny in h.patches(level):
        parts.append(dense[:, jlo:jlo + ny, ilo:ilo + nx].reshape(-1))
    h.write_level(level, np.concatenate(parts))


def _homog_1d(N, tf, bc=W.BC_EXTRAP):
    wl = W.config1(n0=N, tf=tf, bc=(bc, bc))
    wl.medium = W.Medium(kind="layered", axis=0, iface=np.array([0.0]), rho=np.array([1.0, 1.0]),
                         K=np.array([1.0, 1.0]), cmax=1.0)
    return wl


def test_dalembert_convergence_1d():
    """Homogeneous medium (c = 1, Z = 1): p = [f(x-ct) + f(x+ct)]/2,
    u = [f(x-ct) - f(x+ct)]/(2Z) with exact cell averages of the Gaussian
    f = exp(-20 x^2).  L1 errors over 3 grids converge at order >= 1.5 and
    the hump splits into two halves of amplitude 1/2 (Sec. 5.1)."""
    beta, t = 20.0, 1.5
    errs = []
    for N in (200, 400, 800):
        wl = _homog_1d(N, t)
        h = O.OracleHierarchy(wl, nlevels=1, with_qinit=False)
        dx = 8.0 / N
        xl = -4.0 + np.arange(N) * dx
        f0 = np.array([_gauss_avg(a, a + dx, beta) for a in xl])
        _scatter_write(h, 0, np.stack([f0, np.zeros(N)])[:, None, :])
        h.advance(h.nsteps_total())
        q = h.level_dense(0)[:, 0, :]
        fm = np.array([_gauss_avg(a - t, a - t + dx, beta) for a in xl])
        fp = np.array([_gauss_avg(a + t, a + t + dx, beta) for a in xl])
        pe, ue = 0.5 * (fm + fp), 0.5 * (fm - fp)
        errs.append(dx * (np.abs(q[0] - pe).sum() + np.abs(q[1] - ue).sum()))
        if N == 800:
            x = xl + 0.5 * dx
            assert abs(q[0][x < 0].max() - 0.5) < 5e-3
            assert abs(q[0][x > 0].max() - 0.5) < 5e-3
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 1.5, (errs, orders)


def test_standing_wave_convergence_2d_diagonal():
    """2D homogeneous acoustics (c = 1) on a periodic box with the diagonal
    standing wave p = cos(pi (x+y)/2) cos(omega t), omega = pi/sqrt(2):
    exercises the transverse corrections (wave travelling at 45 degrees).
    Point-value errors converge at order >= 1.5."""
    t = 1.0
    errs = []
    for N in (32, 64, 128):
        wl = W.config2(n0=N, lo=-2.0, hi=2.0, bc=(W.BC_PERIODIC,) * 4)
        wl.medium = W.Medium(kind="layered", axis=1, iface=np.array([0.0]), rho=np.ones(2), K=np.ones(2),
                             cmax=1.0)
        wl.tf = t
        h = O.OracleHierarchy(wl, nlevels=1, with_qinit=False)
        dx = 4.0 / N
        xc = -2.0 + (np.arange(N) + 0.5) * dx
        X, Y = np.meshgrid(xc, xc)
        p0 = np.cos(np.pi * (X + Y) / 2.0)
        _scatter_write(h, 0, np.stack([p0, 0 * p0, 0 * p0]))
        h.advance(h.nsteps_total())
        q = h.level_dense(0)
        pe = p0 * math.cos(math.pi / math.sqrt(2.0) * t)
        errs.append(dx * dx * np.abs(q[0] - pe).sum())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 1.5, (errs, orders)


# ----------------------------------------------------------- conservation
def _dense_workload(dim, eqn, N, fields, bc=W.BC_PERIODIC, cmax=None, L=8.0, tf=1.0):
    wl = W.config2(n0=N, lo=-L / 2, hi=L / 2, bc=(bc,) * 4) if dim == 2 else W.config1(n0=N, bc=(bc, bc))
    if dim == 1:
        wl.lo, wl.hi = (-L / 2, 0.0), (L / 2, 1.0)
    wl.eqn = eqn
    if cmax is None:
        if eqn in (W.EQ_SW, W.EQ_SW_ADJ):
            cmax = float(np.sqrt(W.GRAV * fields.max()))
        else:
            cmax = float(np.sqrt(fields[1] / fields[0]).max())
    wl.medium = W.Medium(kind="dense", fields=[fields], cmax=cmax)
    wl.tf = tf
    return wl


def _smooth_field(rng, shape, k=3):
    M, N = shape
    x = np.arange(N) / N
    y = np.arange(M) / M
    X, Y = np.meshgrid(x, y)
    f = np.zeros(shape)
    for _ in range(k):
        a, b, ph = rng.integers(1, 3), rng.integers(0, 3), rng.uniform(0, 2 * np.pi)
        f += rng.normal() * np.cos(2 * np.pi * (a * X + b * Y) + ph)
    return f


@pytest.mark.parametrize("case", ["acoustics_homog", "acoustics_adj_layered", "sw_eta", "sw_adj"])
def test_conservation_periodic_2d(case):
    """Periodic grids: every fluctuation telescopes when the flux difference
    of an edge is split exactly (constant-coefficient wave form, and any
    f-wave form), so cell sums are conserved to round-off:
    homogeneous acoustics: sum p, u, v; adjoint (f-wave) acoustics in a
    variable medium: sum of all fields; shallow water over bathymetry:
    sum eta (momentum has the bathymetry source); adjoint shallow water:
    all fields."""
    rng = np.random.default_rng(7)
    N = 24
    if case == "acoustics_homog":
        eqn, fields, keep = W.EQ_ACOUSTICS, np.stack([np.full((N, N), 1.7), np.full((N, N), 4.2)]), [0, 1, 2]
    elif case == "acoustics_adj_layered":
        eqn = W.EQ_ACOUSTICS_ADJ
        fields = np.stack([rng.uniform(1, 3, (N, N)), rng.uniform(1, 20, (N, N))])
        keep = [0, 1, 2]
    elif case == "sw_eta":
        eqn, fields, keep = W.EQ_SW, rng.uniform(100, 4000, (1, N, N)), [0]
    else:
        eqn, fields, keep = W.EQ_SW_ADJ, rng.uniform(100, 4000, (1, N, N)), [0, 1, 2]
    L = 8.0 if eqn in (W.EQ_ACOUSTICS, W.EQ_ACOUSTICS_ADJ) else 8.0e5
    wl = _dense_workload(2, eqn, N, fields, L=L, tf=40 * 0.9 * (L / N) / 1.0)
    h = O.OracleHierarchy(wl, nlevels=1, with_qinit=False)
    q0 = np.stack([_smooth_field(rng, (N, N)) for _ in range(3)])
    _scatter_write(h, 0, q0)
    s0 = q0.sum(axis=(1, 2))
    h.advance(30)
    q1 = h.level_dense(0)
    s1 = q1.sum(axis=(1, 2))
    scale = np.abs(q0).sum(axis=(1, 2))
    for f in keep:
        assert abs(s1[f] - s0[f]) <= 1e-13 * scale[f], (f, s0[f], s1[f])
    assert np.abs(q1).max() > 1e-3


def test_well_balanced_lake_at_rest_bitwise():
    """Shallow water at rest (eta = mu = gamma = 0) over seamount bathymetry:
    the f-wave flux difference (d mu, g hbar_edge d eta) is exactly zero, so
    the state stays bitwise zero (Sec. 3, f-wave formulation)."""
    rng = np.random.default_rng(3)
    N = 20
    hb = W.bathymetry(*np.meshgrid(np.linspace(0, 2e6, N), np.linspace(0, 2e6, N)),
                      mounts=np.array([[2000.0, 3e5, 1e6, 1e6], [1500.0, 2e5, 5e5, 1.5e6]]))[None]
    for eqn in (W.EQ_SW, W.EQ_SW_ADJ):
        wl = _dense_workload(2, eqn, N, hb, bc=W.BC_WALL, L=2e6)
        wl.lo, wl.hi = (0.0, 0.0), (2e6, 2e6)
        h = O.OracleHierarchy(wl, nlevels=1, with_qinit=False)
        _scatter_write(h, 0, np.zeros((3, N, N)))
        h.advance(10)
        assert np.all(h.level_dense(0) == 0.0)
    del rng


# --------------------------------------------------------------- symmetry
def _run_dense(dim, eqn, fields, q0, nsteps, bc=W.BC_EXTRAP, dt0=0.0):
    if dim == 2:
        M, N = q0.shape[1:]
        assert M == N
    else:
        N = q0.shape[-1]
    wl = _dense_workload(dim, eqn, N, fields, bc=bc)
    h = O.OracleHierarchy(wl, nlevels=1, with_qinit=False, dt0=dt0)
    _scatter_write(h, 0, q0 if dim == 2 else q0[:, None, :] if q0.ndim == 2 else q0)
    h.advance(nsteps)
    return h.level_dense(0)


@pytest.mark.parametrize("eqn", [W.EQ_ACOUSTICS, W.EQ_ACOUSTICS_ADJ])
def test_mirror_symmetry_1d_bitwise(eqn):
    """x -> -x with the medium mirrored and u negated maps solutions to
    solutions; with the written operation order the map is exact in floating
    point (sums and products commute, negation is exact)."""
    rng = np.random.default_rng(11)
    N = 40
    fields = np.stack([rng.uniform(1, 3, N), rng.uniform(1, 30, N)])[:, None, :]
    q0 = np.stack([rng.normal(size=N), rng.normal(size=N)])
    a = _run_dense(1, eqn, fields, q0, 25)
    fm = fields[:, :, ::-1].copy()
    qm = np.stack([q0[0, ::-1], -q0[1, ::-1]])
    b = _run_dense(1, eqn, fm, qm, 25)
    assert np.array_equal(a[0, 0], b[0, 0, ::-1])
    assert np.array_equal(a[1, 0], -b[1, 0, ::-1])


@pytest.mark.parametrize("eqn", [W.EQ_ACOUSTICS, W.EQ_ACOUSTICS_ADJ, W.EQ_SW, W.EQ_SW_ADJ])
def test_transpose_symmetry_2d_bitwise(eqn):
    """x <-> y with u <-> v and the medium transposed: the update
    Q - (X + Y) is symmetric in X and Y, so the transposed run is the
    transpose of the run, bit for bit."""
    rng = np.random.default_rng(12)
    N = 18
    if eqn in (W.EQ_SW, W.EQ_SW_ADJ):
        fields = rng.uniform(100, 4000, (1, N, N))
    else:
        fields = np.stack([rng.uniform(1, 3, (N, N)), rng.uniform(1, 30, (N, N))])
    q0 = rng.normal(size=(3, N, N))
    a = _run_dense(2, eqn, fields, q0, 12)
    ft = fields.transpose(0, 2, 1).copy()
    qt = np.stack([q0[0].T, q0[2].T, q0[1].T]).copy()
    b = _run_dense(2, eqn, ft, qt, 12)
    assert np.array_equal(a[0], b[0].T)
    assert np.array_equal(a[1], b[2].T)
    assert np.array_equal(a[2], b[1].T)


@pytest.mark.parametrize("eqn", [W.EQ_ACOUSTICS, W.EQ_ACOUSTICS_ADJ])
def test_y_independent_2d_equals_1d_bitwise(eqn):
    """y-independent data and medium: every y-jump vanishes, the transverse
    terms cancel exactly, and each row of the 2D run is the 1D run."""
    rng = np.random.default_rng(13)
    N = 30
    rho, K = rng.uniform(1, 3, N), rng.uniform(1, 30, N)
    p0, u0 = rng.normal(size=N), rng.normal(size=N)
    f1 = np.stack([rho, K])[:, None, :]
    dt0 = 0.9 * (8.0 / N) / float(np.sqrt(K / rho).max())
    a = _run_dense(1, eqn, f1, np.stack([p0, u0]), 20, dt0=dt0)
    f2 = np.stack([np.tile(rho, (N, 1)), np.tile(K, (N, 1))])
    q2 = np.stack([np.tile(p0, (N, 1)), np.tile(u0, (N, 1)), np.zeros((N, N))])
    b = _run_dense(2, eqn, f2, q2, 20, dt0=dt0)
    for j in range(N):
        assert np.array_equal(b[0, j], a[0, 0])
        assert np.array_equal(b[1, j], a[1, 0])
    assert np.all(b[2] == 0.0)


def test_walls_conserve_pressure_sec_5_2():
    """The Sec. 5.2 setting (homogeneous K = 4, rho = 1, the pressure hump):
    with walls on all four sides no pressure crosses the boundary (the wall
    Riemann problem has zero normal velocity), so the wave-propagation
    update in this constant-coefficient wave form keeps sum p to round-off
    over the whole run; with the outflow sides of Sec. 5.2.3 the wave leaves
    and most of the pressure with it."""
    sums = {}
    for variant in ("range_walls", "range_mixed"):
        wl = W.paper_5_2(variant)
        h = O.OracleHierarchy(wl, nlevels=1)
        q0 = h.level_dense(0)
        h.advance(h.nsteps_total())
        q1 = h.level_dense(0)
        sums[variant] = (q0[0].sum(), q1[0].sum(), np.abs(q0[0]).sum(), np.abs(q1[1:]).max())
    p0, p1, scale, umax = sums["range_walls"]
    assert p0 > 1.0 and umax > 1e-3
    assert abs(p1 - p0) <= 1e-13 * scale
    p0m, p1m, _, _ = sums["range_mixed"]
    assert p0m == p0 and p1m < 0.5 * p0m
