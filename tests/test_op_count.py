"""The FP64 operation counts per cell-update that bench.py divides by (its
roofline's "algorithmic" work), produced by running the canonical operation
sequence of one edge and one cell update on a counting number type rather
than by hand.  One operation per IEEE operation: + - * / fma min max count
one each; negation and absolute value are free (sign-bit operations); the
comparisons that pick the upwind wave are decisions, not arithmetic."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class Op:
    n = 0

    def __init__(self, v=0.0):
        self.v = float(v)

    @staticmethod
    def _c(x):
        return x if isinstance(x, Op) else Op(x)

    def __add__(self, o):
        Op.n += 1
        return Op()

    __radd__ = __add__

    def __sub__(self, o):
        Op.n += 1
        return Op()

    __rsub__ = __sub__

    def __mul__(self, o):
        Op.n += 1
        return Op()

    __rmul__ = __mul__

    def __truediv__(self, o):
        Op.n += 1
        return Op()

    def __neg__(self):
        return Op()


def fma(a, b, c):
    Op.n += 1
    return Op()


def fmin(a, b):
    Op.n += 1
    return Op()


def fmax(a, b):
    Op.n += 1
    return Op()


def fabs(a):
    return Op()


def decompose(eqn, d0, dn, Zl, Zr, izs, ce, ice):
    if eqn == "ac":
        a1 = fma(Zr, dn, -d0) * izs
        a2 = fma(Zl, dn, d0) * izs
        return (-(Zl * a1), a1), (Zr * a2, a2)
    b1 = fma(-dn, ice, d0) * 0.5
    b2 = fma(dn, ice, d0) * 0.5
    return (b1, -(ce * b1)), (b2, ce * b2)


def mc_phi(w, wu):
    wn = fma(w[0], w[0], w[1] * w[1])
    dot = fma(wu[0], w[0], wu[1] * w[1])
    th = dot / wn
    return fmax(0.0, fmin(fmin(fma(0.5, th, 0.5), 2.0), 2.0 * th))


def edge(eqn, dim):
    """Operations of one edge: jump, decomposition, fluctuations, the two
    limited waves, correction coefficients, second-order flux, CFL and (2D)
    the two transverse splits of the fluctuations entering beside it."""
    x = [Op() for _ in range(8)]
    Zl, Zr, izs, ce, ice, ghe, s1, s2, dtd, hy = (Op() for _ in range(10))
    if eqn == "ac":
        d0, dn = x[0] - x[1], x[2] - x[3]
    else:
        d0, dn = x[2] - x[3], ghe * (x[0] - x[1])
    w1, w2 = decompose(eqn, d0, dn, Zl, Zr, izs, ce, ice)
    if eqn == "ac":
        am = (s1 * w1[0], s1 * w1[1])
        ap = (s2 * w2[0], s2 * w2[1])
    else:
        am, ap = w1, w2
    p1, p2 = mc_phi(w1, w1), mc_phi(w2, w2)
    a1, a2 = fabs(s1), fabs(s2)
    if eqn == "ac":
        cf1, cf2 = a1 * fma(-dtd, a1, 1.0), a2 * fma(-dtd, a2, 1.0)
    else:
        cf1, cf2 = fma(-dtd, a1, 1.0), fma(-dtd, a2, 1.0)
    Fn = [0.5 * (cf1 * (p1 * w1[k]) + cf2 * (p2 * w2[k])) for k in range(2)]
    fmax(Op(), dtd * fmax(fabs(s1), fabs(s2)))  # CFL: running max of dt/dx max |s|
    if dim == 2:
        for delta in (Op(), Op()):           # the entering fluctuations right and left of the edge
            u1, _ = decompose(eqn, delta, 0.0, Zl, Zr, izs, ce, ice)
            (s1 * u1[0], s1 * u1[1])         # one family's part: s_p * w_p(delta)
        for k in range(2):                   # F_k = fma(-h, A-(right) + A+(left), Fn_k)
            fma(-hy, Op() + Op(), Fn[k])
    del am, ap


def cell(dim):
    """Operations of one cell beyond its edges: the entering sums
    (component 0, the one the transverse splits take) and the update."""
    if dim == 2:
        for _ in range(2):                   # Sx_0, Sy_0: (ap - F) + (am + F)
            (Op() - Op()) + (Op() + Op())
        A = [(Op() + Op()) + (Op() - Op()) for _ in range(4)]
        Op() - (Op() * A[0] + Op() * A[2])
        fma(Op(), A[1], Op())
        fma(Op(), A[3], Op())
    else:
        A = [(Op() + Op()) + (Op() - Op()) for _ in range(2)]
        Op() - Op() * A[0]
        fma(Op(), A[1], Op())


def per_cell(eqn, dim):
    Op.n = 0
    for _ in range(dim):
        edge(eqn, dim)
    cell(dim)
    return Op.n


def test_op_counts_match_the_bench_constants():
    sys.path.insert(0, ROOT)
    import bench
    assert per_cell("ac", 2) == bench.OPS_PER_CELL["acoustics2d"]
    assert per_cell("sw", 2) == bench.OPS_PER_CELL["shallow_water2d"]
    assert per_cell("ac", 1) == bench.OPS_PER_CELL["acoustics1d"]
