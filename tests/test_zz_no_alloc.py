"""The allocation-free weighted sum (adjamr_weighted_sum_noalloc) gives the
same J as adjamr_integrate_functional.

It exists for callers that cannot allocate device memory where they need
the sum -- e.g. inside a stream capture or under a fixed memory plan owned
by another framework -- so here the test allocates the input and output
buffers itself (with PyTorch) and hands them over; the entry point works in
its own static scratch.  Two calls in a row, with different term counts,
check that the scratch left behind by one call does not leak into the next.
This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1511_03645_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_03645_gb300 import adjamr
    adjamr.load()
    return adjamr


def _terms(h, wl, t):
    """Values q0 and overlap areas of the cells that make up J, in the order
    the functional sums them: level, patch, row, column; a cell counts only
    where no finer patch covers it."""
    qs, ws = [], []
    for lev in range(wl.nlevels):
        P = h.patches(lev)
        if len(P) == 0:
            break
        dx, dy = wl.level_dx(lev)
        flat = h.read_level(lev)
        fine = h.patches(lev + 1) if lev + 1 < wl.nlevels else np.zeros((0, 4), np.int32)
        r = wl.ratios[lev] if lev + 1 < wl.nlevels else 1
        o = 0
        for ilo, jlo, nx, ny in P:
            q0 = flat[o:o + nx * ny].reshape(ny, nx)
            o += wl.m * nx * ny
            for j in range(ny):
                for i in range(nx):
                    I, J = ilo + i, jlo + j
                    xl, xr = wl.lo[0] + I * dx, wl.lo[0] + (I + 1) * dx
                    ox = min(xr, t.x1) - max(xl, t.x0)
                    if not ox > 0.0:
                        continue
                    yl, yr = wl.lo[1] + J * dy, wl.lo[1] + (J + 1) * dy
                    oy = min(yr, t.y1) - max(yl, t.y0)
                    if not oy > 0.0:
                        continue
                    if any(fi <= I * r < fi + fnx and fj <= J * r < fj + fny for fi, fj, fnx, fny in fine):
                        continue
                    qs.append(q0[j, i])
                    ws.append(ox * oy)
    return np.array(qs), np.array(ws)


def test_noalloc_sum_matches_the_functional_on_two_calls(A):
    import torch
    wl = W.config2(seed=2, n0=24, ratios=(2,), tf=1.0, adj_n=48, nsnap=8, ts=0.0, tol=1e-4)
    h = A.Hierarchy(wl)
    adj = A.solve_adjoint(wl)
    h.set_adjoint(adj)
    h.regrid(0, init=True)
    h.advance(6)
    targets = [W.Target(-0.33, 1.71, -1.1, 0.47, weight=2.0), W.Target(-3.0, -0.5, 0.2, 3.3, weight=0.5)]
    s = torch.cuda.Stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    counts = []
    for t in targets:
        J_ref = h.functional(t)
        qv, wv = _terms(h, wl, t)
        counts.append(qv.size)
        q = torch.tensor(qv, dtype=torch.float64, device="cuda")
        w = torch.tensor(wv, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        A.weighted_sum_noalloc(q.data_ptr(), w.data_ptr(), qv.size, t.weight, out.data_ptr(), s.cuda_stream)
        s.synchronize()
        J = float(out.item())
        assert abs(J - J_ref) <= 1e-12 * max(abs(J_ref), 1e-300), (J, J_ref)
    assert counts[0] != counts[1] and min(counts) > 0


def test_noalloc_sum_rejects_oversized_input_without_launching(A):
    import torch
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(A.AdjamrError) as ei:
        # sizes are checked before any pointer is touched
        A.weighted_sum_noalloc(0, 0, A.NOALLOC_MAX_TERMS + 1, 1.0, out.data_ptr())
    assert ei.value.code == A.EBUDGET
    # an empty sum is zero
    A.weighted_sum_noalloc(0, 0, 0, 1.0, out.data_ptr())
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
