"""Serving loop (GPU): continuous admission by memory budget, overlapping
slots, and results that are the same alone and in the mix."""
import time

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


def _small_requests(n=6, seed=3):
    media, reqs = W.config5(seed=seed, nreq=n, rate=50.0, nmedia=2, nmin=24, nmax=40)
    wls = [W.request_workload(r, media, tf=1.5, tol=1e-4, adj_n=64, nsnap=12) for r in reqs]
    for wl in wls:
        wl.ts = 0.0
    return media, reqs, wls


@pytest.mark.parametrize("flag", ["adjoint", "error"])
def test_results_identical_alone_and_in_the_mix(A, flag):
    """Each request's J and cell-updates are the same served alone, served
    in a mix of concurrent slots, and solved directly; requests flagged by the
    adjoint-weighted error estimate (Sec. 7) too."""
    media, reqs, wls = _small_requests()
    if flag == "error":
        for wl in wls:
            wl.flag_mode, wl.tol = W.FLAG_ERROR, 1e-6
    adjs = {}
    for r, wl in zip(reqs, wls):
        if r.medium_id not in adjs:
            adjs[r.medium_id] = A.solve_adjoint(wl)
    # alone: one slot, one request at a time
    alone = []
    srv = A.Server(budget_bytes=64 << 30, max_slots=1)
    for r, wl in zip(reqs, wls):
        alone.append(srv.wait(srv.submit(wl, adjs[r.medium_id])))
    srv.close()
    # in the mix: 4 slots, all submitted together
    srv = A.Server(budget_bytes=64 << 30, max_slots=4)
    tks = [srv.submit(wl, adjs[r.medium_id]) for r, wl in zip(reqs, wls)]
    mixed = [srv.wait(t) for t in tks]
    srv.close()
    for a, b in zip(alone, mixed):
        assert a["status"] == 0 and b["status"] == 0, (a["error"], b["error"])
        assert a["J"] == b["J"]
        assert a["cell_updates"] == b["cell_updates"]
    # overlap: at some moment more than one request was running
    spans = sorted((m["t_admit"], m["t_finish"]) for m in mixed)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
    # and the same J as a direct (non-served) solve
    h = A.Hierarchy(wls[0])
    h.set_adjoint(adjs[reqs[0].medium_id])
    h.regrid(0, init=True)
    h.advance(h.nsteps_total())
    assert h.functional() == alone[0]["J"]


def test_admission_respects_the_budget(A):
    """Equal-size requests and a budget that holds one of them: they run one
    at a time, in arrival order, and the reserved bytes never exceed the
    budget."""
    media, reqs, wls = _small_requests(n=4, seed=4)
    for wl in wls:
        wl.n0 = (32, 32)
        wl.ratios = (2,)
    adj = A.solve_adjoint(wls[0])
    need = A.estimate_bytes(wls[0])
    assert all(A.estimate_bytes(wl) == need for wl in wls)
    srv = A.Server(budget_bytes=need + 1, max_slots=4)   # room for one request at a time
    tks = [srv.submit(wl, adj) for wl in wls]
    peak_active = 0
    t0 = time.time()
    while time.time() - t0 < 120:
        used, active, queued = srv.info()
        assert used <= need + 1
        peak_active = max(peak_active, active)
        if all(srv.poll(t)["done"] for t in tks):
            break
        time.sleep(0.002)
    res = [srv.wait(t) for t in tks]
    srv.close()
    assert all(r["status"] == 0 for r in res)
    assert peak_active <= 1
    # admissions in arrival order, never overlapping
    spans = [(r["t_admit"], r["t_finish"]) for r in res]
    for k in range(len(spans) - 1):
        assert spans[k + 1][0] >= spans[k][1] - 1e-9


def test_request_larger_than_budget_is_refused(A):
    media, reqs, wls = _small_requests(n=1)
    adj = A.solve_adjoint(wls[0])
    srv = A.Server(budget_bytes=1024, max_slots=1)
    with pytest.raises(A.AdjamrError) as ei:
        srv.submit(wls[0], adj)
    assert ei.value.code == A.EBUDGET
    srv.close()
