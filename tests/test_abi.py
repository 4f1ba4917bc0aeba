"""The C-ABI library builds, loads and exports every entry point that
include/adjamr.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "adjamr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:adjamr_status|void|const char \*|size_t|double)\s*(adjamr_\w+)\s*\(", src,
                                 flags=re.M)))


def test_header_declares_the_boundary_calls():
    d = _declared()
    for name in ["adjamr_init_grid_hierarchy", "adjamr_set_medium", "adjamr_load_adjoint_snapshots",
                 "adjamr_advance_level", "adjamr_flag_cells", "adjamr_regrid", "adjamr_integrate_functional"]:
        assert name in d


def test_library_builds_loads_and_exports_every_symbol():
    from paper_1511_03645_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1511_03645_gb300 import adjamr as A
    assert set(A.SYMBOLS) == set(_declared())
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for n in _declared():
        assert re.search(rf"\bT {n}\b", out), n


def test_kernels_are_built_for_sm_103a():
    from paper_1511_03645_gb300 import build as B
    assert "compute_103a,code=sm_103a" in B.ARCH
    path = B.build()
    assert os.path.getsize(path) > 100_000


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1511_03645_gb300 import adjamr as A
    monkeypatch.setattr(A, "_lib", None)
    monkeypatch.setattr(A, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        A.load(build_if_missing=False)


def test_parameters_are_validated_before_any_device_call():
    """Invalid parameters (here refinement ratios outside 2..16) are refused
    with EINVAL before any CUDA call; the serving byte estimate grows with
    the ratio."""
    from paper_1511_03645_gb300 import adjamr as A, workloads as W
    L = A.load()
    wl = W.config2(seed=1, n0=16, ratios=(2, 4), tf=0.5, adj_n=32, nsnap=4)
    out = ctypes.c_void_p()
    est = {}
    for r, want in ((1, A.EINVAL), (17, A.EINVAL)):
        p = A.make_params(wl)
        p.ratio[1] = r
        assert L.adjamr_init_grid_hierarchy(ctypes.byref(p), ctypes.byref(out)) == want
        assert not out.value
    for r in (2, 4, 16):
        p = A.make_params(wl)
        p.ratio[1] = r
        est[r] = L.adjamr_estimate_bytes(ctypes.byref(p))
    assert 0 < est[2] < est[4] < est[16]
    # the serving admission estimate refuses the same ratios (0 bytes; the
    # server then refuses the request with EINVAL), and the fix-up flag must be 0 or 1
    for r in (0, 1, 17):
        p = A.make_params(wl)
        p.ratio[1] = r
        assert L.adjamr_estimate_bytes(ctypes.byref(p)) == 0
    p = A.make_params(wl)
    p.reflux = 2
    assert L.adjamr_init_grid_hierarchy(ctypes.byref(p), ctypes.byref(out)) == A.EINVAL
    assert not out.value
    p.reflux = 1
    assert L.adjamr_estimate_bytes(ctypes.byref(p)) > est[4]
    # flag modes 0..5 (4, 5: flagging by the Richardson error estimate,
    # adjoint-weighted or not, whose scratch the estimate counts); anything
    # else is refused
    p = A.make_params(wl)
    p.flag_mode = 6
    assert L.adjamr_init_grid_hierarchy(ctypes.byref(p), ctypes.byref(out)) == A.EINVAL
    assert not out.value
    p.flag_mode = W.FLAG_ERROR
    assert L.adjamr_estimate_bytes(ctypes.byref(p)) > est[4]


def test_every_entry_point_cites_its_passage_or_says_it_has_none():
    """Each function declared in include/adjamr.h is preceded by a comment
    that cites the passage of the paper it implements (a section or an
    equation) or states that it has no counterpart in the paper."""
    import re
    lines = open(os.path.join(ROOT, "include", "adjamr.h")).read().splitlines()
    missing = []
    for i, line in enumerate(lines):
        m = re.match(r"^(?:adjamr_status|void|size_t|double|int|const char \*)\s*(adjamr_\w+)\(", line)
        if not m:
            continue
        j, com = i - 1, []
        while j >= 0 and (lines[j].strip().startswith(("*", "/*", "#define")) or lines[j].strip().endswith("*/")):
            com.insert(0, lines[j])
            j -= 1
        text = re.sub(r"\s+", " ", re.sub(r"(/\*|\*/|^\s*\*)", " ", "\n".join(com), flags=re.M))
        if not re.search(r"Secs?\.|Eq\.|[Nn]o counterpart", text):
            missing.append(m.group(1))
    assert not missing, missing
