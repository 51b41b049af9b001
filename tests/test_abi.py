"""The C ABI library builds for sm_103a, loads and exports every declared entry
point; the Python binding covers each one.  No GPU calls."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(mds_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_2206_03203_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    names = declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(built)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2206_03203_gb300 import mdsolve
    assert declared_functions() == set(mdsolve._SIGS)


def test_binding_loads_without_gpu(built):
    from paper_2206_03203_gb300 import mdsolve
    L = mdsolve.lib()
    assert L.mds_error_string(0) == b"ok"
    assert L.mds_error_string(-7) == b"row capacity exceeded"
    # no device: creating a context fails with a status, never a crash
    import torch
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        assert L.mds_create(ctypes.byref(h), 0, None, None) < 0


def test_default_options(built):
    from paper_2206_03203_gb300 import mdsolve
    o = mdsolve.setup_opts()
    assert o.theta < 0 and o.n_coarse == 512 and o.max_levels == 25  # theta resolved by mds_setup
    assert o.level_form == 0 and o.cheb_degree == 2 and mdsolve.setup_opts(level_form="stored").level_form == 2
    s = mdsolve.solve_opts()
    assert s.restart == 30 and s.rtol == 1e-8 and s.x0_zero == 0


def test_sm103a_target_in_build_flags():
    from paper_2206_03203_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2206_03203_gb300 import mdsolve
    monkeypatch.setattr(mdsolve, "_lib", None)
    monkeypatch.setattr(mdsolve, "LIB_PATH", "/nonexistent/libmdsolve.so")
    with pytest.raises(ImportError):
        mdsolve.lib()


def test_null_handles_are_rejected_without_touching_a_device(built):
    """Every entry point that takes a handle returns MDS_ERR_INVALID (-1) for
    a NULL one, before any CUDA call (so this runs without a GPU)."""
    from paper_2206_03203_gb300 import mdsolve
    L = mdsolve.lib()
    N = None
    st = mdsolve.RhsStats()
    cand = mdsolve.TuneCandidate()
    best = ctypes.c_int()
    out = ctypes.c_void_p()
    calls = [
        lambda: L.mds_destroy(N),
        lambda: L.mds_set_stream(N, N),
        lambda: L.mds_assemble(N, N, ctypes.byref(out)),
        lambda: L.mds_assemble_flux(N, N, ctypes.byref(out)),
        lambda: L.mds_assemble_batch(N, N, 1, ctypes.byref(out)),
        lambda: L.mds_system_destroy(N),
        lambda: L.mds_setup(N, N, N, ctypes.byref(out)),
        lambda: L.mds_precond_destroy(N),
        lambda: L.mds_precond_apply(N, N, N, N),
        lambda: L.mds_vcycle(N, N, 0, N, N),
        lambda: L.mds_spmv(N, N, N, N),
        lambda: L.mds_solve(N, N, N, N, N, 1, N, ctypes.byref(st)),
        lambda: L.mds_solve_async(N, N, N, N, N, 1, N),
        lambda: L.mds_solve_done(N),
        lambda: L.mds_solve_wait(N, ctypes.byref(st), 1),
        lambda: L.mds_tune(N, N, N, N, N, ctypes.byref(cand), 1, ctypes.byref(best)),
        lambda: L.mds_timing_reset(N),
    ]
    for k, f in enumerate(calls):
        assert f() == -1, k
    for code in range(-9, 2):
        assert L.mds_error_string(code)


def test_refinement_growth_flag():
    """bench.py --table1 flags iteration counts that more than double from
    the coarsest to the finest grid of a dimension."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    cols = ["2d n=64", "2d n=128", "2d n=256", "3d n=16", "3d n=32", "3d n=64"]
    g = bench.refinement_growth(cols, [10, 14, 21, 14, 20, 28])
    assert g["2d"] == {"ratio": 2.1, "over_2x": True} and g["3d"] == {"ratio": 2.0, "over_2x": False}
    g = bench.refinement_growth(cols, [10, "set-up: failed", None, 14, 20, 28])
    assert g["2d"]["ratio"] is None and not g["2d"]["over_2x"]
