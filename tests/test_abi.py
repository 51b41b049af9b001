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
    assert o.theta == 0.08 and o.n_coarse == 512 and o.max_levels == 25
    s = mdsolve.solve_opts()
    assert s.restart == 30 and s.rtol == 1e-8


def test_sm103a_target_in_build_flags():
    from paper_2206_03203_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2206_03203_gb300 import mdsolve
    monkeypatch.setattr(mdsolve, "_lib", None)
    monkeypatch.setattr(mdsolve, "LIB_PATH", "/nonexistent/libmdsolve.so")
    with pytest.raises(ImportError):
        mdsolve.lib()
