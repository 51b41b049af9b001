"""The C ABI is usable from plain C: `paper_2206_03203_gb300/examples/solve_c.c`
compiles against `include/mdsolve.h` and links against the library.  Without
a GPU the program stops cleanly at context creation (exit status 2); the
solve itself is checked in `tests/test_gpu_c_example.py`."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2206_03203_gb300", "examples", "solve_c.c")


def compile_example(tmp_path):
    from paper_2206_03203_gb300 import build
    lib = build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "solve_c")
    libdir = os.path.dirname(lib)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), SRC,
                        "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_example_builds_and_fails_cleanly_without_gpu(tmp_path):
    exe = compile_example(tmp_path)
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the solve runs in the GPU test")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "mds_create failed" in r.stderr
