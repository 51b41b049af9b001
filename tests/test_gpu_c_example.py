"""The plain-C example solves the four-fracture 64 x 64 instance through the
C ABI and agrees with the oracle (iterations within one, residual <= 1e-8)."""
import re
import subprocess

import pytest

from paper_2206_03203_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_c_example_solves(tmp_path, oracle_mod):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from test_c_example import compile_example
    exe = compile_example(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.stdout, r.stderr)
    m = re.search(r"n_m (\d+) n_f (\d+) nnz (\d+) status (-?\d+) iterations (\d+) relres (\S+)", r.stdout)
    assert m, r.stdout
    n_m, n_f, nnz, status, its, relres = int(m[1]), int(m[2]), int(m[3]), int(m[4]), int(m[5]), float(m[6])
    inst = inputs.fixed_2d(n=64)
    A, b = oracle_mod.assemble(inst)
    assert (n_m, n_f, nnz) == (inst.n_m, inst.n_f, A.nnz)
    res, *_ = oracle_mod.solve(inst)
    assert status == 0 and relres <= 1e-8 and abs(its - res.iterations) <= 1, (its, res.iterations)
