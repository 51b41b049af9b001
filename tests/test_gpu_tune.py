"""The solver tuner (mds_tune): every candidate is set up and solved, its
outcome recorded, and the converged candidate with the least set-up + solve
time chosen; invalid candidates and non-convergence are reported, not fatal.
"""
import numpy as np
import pytest

from paper_2206_03203_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_03203_gb300 import build, mdsolve
    build.build()
    return torch, mdsolve, mdsolve.Context(0)


def test_tune_picks_fastest_converged_candidate(env):
    torch, mdsolve, ctx = env
    inst = inputs.random_segments_2d(n=256, n_seg=20, contrast=1e3)
    sys_ = ctx.assemble(inst)
    cands = [("l1jacobi", 1, 2, "fp64"), ("chebyshev", 1, 3, "fp64"), ("l1jacobi", 2, 2, "fp32"),
             ("chebyshev", 9, 2, "fp64")]  # the last one is invalid (sweeps 1..8)
    best, res = ctx.tune(sys_, cands, base={"format": "csr"}, rtol=1e-8, max_iters=3000)
    assert res[3]["status"] < 0
    ok = [k for k, r in enumerate(res) if r["status"] == 0]
    assert ok == [0, 1, 2]
    t = [res[k]["setup_ms"] + res[k]["solve_ms"] for k in ok]
    assert best == ok[int(np.argmin(t))]
    # each recorded iteration count is that of a plain set-up + solve with the same options
    for k in ok:
        sm, sw, dg, pr = cands[k]
        p = ctx.setup(sys_, format="csr", smoother=sm, sweeps=sw, cheb_degree=dg, precision=pr)
        x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
        code, st = ctx.solve(sys_, p, None, x, rtol=1e-8, max_iters=3000)
        assert code == 0 and st[0].iterations == res[k]["iterations"], (k, st[0].iterations, res[k])
        p.close()


def test_tune_reports_no_convergence(env):
    torch, mdsolve, ctx = env
    sys_ = ctx.assemble(inputs.fixed_2d(n=32))
    best, res = ctx.tune(sys_, [("l1jacobi", 1, 2, "fp64")], max_iters=2)
    assert best == -1 and res[0]["status"] == 1 and res[0]["iterations"] == 2


def test_tune_coarsest_size(env):
    """The coarsest-level size N_c as a tuned option: each candidate's count is
    that of a plain set-up with that N_c, and a larger N_c (an exact solve on
    a bigger coarsest level) never needs more iterations here."""
    torch, mdsolve, ctx = env
    inst = inputs.random_rects_3d(24, 22060304, 3, 4, nrhs=1)
    sys_ = ctx.assemble(inst)
    cands = [("l1jacobi", 1, 2, "fp64", nc) for nc in (64, 256, 1024)]
    best, res = ctx.tune(sys_, cands, base={"format": "csr"}, rtol=1e-8, max_iters=3000)
    assert all(r["status"] == 0 for r in res) and best >= 0
    for k, nc in enumerate((64, 256, 1024)):
        p = ctx.setup(sys_, format="csr", n_coarse=nc)
        x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
        code, st = ctx.solve(sys_, p, None, x, rtol=1e-8, max_iters=3000)
        assert code == 0 and st[0].iterations == res[k]["iterations"]
        p.close()
    assert res[2]["iterations"] <= res[0]["iterations"]
