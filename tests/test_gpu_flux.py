"""GPU parity in the paper's own partition (Sec. 3.1, Eq. (4)): unknowns
[pressures of all cells; interface fluxes], assembled by mds_assemble_flux.

Bit-exact against the oracle: the assembled matrix and right-hand sides,
the four blocks, S~ (Eq. (7), exact here because A_GG is diagonal) and every
level of both hierarchies; the flux block's hierarchy is one level solved by
x = b / a_ii on both sides.  Tolerance: one application of M_L, B_D and B_U
(1e-12 relative in FP64, 2e-5 in FP32), and the solves (iteration count
within one of the oracle's for FGMRES, MINRES as in the primal tests, true
relative residual <= rtol).
"""
import numpy as np
from conftest import maxrel
import pytest

from paper_2206_03203_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = {
    "fixed2d-37": lambda: inputs.fixed_2d(n=37),
    "seg2d-96": lambda: inputs.random_segments_2d(n=96, n_seg=12),
    "planes3d-13-kf1": lambda: inputs.planes_3d(n=13, kf=1.0),
    "rects3d-18": lambda: inputs.random_rects_3d(18, 22060305, 0, 6, sigma=2.0),
}


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_mod):
    from paper_2206_03203_gb300 import build, mdsolve
    build.build()
    return mdsolve.Context(0)


def dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def same_csr(A, B):
    return (A.shape == B.shape and np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
            and np.array_equal(A.data, B.data))


@pytest.mark.parametrize("case", list(CASES))
def test_flux_assembly_bit_exact(ctx, oracle_mod, case):
    inst = CASES[case]()
    sys_ = ctx.assemble(inst, form="flux")
    N = inst.n_m + inst.n_f
    assert sys_.n_m == N and sys_.n_f == 2 * inst.n_f
    (Aoo, Aog, Ago, Agg, A), b = sys_.to_host()
    Ao, bo = oracle_mod.assemble(inst, form="flux")
    assert same_csr(A, Ao)
    assert np.array_equal(b, bo)
    for G, O in zip((Aoo, Aog, Ago, Agg), oracle_mod.split(Ao, N)):
        assert same_csr(G, O)


@pytest.mark.parametrize("case", list(CASES))
def test_flux_hierarchies_bit_exact(ctx, oracle_mod, case):
    inst = CASES[case]()
    N = inst.n_m + inst.n_f
    sys_ = ctx.assemble(inst, form="flux")
    prec = ctx.setup(sys_)
    Ao, _ = oracle_mod.assemble(inst, form="flux")
    M = oracle_mod.ML(Ao, N)
    S_gpu, _, _ = prec.level_host(0, 0)
    assert same_csr(S_gpu, M.schur)
    for block in (0, 1):
        amg = M.amg(block)
        info = prec.info(block)
        assert info["nlevels"] == amg.nlevels
        assert info["dense"] == amg.coarsest_dense and info["diagonal"] == amg.coarsest_diagonal
        for l in range(amg.nlevels):
            Ag, agg, roots = prec.level_host(block, l)
            assert same_csr(Ag, amg.level_A(l)), (block, l)
            ao = amg.agg(l)
            assert (agg is None and ao is None) or np.array_equal(agg, ao), (block, l)
    # the flux block: one level without couplings, whatever its size
    info = prec.info(1)
    assert info["nlevels"] == 1 and info["diagonal"] and not info["dense"]


@pytest.mark.parametrize("prec_name,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_flux_block_solve_is_exact(ctx, oracle_mod, torch_mod, prec_name, tol):
    """One V-cycle on the flux block is x = b / a_ii (to the vector
    precision's rounding)."""
    torch = torch_mod
    inst = CASES["seg2d-96"]()
    N = inst.n_m + inst.n_f
    sys_ = ctx.assemble(inst, form="flux")
    prec = ctx.setup(sys_, precision=prec_name)
    Ao, _ = oracle_mod.assemble(inst, form="flux")
    d = Ao.tocsr()[N:, N:].diagonal()
    b = np.random.default_rng(11).standard_normal(2 * inst.n_f)
    x = torch.zeros(2 * inst.n_f, dtype=torch.float64, device="cuda")
    ctx.vcycle(prec, 1, dev(torch, b), x)
    xo = oracle_mod.ML(Ao, N, prec=64 if prec_name == "fp64" else 32).amg(1).vcycle(b)
    xg = x.cpu().numpy()
    assert maxrel(xg, xo) <= tol
    assert maxrel(xg, b / d) <= tol
    if prec_name == "fp64":
        assert np.array_equal(xg, xo)


@pytest.mark.parametrize("kind", ["lower", "diag", "upper"])
@pytest.mark.parametrize("prec_name,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_flux_precond_apply_parity(ctx, oracle_mod, torch_mod, kind, prec_name, tol):
    torch = torch_mod
    inst = CASES["rects3d-18"]()
    N = inst.n_m + inst.n_f
    sys_ = ctx.assemble(inst, form="flux")
    prec = ctx.setup(sys_, precision=prec_name, kind=kind)
    Ao, _ = oracle_mod.assemble(inst, form="flux")
    M = oracle_mod.ML(Ao, N, kind=kind, prec=64 if prec_name == "fp64" else 32)
    r = np.random.default_rng(12).standard_normal(sys_.N)
    z = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    ctx.precond_apply(prec, dev(torch, r), z)
    zo = M.apply(r)
    zg = z.cpu().numpy()
    assert maxrel(zg, zo) <= tol
    if kind == "diag":  # -Q_ff on the negative definite flux block: B_D is positive
        assert r @ zg > 0.0 and np.all(zg[N:] * r[N:] > 0.0)


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_flux_fgmres_parity(ctx, oracle_mod, torch_mod, case, prec_name):
    """M_L + FGMRES(30) on the saddle-point system: iterations within one of
    the oracle's; the pressures solve the primal system to the same bound."""
    torch = torch_mod
    inst = CASES[case]()
    N = inst.n_m + inst.n_f
    sys_ = ctx.assemble(inst, form="flux")
    prec = ctx.setup(sys_, precision=prec_name)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, rtol=1e-8, max_iters=3000)
    Ao, bo = oracle_mod.assemble(inst, form="flux")
    M = oracle_mod.ML(Ao, N, prec=64 if prec_name == "fp64" else 32)
    res = oracle_mod.fgmres(Ao, bo[0], M, rtol=1e-8, maxit=3000)
    assert code == 0 and res.converged
    assert abs(st[0].iterations - res.iterations) <= 1, (st[0].iterations, res.iterations)
    xg = x.cpu().numpy()
    rel = np.linalg.norm(bo[0] - Ao @ xg) / np.linalg.norm(bo[0])
    assert rel <= 1e-8 * 1.01 and abs(rel - st[0].relres_true) <= 1e-3 * rel + 1e-15
    assert np.linalg.norm(Ao @ (xg - res.x)) / np.linalg.norm(bo[0]) <= 2.1e-8


@pytest.mark.parametrize("case", ["fixed2d-37", "seg2d-96", "planes3d-13-kf1"])
def test_flux_minres_block_diagonal(ctx, oracle_mod, torch_mod, case):
    """MINRES with B_D (flux block -Q_ff) on the symmetric indefinite system."""
    torch = torch_mod
    inst = CASES[case]()
    N = inst.n_m + inst.n_f
    sys_ = ctx.assemble(inst, form="flux")
    prec = ctx.setup(sys_, kind="diag")
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, krylov="minres", max_iters=5000)
    Ao, bo = oracle_mod.assemble(inst, form="flux")
    res = oracle_mod.minres(Ao, bo[0], oracle_mod.ML(Ao, N, kind="diag"), rtol=1e-8, maxit=5000)
    assert code == 0 and res.converged
    tol = max(1, res.iterations // 100)
    assert abs(st[0].iterations - res.iterations) <= tol, (st[0].iterations, res.iterations)
    assert st[0].relres_true <= 1e-8
    err = np.linalg.norm(x.cpu().numpy() - res.x) / np.linalg.norm(res.x)
    assert err <= 1e-6, err


def test_flux_no_fractures_is_primal(ctx, oracle_mod):
    inst = inputs.make_instance("plain", 2, 12, np.linspace(1, 3, 144), [])
    a = ctx.assemble(inst)
    f = ctx.assemble(inst, form="flux")
    (_, _, _, _, A), b = a.to_host()
    (_, _, _, _, Af), bf = f.to_host()
    assert same_csr(A, Af) and np.array_equal(b, bf) and f.n_f == 0


def test_flux_full_size_random_segments(ctx, oracle_mod, torch_mod):
    """1024 x 1024, 64 segments, contrast 1e4 in the flux form: assembly and
    both hierarchies bit-exact; M_L + FGMRES meets the stopping rule on an
    independent residual; one application of M_L against the oracle."""
    torch = torch_mod
    inst = inputs.random_segments_2d()
    N = inst.n_m + inst.n_f
    sys_ = ctx.assemble(inst, form="flux")
    (_, _, _, _, A), b = sys_.to_host()
    Ao, bo = oracle_mod.assemble(inst, form="flux")
    assert same_csr(A, Ao) and np.array_equal(b, bo)
    prec = ctx.setup(sys_)
    M = oracle_mod.ML(Ao, N)
    for block in (0, 1):
        amg = M.amg(block)
        assert prec.info(block)["nlevels"] == amg.nlevels
        for l in range(amg.nlevels):
            Ag, agg, _ = prec.level_host(block, l)
            assert same_csr(Ag, amg.level_A(l))
            ao = amg.agg(l)
            assert (agg is None and ao is None) or np.array_equal(agg, ao)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, max_iters=5000)
    xg = x.cpu().numpy()
    rel = np.linalg.norm(bo[0] - Ao @ xg) / np.linalg.norm(bo[0])
    assert code == 0 and rel <= 1.01e-8
    r = np.random.default_rng(5).standard_normal(sys_.N)
    z = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    ctx.precond_apply(prec, dev(torch, r), z)
    zo = M.apply(r)
    assert maxrel(z.cpu().numpy(), zo) <= 1e-12


@pytest.mark.parametrize("form", ["primal", "flux"])
@pytest.mark.parametrize("case", ["seg2d-96", "rects3d-18"])
def test_normal_permeability_bit_exact(ctx, oracle_mod, torch_mod, case, form):
    """A normal permeability k_n independent of k_f (kappa = 2 k_n / a): the
    GPU assembly equals the oracle's, and M_L + FGMRES matches its iteration
    count."""
    import dataclasses
    torch = torch_mod
    inst = CASES[case]()
    kn = np.exp(np.random.default_rng(21).uniform(np.log(1e-4), np.log(1e4), inst.n_f))
    inst = dataclasses.replace(inst, fc_kn=kn)
    sys_ = ctx.assemble(inst, form=form)
    (_, _, _, _, A), b = sys_.to_host()
    Ao, bo, no = oracle_mod.assemble(inst, form=form, with_split=True)
    assert same_csr(A, Ao) and np.array_equal(b, bo)
    prec = ctx.setup(sys_)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, rtol=1e-8, max_iters=3000)
    res = oracle_mod.fgmres(Ao, bo[0], oracle_mod.ML(Ao, no), rtol=1e-8, maxit=3000)
    assert code == 0 and res.converged and abs(st[0].iterations - res.iterations) <= 1
