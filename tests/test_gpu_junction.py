"""GPU parity of the junction rules (Sec. 2.1 intersections): star-delta in
the primal form and intersection cells with their own interface fluxes in
the flux form, through the C ABI against the oracle.

Bit-exact: assembled matrices and right-hand sides, block splits, S~ and
every AMG level.  Tolerance: iteration counts within one of the oracle's for
FGMRES (MINRES: one or 1% of the count), true relative residual <= rtol.
"""
import numpy as np
import pytest

from paper_2206_03203_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = {
    "fixed2d-37": lambda: inputs.fixed_2d(n=37),
    "seg2d-96": lambda: inputs.random_segments_2d(n=96, n_seg=12),
    "planes3d-13-kf1": lambda: inputs.planes_3d(n=13, kf=1.0),
    "planes3d-16": lambda: inputs.planes_3d(n=16),
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


def same_csr(A, B):
    return (A.shape == B.shape and np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
            and np.array_equal(A.data, B.data))


@pytest.mark.parametrize("case", list(CASES))
def test_star_delta_assembly_bit_exact(ctx, oracle_mod, case):
    inst = CASES[case]()
    sys_ = ctx.assemble(inst, junction="star")
    (_, _, _, _, A), b = sys_.to_host()
    Ao, bo = oracle_mod.assemble(inst, junction=1)
    assert same_csr(A, Ao) and np.array_equal(b, bo)


@pytest.mark.parametrize("case", list(CASES))
def test_intersection_form_bit_exact(ctx, oracle_mod, case):
    """Assembly, blocks, S~ and both hierarchies of the flux form with
    intersection cells."""
    inst = CASES[case]()
    sys_ = ctx.assemble(inst, form="flux", junction="star")
    Ao, bo, no = oracle_mod.assemble(inst, form="flux", junction=1, with_split=True)
    assert sys_.n_m == no and sys_.N == Ao.shape[0]
    (B0, B1, B2, B3, A), b = sys_.to_host()
    assert same_csr(A, Ao) and np.array_equal(b, bo)
    for G, O in zip((B0, B1, B2, B3), oracle_mod.split(Ao, no)):
        assert same_csr(G, O)
    prec = ctx.setup(sys_)
    M = oracle_mod.ML(Ao, no)
    S_gpu, _, _ = prec.level_host(0, 0)
    assert same_csr(S_gpu, M.schur)
    for block in (0, 1):
        amg = M.amg(block)
        info = prec.info(block)
        assert info["nlevels"] == amg.nlevels and info["diagonal"] == amg.coarsest_diagonal
        for l in range(amg.nlevels):
            Ag, agg, roots = prec.level_host(block, l)
            assert same_csr(Ag, amg.level_A(l)), (block, l)
            ao = amg.agg(l)
            assert (agg is None and ao is None) or np.array_equal(agg, ao), (block, l)


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["fixed2d-37", "planes3d-16", "rects3d-18"])
def test_intersection_form_fgmres_parity(ctx, oracle_mod, torch_mod, case, prec_name):
    torch = torch_mod
    inst = CASES[case]()
    sys_ = ctx.assemble(inst, form="flux", junction="star")
    prec = ctx.setup(sys_, precision=prec_name)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, rtol=1e-8, max_iters=3000)
    Ao, bo, no = oracle_mod.assemble(inst, form="flux", junction=1, with_split=True)
    res = oracle_mod.fgmres(Ao, bo[0], oracle_mod.ML(Ao, no, prec=64 if prec_name == "fp64" else 32), rtol=1e-8,
                            maxit=3000)
    assert code == 0 and res.converged
    assert abs(st[0].iterations - res.iterations) <= 1, (st[0].iterations, res.iterations)
    xg = x.cpu().numpy()
    rel = np.linalg.norm(bo[0] - Ao @ xg) / np.linalg.norm(bo[0])
    assert rel <= 1.01e-8
    assert np.linalg.norm(Ao @ (xg - res.x)) / np.linalg.norm(bo[0]) <= 2.1e-8


@pytest.mark.parametrize("case", ["fixed2d-37", "planes3d-13-kf1"])
def test_intersection_form_minres(ctx, oracle_mod, torch_mod, case):
    torch = torch_mod
    inst = CASES[case]()
    sys_ = ctx.assemble(inst, form="flux", junction="star")
    prec = ctx.setup(sys_, kind="diag")
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, krylov="minres", max_iters=5000)
    Ao, bo, no = oracle_mod.assemble(inst, form="flux", junction=1, with_split=True)
    res = oracle_mod.minres(Ao, bo[0], oracle_mod.ML(Ao, no, kind="diag"), rtol=1e-8, maxit=5000)
    assert code == 0 and res.converged
    assert abs(st[0].iterations - res.iterations) <= max(1, res.iterations // 100)
    assert st[0].relres_true <= 1e-8


def test_star_delta_primal_solve_parity(ctx, oracle_mod, torch_mod):
    """M_L + FGMRES on the star-delta primal system (the partition of the
    workloads, only the junction rule changed)."""
    torch = torch_mod
    inst = CASES["planes3d-16"]()
    sys_ = ctx.assemble(inst, junction="star")
    prec = ctx.setup(sys_)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, rtol=1e-8, max_iters=3000)
    Ao, bo = oracle_mod.assemble(inst, junction=1)
    res = oracle_mod.fgmres(Ao, bo[0], oracle_mod.ML(Ao, inst.n_m), rtol=1e-8, maxit=3000)
    assert code == 0 and res.converged and abs(st[0].iterations - res.iterations) <= 1


def test_star_delta_packed_batch(ctx, oracle_mod):
    """A packed batch with the star rule: each instance cut out of the packed
    system equals the oracle's star-delta assembly."""
    batch = [inputs.planes_3d(n=8, kf=10.0), inputs.fixed_2d(n=12), inputs.random_rects_3d(9, 22060305, 1, 5)]
    sys_ = ctx.assemble_batch(batch, junction="star")
    (_, _, _, _, A), b = sys_.to_host()
    mo, fo = sys_.instances()
    NM = sys_.n_m
    for k, inst in enumerate(batch):
        rows = np.concatenate([np.arange(mo[k], mo[k + 1]), NM + np.arange(fo[k], fo[k + 1])])
        Ak = A[rows][:, rows].tocsr()
        Ak.sort_indices()
        Ao, bo = oracle_mod.assemble(inst, junction=1)
        assert same_csr(Ak, Ao) and np.array_equal(b[:, rows], bo)


def test_rejects_unknown_junction_rule(ctx):
    from paper_2206_03203_gb300 import mdsolve
    inst = inputs.fixed_2d(n=8)
    mdsolve.JUNCTION[7] = 7
    try:
        with pytest.raises(mdsolve.MDSError):
            ctx.assemble(inst, junction=7)
    finally:
        del mdsolve.JUNCTION[7]


def test_intersection_form_full_size_planes3d(ctx, oracle_mod, torch_mod):
    """128^3 with nine fracture planes (k_f = 1e4): 3,456 intersection cells
    (edges where two planes cross) with four fluxes each; assembly bit-exact,
    M_L + FGMRES meets the stopping rule on an independent residual."""
    torch = torch_mod
    inst = inputs.planes_3d(128, kf=1e4)
    sys_ = ctx.assemble(inst, form="flux", junction="star")
    Ao, bo, no = oracle_mod.assemble(inst, form="flux", junction=1, with_split=True)
    N = inst.n_m + inst.n_f
    assert no - N == 3456 and Ao.shape[0] == no + 2 * inst.n_f + 4 * 3456
    (_, _, _, _, A), b = sys_.to_host()
    assert same_csr(A, Ao) and np.array_equal(b, bo)
    prec = ctx.setup(sys_)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, max_iters=5000)
    xg = x.cpu().numpy()
    rel = np.linalg.norm(bo[0] - Ao @ xg) / np.linalg.norm(bo[0])
    assert code == 0 and rel <= 1.01e-8
