"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded instances.

Bit-exact: sparsity, FP64 matrix values, right-hand sides, the Schur
complement, every AMG level's matrix, MIS-2 roots and aggregates (integer and
set-up work with a fixed summation order on both sides).  Tolerance: V-cycle
and preconditioner outputs element by element (max |x - x_o| <= tol max |x_o|
with tol 1e-12 in FP64, 2e-5 in FP32), solves (iteration count within one of
the oracle, true relative residual <= rtol).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
from conftest import maxrel

from paper_2206_03203_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = {
    "fixed2d-64": lambda: inputs.fixed_2d(),
    "fixed2d-37": lambda: inputs.fixed_2d(n=37),
    "seg2d-96": lambda: inputs.random_segments_2d(n=96, n_seg=12),
    "seg2d-61-c1": lambda: inputs.random_segments_2d(n=61, n_seg=9, contrast=1.0),
    "planes3d-16": lambda: inputs.planes_3d(n=16),
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
def test_assembly_bit_exact(ctx, oracle_mod, case):
    inst = CASES[case]()
    sys_ = ctx.assemble(inst)
    (Amm, Amf, Afm, Aff, A), b = sys_.to_host()
    Ao, bo = oracle_mod.assemble(inst)
    assert same_csr(A, Ao)
    assert np.array_equal(b, bo)
    for G, O in zip((Amm, Amf, Afm, Aff), oracle_mod.split(Ao, inst.n_m)):
        assert same_csr(G, O)


@pytest.mark.parametrize("case", list(CASES))
def test_schur_and_hierarchies_bit_exact(ctx, oracle_mod, case):
    inst = CASES[case]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_)
    Ao, _ = oracle_mod.assemble(inst)
    M = oracle_mod.ML(Ao, inst.n_m)
    S_gpu, _, _ = prec.level_host(0, 0)
    assert same_csr(S_gpu, M.schur)
    for block in (0, 1):
        amg = M.amg(block)
        info = prec.info(block)
        assert info["nlevels"] == amg.nlevels
        assert info["dense"] == amg.coarsest_dense
        for l in range(amg.nlevels):
            Ag, agg, roots = prec.level_host(block, l)
            assert same_csr(Ag, amg.level_A(l)), (block, l)
            assert np.array_equal(roots, amg.roots(l)), (block, l)
            ao = amg.agg(l)
            if ao is None:
                assert agg is None
            else:
                assert np.array_equal(agg, ao), (block, l)


@pytest.mark.parametrize("prec_name", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("case", ["seg2d-96", "planes3d-16", "rects3d-18"])
def test_stored_levels_bit_exact(ctx, oracle_mod, case, prec_name):
    """What each V-cycle level multiplies by, bit for bit: FP32 values, or
    the bf16 / fp16 values q_ij with their power-of-two row scales s_i
    (s_i q_ij equal to the oracle's stored value), and 1/D1."""
    inst = CASES[case]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, precision=prec_name, format="csr")
    Ao, _ = oracle_mod.assemble(inst)
    code = {"fp32": 32, "bf16": 16, "fp16": 17}[prec_name]
    M = oracle_mod.ML(Ao, inst.n_m, prec=code)
    lowp_levels = 0
    for block in (0, 1):
        amg = M.amg(block)
        for l in range(amg.nlevels):
            av, rs, dv, lowp = amg.stored(l)
            vt, v, r, d = prec.level_storage_host(block, l)
            assert np.array_equal(d, dv), (block, l)
            if l == amg.nlevels - 1 and amg.coarsest_dense:
                assert v is None
                continue
            assert vt == (code if lowp else 32), (block, l, vt)
            if lowp:
                lowp_levels += 1
                assert np.array_equal(r, rs), (block, l)
                assert np.array_equal(v * r[np.repeat(np.arange(len(r)), np.diff(amg.level_A(l).indptr))], av)
            else:
                assert r is None and np.array_equal(v, av), (block, l)
    assert lowp_levels > 0 or prec_name == "fp32"


@pytest.mark.parametrize("prec_name,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("case", ["fixed2d-64", "seg2d-96", "planes3d-16", "rects3d-18"])
def test_vcycle_parity(ctx, oracle_mod, torch_mod, case, prec_name, tol):
    torch = torch_mod
    inst = CASES[case]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, precision=prec_name)
    Ao, _ = oracle_mod.assemble(inst)
    M = oracle_mod.ML(Ao, inst.n_m, prec=64 if prec_name == "fp64" else 32)
    rng = np.random.default_rng(7)
    for block, n in ((0, inst.n_m), (1, inst.n_f)):
        b = rng.standard_normal(n)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.vcycle(prec, block, dev(torch, b), x)
        xo = M.amg(block).vcycle(b)
        err = maxrel(x.cpu().numpy(), xo)
        assert err < tol, (block, err)


@pytest.mark.parametrize("kind", ["lower", "diag", "upper"])
@pytest.mark.parametrize("prec_name,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_precond_apply_parity(ctx, oracle_mod, torch_mod, kind, prec_name, tol):
    torch = torch_mod
    inst = CASES["seg2d-96"]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, precision=prec_name, kind=kind)
    Ao, _ = oracle_mod.assemble(inst)
    M = oracle_mod.ML(Ao, inst.n_m, kind=kind, prec=64 if prec_name == "fp64" else 32)
    r = np.random.default_rng(3).standard_normal(sys_.N)
    z = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    ctx.precond_apply(prec, dev(torch, r), z)
    zo = M.apply(r)
    err = maxrel(z.cpu().numpy(), zo)
    assert err < tol, err


def test_spmv_parity(ctx, oracle_mod, torch_mod):
    torch = torch_mod
    inst = CASES["rects3d-18"]()
    sys_ = ctx.assemble(inst)
    Ao, _ = oracle_mod.assemble(inst)
    x = np.random.default_rng(1).standard_normal(sys_.N)
    y = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    ctx.spmv(sys_, dev(torch, x), y)
    yo = oracle_mod.spmv(Ao, x)
    assert np.max(np.abs(y.cpu().numpy() - yo)) <= 1e-13 * np.max(np.abs(yo))


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_solve_parity(ctx, oracle_mod, torch_mod, case, prec_name):
    torch = torch_mod
    inst = CASES[case]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, precision=prec_name)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, rtol=1e-8, max_iters=3000)
    res, Ao, bo, _ = oracle_mod.solve(inst, prec=64 if prec_name == "fp64" else 32, maxit=3000)
    assert code == 0 and res.converged
    assert abs(st[0].iterations - res.iterations) <= 1, (st[0].iterations, res.iterations)
    xg = x.cpu().numpy()
    rel = np.linalg.norm(bo[0] - Ao @ xg) / np.linalg.norm(bo[0])
    assert rel <= 1e-8 * 1.01 and abs(rel - st[0].relres_true) <= 1e-3 * rel + 1e-15
    # both solutions are within the same residual bound of the exact one
    assert np.linalg.norm(Ao @ (xg - res.x)) / np.linalg.norm(bo[0]) <= 2.1e-8


def test_solve_matches_direct(ctx, oracle_mod, torch_mod):
    torch = torch_mod
    inst = CASES["fixed2d-64"]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    ctx.solve(sys_, prec, None, x, rtol=1e-12)
    Ao, bo = oracle_mod.assemble(inst)
    xd = spla.spsolve(Ao.tocsc(), bo[0])
    assert np.max(np.abs(x.cpu().numpy() - xd)) < 1e-8


def test_pcg_block_diagonal(ctx, oracle_mod, torch_mod):
    torch = torch_mod
    inst = CASES["planes3d-13-kf1"]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, kind="diag")
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, krylov="pcg", max_iters=2000)
    res, Ao, bo, _ = oracle_mod.solve(inst, kind="diag", krylov="pcg", maxit=2000)
    assert code == 0 and abs(st[0].iterations - res.iterations) <= 1
    assert st[0].relres_true <= 1e-8


@pytest.mark.parametrize("case,precision", [("planes3d-13-kf1", "fp64"), ("seg2d-96", "fp64"),
                                            ("rects3d-18", "fp64"), ("planes3d-13-kf1", "fp32")])
def test_minres_block_diagonal(ctx, oracle_mod, torch_mod, case, precision):
    """Preconditioned MINRES with B_D (symmetric V-cycles) through the C ABI:
    iteration count within one of the oracle's (same stopping rule), the
    solution within the solve tolerance of the oracle's."""
    torch = torch_mod
    inst = CASES[case]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, kind="diag", precision=precision)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, krylov="minres", max_iters=3000)
    kw = {"prec": 32} if precision == "fp32" else {}
    res, Ao, bo, _ = oracle_mod.solve(inst, kind="diag", krylov="minres", maxit=3000, **kw)
    assert code == 0 and res.converged
    # the three-term Lanczos recurrence is not reorthogonalised: rounding that
    # differs in order (FMA, reduction trees) shifts when lost orthogonality
    # delays convergence, so long runs may differ by 1% of the count
    tol = max(1 if precision == "fp64" else 2, res.iterations // 100)
    assert abs(st[0].iterations - res.iterations) <= tol, (st[0].iterations, res.iterations)
    assert st[0].relres_true <= 1e-8
    xo = res.x
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-6, err


def test_minres_identity_and_restart(ctx, oracle_mod, torch_mod):
    """MINRES without preconditioner on the assembled system: the same
    iteration count as the oracle; a nonzero initial guess equal to the
    solution returns at once."""
    torch = torch_mod
    inst = inputs.fixed_2d(n=12)
    sys_ = ctx.assemble(inst)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, None, None, x, krylov="minres", use_precond=0, max_iters=5000)
    Ao, bo = oracle_mod.assemble(inst)
    res = oracle_mod.minres(Ao, bo[0], "identity", maxit=5000)
    assert code == 0 and abs(st[0].iterations - res.iterations) <= 1 and st[0].relres_true <= 1e-8
    code, st2 = ctx.solve(sys_, None, None, x, krylov="minres", use_precond=0, max_iters=5000)
    assert code == 0 and st2[0].iterations == 0


def test_identity_preconditioner(ctx, oracle_mod, torch_mod):
    torch = torch_mod
    inst = inputs.fixed_2d(n=12)
    sys_ = ctx.assemble(inst)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, None, None, x, use_precond=0, max_iters=5000, restart=30)
    Ao, bo = oracle_mod.assemble(inst)
    res = oracle_mod.fgmres(Ao, bo[0], "identity", restart=30, maxit=5000)
    assert abs(st[0].iterations - res.iterations) <= 1 and st[0].relres_true <= 1e-8


def test_system_from_csr(ctx, oracle_mod, torch_mod):
    torch = torch_mod
    inst = CASES["seg2d-61-c1"]()
    Ao, bo = oracle_mod.assemble(inst)
    blocks = []
    for B in oracle_mod.split(Ao, inst.n_m):
        blocks.append((dev(torch, B.indptr.astype(np.int32)), dev(torch, B.indices.astype(np.int32)),
                       dev(torch, B.data), B.shape[0], B.shape[1]))
    b = dev(torch, bo[0])
    sys_ = ctx.system_from_csr(blocks, b)
    (_, _, _, _, A), bh = sys_.to_host()
    assert same_csr(A, Ao) and np.array_equal(bh[0], bo[0])
    prec = ctx.setup(sys_)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x)
    res, *_ = oracle_mod.solve(inst)
    assert code == 0 and abs(st[0].iterations - res.iterations) <= 1


def test_host_buffers_and_nonzero_x0(ctx, oracle_mod):
    inst = CASES["fixed2d-37"]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_)
    Ao, bo = oracle_mod.assemble(inst)
    x = np.zeros(sys_.N)
    code, st = ctx.solve(sys_, prec, np.ascontiguousarray(bo[0]), x)
    assert code == 0 and np.linalg.norm(bo[0] - Ao @ x) / np.linalg.norm(bo[0]) <= 1e-8
    # restart from the solution: zero iterations
    code, st = ctx.solve(sys_, prec, np.ascontiguousarray(bo[0]), x)
    assert st[0].iterations == 0


def test_multiple_rhs(ctx, oracle_mod):
    inst = inputs.random_rects_3d(12, 5, 1, 4, nrhs=3, random_dirichlet=True)
    sys_ = ctx.assemble(inst)
    assert sys_.nrhs == 3
    prec = ctx.setup(sys_)
    x = np.zeros(3 * sys_.N)
    code, st = ctx.solve(sys_, prec, None, x, nrhs=3)
    Ao, bo = oracle_mod.assemble(inst)
    for k in range(3):
        xk = x[k * sys_.N:(k + 1) * sys_.N]
        assert np.linalg.norm(bo[k] - Ao @ xk) / np.linalg.norm(bo[k]) <= 1e-8
        r = oracle_mod.fgmres(Ao, bo[k], oracle_mod.ML(Ao, inst.n_m))
        assert abs(st[k].iterations - r.iterations) <= 1


# ---------------------------------------------------------------- edge cases

def test_no_fractures(ctx, oracle_mod, torch_mod):
    torch = torch_mod
    inst = inputs.make_instance("plain", 2, 40, inputs.lognormal_km(1, 0, 1600, 1.0), [])
    sys_ = ctx.assemble(inst)
    assert sys_.n_f == 0
    prec = ctx.setup(sys_)
    assert prec.info(1)["nlevels"] == 0
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x)
    res, *_ = oracle_mod.solve(inst)
    assert code == 0 and abs(st[0].iterations - res.iterations) <= 1


def test_tiny_grids(ctx, oracle_mod, torch_mod):
    torch = torch_mod
    for inst in (inputs.make_instance("one", 2, 1, np.ones(1), []),
                 inputs.make_instance("two", 3, 2, np.array([1., 2, 3, 4, 5, 6, 7, 8]),
                                      [inputs.Rect(2, 1, (0, 0), (1, 2), 3.0, 0.1)])):
        sys_ = ctx.assemble(inst)
        (_, _, _, _, A), b = sys_.to_host()
        Ao, bo = oracle_mod.assemble(inst)
        assert same_csr(A, Ao) and np.array_equal(b, bo)
        prec = ctx.setup(sys_)
        x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
        code, st = ctx.solve(sys_, prec, None, x)
        assert code == 0 and st[0].relres_true <= 1e-8


def test_coarsening_stall_is_smoother_only(ctx, oracle_mod, torch_mod):
    """Blocking fractures make A_ff strongly diagonal: no strong couplings, the
    hierarchy stops at level 0 and the V-cycle is two L1-Jacobi sweeps."""
    torch = torch_mod
    inst = inputs.random_segments_2d(n=200, n_seg=20, contrast=1e-4)
    inst.fc_kf[:] = 1e-4
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, n_coarse=16)
    Ao, _ = oracle_mod.assemble(inst)
    M = oracle_mod.ML(Ao, inst.n_m, n_coarse=16)
    info = prec.info(1)
    assert info["nlevels"] == M.amg(1).nlevels and info["dense"] == M.amg(1).coarsest_dense
    b = np.random.default_rng(0).standard_normal(inst.n_f)
    x = torch.zeros(inst.n_f, dtype=torch.float64, device="cuda")
    ctx.vcycle(prec, 1, dev(torch, b), x)
    xo = M.amg(1).vcycle(b)
    assert maxrel(x.cpu().numpy(), xo) <= 1e-12


def test_rejects_duplicate_fracture_face(ctx):
    from paper_2206_03203_gb300 import mdsolve
    inst = inputs.make_instance("d", 2, 8, np.ones(64), [inputs.Rect(0, 4, (0,), (2,), 1.0, 1.0)])
    inst.fc_pos = np.vstack([inst.fc_pos, inst.fc_pos[:1]])
    inst.fc_axis = np.concatenate([inst.fc_axis, inst.fc_axis[:1]])
    inst.fc_kf = np.concatenate([inst.fc_kf, inst.fc_kf[:1]])
    inst.fc_a = np.concatenate([inst.fc_a, inst.fc_a[:1]])
    with pytest.raises(mdsolve.MDSError) as e:
        ctx.assemble(inst)
    assert e.value.code == -1
    # the context stays usable
    ctx.assemble(inputs.fixed_2d(n=8))


def test_rejects_interior_plane_violation(ctx):
    from paper_2206_03203_gb300 import mdsolve
    inst = inputs.make_instance("b", 2, 8, np.ones(64), [inputs.Rect(0, 4, (0,), (2,), 1.0, 1.0)])
    inst.fc_pos = inst.fc_pos.copy()
    inst.fc_pos[0, 0] = 8  # boundary plane
    with pytest.raises(mdsolve.MDSError):
        ctx.assemble(inst)


def test_nonfinite_rhs_reports_error(ctx, torch_mod):
    torch = torch_mod
    inst = inputs.fixed_2d(n=16)
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_)
    b = torch.full((sys_.N,), float("nan"), dtype=torch.float64, device="cuda")
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    from paper_2206_03203_gb300 import mdsolve
    with pytest.raises(mdsolve.MDSError):
        ctx.solve(sys_, prec, b, x)


def test_iteration_cap_warns(ctx, torch_mod):
    torch = torch_mod
    inst = inputs.fixed_2d(n=32)
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, max_iters=3)
    assert code == 1 and st[0].status == 1 and st[0].iterations == 3


# ---------------------------------------------------------------- full size

def test_full_size_random_segments(ctx, oracle_mod, torch_mod):
    """1024 x 1024, 64 segments, contrast 1e4: assembly, S~ and every AMG level
    bit-exact; the solve meets the stopping rule on an independent residual."""
    torch = torch_mod
    inst = inputs.random_segments_2d()
    sys_ = ctx.assemble(inst)
    (Amm, Amf, Afm, Aff, A), b = sys_.to_host()
    Ao, bo = oracle_mod.assemble(inst)
    assert same_csr(A, Ao) and np.array_equal(b, bo)
    prec = ctx.setup(sys_)
    M = oracle_mod.ML(Ao, inst.n_m)
    for block in (0, 1):
        amg = M.amg(block)
        assert prec.info(block)["nlevels"] == amg.nlevels
        for l in range(amg.nlevels):
            Ag, agg, roots = prec.level_host(block, l)
            assert same_csr(Ag, amg.level_A(l))
            ao = amg.agg(l)
            assert (agg is None and ao is None) or np.array_equal(agg, ao)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, max_iters=5000)
    xg = x.cpu().numpy()
    rel = np.linalg.norm(bo[0] - Ao @ xg) / np.linalg.norm(bo[0])
    assert code == 0 and rel <= 1.01e-8
    # sampled rows of M_L: one application against the oracle
    r = np.random.default_rng(5).standard_normal(sys_.N)
    z = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    ctx.precond_apply(prec, dev(torch, r), z)
    zo = M.apply(r)
    assert maxrel(z.cpu().numpy(), zo) <= 1e-12


# ---------------------------------------------------------------- storage and smoother options

PREC_CODE = {"fp64": 64, "fp32": 32, "bf16": 16, "fp16": 17}
OPTION_CASES = [
    dict(precision="fp64", smoother="chebyshev"),
    dict(precision="fp32", smoother="chebyshev"),
    dict(precision="fp64", sweeps=2),
    dict(precision="fp32", sweeps=2),
    dict(precision="bf16"),
    dict(precision="fp16"),
    dict(precision="fp16", lowp_from_level=0),
    dict(precision="fp32", format="sell"),
    dict(precision="fp32", format="sell", sell_c=16, sell_sigma=64),
    dict(precision="fp64", format="sell", sell_c=8, sell_sigma=32),
    dict(precision="bf16", format="sell", sell_sigma=256),
    dict(precision="fp32", format="auto"),
    dict(precision="fp64", format="auto", smoother="chebyshev"),
    dict(precision="fp64", smoother="chebyshev", cheb_degree=1),
    dict(precision="fp64", smoother="chebyshev", cheb_degree=3),
    dict(precision="fp32", smoother="chebyshev", cheb_degree=4, sweeps=2),
]


def oracle_kw(cfg):
    return dict(prec=PREC_CODE[cfg.get("precision", "fp64")], smoother=1 if cfg.get("smoother") == "chebyshev" else 0,
                sweeps=cfg.get("sweeps", 1), lowp_from_level=cfg.get("lowp_from_level", 1),
                cheb_degree=cfg.get("cheb_degree", 2))


def tol_of(cfg):
    return {"fp64": 1e-12, "fp32": 2e-5}.get(cfg.get("precision"), 5e-5)


@pytest.mark.parametrize("cfg", OPTION_CASES, ids=lambda c: "-".join(f"{k}={v}" for k, v in c.items()))
@pytest.mark.parametrize("case", ["seg2d-256", "rects3d-18"])
def test_vcycle_options_parity(ctx, oracle_mod, torch_mod, case, cfg):
    torch = torch_mod
    inst = inputs.random_segments_2d(n=256, n_seg=20) if case == "seg2d-256" else CASES[case]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, **cfg)
    Ao, _ = oracle_mod.assemble(inst)
    M = oracle_mod.ML(Ao, inst.n_m, **oracle_kw(cfg))
    rng = np.random.default_rng(11)
    for block, n in ((0, inst.n_m), (1, inst.n_f)):
        b = rng.standard_normal(n)
        for rep in range(2):  # repeated application uses the same stored state
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            ctx.vcycle(prec, block, dev(torch, b), x)
            xo = M.amg(block).vcycle(b)
            err = maxrel(x.cpu().numpy(), xo)
            assert err < tol_of(cfg), (block, rep, err)


@pytest.mark.parametrize("cfg", [dict(precision="bf16"), dict(precision="fp16"), dict(smoother="chebyshev"),
                                 dict(precision="fp32", smoother="chebyshev", format="sell"),
                                 dict(precision="fp32", sweeps=2, format="auto"),
                                 dict(smoother="chebyshev", cheb_degree=3)],
                         ids=lambda c: "-".join(f"{k}={v}" for k, v in c.items()))
@pytest.mark.parametrize("case", ["seg2d-96", "planes3d-16", "rects3d-18"])
def test_solve_options_parity(ctx, oracle_mod, torch_mod, case, cfg):
    torch = torch_mod
    inst = CASES[case]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, **cfg)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, max_iters=3000)
    res, Ao, bo, _ = oracle_mod.solve(inst, maxit=3000, **oracle_kw(cfg))
    assert code == 0 and res.converged
    assert abs(st[0].iterations - res.iterations) <= 1, (st[0].iterations, res.iterations)
    xg = x.cpu().numpy()
    assert np.linalg.norm(bo[0] - Ao @ xg) / np.linalg.norm(bo[0]) <= 1.01e-8


def test_autotuner_cache_reuses_choice(ctx, torch_mod):
    inst = inputs.random_segments_2d(n=256, n_seg=20)
    s1 = ctx.assemble(inst)
    p1 = ctx.setup(s1, precision="fp32", format="auto")
    p2 = ctx.setup(s1, precision="fp32", format="auto")
    r = np.random.default_rng(0).standard_normal(s1.N)
    z1 = torch_mod.zeros(s1.N, dtype=torch_mod.float64, device="cuda")
    z2 = torch_mod.zeros_like(z1)
    ctx.precond_apply(p1, dev(torch_mod, r), z1)
    ctx.precond_apply(p2, dev(torch_mod, r), z2)
    assert torch_mod.equal(z1, z2)


@pytest.mark.parametrize("krylov,kind,precision", [("fgmres", "lower", "fp64"), ("fgmres", "lower", "fp32"),
                                                    ("pcg", "diag", "fp64")])
def test_graphs_match_direct_launches(ctx, torch_mod, krylov, kind, precision):
    """Replaying captured Krylov steps gives bit-identical results and the same
    launch accounting as launching every kernel directly."""
    torch = torch_mod
    inst = CASES["planes3d-13-kf1"]() if krylov == "pcg" else CASES["seg2d-96"]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, kind=kind, precision=precision)
    out = []
    for graphs in (0, 1):
        x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
        ctx.timing_reset()
        code, st = ctx.solve(sys_, prec, None, x, krylov=krylov, restart=10, graphs=graphs, max_iters=2000)
        out.append((x, st[0], ctx.launch_count(), ctx.timing_query("gs_dot")[0], ctx.timing_query("spmv")[0]))
    (x0, s0, l0, d0, p0), (x1, s1, l1, d1, p1) = out
    assert torch.equal(x0, x1)
    assert s0.iterations == s1.iterations and s0.relres_true == s1.relres_true
    assert l0 == l1 and d0 == d1 and p0 == p1


@pytest.mark.parametrize("case,precision,nr", [("seg2d-96", "fp64", 1), ("planes3d-16", "fp64", 1),
                                               ("rects3d-18", "fp32", 1), ("seg2d-96", "fp64", 4)])
def test_coarse_tail_matches_per_level_launches(ctx, torch_mod, case, precision, nr):
    """The coarse end of the V-cycle run as one cluster kernel gives the same
    V-cycle (to rounding) and the same solve as one launch per level op."""
    torch = torch_mod
    inst = CASES[case]()
    sys_ = ctx.assemble(inst)
    pre = [ctx.setup(sys_, precision=precision, coarse_tail=t) for t in (0, 1)]
    gen = torch.Generator(device="cpu").manual_seed(7)
    for blk, n in ((0, sys_.n_m), (1, sys_.n_f)):
        if n == 0:
            continue
        b = torch.rand(n, generator=gen, dtype=torch.float64).to("cuda")
        xs = []
        for p in pre:
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            ctx.vcycle(p, blk, b, x)
            xs.append(x)
        rel = (torch.linalg.norm(xs[0] - xs[1]) / torch.linalg.norm(xs[0])).item()
        assert rel <= (1e-13 if precision == "fp64" else 2e-6), (blk, rel)
    its = []
    for p in pre:
        x = torch.zeros(sys_.N * nr, dtype=torch.float64, device="cuda")
        B = torch.rand(sys_.N * nr, generator=gen.manual_seed(3), dtype=torch.float64).to("cuda")
        code, st = ctx.solve(sys_, p, B, x, nrhs=nr, max_iters=3000)
        assert code == 0
        its.append([s_.iterations for s_ in st])
    assert all(abs(a - b) <= 1 for a, b in zip(*its)), its


def test_sampled_timing(ctx, torch_mod):
    """With timing sampled every 4th restart cycle the solution is unchanged,
    only some launches are bracketed, and the per-launch averages of the
    bracketed subset are positive and consistent with the class totals."""
    torch = torch_mod
    inst = CASES["seg2d-96"]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_)
    out = []
    for every in (1, 4):
        ctx.timing_enable("gs_dot", True)
        ctx.timing_sample_every(every)
        ctx.timing_reset()
        x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
        code, st = ctx.solve(sys_, prec, None, x, restart=5, max_iters=2000)
        assert code == 0
        out.append((x, st[0], ctx.timing_query("gs_dot"), ctx.timing_sampled("gs_dot")))
    ctx.timing_sample_every(1)
    ctx.timing_enable("gs_dot", False)
    (x1, s1, q1, t1), (x4, s4, q4, t4) = out
    assert torch.equal(x1, x4) and s1.iterations == s4.iterations
    assert q1[0] == t1[0] == s1.iterations  # every launch bracketed
    assert q4[0] == s4.iterations and 0 < t4[0] < q4[0]
    assert t4[1] > 0 and t4[2] > 0 and t4[2] < q4[2]


def test_context_outlives_dependents_in_any_order(torch_mod):
    """mds_destroy with live systems/preconditioners defers the release until
    the last of them is destroyed (any finalisation order is safe)."""
    from paper_2206_03203_gb300 import mdsolve
    L = mdsolve.lib()
    c2 = mdsolve.Context(0)
    s = c2.assemble(inputs.fixed_2d(n=16))
    p = c2.setup(s)
    h_ctx, h_s, h_p = c2.h, s.h, p.h
    c2.h = s.h = p.h = None  # detach the Python wrappers
    assert L.mds_destroy(h_ctx) == 0
    assert L.mds_system_destroy(h_s) == 0
    assert L.mds_precond_destroy(h_p) == 0


# ---------------------------------------------------------------- batching (multi-RHS, packed instances)

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multi_rhs_lockstep(ctx, oracle_mod, torch_mod, precision):
    """Several right-hand sides solved together (shared SpMV / V-cycle reads,
    per-column FGMRES) agree with column-by-column solves and the oracle."""
    inst = inputs.random_rects_3d(14, 7, 2, 5, nrhs=5, random_dirichlet=True)
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, precision=precision)
    xb = np.zeros(5 * sys_.N)
    code, stb = ctx.solve(sys_, prec, None, xb, nrhs=5)
    xs = np.zeros(5 * sys_.N)
    code2, sts = ctx.solve(sys_, prec, None, xs, nrhs=5, batched=0)
    assert code == 0 and code2 == 0
    Ao, bo = oracle_mod.assemble(inst)
    M = oracle_mod.ML(Ao, inst.n_m, prec=64 if precision == "fp64" else 32)
    for k in range(5):
        xk = xb[k * sys_.N:(k + 1) * sys_.N]
        assert np.linalg.norm(bo[k] - Ao @ xk) / np.linalg.norm(bo[k]) <= 1.01e-8
        assert abs(stb[k].iterations - sts[k].iterations) <= 1
        r = oracle_mod.fgmres(Ao, bo[k], M)
        assert abs(stb[k].iterations - r.iterations) <= 1, (k, stb[k].iterations, r.iterations)


def packed_oracle(oracle_mod, insts):
    """Block-diagonal packing [m_0..m_K-1; f_0..f_K-1] of oracle assemblies."""
    import scipy.sparse as sp
    blocks = [oracle_mod.split(*oracle_mod.assemble(i)[:1], i.n_m) for i in insts]
    bs = [oracle_mod.assemble(i)[1] for i in insts]
    Amm = sp.block_diag([b[0] for b in blocks], format="csr")
    Amf = sp.block_diag([b[1] for b in blocks], format="csr")
    Afm = sp.block_diag([b[2] for b in blocks], format="csr")
    Aff = sp.block_diag([b[3] for b in blocks], format="csr")
    A = sp.bmat([[Amm, Amf], [Afm, Aff]], format="csr")
    A.sort_indices()
    nrhs = insts[0].nrhs
    b = np.stack([np.concatenate([bs[k][r][:insts[k].n_m] for k in range(len(insts))] +
                                 [bs[k][r][insts[k].n_m:] for k in range(len(insts))]) for r in range(nrhs)])
    return A, b, Amm.shape[0]


def test_packed_batch_of_uneven_instances(ctx, oracle_mod, torch_mod):
    insts = [inputs.random_rects_3d(n, 22060304, k, 1 + k % 4, nrhs=2, random_dirichlet=True)
             for k, n in enumerate([9, 12, 8, 14, 11])]
    sys_ = ctx.assemble_batch(insts)
    assert sys_.n_inst == 5
    (_, _, _, _, A), b = sys_.to_host()
    Ao, bo, NM = packed_oracle(oracle_mod, insts)
    assert same_csr(A, Ao) and np.array_equal(b, bo)
    mo, fo = sys_.instances()
    prec = ctx.setup(sys_)
    x = np.zeros(2 * sys_.N)
    code, st = ctx.solve(sys_, prec, None, x, nrhs=2)
    assert code == 0 and len(st) == 10
    M = oracle_mod.ML(Ao, NM, segments=(mo, fo))
    for k in range(5):
        rows = np.r_[mo[k]:mo[k + 1], NM + fo[k]:NM + fo[k + 1]]
        for c in range(2):
            be = np.zeros(sys_.N)
            be[rows] = bo[c][rows]
            r = oracle_mod.fgmres(Ao, be, M)
            s = st[k * 2 + c]
            assert s.status == 0 and abs(s.iterations - r.iterations) <= 1, (k, c, s.iterations, r.iterations)
            xk = x[c * sys_.N:(c + 1) * sys_.N][rows]
            Ak = Ao[rows][:, rows]
            assert np.linalg.norm(be[rows] - Ak @ xk) / np.linalg.norm(be[rows]) <= 1.01e-8


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_packed_hierarchies_bit_exact(ctx, oracle_mod, precision):
    """A packed batch is coarsened instance by instance: every level, aggregate
    map and root set of both hierarchies equals the oracle's segmented set-up,
    and the last level holds at most n_coarse rows of each instance."""
    insts = [inputs.random_rects_3d(n, 22060304, k, 1 + k % 4, nrhs=1, random_dirichlet=True)
             for k, n in enumerate([9, 12, 8, 14, 11, 10])]
    sys_ = ctx.assemble_batch(insts)
    mo, fo = sys_.instances()
    Ao, _, NM = packed_oracle(oracle_mod, insts)
    code = {"fp64": 64, "bf16": 16}[precision]
    prec = ctx.setup(sys_, precision=precision, n_coarse=48, format="csr")
    M = oracle_mod.ML(Ao, NM, segments=(mo, fo), n_coarse=48, prec=code)
    for block in (0, 1):
        amg = M.amg(block)
        assert prec.info(block)["nlevels"] == amg.nlevels
        assert np.all(np.diff(amg.segments(amg.nlevels - 1)) <= 48)
        for l in range(amg.nlevels):
            Ag, agg, roots = prec.level_host(block, l)
            assert same_csr(Ag, amg.level_A(l)), (block, l)
            assert np.array_equal(roots, amg.roots(l)), (block, l)
            ao = amg.agg(l)
            assert (agg is None and ao is None) or np.array_equal(agg, ao), (block, l)
    rng = np.random.default_rng(2)
    for block, n in ((0, NM), (1, sys_.n_f)):
        b = rng.standard_normal(n)
        import torch
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.vcycle(prec, block, torch.as_tensor(b, device="cuda"), x)
        assert maxrel(x.cpu().numpy(), M.amg(block).vcycle(b)) < (1e-12 if precision == "fp64" else 5e-5)


def test_packed_coarsest_tiles_many_instances(ctx, oracle_mod, torch_mod):
    """A batch with more coarsest-level tiles than the GPU has SMs takes the
    tiled coarsest inverse (symmetric, mirrored) and the tiled apply: its
    V-cycles agree with the oracle's segmented ones (FP64), and sampled
    problems of the batched solve converge as the oracle's do."""
    import torch
    insts = [inputs.random_rects_3d(6 + k % 3, 22060304, k, 1, nrhs=1, random_dirichlet=True)
             for k in range(160)]
    sys_ = ctx.assemble_batch(insts)
    mo, fo = sys_.instances()
    Ao, bo, NM = packed_oracle(oracle_mod, insts)
    prec = ctx.setup(sys_, precision="fp64", format="csr")
    M = oracle_mod.ML(Ao, NM, segments=(mo, fo))
    rng = np.random.default_rng(5)
    for block, n in ((0, NM), (1, sys_.n_f)):
        assert prec.info(block)["dense"]
        b = rng.standard_normal(n)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.vcycle(prec, block, torch.as_tensor(b, device="cuda"), x)
        assert maxrel(x.cpu().numpy(), M.amg(block).vcycle(b)) < 1e-12, block
    x = np.zeros(sys_.N)
    code, st = ctx.solve(sys_, prec, None, x, nrhs=1, rtol=1e-8)
    assert code == 0
    for k in (0, 57, 101, 159):
        rows = np.r_[mo[k]:mo[k + 1], NM + fo[k]:NM + fo[k + 1]]
        be = np.zeros(sys_.N)
        be[rows] = bo[0][rows]
        r = oracle_mod.fgmres(Ao, be, M)
        assert abs(st[k].iterations - r.iterations) <= 1, (k, st[k].iterations, r.iterations)


def test_packed_batch_per_problem_iteration_cap(ctx, torch_mod):
    insts = [inputs.random_rects_3d(n, 3, k, 2, nrhs=1) for k, n in enumerate([8, 10])]
    sys_ = ctx.assemble_batch(insts)
    prec = ctx.setup(sys_)
    x = np.zeros(sys_.N)
    code, st = ctx.solve(sys_, prec, None, x, max_iters=4)
    assert code == 1 and all(s.iterations == 4 and s.status == 1 for s in st)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_packed_batch_four_columns_uneven_convergence(ctx, torch_mod, precision):
    """Problems stop at different steps; the stopped ones must not disturb the
    others (shared coarsest dense solve) nor their own solution."""
    insts = [inputs.random_rects_3d(n, 22060304, k, 2 + k, nrhs=4, random_dirichlet=True)
             for k, n in enumerate([16, 11, 14, 9])]
    sys_ = ctx.assemble_batch(insts)
    prec = ctx.setup(sys_, precision=precision)
    x = np.zeros(4 * sys_.N)
    code, st = ctx.solve(sys_, prec, None, x, nrhs=4)
    assert code == 0 and all(s.status == 0 and s.relres_true <= 1.01e-8 for s in st)
    assert np.all(np.isfinite(x))
    # problems of one instance differ only in their boundary data: similar counts
    for k in range(4):
        its = [st[k * 4 + c].iterations for c in range(4)]
        assert max(its) - min(its) <= max(3, min(its) // 4), its


@pytest.mark.parametrize("eta2", [0.0, 0.5, 2.0])
def test_reorthogonalisation_threshold(ctx, oracle_mod, torch_mod, eta2):
    """One classical Gram-Schmidt pass (eta2 = 0), the DGKS rule (0.5) and
    always two passes (>= 1) all reach the stopping rule within one iteration
    of the oracle's modified Gram-Schmidt."""
    torch = torch_mod
    inst = CASES["rects3d-18"]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, reorth_eta2=eta2)
    res, Ao, bo, _ = oracle_mod.solve(inst)
    assert code == 0 and abs(st[0].iterations - res.iterations) <= 1
    assert st[0].relres_true <= 1e-8


# ---------------------------------------------------------------- smoothed aggregation

@pytest.mark.parametrize("case", ["fixed2d-37", "seg2d-96", "planes3d-13-kf1", "rects3d-18"])
def test_smoothed_hierarchy_bit_exact(ctx, oracle_mod, case):
    inst = CASES[case]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, prolongation="smoothed")
    Ao, _ = oracle_mod.assemble(inst)
    M = oracle_mod.ML(Ao, inst.n_m, smoothed=1)
    for block in (0, 1):
        amg = M.amg(block)
        assert prec.info(block)["nlevels"] == amg.nlevels
        for l in range(amg.nlevels):
            Ag, agg, roots = prec.level_host(block, l)
            assert same_csr(Ag, amg.level_A(l)), (block, l)
            Po = amg.P(l)
            Pg = prec.prolongator_host(block, l)
            assert (Po is None and Pg is None) or same_csr(Pg, Po), (block, l)


@pytest.mark.parametrize("prec_name,tol", [("fp64", 1e-12), ("fp32", 2e-5), ("bf16", 5e-5)])
def test_smoothed_vcycle_and_solve_parity(ctx, oracle_mod, torch_mod, prec_name, tol):
    torch = torch_mod
    inst = CASES["rects3d-18"]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, precision=prec_name, prolongation="smoothed", format="auto")
    Ao, bo = oracle_mod.assemble(inst)
    code_p = {"fp64": 64, "fp32": 32, "bf16": 16}[prec_name]
    M = oracle_mod.ML(Ao, inst.n_m, prec=code_p, smoothed=1)
    b = np.random.default_rng(4).standard_normal(inst.n_m)
    x = torch.zeros(inst.n_m, dtype=torch.float64, device="cuda")
    ctx.vcycle(prec, 0, dev(torch, b), x)
    xo = M.amg(0).vcycle(b)
    assert maxrel(x.cpu().numpy(), xo) < tol
    xs = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, xs)
    r = oracle_mod.fgmres(Ao, bo[0], M)
    assert code == 0 and abs(st[0].iterations - r.iterations) <= 1


def test_smoothed_batched_multi_rhs(ctx, torch_mod):
    inst = inputs.random_rects_3d(14, 7, 2, 5, nrhs=4, random_dirichlet=True)
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, precision="fp32", prolongation="smoothed")
    x = np.zeros(4 * sys_.N)
    code, st = ctx.solve(sys_, prec, None, x, nrhs=4)
    xs = np.zeros(4 * sys_.N)
    code2, st2 = ctx.solve(sys_, prec, None, xs, nrhs=4, batched=0)
    assert code == 0 and code2 == 0
    assert all(abs(a.iterations - b.iterations) <= 1 for a, b in zip(st, st2))


def test_rejects_sizes_beyond_int32_indices(ctx, torch_mod):
    """1300^3 cells exceed the int32 row and column indices: the assembly is
    refused before any instance array is read (the device arrays here are
    placeholders of one element)."""
    import types
    torch = torch_mod
    from paper_2206_03203_gb300 import mdsolve
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    onei = torch.zeros(3, dtype=torch.int32, device="cuda")
    inst = types.SimpleNamespace(dim=3, n=1300, n_f=0, nrhs=1)
    arrs = dict(km=one, fc_axis=onei, fc_pos=onei, fc_kf=one, fc_a=one, pD_left=one, pD_right=one)
    with pytest.raises(mdsolve.MDSError) as e:
        ctx.assemble(inst, device_arrays=arrs)
    assert "int32" in str(e.value)


@pytest.mark.parametrize("case", ["fixed2d-64", "seg2d-96", "planes3d-16", "rects3d-18"])
def test_fp64_path_agrees_with_oracle_to_1e10(ctx, oracle_mod, torch_mod, case):
    """The FP64 path and the oracle, both solved to a relative residual of
    1e-12, agree to 1e-10 in the relative residual of their difference (and
    to 1e-9 in the solution against a sparse direct solve)."""
    torch = torch_mod
    inst = CASES[case]()
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, format="csr")
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, rtol=1e-12, max_iters=5000)
    res, Ao, bo, _ = oracle_mod.solve(inst, rtol=1e-12, maxit=5000)
    assert code == 0 and res.converged
    xg = x.cpu().numpy()
    nb = np.linalg.norm(bo[0])
    assert np.linalg.norm(Ao @ (xg - res.x)) / nb <= 1e-10
    xd = spla.spsolve(Ao.tocsc(), bo[0])
    assert np.linalg.norm(xg - xd) <= 1e-9 * np.linalg.norm(xd)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("case", ["fixed2d-37", "planes3d-13-kf1", "rects3d-18", "packed"])
def test_stencil_storage_is_csr_bit_for_bit(ctx, torch_mod, case, precision):
    """The finest S~ level stored by diagonals (no column indices) gives the
    one-thread-per-row CSR results bit for bit: V-cycles, M_L and whole
    solves (same iteration counts, identical solutions), single instances in
    2D and 3D and a packed batch of instances of different sizes."""
    torch = torch_mod
    if case == "packed":
        insts = [inputs.random_rects_3d(n, 22060304, k, 1 + k % 3, nrhs=2, random_dirichlet=True)
                 for k, n in enumerate([9, 12, 7, 10])]
        sys_ = ctx.assemble_batch(insts)
    else:
        sys_ = ctx.assemble(CASES[case]())
    nr = sys_.nrhs
    ps = ctx.setup(sys_, precision=precision, format="stencil")
    pc = ctx.setup(sys_, precision=precision, format="csr")
    assert ps.level_format(0, 0) == "stencil" and pc.level_format(0, 0) == "csr"
    rng = np.random.default_rng(5)
    r = dev(torch, rng.standard_normal(sys_.N))
    zs = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    zc = torch.zeros_like(zs)
    ctx.precond_apply(ps, r, zs)
    ctx.precond_apply(pc, r, zc)
    assert torch.equal(zs, zc)
    xs = torch.zeros(sys_.N * nr, dtype=torch.float64, device="cuda")
    xc = torch.zeros_like(xs)
    c1, s1 = ctx.solve(sys_, ps, None, xs, nrhs=nr, max_iters=3000)
    c2, s2 = ctx.solve(sys_, pc, None, xc, nrhs=nr, max_iters=3000)
    assert c1 == c2 == 0
    assert [q.iterations for q in s1] == [q.iterations for q in s2]
    assert torch.equal(xs, xc)


@pytest.mark.parametrize("precision,nr", [("bf16", 4), ("fp32", 4), ("fp64", 2), ("fp64", 4)])
def test_stencil_bulk_staging_is_csr_bit_for_bit(ctx, torch_mod, precision, nr):
    """The stencil kernel that stages each row block's planes and its
    neighbours' window by bulk asynchronous copies (vectors of 16-byte
    rows: FP32 with 4 columns, FP64 with 2 or 4) gives the CSR results bit
    for bit: a packed batch of uneven 3D instances (instances of different
    cells per side, blocks straddling two instances), whole lockstep solves."""
    torch = torch_mod
    insts = [inputs.random_rects_3d(n, 22060304, k, 1 + k % 3, nrhs=nr, random_dirichlet=True)
             for k, n in enumerate([9, 12, 7, 10, 23])]
    sys_ = ctx.assemble_batch(insts)
    ps = ctx.setup(sys_, precision=precision, format="stencil-bulk")
    pc = ctx.setup(sys_, precision=precision, format="csr")
    assert ps.level_format(0, 0) == "stencil-bulk" and pc.level_format(0, 0) == "csr"
    xs = torch.zeros(sys_.N * nr, dtype=torch.float64, device="cuda")
    xc = torch.zeros_like(xs)
    c1, s1 = ctx.solve(sys_, ps, None, xs, nrhs=nr, max_iters=3000)
    c2, s2 = ctx.solve(sys_, pc, None, xc, nrhs=nr, max_iters=3000)
    assert c1 == c2 == 0
    assert [q.iterations for q in s1] == [q.iterations for q in s2]
    assert torch.equal(xs, xc)


@pytest.mark.parametrize("precision,nr,fmt", [("bf16", 4, "csr"), ("bf16", 4, "stencil"), ("fp32", 1, "sell"),
                                               ("fp64", 4, "stencil"), ("fp64", 1, "csr")])
def test_stored_level_form_is_fused_bit_for_bit(ctx, torch_mod, precision, nr, fmt):
    """The stored form of a level's smoothing (y = D1^-1 b, residual, y +=
    P x_c, smoothing from y: four launches) rounds as the fused pair does,
    which forms y per neighbour: whole lockstep solves of a packed batch of
    uneven 3D instances are equal bit for bit, on CSR, SELL and stencil
    storage, with BF16, FP32 and FP64 levels."""
    torch = torch_mod
    from paper_2206_03203_gb300 import mdsolve
    insts = [inputs.random_rects_3d(n, 22060304, k, 1 + k % 3, nrhs=nr, random_dirichlet=True)
             for k, n in enumerate([9, 12, 7, 10, 23])]
    sys_ = ctx.assemble_batch(insts)
    with pytest.raises(mdsolve.MDSError) as e:
        ctx.setup(sys_, precision=precision, format=fmt, level_form=3)
    assert e.value.code == -1
    pf = ctx.setup(sys_, precision=precision, format=fmt, level_form="fused")
    ps = ctx.setup(sys_, precision=precision, format=fmt, level_form="stored")
    xf = torch.zeros(sys_.N * nr, dtype=torch.float64, device="cuda")
    xs = torch.zeros_like(xf)
    c1, s1 = ctx.solve(sys_, pf, None, xf, nrhs=nr, max_iters=3000)
    c2, s2 = ctx.solve(sys_, ps, None, xs, nrhs=nr, max_iters=3000)
    assert c1 == c2 == 0
    assert [q.iterations for q in s1] == [q.iterations for q in s2]
    assert torch.equal(xf, xs)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_batched_graphs_match_direct_launches(ctx, torch_mod, precision):
    """The lockstep batched FGMRES replays each Arnoldi step as a CUDA graph
    (captured on its second use): solutions and iteration counts equal, bit
    for bit, those of the same solve with every kernel launched directly, on
    a packed batch whose problems stop at different steps and restart."""
    torch = torch_mod
    insts = [inputs.random_rects_3d(n, 22060304, k, 2 + k, nrhs=4, random_dirichlet=True)
             for k, n in enumerate([14, 9, 12, 10, 8])]
    sys_ = ctx.assemble_batch(insts)
    prec = ctx.setup(sys_, precision=precision)
    xs = []
    its = []
    for graphs in (1, 0):
        x = torch.zeros(sys_.N * 4, dtype=torch.float64, device="cuda")
        code, st = ctx.solve(sys_, prec, None, x, nrhs=4, restart=10, max_iters=3000, graphs=graphs)
        assert code == 0
        xs.append(x)
        its.append([q.iterations for q in st])
    assert its[0] == its[1] and max(its[0]) > 20  # several restart cycles replayed
    assert torch.equal(xs[0], xs[1])


def test_zero_initial_guess_option(ctx, torch_mod):
    """x0_zero: x is output only.  Host and device x filled with garbage give,
    bit for bit, the solution of the solve from an explicitly zeroed x, for a
    single instance and a packed batch."""
    torch = torch_mod
    for sys_ in (ctx.assemble(CASES["seg2d-96"]()),
                 ctx.assemble_batch([inputs.random_rects_3d(n, 7, k, 2, nrhs=2) for k, n in enumerate([9, 11, 8])])):
        nr = sys_.nrhs
        prec = ctx.setup(sys_, precision="bf16")
        ref = torch.zeros(sys_.N * nr, dtype=torch.float64, device="cuda")
        c0, s0 = ctx.solve(sys_, prec, None, ref, nrhs=nr)
        xd = torch.full_like(ref, float("nan"))
        c1, s1 = ctx.solve(sys_, prec, None, xd, nrhs=nr, x0_zero=True)
        xh = np.full(sys_.N * nr, 1e300)
        c2, s2 = ctx.solve(sys_, prec, None, xh, nrhs=nr, x0_zero=True)
        assert c0 == c1 == c2 == 0
        assert [q.iterations for q in s0] == [q.iterations for q in s1] == [q.iterations for q in s2]
        assert torch.equal(xd, ref)
        assert np.array_equal(xh, ref.cpu().numpy())


def test_pinned_host_batch_paths(ctx, oracle_mod, torch_mod):
    """A packed batch from page-locked host arrays (gathered by one kernel
    that reads host memory) assembles the oracle's system bit for bit, and a
    lockstep solve into a page-locked host x (written in place by the device)
    equals the solve into a device x bit for bit, with x0 read from the
    buffer and with x0_zero."""
    torch = torch_mod

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    insts = [inputs.random_rects_3d(n, 22060304, k, 1 + k % 4, nrhs=2, random_dirichlet=True)
             for k, n in enumerate([9, 12, 8, 14, 11])]
    import dataclasses
    ph = [dataclasses.replace(b, km=pinned(b.km), fc_axis=pinned(b.fc_axis), fc_pos=pinned(b.fc_pos),
                              fc_kf=pinned(b.fc_kf), fc_a=pinned(b.fc_a), pD_left=pinned(b.pD_left),
                              pD_right=pinned(b.pD_right)) for b in insts]
    sys_ = ctx.assemble_batch(ph)
    (_, _, _, _, A), b = sys_.to_host()
    Ao, bo, NM = packed_oracle(oracle_mod, insts)
    assert same_csr(A, Ao) and np.array_equal(b, bo)
    prec = ctx.setup(sys_, precision="bf16")
    xd = torch.zeros(2 * sys_.N, dtype=torch.float64, device="cuda")
    c0, s0 = ctx.solve(sys_, prec, None, xd, nrhs=2)
    xh = pinned(np.zeros(2 * sys_.N))
    c1, s1 = ctx.solve(sys_, prec, None, xh, nrhs=2)
    xz = pinned(np.full(2 * sys_.N, np.nan))
    c2, s2 = ctx.solve(sys_, prec, None, xz, nrhs=2, x0_zero=True)
    assert c0 == c1 == c2 == 0
    assert [q.iterations for q in s0] == [q.iterations for q in s1] == [q.iterations for q in s2]
    ref = xd.cpu().numpy()
    assert np.array_equal(xh, ref) and np.array_equal(xz, ref)
