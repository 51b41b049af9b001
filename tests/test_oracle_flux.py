"""Pins of the oracle's assembly in the paper's own partition (Sec. 3.1,
Eq. (4)): unknowns [pressures of every cell; interface fluxes], and of the
solver on that symmetric saddle-point system.

The flux form must reduce to the primal two-point-flux system when the
interface fluxes are eliminated (the Schur complement of the diagonal flux
block is exact), which pins every block against the independently pinned
primal assembly."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2206_03203_gb300 import inputs

CASES = {
    "fixed2d-16": lambda: inputs.fixed_2d(n=16),
    "seg2d-40": lambda: inputs.random_segments_2d(n=40, n_seg=8, contrast=1e3),
    "planes3d-8": lambda: inputs.planes_3d(n=8, kf=1e-2),
    "rects3d-10": lambda: inputs.random_rects_3d(10, 22060305, 0, 4, sigma=2.0),
}


def blocks(A, n):
    A = A.tocsr()
    return A[:n, :n], A[:n, n:], A[n:, :n], A[n:, n:]


@pytest.mark.parametrize("case", list(CASES))
def test_flux_form_structure(oracle_mod, case):
    inst = CASES[case]()
    Af, bf = oracle_mod.assemble(inst, form="flux")
    N, nf = inst.n_m + inst.n_f, inst.n_f
    assert Af.shape == (N + 2 * nf, N + 2 * nf)
    assert abs(Af - Af.T).max() == 0.0  # exactly symmetric
    Aoo, Aog, Ago, Agg = blocks(Af, N)
    assert (Agg - sp.diags(Agg.diagonal())).nnz == 0 and np.all(Agg.diagonal() < 0)
    # every flux couples one matrix cell (+1) and one fracture cell (-1)
    G = Ago.tocsr()
    for j in range(2 * nf):
        cols, vals = G.indices[G.indptr[j]:G.indptr[j + 1]], G.data[G.indptr[j]:G.indptr[j + 1]]
        assert len(cols) == 2 and cols[0] < inst.n_m <= cols[1] and list(vals) == [1.0, -1.0]
        assert cols[1] == inst.n_m + j // 2
    # pressure block: no matrix-fracture coupling left
    assert Aoo[:inst.n_m, inst.n_m:].nnz == 0
    assert np.all(bf[:, N:] == 0.0)


@pytest.mark.parametrize("case", list(CASES))
def test_flux_elimination_gives_primal(oracle_mod, case):
    """A_OO - A_OG A_GG^-1 A_GO is the primal matrix (to rounding) and the
    pressure right-hand side is the primal one exactly."""
    inst = CASES[case]()
    A, b = oracle_mod.assemble(inst)
    Af, bf = oracle_mod.assemble(inst, form="flux")
    N = inst.n_m + inst.n_f
    Aoo, Aog, Ago, Agg = blocks(Af, N)
    S = (Aoo - Aog @ sp.diags(1.0 / Agg.diagonal()) @ Ago).tocsr()
    D = (S - A).tocsr()
    assert np.max(np.abs(D.data), initial=0.0) <= 1e-13 * np.max(np.abs(A.data))
    assert np.array_equal(bf[:, :N], b)
    # Eq. (7) on this partition is exact (A_GG is diagonal): the oracle's S~
    St = oracle_mod.schur(Aoo, Aog, Ago, Agg)
    D2 = (St - A).tocsr()
    assert np.max(np.abs(D2.data), initial=0.0) <= 1e-13 * np.max(np.abs(A.data))


@pytest.mark.parametrize("case", list(CASES))
def test_flux_solution_is_primal_solution(oracle_mod, case):
    """Direct solves: the pressures agree with the primal solution and each
    flux is T (p_i - p_k)."""
    inst = CASES[case]()
    A, b = oracle_mod.assemble(inst)
    Af, bf = oracle_mod.assemble(inst, form="flux")
    N = inst.n_m + inst.n_f
    p = spla.spsolve(A.tocsc(), b[0])
    y = spla.spsolve(Af.tocsc(), bf[0])
    assert np.max(np.abs(y[:N] - p)) <= 1e-9 * max(1.0, np.max(np.abs(p)))
    Agg = Af.tocsr()[N:, N:].diagonal()
    Ago = Af.tocsr()[N:, :N]
    lam = (Ago @ p) / (-Agg)  # lambda_j = T_j (p_i - p_k)
    assert np.max(np.abs(y[N:] - lam)) <= 1e-8 * max(1.0, np.max(np.abs(lam)))


def test_no_fractures_flux_form_is_primal(oracle_mod):
    inst = inputs.make_instance("plain", 2, 12, np.linspace(1, 3, 144), [])
    A, b = oracle_mod.assemble(inst)
    Af, bf = oracle_mod.assemble(inst, form="flux")
    assert (A != Af).nnz == 0 and np.array_equal(b, bf)


def test_flux_block_hierarchy_is_exact_diagonal(oracle_mod):
    """The flux block has no couplings: its hierarchy is one level solved by
    x = b / a_ii (neither coarsened nor factored, whatever its size)."""
    for inst in (inputs.fixed_2d(n=16), inputs.random_segments_2d(n=64, n_seg=12)):
        Af, bf = oracle_mod.assemble(inst, form="flux")
        N = inst.n_m + inst.n_f
        M = oracle_mod.ML(Af, N)
        amg = M.amg(1)
        assert amg.nlevels == 1 and amg.coarsest_diagonal and not amg.coarsest_dense
        r = np.random.default_rng(3).standard_normal(2 * inst.n_f)
        d = Af.tocsr()[N:, N:].diagonal()
        assert np.array_equal(amg.vcycle(r), d ** -1 * r) or np.allclose(amg.vcycle(r), r / d, rtol=1e-15)


@pytest.mark.parametrize("case", ["fixed2d-16", "seg2d-40", "planes3d-8"])
def test_flux_form_solves(oracle_mod, case):
    """M_L + FGMRES and B_D + MINRES (B_D positive definite: its flux block is
    -A_GG^-1) reach the direct solution of the saddle-point system."""
    inst = CASES[case]()
    Af, bf = oracle_mod.assemble(inst, form="flux")
    N = inst.n_m + inst.n_f
    y = spla.spsolve(Af.tocsc(), bf[0])
    ML = oracle_mod.ML(Af, N)
    r1 = oracle_mod.fgmres(Af, bf[0], ML, rtol=1e-10, maxit=3000)
    assert r1.converged and np.max(np.abs(r1.x - y)) <= 1e-6 * max(1.0, np.max(np.abs(y)))
    BD = oracle_mod.ML(Af, N, kind="diag")
    rng = np.random.default_rng(4)
    for _ in range(3):
        v = rng.standard_normal(Af.shape[0])
        assert v @ BD.apply(v) > 0.0
    r2 = oracle_mod.minres(Af, bf[0], BD, rtol=1e-10, maxit=5000)
    assert r2.converged and np.max(np.abs(r2.x - y)) <= 1e-6 * max(1.0, np.max(np.abs(y)))
