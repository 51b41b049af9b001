"""Pins of the oracle's block preconditioners (Sec. 3.2, Eq. (8), Algorithm 1)
and Krylov solvers (right-preconditioned FGMRES, PCG)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2206_03203_gb300 import inputs


def isolated_instance():
    """One-cell fractures that touch nothing: A_ff is diagonal, so S~ = S."""
    n = 12
    rects = [inputs.Rect(0, 3, (2,), (3,), 50.0, 1e-2), inputs.Rect(1, 7, (5,), (6,), 1e-3, 1e-2),
             inputs.Rect(0, 9, (8,), (9,), 7.0, 1e-3)]
    return inputs.make_instance("iso", 2, n, np.linspace(0.5, 2, n * n), rects)


def test_exact_block_lower_converges_in_two_steps(oracle_mod):
    """A B_L = U has (U - I)^2 = 0 (Sec. 3.2): GMRES stops after <= 2 steps."""
    inst = inputs.fixed_2d(n=16)
    A, b = oracle_mod.assemble(inst)
    nm = inst.n_m
    Amm, Amf, Afm, Aff = oracle_mod.split(A, nm)
    S = Amm.toarray() - Amf.toarray() @ np.linalg.solve(Aff.toarray(), Afm.toarray())
    Fi = np.linalg.inv(Aff.toarray())
    Si = np.linalg.inv(S)
    Afm_d = Afm.toarray()

    def BL(r):
        zm = Si @ r[:nm]
        return np.concatenate([zm, Fi @ (r[nm:] - Afm_d @ zm)])

    res = oracle_mod.fgmres(A, b[0], BL, rtol=1e-12, maxit=50)
    assert res.converged and res.iterations <= 2


def test_oracle_ML_is_block_lower_solve(oracle_mod):
    """With one-level (exact) block solves, Algorithm 1 applies
    [S~ 0; A_fm A_ff]^-1 exactly."""
    inst = inputs.fixed_2d(n=16)
    A, b = oracle_mod.assemble(inst)
    nm = inst.n_m
    M = oracle_mod.ML(A, nm, n_coarse=100000)
    Amm, Amf, Afm, Aff = oracle_mod.split(A, nm)
    S = oracle_mod.schur(Amm, Amf, Afm, Aff).toarray()
    N = A.shape[0]
    BL = np.zeros((N, N))
    BL[:nm, :nm] = S
    BL[nm:, :nm] = Afm.toarray()
    BL[nm:, nm:] = Aff.toarray()
    r = np.random.default_rng(3).standard_normal(N)
    z = M.apply(r)
    assert np.max(np.abs(BL @ z - r)) < 1e-11 * np.max(np.abs(r))
    # block diagonal and block upper variants
    D = oracle_mod.ML(A, nm, kind="diag", n_coarse=100000).apply(r)
    BD = BL.copy()
    BD[nm:, :nm] = 0
    assert np.max(np.abs(BD @ D - r)) < 1e-11 * np.max(np.abs(r))
    U = oracle_mod.ML(A, nm, kind="upper", n_coarse=100000).apply(r)
    BU = BD.copy()
    BU[:nm, nm:] = Amf.toarray()
    assert np.max(np.abs(BU @ U - r)) < 1e-11 * np.max(np.abs(r))


def test_oracle_ML_two_steps_when_schur_is_exact(oracle_mod):
    inst = isolated_instance()
    A, b = oracle_mod.assemble(inst)
    M = oracle_mod.ML(A, inst.n_m, n_coarse=100000)
    res = oracle_mod.fgmres(A, b[0], M, rtol=1e-12, maxit=50)
    assert res.converged and res.iterations <= 2


def test_identity_fgmres_is_gmres_finite_termination(oracle_mod):
    rng = np.random.default_rng(1)
    n = 25
    A = sp.csr_matrix(np.diag(np.arange(1, n + 1.0)) + 0.3 * rng.standard_normal((n, n)))
    b = rng.standard_normal(n)
    res = oracle_mod.fgmres(A, b, "identity", restart=30, rtol=1e-12, maxit=100)
    assert res.converged and res.iterations <= n
    assert np.allclose(res.x, np.linalg.solve(A.toarray(), b), rtol=1e-9, atol=1e-9)
    # estimates are monotone within the cycle
    assert np.all(np.diff(res.history) <= 1e-14)


def test_fgmres_restarted_matches_direct_solve(oracle_mod):
    inst = inputs.fixed_2d(n=32)
    A, b = oracle_mod.assemble(inst)
    M = oracle_mod.ML(A, inst.n_m)
    res = oracle_mod.fgmres(A, b[0], M, restart=5, rtol=1e-10, maxit=500)
    assert res.converged and res.restarts >= 2
    xd = spla.spsolve(A.tocsc(), b[0])
    assert np.linalg.norm(A @ res.x - b[0]) <= 1e-10 * np.linalg.norm(b[0]) * 1.0001
    assert np.max(np.abs(res.x - xd)) < 1e-6
    assert res.relres <= 1e-10


def test_fgmres_nonzero_initial_guess(oracle_mod):
    inst = inputs.fixed_2d(n=16)
    A, b = oracle_mod.assemble(inst)
    M = oracle_mod.ML(A, inst.n_m)
    xd = spla.spsolve(A.tocsc(), b[0])
    res = oracle_mod.fgmres(A, b[0], M, x0=xd, rtol=1e-8)
    assert res.iterations == 0 and res.converged


def test_pcg_block_diagonal(oracle_mod):
    inst = inputs.planes_3d(n=8, kf=1.0)
    A, b = oracle_mod.assemble(inst)
    M = oracle_mod.ML(A, inst.n_m, kind="diag")
    res = oracle_mod.pcg(A, b[0], M, rtol=1e-8, maxit=500)
    assert res.converged
    xd = spla.spsolve(A.tocsc(), b[0])
    assert np.max(np.abs(res.x - xd)) < 1e-6
    # PCG with identity on an SPD system: finite termination in exact arithmetic
    rng = np.random.default_rng(2)
    Q = rng.standard_normal((20, 20))
    S = sp.csr_matrix(Q @ Q.T + 20 * np.eye(20))
    r2 = oracle_mod.pcg(S, rng.standard_normal(20), "identity", rtol=1e-12, maxit=40)
    assert r2.converged and r2.iterations <= 20


@pytest.mark.parametrize("make", [lambda: inputs.fixed_2d(), lambda: inputs.planes_3d(n=16)])
def test_solve_against_direct(oracle_mod, make):
    inst = make()
    res, A, b, M = oracle_mod.solve(inst)
    assert res.converged and res.relres <= 1e-8
    xd = spla.spsolve(A.tocsc(), b[0])
    assert np.max(np.abs(res.x - xd)) < 1e-5


def test_mixed_precision_emulation_converges(oracle_mod):
    inst = inputs.fixed_2d()
    r64, A, b, _ = oracle_mod.solve(inst)
    r32, *_ = oracle_mod.solve(inst, prec=32)
    r16, *_ = oracle_mod.solve(inst, prec=16)
    assert r32.converged and r16.converged
    assert abs(r32.iterations - r64.iterations) <= 3
    assert r16.iterations <= r64.iterations + 10


def _krylov_lsq(A, b, k):
    """argmin ||b - A x||_2 over x in span{b, A b, ..., A^(k-1) b}, by an
    explicit QR of the Krylov matrix (brute force, small k)."""
    K = np.empty((A.shape[0], k))
    v = b.copy()
    for j in range(k):
        K[:, j] = v / np.linalg.norm(v)
        v = A @ K[:, j]
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
    return Q @ y


def test_minres_minimises_residual_over_krylov_space(oracle_mod):
    """MINRES with the identity preconditioner: the k-th iterate is the
    minimum-residual point of the k-th Krylov space (symmetric indefinite
    matrix, where CG has no such property), and the 2-norm residual never
    grows."""
    rng = np.random.default_rng(11)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([np.linspace(-3.0, -0.5, 12), np.linspace(0.7, 5.0, n - 12)])
    Ad = (Q * lam) @ Q.T
    Ad = 0.5 * (Ad + Ad.T)
    A = sp.csr_matrix(Ad)
    b = rng.standard_normal(n)
    for k in (1, 3, 6, 10):
        res = oracle_mod.minres(A, b, "identity", rtol=1e-300, maxit=k)
        assert res.iterations == k
        xk = _krylov_lsq(Ad, b, k)
        assert np.linalg.norm(res.x - xk) <= 1e-8 * (1 + np.linalg.norm(xk)), k
    full = oracle_mod.minres(A, b, "identity", rtol=1e-10, maxit=200)
    assert full.converged
    assert np.all(np.diff(full.history) <= 1e-12)
    assert np.linalg.norm(full.x - np.linalg.solve(Ad, b)) <= 1e-7 * np.linalg.norm(np.linalg.solve(Ad, b))


def test_minres_preconditioned_norm_decreases(oracle_mod):
    """With an SPD preconditioner M, the iterates minimise the residual in the
    M-inverse norm over the preconditioned Krylov space: that norm never
    grows with k (checked by restarting the solve with more steps)."""
    rng = np.random.default_rng(5)
    n = 24
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([np.linspace(-2.0, -0.3, 8), np.linspace(0.4, 6.0, n - 8)])
    Ad = (Q * lam) @ Q.T
    Ad = 0.5 * (Ad + Ad.T)
    A = sp.csr_matrix(Ad)
    G = rng.standard_normal((n, n))
    Md = G @ G.T / n + np.eye(n)  # SPD preconditioner (applied as M^-1 = Md)
    Mi = np.linalg.inv(Md)
    b = rng.standard_normal(n)
    norms = []
    for k in range(1, 14):
        res = oracle_mod.minres(A, b, lambda r: Md @ r, rtol=1e-300, maxit=k)
        r = b - Ad @ res.x
        norms.append(np.sqrt(r @ (Md @ r)))
    assert all(b_ <= a_ * (1 + 1e-10) for a_, b_ in zip(norms, norms[1:]))
    full = oracle_mod.minres(A, b, lambda r: Md @ r, rtol=1e-10, maxit=400)
    assert full.converged
    assert np.linalg.norm(full.x - np.linalg.solve(Ad, b)) <= 1e-7 * np.linalg.norm(np.linalg.solve(Ad, b))
    del Mi


def test_minres_block_diagonal_on_assembled_system(oracle_mod):
    """B_D (one symmetric V-cycle per block) with MINRES on the assembled
    mixed-dimensional system reaches the direct solution."""
    inst = inputs.planes_3d(n=8, kf=1.0)
    res, A, b, M = oracle_mod.solve(inst, kind="diag", krylov="minres", maxit=500)
    assert res.converged and res.relres <= 1e-8
    xd = spla.spsolve(A.tocsc(), b[0])
    assert np.max(np.abs(res.x - xd)) < 1e-6
    pc, *_ = oracle_mod.solve(inst, kind="diag", krylov="pcg", maxit=500)
    assert abs(res.iterations - pc.iterations) <= max(3, pc.iterations // 4)
