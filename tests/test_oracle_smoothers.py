"""Pins of the oracle's smoothers (Sec. 3.3: one V-cycle per block; Sec. 4
uses Gauss-Seidel, this solver L1-Jacobi or Chebyshev).

On a one-level hierarchy the V-cycle is pre-smoothing from zero followed by
post-smoothing, so its residual has a closed form: for Chebyshev of degree k
on D1^-1 A over [0.3, 1] the residual polynomial is
R_k(t) = T_k((theta - t) / delta) / T_k(theta / delta), applied twice; for
Gauss-Seidel it is a forward then a backward triangular solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2206_03203_gb300 import inputs


def small_matrix(oracle_mod):
    inst = inputs.random_segments_2d(n=12, n_seg=4, contrast=10.0)
    A, _ = oracle_mod.assemble(inst)
    return A.tocsr()


def l1_diag(A):
    d = A.diagonal()
    off = abs(A).sum(axis=1).A1 - np.abs(d)
    return d + off


@pytest.mark.parametrize("degree", [1, 2, 3, 4, 6])
def test_chebyshev_residual_polynomial(oracle_mod, degree):
    A = small_matrix(oracle_mod)
    amg = oracle_mod.AMG(A, max_levels=1, n_coarse=1, smoother=1, cheb_degree=degree)
    assert amg.nlevels == 1 and not amg.coarsest_dense
    b = np.random.default_rng(degree).standard_normal(A.shape[0])
    x = amg.vcycle(b)
    D = l1_diag(A)
    Dh = np.sqrt(D)
    S = (A.toarray() / Dh[:, None]) / Dh[None, :]
    lam, Q = np.linalg.eigh(S)
    assert lam.max() <= 1.0 + 1e-12  # L1 diagonal bound
    theta, delta = 0.65, 0.35
    R = np.polynomial.chebyshev.chebval((theta - lam) / delta, [0] * degree + [1]) / \
        np.polynomial.chebyshev.chebval(theta / delta, [0] * degree + [1])
    r_expected = Dh * (Q @ (R ** 2 * (Q.T @ (b / Dh))))
    r = b - A @ x
    assert np.linalg.norm(r - r_expected) <= 1e-11 * np.linalg.norm(b)


def test_gauss_seidel_one_level_is_forward_then_backward(oracle_mod):
    A = small_matrix(oracle_mod)
    amg = oracle_mod.AMG(A, max_levels=1, n_coarse=1, smoother=2)
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    x = amg.vcycle(b)
    lower = sp.tril(A, format="csr")
    upper = sp.triu(A, format="csr")
    x1 = spla.spsolve_triangular(lower, b, lower=True)
    x2 = x1 + spla.spsolve_triangular(upper, b - A @ x1, lower=False)
    assert np.linalg.norm(x - x2) <= 1e-13 * np.linalg.norm(x2)


@pytest.mark.parametrize("smoother,kw", [(2, {}), (1, {"cheb_degree": 3}), (0, {})])
def test_multilevel_vcycle_is_symmetric(oracle_mod, smoother, kw):
    """Forward Gauss-Seidel before and backward after the coarse correction
    (and the same polynomial for Chebyshev / L1-Jacobi) make the V-cycle a
    symmetric operator."""
    inst = inputs.fixed_2d(n=32)
    A, _ = oracle_mod.assemble(inst)
    amg = oracle_mod.AMG(A.tocsr(), n_coarse=16, smoother=smoother, **kw)
    assert amg.nlevels >= 3
    rng = np.random.default_rng(9)
    v, w = rng.standard_normal((2, A.shape[0]))
    a, c = v @ amg.vcycle(w), w @ amg.vcycle(v)
    assert abs(a - c) <= 1e-12 * max(abs(a), abs(c))
    assert v @ amg.vcycle(v) > 0.0


def test_smoother_iteration_counts(oracle_mod, capsys):
    """M_L + FGMRES with each smoother on a 128^2 random-segment instance at
    three contrasts: all converge; the counts are recorded for comparison
    with the paper's Gauss-Seidel."""
    rows = []
    for c in (1e-4, 1.0, 1e4):
        inst = inputs.random_segments_2d(n=128, n_seg=16, contrast=c)
        A, b = oracle_mod.assemble(inst)
        its = []
        for smoother, kw in ((0, {}), (1, {}), (1, {"cheb_degree": 3}), (2, {})):
            M = oracle_mod.ML(A, inst.n_m, smoother=smoother, **kw)
            res = oracle_mod.fgmres(A, b[0], M, rtol=1e-8, maxit=3000)
            assert res.converged
            its.append(res.iterations)
        rows.append((c, its))
    with capsys.disabled():
        for c, its in rows:
            print(f"\n  contrast {c:g}: L1-Jacobi {its[0]}, Chebyshev-2 {its[1]}, Chebyshev-3 {its[2]}, "
                  f"Gauss-Seidel {its[3]}", end="")
