"""Pins of the oracle's two-point-flux assembly (Sec. 2.1, Eq. (1)-(3), and the
block system of Eq. (4)) against closed forms and invariants."""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2206_03203_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def solve(A, b):
    return spla.spsolve(A.tocsc(), b)


def centres(n, dim):
    c = (np.arange(n) + 0.5) / n
    if dim == 2:
        return np.tile(c, n)
    return np.tile(c, n * n)


@pytest.mark.parametrize("dim,n", [(2, 8), (2, 16), (3, 6)])
def test_linear_field_exact_without_fractures(oracle_mod, dim, n):
    inst = inputs.make_instance("lin", dim, n, np.ones(n ** dim), [])
    A, b = oracle_mod.assemble(inst)
    p = solve(A, b[0])
    assert np.max(np.abs(p - (1.0 - centres(n, dim)))) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_parallel_fractures_keep_linear_field(oracle_mod, dim):
    """Fractures spanning x between the two Dirichlet faces carry flow in
    parallel with the matrix; the field stays linear in x."""
    n = 8
    kf, a = 37.0, 1e-2
    if dim == 2:
        rects = [inputs.Rect(1, 3, (0,), (n,), kf, a), inputs.Rect(1, 6, (0,), (n,), 2 * kf, a)]
    else:
        rects = [inputs.Rect(1, 3, (0, 0), (n, n), kf, a)]
    inst = inputs.make_instance("par", dim, n, np.ones(n ** dim), rects)
    A, b = oracle_mod.assemble(inst)
    p = solve(A, b[0])
    nm = inst.n_m
    assert np.max(np.abs(p[:nm] - (1.0 - centres(n, dim)))) < 1e-12
    # fracture cells sit at the centres of their x-cells
    xf = (inst.fc_pos[:, 0] + 0.5) / n
    assert np.max(np.abs(p[nm:] - (1.0 - xf))) < 1e-12
    # total inflow at x=0: matrix k_m |boundary| + sum k_f a (per unit height in 2D, per
    # unit length of intersection line with the boundary in 3D)
    r = A @ p - b[0]
    left = np.zeros(A.shape[0], dtype=bool)
    left[:nm] = centres(n, dim) < 1.0 / n
    left[nm:] = inst.fc_pos[:, 0] == 0
    # A p - b = 0 everywhere; inflow is the Dirichlet term b_i - T_b p_i summed over left rows
    Tb = np.asarray(A.sum(axis=1)).ravel()  # row sums equal the Dirichlet coefficients
    inflow = np.sum((Tb * (1.0 - p))[left])
    expected = 1.0 + (sum(r_.kf * r_.a for r_ in rects) if dim == 2 else kf * a * 1.0)
    assert abs(inflow - expected) < 1e-10 * expected
    assert np.max(np.abs(r)) < 1e-10


@pytest.mark.parametrize("kf,a", [(1e-4, 1e-4), (3.0, 0.05), (1e4, 1e-4)])
def test_series_fracture_closed_form(oracle_mod, kf, a):
    """A full-height fracture normal to x is a resistance a/k_f in series with
    the matrix (kappa = 2 k_f / a on each side): q = 1 / (1/k_m + a/k_f)."""
    n = 8
    inst = inputs.make_instance("ser", 2, n, np.ones(n * n), [inputs.Rect(0, 4, (0,), (n,), kf, a)])
    A, b = oracle_mod.assemble(inst)
    p = solve(A, b[0])
    q = 1.0 / (1.0 + a / kf)
    h = 1.0 / n
    # inflow through x=0 (total boundary length 1)
    pl = p[:inst.n_m].reshape(n, n)[:, 0]
    inflow = np.sum(2.0 * (1.0 - pl))  # T_b = |F| 2 k / h = 2 with |F| = h, k = 1
    assert abs(inflow - q) < 1e-12
    # jump across the fracture: q a / k_f between the two matrix cells beyond half cells
    pm = p[:inst.n_m].reshape(n, n)
    jump = pm[:, 3] - pm[:, 4]
    assert np.max(np.abs(jump - q * (h + a / kf))) < 1e-12
    assert np.max(np.abs(p[inst.n_m:] - 0.5 * (pm[:, 3] + pm[:, 4]))) < 1e-12


def test_layered_permeability_harmonic(oracle_mod):
    n = 8
    kx = np.array([1.0, 4.0, 0.25, 2.0, 8.0, 1.0, 0.5, 3.0])
    km = np.tile(kx, n)
    inst = inputs.make_instance("lay", 2, n, km, [])
    A, b = oracle_mod.assemble(inst)
    p = solve(A, b[0])
    h = 1.0 / n
    q = 1.0 / np.sum(h / kx)
    # p at centre of cell i: 1 - q (h/(2k_0) + sum_{j<i} h/k_j ... ) with half cells
    pc = np.empty(n)
    acc = h / (2 * kx[0])
    pc[0] = 1.0 - q * acc
    for i in range(1, n):
        acc += h / (2 * kx[i - 1]) + h / (2 * kx[i])
        pc[i] = 1.0 - q * acc
    assert np.max(np.abs(p.reshape(n, n) - pc[None, :])) < 1e-12


def test_counts_match_hand_derivation(oracle_mod):
    gold = dict(l.split() for l in open(os.path.join(GOLD, "fixed_2d_64_counts.txt")) if not l.startswith("#"))
    inst = inputs.fixed_2d()
    A, _ = oracle_mod.assemble(inst)
    Amm, Amf, Afm, Aff = oracle_mod.split(A, inst.n_m)
    assert inst.n_m == int(gold["n_m"]) and inst.n_f == int(gold["n_f"])
    assert (Amm.nnz, Amf.nnz, Afm.nnz, Aff.nnz) == tuple(int(gold[k]) for k in ("nnz_mm", "nnz_mf", "nnz_fm", "nnz_ff"))


def test_planes_3d_counts_closed_form(oracle_mod):
    n = 8
    inst = inputs.planes_3d(n=n)
    A, _ = oracle_mod.assemble(inst)
    Amm, Amf, Afm, Aff = oracle_mod.split(A, inst.n_m)
    assert Amm.nnz == n ** 3 + 2 * (3 * n * n * (n - 1) - 9 * n * n)
    assert Amf.nnz == 2 * 9 * n * n
    pairs = 18 * n * (n - 1) + 108 * n  # in-plane pairs plus 6 pairs on 27 n crossing edges
    assert Aff.nnz == 9 * n * n + 2 * pairs


@pytest.mark.parametrize("make", [lambda: inputs.fixed_2d(n=16), lambda: inputs.planes_3d(n=8, kf=1.0),
                                  lambda: inputs.random_segments_2d(n=32, n_seg=8),
                                  lambda: inputs.random_rects_3d(8, 5, 0, 4)])
def test_invariants(oracle_mod, make):
    inst = make()
    A, b = oracle_mod.assemble(inst)
    nm = inst.n_m
    # exact symmetry, A_mf = A_fm^T (Sec. 3.1)
    assert (A - A.T).nnz == 0 or np.max(np.abs((A - A.T).data)) == 0.0
    Amm, Amf, Afm, Aff = oracle_mod.split(A, nm)
    assert np.array_equal((Amf - Afm.T).toarray(), np.zeros(Amf.shape))
    # M-matrix signs
    d = A.diagonal()
    assert np.all(d > 0)
    off = A - sp.diags(d)
    assert np.all(off.data <= 0)
    # row sums are the Dirichlet coefficients: zero for interior rows
    rs = np.asarray(A.sum(axis=1)).ravel()
    assert np.all(rs > -1e-12 * d)
    has_dir = np.zeros(A.shape[0], dtype=bool)
    has_dir[:nm] = (np.arange(nm) % inst.n == 0) | (np.arange(nm) % inst.n == inst.n - 1)
    has_dir[nm:] = (inst.fc_axis != 0) & ((inst.fc_pos[:, 0] == 0) | (inst.fc_pos[:, 0] == inst.n - 1))
    assert np.all(np.abs(rs[~has_dir]) <= 1e-12 * d[~has_dir])
    assert np.all(rs[has_dir] > 0)
    # SPD (dense Cholesky) on small systems
    if A.shape[0] < 3000:
        np.linalg.cholesky(A.toarray())
    # mass conservation of the solution: inflow = outflow
    p = solve(A, b[0])
    res = A @ p - b[0]
    assert np.max(np.abs(res)) < 1e-9 * np.max(np.abs(b[0]))


def test_crossing_pairwise_transmissibility(oracle_mod):
    """At a crossing, each of the four fracture cells is linked to the other
    three by t_i t_j / (t_i + t_j) with t = k_f a / (h/2) in 2D."""
    n = 8
    kf1, kf2, a = 2.0, 6.0, 0.1
    rects = [inputs.Rect(0, 4, (0,), (n,), kf1, a), inputs.Rect(1, 4, (0,), (n,), kf2, a)]
    inst = inputs.make_instance("x", 2, n, np.ones(n * n), rects)
    A, _ = oracle_mod.assemble(inst)
    nm = inst.n_m
    h = 1.0 / n
    t1, t2 = kf1 * a / (h / 2), kf2 * a / (h / 2)
    pos = {(int(ax), int(p[0]), int(p[1])): k for k, (ax, p) in enumerate(zip(inst.fc_axis, inst.fc_pos))}
    v_lo, v_hi = pos[(0, 4, 3)], pos[(0, 4, 4)]     # x-normal cells below/above y=4
    h_lo, h_hi = pos[(1, 3, 4)], pos[(1, 4, 4)]     # y-normal cells left/right of x=4
    Ad = A.toarray()
    f = lambda i, j: -Ad[nm + i, nm + j]
    assert f(v_lo, v_hi) == pytest.approx(t1 / 2, rel=1e-15)
    assert f(h_lo, h_hi) == pytest.approx(t2 / 2, rel=1e-15)
    assert f(v_lo, h_lo) == pytest.approx(t1 * t2 / (t1 + t2), rel=1e-15)
    assert f(v_hi, h_hi) == pytest.approx(t1 * t2 / (t1 + t2), rel=1e-15)
    # the crossing links are the only extra couplings of a crossing cell
    assert np.count_nonzero(Ad[nm + v_lo, nm:]) == 1 + 1 + 1 + 2  # self, below, above, 2 horizontals


def test_fracture_end_on_dirichlet_face(oracle_mod):
    """A fracture cell whose end edge lies on x=0 gets T_b = t and b = t p_D."""
    n = 8
    kf, a = 5.0, 0.02
    inst = inputs.make_instance("e", 2, n, np.ones(n * n), [inputs.Rect(1, 4, (0,), (2,), kf, a)])
    A, b = oracle_mod.assemble(inst)
    nm = inst.n_m
    t = kf * a / (0.5 / n)
    assert b[0][nm + 0] == pytest.approx(t * 1.0, rel=1e-15)
    assert A.sum(axis=1)[nm + 0, 0] == pytest.approx(t, rel=1e-12)
    assert b[0][nm + 1] == 0.0


def test_rejects_duplicate_face(oracle_mod):
    inst = inputs.make_instance("d", 2, 8, np.ones(64), [inputs.Rect(0, 4, (0,), (2,), 1.0, 1.0)])
    inst.fc_pos = np.vstack([inst.fc_pos, inst.fc_pos[:1]])
    inst.fc_axis = np.concatenate([inst.fc_axis, inst.fc_axis[:1]])
    inst.fc_kf = np.concatenate([inst.fc_kf, inst.fc_kf[:1]])
    inst.fc_a = np.concatenate([inst.fc_a, inst.fc_a[:1]])
    with pytest.raises(ValueError):
        oracle_mod.assemble(inst)
