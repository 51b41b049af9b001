"""Pins of the oracle's Schur complement (Eq. (7)) and aggregation AMG
(Sec. 3.3) against dense brute force, textbook identities and invariants."""
from collections import deque

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2206_03203_gb300 import inputs


def blocks(oracle_mod, inst):
    A, b = oracle_mod.assemble(inst)
    return (A, b) + tuple(oracle_mod.split(A, inst.n_m))


@pytest.mark.parametrize("make", [lambda: inputs.fixed_2d(n=16), lambda: inputs.planes_3d(n=8),
                                  lambda: inputs.random_segments_2d(n=32, n_seg=8)])
def test_schur_dense_brute_force(oracle_mod, make):
    inst = make()
    A, b, Amm, Amf, Afm, Aff = blocks(oracle_mod, inst)
    S = oracle_mod.schur(Amm, Amf, Afm, Aff).toarray()
    d = Aff.diagonal()
    ref = Amm.toarray() - Amf.toarray() @ np.diag(1.0 / d) @ Afm.toarray()
    assert np.max(np.abs(S - ref)) <= 1e-14 * np.max(np.abs(ref))
    # symmetric weakly diagonally dominant M-matrix
    assert np.array_equal(S, S.T)
    assert np.all(np.diag(S) > 0)
    off = S - np.diag(np.diag(S))
    assert np.all(off <= 0)
    assert np.all(S.sum(axis=1) >= -1e-12 * np.diag(S))


def test_schur_sparsity_is_uncut_stencil(oracle_mod):
    inst = inputs.fixed_2d(n=16)
    A, b, Amm, Amf, Afm, Aff = blocks(oracle_mod, inst)
    S = oracle_mod.schur(Amm, Amf, Afm, Aff)
    plain = inputs.make_instance("p", 2, 16, np.ones(256), [])
    A0, _ = oracle_mod.assemble(plain)
    assert np.array_equal(S.indptr, A0.indptr) and np.array_equal(S.indices, A0.indices)


def test_schur_exact_when_fracture_block_is_diagonal(oracle_mod):
    """Isolated one-cell fractures (no fracture-fracture links): A_ff is
    diagonal, so S~ equals the exact Schur complement of Eq. (6)."""
    n = 12
    rects = [inputs.Rect(0, 3, (2,), (3,), 50.0, 1e-2), inputs.Rect(1, 7, (5,), (6,), 1e-3, 1e-2),
             inputs.Rect(0, 9, (8,), (9,), 7.0, 1e-3)]
    inst = inputs.make_instance("iso", 2, n, np.linspace(0.5, 2, n * n), rects)
    A, b, Amm, Amf, Afm, Aff = blocks(oracle_mod, inst)
    assert Aff.nnz == Aff.shape[0]
    S = oracle_mod.schur(Amm, Amf, Afm, Aff).toarray()
    exact = Amm.toarray() - Amf.toarray() @ np.linalg.inv(Aff.toarray()) @ Afm.toarray()
    assert np.max(np.abs(S - exact)) <= 1e-13 * np.max(np.abs(exact))


def test_schur_entry_closed_form(oracle_mod):
    """One fracture cell k between matrix cells i, j: S_ij = A_ij - T_ik T_jk / d_k
    with A_ij = 0 (the link is cut)."""
    n = 6
    inst = inputs.make_instance("one", 2, n, np.ones(n * n), [inputs.Rect(0, 3, (2,), (3,), 4.0, 0.01)])
    A, b, Amm, Amf, Afm, Aff = blocks(oracle_mod, inst)
    S = oracle_mod.schur(Amm, Amf, Afm, Aff).toarray()
    i, j = 2 + n * 2, 3 + n * 2
    h = 1.0 / n
    T = h / (h / 2 + 1.0 / (2 * 4.0 / 0.01))
    d = 2 * T
    assert Amm[i, j] == 0.0
    assert S[i, j] == pytest.approx(-T * T / d, rel=1e-14)


def lap2(n, eps=1.0):
    e = np.ones(n)
    T = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1]).tolil()
    T[0, 0] = 3
    T[n - 1, n - 1] = 3
    Nn = sp.diags([-e[:-1], np.r_[1, 2 * np.ones(n - 2), 1], -e[:-1]], [-1, 0, 1])
    return (sp.kron(sp.eye(n), T) + eps * sp.kron(Nn, sp.eye(n))).tocsr()


def test_strength_anisotropic(oracle_mod):
    """With y-couplings 1e-3 of the x-couplings only x-neighbours are strong."""
    n = 10
    A = lap2(n, eps=1e-3)
    G = oracle_mod.strength(A, 0.08)
    rows, cols = G.nonzero()
    assert len(rows) > 0 and np.all(np.abs(rows - cols) == 1)
    assert (G - G.T).nnz == 0 or np.all((abs(G) - abs(G.T)).data == 0)


def bfs_dist(G, src, limit):
    dist = {src: 0}
    q = deque([src])
    while q:
        u = q.popleft()
        if dist[u] == limit:
            continue
        for v in G.indices[G.indptr[u]:G.indptr[u + 1]]:
            if v not in dist:
                dist[v] = dist[u] + 1
                q.append(v)
    return dist


def greedy_mis2(G, keys):
    n = G.shape[0]
    state = np.zeros(n, dtype=int)
    deg = np.diff(G.indptr)
    state[deg == 0] = 2
    for v in sorted(range(n), key=lambda i: -keys[i]):
        if state[v]:
            continue
        state[v] = 1
        for u, dd in bfs_dist(G, v, 2).items():
            if u != v and state[u] == 0:
                state[u] = 2
    return state == 1


def test_mis_key_definition(oracle_mod):
    """key = (top 32 bits of the SplitMix64 finaliser of (level key + (i+1) gamma)) | i."""
    seed = 12345
    g = inputs.GOLDEN
    with np.errstate(over="ignore"):
        lk = inputs.splitmix64_mix(np.uint64(seed) + g * np.uint64(3 + 1))
        hv = int(inputs.splitmix64_mix(lk + g * np.uint64(7 + 1)))
    assert oracle_mod.mis_key(seed, 3, 7) == ((hv >> 32) << 32) | 7


@pytest.mark.parametrize("make", [lambda: lap2(12), lambda: lap2(9, eps=1e-3),
                                  lambda: None])
def test_mis2_and_aggregates(oracle_mod, make):
    A = make()
    if A is None:
        inst = inputs.random_segments_2d(n=24, n_seg=6)
        Af, b = oracle_mod.assemble(inst)
        Amm, Amf, Afm, Aff = oracle_mod.split(Af, inst.n_m)
        A = oracle_mod.schur(Amm, Amf, Afm, Aff)
    amg = oracle_mod.AMG(A, n_coarse=8)
    assert amg.nlevels >= 2
    for l in range(amg.nlevels - 1):
        Al = amg.level_A(l)
        G = oracle_mod.strength(Al, 0.08)
        roots = amg.roots(l)
        agg = amg.agg(l)
        n = Al.shape[0]
        keys = [oracle_mod.mis_key(oracle_mod.DEFAULT_SEED, l, i) for i in range(n)]
        # equals the sequential greedy definition on G^2 in descending key order
        assert np.array_equal(roots, greedy_mis2(G, keys))
        deg = np.diff(G.indptr)
        rl = np.nonzero(roots)[0]
        # roots pairwise at distance >= 3; every non-isolated vertex within 2 of a root
        covered = np.zeros(n, dtype=bool)
        for r in rl:
            d = bfs_dist(G, r, 2)
            for u in d:
                covered[u] = True
                if u != r:
                    assert not roots[u]
        assert np.all(covered[deg > 0])
        # aggregates: a partition of the non-isolated vertices, roots numbered ascending
        assert np.all(agg[deg == 0] == -1)
        assert np.all(agg[deg > 0] >= 0)
        assert np.array_equal(agg[rl], np.arange(len(rl)))
        # each aggregate is connected in G and contains its root
        for I in range(len(rl)):
            mem = set(np.nonzero(agg == I)[0])
            seen = {rl[I]}
            q = deque([rl[I]])
            while q:
                u = q.popleft()
                for v in G.indices[G.indptr[u]:G.indptr[u + 1]]:
                    if v in mem and v not in seen:
                        seen.add(v)
                        q.append(v)
            assert seen == mem
        # Galerkin operator against the dense product P^T A P
        P = np.zeros((n, len(rl)))
        P[np.nonzero(agg >= 0)[0], agg[agg >= 0]] = 1.0
        Ac = amg.level_A(l + 1).toarray()
        ref = P.T @ Al.toarray() @ P
        assert np.max(np.abs(Ac - ref)) <= 1e-13 * np.max(np.abs(ref))
        # row sums: A_c 1 = P^T A (P 1), P 1 the indicator of aggregated vertices
        ind = (agg >= 0).astype(float)
        assert np.allclose(Ac.sum(axis=1), P.T @ (Al @ ind), rtol=1e-12, atol=1e-12 * np.abs(Ac).max())
        np.linalg.cholesky(Ac)


def test_aggregate_distance2_tie_break(oracle_mod):
    """1D chain 0-1-2-3-4 with equal weights: a vertex at distance 2 from two
    roots' first rings goes to the smaller aggregate id."""
    n = 7
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    amg = oracle_mod.AMG(A, n_coarse=1)
    agg, roots = amg.agg(0), amg.roots(0)
    rl = np.nonzero(roots)[0]
    for i in range(n):
        if agg[i] < 0:
            continue
        if roots[i]:
            continue
        nb = [j for j in (i - 1, i + 1) if 0 <= j < n]
        if any(roots[j] for j in nb):
            assert agg[i] == agg[[j for j in nb if roots[j]][0]]
        else:
            cands = [agg[j] for j in nb if agg[j] >= 0 and any(roots[k] for k in (j - 1, j + 1) if 0 <= k < n)]
            assert agg[i] == min(cands)
    assert len(rl) >= 2


def test_vcycle_single_level_is_exact(oracle_mod):
    A = lap2(10)
    amg = oracle_mod.AMG(A, n_coarse=1000)
    assert amg.nlevels == 1 and amg.coarsest_dense
    b = np.random.default_rng(0).standard_normal(100)
    x = amg.vcycle(b)
    assert np.max(np.abs(A @ x - b)) < 1e-12 * np.max(np.abs(b))


def dense_operator(f, n):
    return np.column_stack([f(np.eye(n)[:, j]) for j in range(n)])


@pytest.mark.parametrize("smoother", [0, 1])
def test_vcycle_two_grid_error_propagation(oracle_mod, smoother):
    """E = I - V A of the two-level cycle equals the textbook product
    (I - M^-1 A)(I - P A_c^-1 P^T A)(I - M^-1 A) for L1-Jacobi M."""
    A = lap2(8, eps=0.7) + sp.diags(np.linspace(0, 0.3, 64))
    A = sp.csr_matrix(A)
    amg = oracle_mod.AMG(A, n_coarse=20, smoother=smoother)
    assert amg.nlevels == 2 and amg.coarsest_dense
    n = 64
    Ad = A.toarray()
    V = dense_operator(amg.vcycle, n)
    E = np.eye(n) - V @ Ad
    agg = amg.agg(0)
    P = np.zeros((n, agg.max() + 1))
    P[np.nonzero(agg >= 0)[0], agg[agg >= 0]] = 1.0
    Ac = P.T @ Ad @ P
    CG = np.eye(n) - P @ np.linalg.solve(Ac, P.T @ Ad)
    Minv = np.diag(1.0 / amg.l1(0))
    if smoother == 0:
        Sm = np.eye(n) - Minv @ Ad
    else:
        # degree-2 Chebyshev error polynomial on [0.3, 1]: p(t) = T2((1+0.3-2t)/(1-0.3)) / T2((1+0.3)/(1-0.3))
        lo, hi = 0.3, 1.0
        X = Minv @ Ad
        Y = ((hi + lo) * np.eye(n) - 2 * X) / (hi - lo)
        T2 = 2 * Y @ Y - np.eye(n)
        s = (hi + lo) / (hi - lo)
        Sm = T2 / (2 * s * s - 1)
    assert np.max(np.abs(E - Sm @ CG @ Sm)) < 1e-12
    # symmetric operator, error reduction < 1 in the energy norm
    assert np.max(np.abs(V - V.T)) < 1e-12 * np.max(np.abs(V))
    ev = np.linalg.eigvals(E)
    assert np.max(np.abs(ev)) < 1.0


def test_l1_diagonal(oracle_mod):
    A = lap2(6, eps=0.5)
    amg = oracle_mod.AMG(A, n_coarse=1)
    assert np.array_equal(amg.l1(0), np.asarray(abs(A).sum(axis=1)).ravel())


def test_lowp_rounding(oracle_mod):
    """bf16 keeps 8 significant bits, fp16 11, both round to nearest even."""
    r = oracle_mod.round_lowp
    # bf16: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> even (1); 1 + 3 2^-8 -> 1 + 2^-6
    assert r(1 + 2 ** -8, 16) == 1.0
    assert r(1 + 3 * 2 ** -8, 16) == 1 + 2 ** -6
    assert r(1 + 2 ** -8 + 2 ** -20, 16) == 1 + 2 ** -7
    assert r(-3.0, 16) == -3.0 and r(2.0 ** -130, 16) == 2.0 ** -130
    # fp16 against numpy's IEEE binary16 conversion of the float
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.uniform(-9, 5, 2000), [65519.0, 65520.0, 6e-8,
                                                                                       2 ** -25, 3 * 2 ** -26]])
    for x in xs:
        ref = float(np.float16(np.float32(x)))
        assert r(x, 17) == ref or (np.isinf(ref) and np.isinf(r(x, 17))), x
    assert r(1.0 / 3.0, 32) == float(np.float32(1.0 / 3.0))


@pytest.mark.parametrize("smoother", [0, 1])
def test_vcycle_two_sweeps(oracle_mod, smoother):
    """Two sweeps: E = S^2 (I - P A_c^-1 P^T A) S^2 for the two-level cycle."""
    A = sp.csr_matrix(lap2(8, eps=0.7) + sp.diags(np.linspace(0, 0.3, 64)))
    amg = oracle_mod.AMG(A, n_coarse=20, smoother=smoother, sweeps=2)
    n = 64
    Ad = A.toarray()
    V = dense_operator(amg.vcycle, n)
    E = np.eye(n) - V @ Ad
    agg = amg.agg(0)
    P = np.zeros((n, agg.max() + 1))
    P[np.nonzero(agg >= 0)[0], agg[agg >= 0]] = 1.0
    CG = np.eye(n) - P @ np.linalg.solve(P.T @ Ad @ P, P.T @ Ad)
    Minv = np.diag(1.0 / amg.l1(0))
    if smoother == 0:
        Sm = np.eye(n) - Minv @ Ad
    else:
        lo, hi = 0.3, 1.0
        Y = ((hi + lo) * np.eye(n) - 2 * Minv @ Ad) / (hi - lo)
        s = (hi + lo) / (hi - lo)
        Sm = (2 * Y @ Y - np.eye(n)) / (2 * s * s - 1)
    S2 = Sm @ Sm
    assert np.max(np.abs(E - S2 @ CG @ S2)) < 1e-12


def sa_reference(A, G, agg, nc):
    """P = P0 - (4/3) D1F^-1 AF P0 written densely: AF keeps the strong
    off-diagonals and moves the weak ones to the diagonal."""
    n = A.shape[0]
    Ad = A.toarray()
    S = np.zeros((n, n), dtype=bool)
    S[G.nonzero()] = True
    AF = np.where(S, Ad, 0.0)
    weak = ~S & ~np.eye(n, dtype=bool) & (Ad != 0)
    np.fill_diagonal(AF, np.diag(Ad) + np.where(weak, Ad, 0.0).sum(axis=1))
    d1 = np.diag(AF) + np.abs(AF - np.diag(np.diag(AF))).sum(axis=1)
    P0 = np.zeros((n, nc))
    P0[np.nonzero(agg >= 0)[0], agg[agg >= 0]] = 1.0
    return P0 - (4.0 / 3.0) * (AF / d1[:, None]) @ P0


@pytest.mark.parametrize("make", [lambda: lap2(12), lambda: lap2(10, eps=1e-3), lambda: None])
def test_smoothed_prolongator_and_galerkin(oracle_mod, make):
    A = make()
    if A is None:
        inst = inputs.random_segments_2d(n=20, n_seg=5)
        Af, _ = oracle_mod.assemble(inst)
        A = oracle_mod.schur(*oracle_mod.split(Af, inst.n_m))
    amg = oracle_mod.AMG(A, n_coarse=8, smoothed=1)
    assert amg.nlevels >= 2
    for l in range(amg.nlevels - 1):
        Al = amg.level_A(l)
        G = oracle_mod.strength(Al, amg.opts.theta)
        agg = amg.agg(l)
        nc = amg.level_A(l + 1).shape[0]
        P = amg.P(l)
        ref = sa_reference(Al, G, agg, nc)
        assert np.max(np.abs(P.toarray() - ref)) <= 1e-14 * max(1.0, np.abs(ref).max())
        Ac = amg.level_A(l + 1).toarray()
        Pd = P.toarray()
        cref = Pd.T @ Al.toarray() @ Pd
        assert np.max(np.abs(Ac - cref)) <= 1e-12 * np.abs(cref).max()
        np.linalg.cholesky(Ac)


def test_smoothed_two_grid_error_propagation(oracle_mod):
    A = sp.csr_matrix(lap2(8, eps=0.7) + sp.diags(np.linspace(0, 0.3, 64)))
    amg = oracle_mod.AMG(A, n_coarse=20, smoothed=1)
    assert amg.nlevels == 2 and amg.coarsest_dense
    n = 64
    Ad = A.toarray()
    E = np.eye(n) - dense_operator(amg.vcycle, n) @ Ad
    P = amg.P(0).toarray()
    CG = np.eye(n) - P @ np.linalg.solve(P.T @ Ad @ P, P.T @ Ad)
    Sm = np.eye(n) - np.diag(1.0 / amg.l1(0)) @ Ad
    assert np.max(np.abs(E - Sm @ CG @ Sm)) < 1e-12
