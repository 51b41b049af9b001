"""Pins of the junction rules of the oracle's assembly (Sec. 2.1: fractures
meeting at intersections, which the paper models as subdomains of dimension
N-2 with their own pressures and interface fluxes).

junction=0 links every pair of fracture cells at a junction by
t_i t_j / (t_i + t_j).  junction=1 joins the cells of a junction of three or
more to a node by their half transmissibilities t_l: in the primal form the
node is eliminated (star-delta, T_ij = t_i t_j / sum t), in the flux form it
is an intersection cell with one interface flux per member cell.
"""
import itertools

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


def half_t(inst, k):
    h = 1.0 / inst.n
    elen = 1.0 if inst.dim == 2 else h
    return inst.fc_kf[k] * inst.fc_a[k] * elen / (0.5 * h)


def junctions_brute_force(inst):
    """Every grid vertex (2D) or edge (3D) with the fracture faces containing
    it, found by scanning the geometry (not the cells' neighbourhoods)."""
    n, dim = inst.n, inst.dim
    faces = {}
    for k, (d, p) in enumerate(zip(inst.fc_axis, inst.fc_pos)):
        faces[(int(d),) + tuple(int(v) for v in p[:dim])] = k
    out = {}
    if dim == 2:
        for x, y in itertools.product(range(n + 1), repeat=2):
            mem = []
            for yy in (y - 1, y):  # x-normal faces at plane x, cells y-1 and y
                k = faces.get((0, x, yy))
                if k is not None:
                    mem.append(k)
            for xx in (x - 1, x):
                k = faces.get((1, xx, y))
                if k is not None:
                    mem.append(k)
            if mem:
                out[(x, y)] = sorted(mem)
        return out
    for a in range(3):  # edges along axis a
        b, c = [q for q in range(3) if q != a]
        for u, v, w in itertools.product(range(n + 1), range(n + 1), range(n)):
            mem = []
            # faces normal to b at plane u, and normal to c at plane v
            for dv in (v - 1, v):
                pos = [0, 0, 0]
                pos[a], pos[b], pos[c] = w, u, dv
                k = faces.get((b,) + tuple(pos))
                if k is not None:
                    mem.append(k)
            for du in (u - 1, u):
                pos = [0, 0, 0]
                pos[a], pos[b], pos[c] = w, du, v
                k = faces.get((c,) + tuple(pos))
                if k is not None:
                    mem.append(k)
            if mem:
                out[(a, u, v, w)] = sorted(mem)
    return out


def test_star_delta_is_the_eliminated_star():
    """The star-delta rule is the Schur complement of a star network: a node
    joined to m cells by t_l, eliminated (checked on a dense Laplacian)."""
    t = np.array([2.0, 3.0, 5.0, 7.0])
    m = len(t)
    L = np.zeros((m + 1, m + 1))
    for i, ti in enumerate(t):
        L[i, i] += ti
        L[m, m] += ti
        L[i, m] -= ti
        L[m, i] -= ti
    S = L[:m, :m] - np.outer(L[:m, m], L[m, :m]) / L[m, m]
    for i, j in itertools.combinations(range(m), 2):
        assert -S[i, j] == pytest.approx(t[i] * t[j] / t.sum(), rel=1e-15)


def test_crossing_star_delta_closed_form(oracle_mod):
    """Two fractures crossing at one vertex (2D): the four cells around it are
    linked by t_i t_j / (2 t_1 + 2 t_2) instead of the pairwise rule."""
    n = 8
    kf1, kf2, a = 2.0, 6.0, 0.1
    rects = [inputs.Rect(0, 4, (0,), (n,), kf1, a), inputs.Rect(1, 4, (0,), (n,), kf2, a)]
    inst = inputs.make_instance("x", 2, n, np.ones(n * n), rects)
    A, _ = oracle_mod.assemble(inst, junction=1)
    nm = inst.n_m
    h = 1.0 / n
    t1, t2 = kf1 * a / (h / 2), kf2 * a / (h / 2)
    S = 2 * t1 + 2 * t2
    pos = {(int(ax), int(p[0]), int(p[1])): k for k, (ax, p) in enumerate(zip(inst.fc_axis, inst.fc_pos))}
    v_lo, v_hi = pos[(0, 4, 3)], pos[(0, 4, 4)]
    h_lo, h_hi = pos[(1, 3, 4)], pos[(1, 4, 4)]
    Ad = A.toarray()
    f = lambda i, j: -Ad[nm + i, nm + j]
    assert f(v_lo, v_hi) == pytest.approx(t1 * t1 / S, rel=1e-15)
    assert f(h_lo, h_hi) == pytest.approx(t2 * t2 / S, rel=1e-15)
    assert f(v_lo, h_lo) == pytest.approx(t1 * t2 / S, rel=1e-15)
    assert f(v_hi, h_hi) == pytest.approx(t1 * t2 / S, rel=1e-15)
    # away from the crossing, coplanar neighbours keep t/2
    assert f(pos[(0, 4, 1)], pos[(0, 4, 2)]) == t1 * t1 / (t1 + t1)


@pytest.mark.parametrize("case", list(CASES))
def test_star_delta_differs_only_at_intersections(oracle_mod, case):
    """Junctions of two cells give the pairwise value bit for bit; only rows
    of cells at junctions of three or more change."""
    inst = CASES[case]()
    A0, b0 = oracle_mod.assemble(inst)
    A1, b1 = oracle_mod.assemble(inst, junction=1)
    assert np.array_equal(b0, b1)
    assert np.array_equal(A0.indptr, A1.indptr) and np.array_equal(A0.indices, A1.indices)
    at_int = set()
    for mem in junctions_brute_force(inst).values():
        if len(mem) >= 3:
            at_int.update(mem)
    rows = set(np.nonzero(np.any((A0 != A1).toarray(), axis=1))[0]) if A0.shape[0] < 6000 else None
    if rows is not None:
        assert rows <= {inst.n_m + k for k in at_int}
    # symmetry, M-matrix signs, zero row sums away from Dirichlet ends
    assert abs(A1 - A1.T).max() == 0.0
    off = A1 - sp.diags(A1.diagonal())
    assert off.nnz == 0 or off.data.max() <= 0.0
    rs0 = np.asarray(A0.sum(axis=1)).ravel()
    rs1 = np.asarray(A1.sum(axis=1)).ravel()
    assert np.allclose(rs0, rs1, rtol=0, atol=1e-12 * np.abs(A1.diagonal()).max())


@pytest.mark.parametrize("case", list(CASES))
def test_intersection_form_structure(oracle_mod, case):
    inst = CASES[case]()
    A, b, no = oracle_mod.assemble(inst, form="flux", junction=1, with_split=True)
    N, nf = inst.n_m + inst.n_f, inst.n_f
    junc = {k: v for k, v in junctions_brute_force(inst).items() if len(v) >= 3}
    nI = len(junc)
    nIF = sum(len(v) for v in junc.values())
    assert no == N + nI and A.shape == (N + nI + 2 * nf + nIF,) * 2
    assert abs(A - A.T).max() == 0.0
    A = A.tocsr()
    G = A[no:, no:]
    assert (G - sp.diags(G.diagonal())).count_nonzero() == 0 and np.all(G.diagonal() < 0)
    # intersection rows: an explicit zero diagonal and -1 per member flux
    members_seen = []
    for I in range(nI):
        r = N + I
        cols, vals = A.indices[A.indptr[r]:A.indptr[r + 1]], A.data[A.indptr[r]:A.indptr[r + 1]]
        assert cols[0] == r and vals[0] == 0.0 and np.all(vals[1:] == -1.0) and np.all(cols[1:] >= no + 2 * nf)
        mem = []
        for j in cols[1:]:
            c2, v2 = A.indices[A.indptr[j]:A.indptr[j + 1]], A.data[A.indptr[j]:A.indptr[j + 1]]
            # flux row: +1 at the member fracture cell, -1 at the intersection, -1/t_l
            assert len(c2) == 3 and v2[0] == 1.0 and c2[1] == r and v2[1] == -1.0 and c2[2] == j
            l = c2[0] - inst.n_m
            assert 0 <= l < nf and v2[2] == -1.0 / half_t(inst, l)
            mem.append(int(l))
        assert mem == sorted(mem)
        members_seen.append(tuple(mem))
    assert sorted(members_seen) == sorted(tuple(v) for v in junc.values())
    assert np.all(b[:, N:] == 0.0)


@pytest.mark.parametrize("case", list(CASES))
def test_intersection_form_eliminates_to_star_delta(oracle_mod, case):
    """Eliminating the fluxes (exact: A_GG is diagonal) and then the
    intersection pressures gives the star-delta primal system."""
    inst = CASES[case]()
    A1, b1 = oracle_mod.assemble(inst, junction=1)
    A, b, no = oracle_mod.assemble(inst, form="flux", junction=1, with_split=True)
    N = inst.n_m + inst.n_f
    A = A.tocsr()
    Aoo, Aog, Ago, Agg = A[:no, :no], A[:no, no:], A[no:, :no], A[no:, no:]
    S = (Aoo - Aog @ sp.diags(1.0 / Agg.diagonal()) @ Ago).tocsr()
    # the oracle's Eq. (7) on this partition is the same exact elimination
    St = oracle_mod.schur(*oracle_mod.split(A, no))
    assert np.max(np.abs((St - S).data), initial=0.0) <= 1e-13 * np.max(np.abs(S.data))
    if no > N:
        Sii = S[N:, N:]
        assert (Sii - sp.diags(Sii.diagonal())).count_nonzero() == 0  # intersections do not touch
        P = (S[:N, :N] - S[:N, N:] @ sp.diags(1.0 / Sii.diagonal()) @ S[N:, :N]).tocsr()
    else:
        P = S
    assert np.max(np.abs((P - A1).data), initial=0.0) <= 1e-13 * np.max(np.abs(A1.data))
    assert np.array_equal(b[:, :N], b1)


@pytest.mark.parametrize("case", ["fixed2d-16", "planes3d-8"])
def test_intersection_pressure_is_weighted_mean(oracle_mod, case):
    """Direct solve of the intersection form: pressures of all cells equal
    the star-delta primal solution; at each intersection the member fluxes sum
    to zero, each is t_l (p_l - p_I), and p_I is the t-weighted mean."""
    inst = CASES[case]()
    A1, b1 = oracle_mod.assemble(inst, junction=1)
    A, b, no = oracle_mod.assemble(inst, form="flux", junction=1, with_split=True)
    N = inst.n_m + inst.n_f
    p = spla.spsolve(A1.tocsc(), b1[0])
    y = spla.spsolve(A.tocsc(), b[0])
    scale = max(1.0, np.max(np.abs(p)))
    assert np.max(np.abs(y[:N] - p)) <= 1e-9 * scale
    A = A.tocsr()
    for I in range(no - N):
        r = N + I
        flux_cols = A.indices[A.indptr[r] + 1:A.indptr[r + 1]]
        lam = y[flux_cols]
        assert abs(lam.sum()) <= 1e-9 * max(1.0, np.abs(lam).max())
        mem = [A.indices[A.indptr[j]] - inst.n_m for j in flux_cols]
        t = np.array([half_t(inst, l) for l in mem])
        pl = y[[inst.n_m + l for l in mem]]
        assert y[r] == pytest.approx(np.dot(t, pl) / t.sum(), rel=1e-9, abs=1e-9 * scale)
        assert np.allclose(lam, t * (pl - y[r]), rtol=1e-7, atol=1e-9 * scale * t.max())


def test_no_intersections_flux_forms_agree(oracle_mod):
    """Without junctions of three or more cells both junction rules give the
    same flux-form system, bit for bit."""
    n = 12
    rects = [inputs.Rect(0, 3, (1,), (9,), 3.0, 0.01), inputs.Rect(1, 8, (4,), (11,), 0.5, 0.01)]
    inst = inputs.make_instance("nx", 2, n, np.linspace(1, 2, n * n), rects)
    assert all(len(v) < 3 for v in junctions_brute_force(inst).values())
    A0, b0 = oracle_mod.assemble(inst, form="flux")
    A1, b1, no = oracle_mod.assemble(inst, form="flux", junction=1, with_split=True)
    assert no == inst.n_m + inst.n_f
    assert (A0 != A1).nnz == 0 and np.array_equal(b0, b1)


@pytest.mark.parametrize("case", ["fixed2d-16", "seg2d-40", "planes3d-8"])
def test_intersection_form_solves(oracle_mod, case):
    """M_L + FGMRES and B_D + MINRES on the intersection form reach its
    direct solution."""
    inst = CASES[case]()
    A, b, no = oracle_mod.assemble(inst, form="flux", junction=1, with_split=True)
    y = spla.spsolve(A.tocsc(), b[0])
    scale = max(1.0, np.max(np.abs(y)))
    r1 = oracle_mod.fgmres(A, b[0], oracle_mod.ML(A, no), rtol=1e-10, maxit=3000)
    assert r1.converged and np.max(np.abs(r1.x - y)) <= 1e-6 * scale
    r2 = oracle_mod.minres(A, b[0], oracle_mod.ML(A, no, kind="diag"), rtol=1e-10, maxit=5000)
    assert r2.converged and np.max(np.abs(r2.x - y)) <= 1e-6 * scale


def test_smoothed_aggregation_on_intersection_cells(oracle_mod):
    """Smoothed aggregation on the paper's partition with intersection cells
    and K_par = 1e4 (coarse operators with positive off-diagonals, where
    lumping weak entries can leave a non-positive diagonal): every level's
    matrix is finite, the V-cycle is symmetric positive definite, and M_L +
    FGMRES reaches the direct solution."""
    import dataclasses
    inst = inputs.planes_3d(16, kf=1e4)
    inst = dataclasses.replace(inst, fc_kn=np.full(inst.n_f, 1.0))
    A, b, no = oracle_mod.assemble(inst, form="flux", junction=1, with_split=True)
    M = oracle_mod.ML(A, no, smoothed=1)
    amg = M.amg(0)
    assert amg.nlevels >= 3
    for l in range(amg.nlevels):
        assert np.all(np.isfinite(amg.level_A(l).data)), l
    rng = np.random.default_rng(17)
    v, w = rng.standard_normal((2, no))
    x, y = v @ amg.vcycle(w), w @ amg.vcycle(v)
    assert abs(x - y) <= 1e-10 * max(abs(x), abs(y)) and v @ amg.vcycle(v) > 0
    y_direct = spla.spsolve(A.tocsc(), b[0])
    r = oracle_mod.fgmres(A, b[0], M, rtol=1e-10, maxit=1000)
    assert r.converged and np.max(np.abs(r.x - y_direct)) <= 1e-6 * max(1.0, np.max(np.abs(y_direct)))
