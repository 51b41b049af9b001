"""Pins of the packed-batch hierarchies: a block-diagonal system of K
instances is coarsened instance by instance (the V-cycle of Sec. 3.3 applied
to each instance of a batch), so every level of the packed hierarchy, cut to
one instance's rows, is that instance's own hierarchy level, and the
coarsest level is solved exactly per instance."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2206_03203_gb300 import inputs


def _instances():
    return [inputs.random_rects_3d(n, 22060304, k, 1 + k % 4, nrhs=1) for k, n in enumerate([9, 12, 8, 11, 10])]


def _schur_blocks(oracle_mod, insts):
    out = []
    for inst in insts:
        A, _ = oracle_mod.assemble(inst)
        out.append(oracle_mod.ML(A, inst.n_m).schur)
    return out


@pytest.mark.parametrize("smoothed", [0, 1])
def test_packed_levels_are_the_instances_own(oracle_mod, smoothed):
    insts = _instances()
    S = _schur_blocks(oracle_mod, insts)
    off = np.cumsum([0] + [s.shape[0] for s in S])
    P = sp.block_diag(S, format="csr")
    packed = oracle_mod.AMG(P, segments=off, n_coarse=40, smoothed=smoothed)
    assert packed.coarsest_dense
    deepest = 0
    for k, Sk in enumerate(S):
        own = oracle_mod.AMG(Sk, n_coarse=40, smoothed=smoothed)
        assert own.coarsest_dense
        deepest = max(deepest, own.nlevels)
        for l in range(own.nlevels):
            seg = packed.segments(l)
            r0, r1 = seg[k], seg[k + 1]
            Al = packed.level_A(l).tocsr()
            Ak = Al[r0:r1][:, r0:r1]
            # nothing couples instance k to another instance
            assert Al[r0:r1].nnz == Ak.nnz
            Ok = own.level_A(l).tocsr()
            assert Ak.shape == Ok.shape and abs(Ak - Ok).max() == 0.0, (k, l)
            assert np.array_equal(packed.roots(l)[r0:r1], own.roots(l)), (k, l)
            if l < own.nlevels - 1:
                pa, oa = packed.agg(l)[r0:r1], own.agg(l)
                nxt = packed.segments(l + 1)[k]
                assert np.array_equal(np.where(pa >= 0, pa - nxt, -1), oa), (k, l)
        # the packed hierarchy stops only once every instance is small enough
        last = packed.segments(packed.nlevels - 1)
        assert np.all(np.diff(last) <= 40)
    assert packed.nlevels >= deepest


def test_packed_coarsest_is_exact_per_instance(oracle_mod):
    """With every instance at most n_coarse rows the packed V-cycle is the
    exact block-diagonal solve."""
    insts = [inputs.random_rects_3d(n, 3, k, 2, nrhs=1) for k, n in enumerate([5, 6, 4])]
    S = _schur_blocks(oracle_mod, insts)
    off = np.cumsum([0] + [s.shape[0] for s in S])
    P = sp.block_diag(S, format="csr")
    amg = oracle_mod.AMG(P, segments=off, n_coarse=256)
    assert amg.nlevels == 1 and amg.coarsest_dense
    b = np.random.default_rng(3).standard_normal(P.shape[0])
    x = amg.vcycle(b)
    xd = spla.spsolve(P.tocsc(), b)
    assert np.max(np.abs(x - xd)) <= 1e-12 * np.max(np.abs(xd))
    # and a single instance through the segmented entry equals the plain one
    one = oracle_mod.AMG(S[1], segments=[0, S[1].shape[0]], n_coarse=20)
    plain = oracle_mod.AMG(S[1], n_coarse=20)
    assert one.nlevels == plain.nlevels
    bb = b[:S[1].shape[0]]
    assert np.array_equal(one.vcycle(bb), plain.vcycle(bb))


def test_packed_ml_solves_each_instance_as_alone(oracle_mod):
    """M_L on a packed batch whose instances all stop at the same depth is M_L
    of each instance: FGMRES on a packed right-hand side that is nonzero on one
    instance takes that instance's own iteration count."""
    insts = [inputs.random_rects_3d(n, 22060304, k, 2, nrhs=1) for k, n in enumerate([10, 10, 10])]
    As, bs = zip(*[oracle_mod.assemble(i) for i in insts])
    blocks = [oracle_mod.split(A, i.n_m) for A, i in zip(As, insts)]
    Amm = sp.block_diag([b[0] for b in blocks], format="csr")
    Amf = sp.block_diag([b[1] for b in blocks], format="csr")
    Afm = sp.block_diag([b[2] for b in blocks], format="csr")
    Aff = sp.block_diag([b[3] for b in blocks], format="csr")
    A = sp.bmat([[Amm, Amf], [Afm, Aff]], format="csr")
    A.sort_indices()
    mo = np.cumsum([0] + [i.n_m for i in insts])
    fo = np.cumsum([0] + [i.n_f for i in insts])
    M = oracle_mod.ML(A, Amm.shape[0], segments=(mo, fo), n_coarse=64)
    compared = 0
    for k, inst in enumerate(insts):
        own = oracle_mod.ML(As[k], inst.n_m, n_coarse=64)
        if any(own.amg(q).nlevels != M.amg(q).nlevels for q in (0, 1)):
            continue  # instance k would stop coarsening earlier than the batch
        compared += 1
        b = np.zeros(A.shape[0])
        rows = np.r_[mo[k]:mo[k + 1], Amm.shape[0] + fo[k]:Amm.shape[0] + fo[k + 1]]
        b[rows] = bs[k][0]
        r_packed = oracle_mod.fgmres(A, b, M, rtol=1e-8, maxit=300)
        r_own = oracle_mod.fgmres(As[k], bs[k][0], own, rtol=1e-8, maxit=300)
        assert r_packed.iterations == r_own.iterations
        assert np.max(np.abs(r_packed.x[rows] - r_own.x)) <= 1e-10 * np.max(np.abs(r_own.x))
    assert compared >= 1
