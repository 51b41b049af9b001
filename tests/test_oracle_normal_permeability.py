"""Pins of the fractures' normal permeability k_n (Eq. (2): the interface law's
kappa = 2 k_n / a), independent of the tangential permeability K_par = k_f
that enters the fracture-fracture transmissibilities (Sec. 4 varies the two
independently, Table 1).

Flow across a fracture sees only k_n; flow along a fracture sees only k_f;
k_n = k_f reproduces the default assembly bit for bit.
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_2206_03203_gb300 import inputs


def with_kn(inst, kn):
    return dataclasses.replace(inst, fc_kn=np.full(inst.n_f, float(kn)))


def test_kn_equal_kf_is_the_default(oracle_mod):
    for inst in (inputs.fixed_2d(n=16), inputs.random_rects_3d(10, 22060305, 0, 4, sigma=2.0)):
        A, b = oracle_mod.assemble(inst)
        A2, b2 = oracle_mod.assemble(dataclasses.replace(inst, fc_kn=inst.fc_kf.copy()))
        assert (A != A2).nnz == 0 and np.array_equal(b, b2)
        Af, bf = oracle_mod.assemble(inst, form="flux")
        Af2, bf2 = oracle_mod.assemble(dataclasses.replace(inst, fc_kn=inst.fc_kf.copy()), form="flux")
        assert (Af != Af2).nnz == 0 and np.array_equal(bf, bf2)


@pytest.mark.parametrize("kf,kn,a", [(1e4, 1e-4, 1e-4), (1e-4, 1e4, 1e-4), (3.0, 0.2, 0.05)])
def test_across_a_fracture_only_kn_counts(oracle_mod, kf, kn, a):
    """A full-height fracture normal to x: resistance a / k_n in series with
    the matrix, q = 1 / (1/k_m + a/k_n), whatever k_f."""
    n = 8
    inst = with_kn(inputs.make_instance("ser", 2, n, np.ones(n * n), [inputs.Rect(0, 4, (0,), (n,), kf, a)]), kn)
    A, b = oracle_mod.assemble(inst)
    p = spla.spsolve(A.tocsc(), b[0])
    pl = p[:inst.n_m].reshape(n, n)[:, 0]
    inflow = np.sum(2.0 * (1.0 - pl))
    assert abs(inflow - 1.0 / (1.0 + a / kn)) < 1e-12
    # the flux form gives the same pressures
    Af, bf = oracle_mod.assemble(inst, form="flux")
    y = spla.spsolve(Af.tocsc(), bf[0])
    assert np.max(np.abs(y[:inst.n_m + inst.n_f] - p)) < 1e-10


@pytest.mark.parametrize("kn", [1e-4, 1.0, 1e4])
def test_along_a_fracture_only_kf_counts(oracle_mod, kn):
    """Fractures spanning x between the Dirichlet faces carry the flow in
    parallel with the matrix: the linear field and the inflow
    1 + sum k_f a do not depend on k_n."""
    n = 8
    kf, a = 37.0, 1e-2
    rects = [inputs.Rect(1, 3, (0,), (n,), kf, a), inputs.Rect(1, 6, (0,), (n,), 2 * kf, a)]
    inst = with_kn(inputs.make_instance("par", 2, n, np.ones(n * n), rects), kn)
    A, b = oracle_mod.assemble(inst)
    p = spla.spsolve(A.tocsc(), b[0])
    xc = (np.arange(n) + 0.5) / n
    assert np.max(np.abs(p[:inst.n_m] - (1.0 - np.tile(xc, n)))) < 1e-10
    rs = np.asarray(A.sum(axis=1)).ravel()
    left = np.zeros(A.shape[0], dtype=bool)
    left[:inst.n_m] = np.tile(xc, n) < 1.0 / n
    left[inst.n_m:] = inst.fc_pos[:, 0] == 0
    inflow = np.sum((rs * (1.0 - p))[left])
    assert abs(inflow - (1.0 + 3 * kf * a)) < 1e-9 * (1.0 + 3 * kf * a)


def test_kn_enters_only_the_coupling_entries(oracle_mod):
    """Changing k_n changes exactly the matrix-fracture entries and the
    diagonals they feed; the matrix-matrix and fracture-fracture entries stay."""
    inst = inputs.fixed_2d(n=16)
    A, _ = oracle_mod.assemble(inst)
    B, _ = oracle_mod.assemble(with_kn(inst, 1e-2))
    Amm, Amf, Afm, Aff = oracle_mod.split(A, inst.n_m)
    Bmm, Bmf, Bfm, Bff = oracle_mod.split(B, inst.n_m)
    for X, Y in ((Amm, Bmm), (Aff, Bff)):
        D = (X - Y).tocsr()
        D.setdiag(0.0)
        D.eliminate_zeros()
        assert D.nnz == 0
    assert (Amf != Bmf).nnz == Amf.nnz
    # the coupling of fracture cell k to each side is |F| / (h/(2 k_m) + a/(2 k_n))
    h = 1.0 / 16
    t = h / (h / 2 + inst.fc_a[0] / (2 * 1e-2))
    assert np.allclose(-Bfm.data, t, rtol=1e-14)
