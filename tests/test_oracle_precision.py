"""Pins of the oracle's precision emulation (the mixed-precision readings of
the V-cycle of Sec. 3.3: FP32 levels, bf16 / fp16 levels with power-of-two
row scales, FP32 vectors).

Two things fix what the emulation must compute, independently of its C code:
  * the storage rule: a bf16 / fp16 row i stores q_ij = round(a_ij / s_i)
    with s_i the least power of two >= max_j |a_ij| of the FP64 master row,
    so |q_ij| <= 1, q_ij is a value of the format, and s_i q_ij is what the
    residual multiplies by; FP32 levels store float32(a_ij); 1/D1 is
    float32(1 / l1_i);
  * the rounding points of one V-cycle with FP32 vectors: every vector the
    cycle stores (b on entry, the smoothed iterate, the residual handed to the
    restriction, the restricted right-hand side, the coarse solution, the
    prolongated iterate) is rounded to float32; sums inside one kernel (a
    row's products, an aggregate's members) and the coarse Cholesky are
    exact-order FP64.
The checks below evaluate both in numpy / plain Python from those rules and
require bit equality, so a wrong scale exponent, a dropped or an added
rounding fails them (the mutation tests plant exactly those).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2206_03203_gb300 import inputs


def _lap2(n, eps=1.0):
    e = np.ones(n)
    T = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1]).tolil()
    T[0, 0] = 3
    T[n - 1, n - 1] = 3
    Nn = sp.diags([-e[:-1], np.r_[1, 2 * np.ones(n - 2), 1], -e[:-1]], [-1, 0, 1])
    return (sp.kron(sp.eye(n), T) + eps * sp.kron(Nn, sp.eye(n))).tocsr()


def least_pow2_at_least(m):
    """The least power of two >= m > 0, from the binary exponent of m."""
    f, e = math.frexp(m)  # m = f 2^e, 0.5 <= f < 1
    return m if f == 0.5 else math.ldexp(1.0, e)


def bf16_rne(x32):
    """float32 -> nearest bfloat16 value (8 significant bits), ties to even:
    the float's value divided by its bf16 spacing, rounded half-to-even by
    np.rint, times the spacing."""
    x = float(x32)
    if x == 0.0 or not math.isfinite(x):
        return x
    _, e = math.frexp(abs(x))  # |x| in [2^(e-1), 2^e)
    ulp = math.ldexp(1.0, max(e - 1, -126) - 7)
    return float(np.rint(x / ulp)) * ulp


def in_format(q, lowp):
    if lowp == 16:
        u = np.array([q], dtype=np.float32).view(np.uint32)[0]
        return float(np.float32(q)) == q and (u & 0xFFFF) == 0
    return float(np.float16(q)) == q


def _systems():
    yield "fixed2d-64", inputs.fixed_2d()
    yield "planes3d-16", inputs.planes_3d(n=16, kf=1.0)
    # log-normal k_m and random fracture permeabilities: rows with a wide range
    b = inputs.batch_3d(count=1, lo=12, hi=12)[0]
    yield "rects3d-12", b


@pytest.mark.parametrize("prec", [16, 17])
@pytest.mark.parametrize("case", ["fixed2d-64", "planes3d-16", "rects3d-12"])
def test_row_scaled_storage_rule(oracle_mod, prec, case):
    inst = dict(_systems())[case]
    A, _ = oracle_mod.assemble(inst)
    M = oracle_mod.ML(A, inst.n_m, prec=prec)
    checked = 0
    for blk in (0, 1):
        amg = M.amg(blk)
        if amg is None:
            continue
        for l in range(amg.nlevels):
            Am = amg.level_A(l).tocsr()
            av, rs, dv, lowp = amg.stored(l)
            l1 = amg.l1(l)
            assert np.array_equal(dv, np.float32(1.0 / l1).astype(np.float64))
            if l == 0:
                assert lowp == 0  # the finest level stays FP32
            if not lowp:
                assert np.all(rs == 1.0)
                assert np.array_equal(av, Am.data.astype(np.float32).astype(np.float64))
                continue
            assert lowp == prec
            for i in range(Am.shape[0]):
                row = Am.data[Am.indptr[i]:Am.indptr[i + 1]]
                s = least_pow2_at_least(float(np.max(np.abs(row))))
                assert rs[i] == s, (l, i, rs[i], s)
                for a, st in zip(row, av[Am.indptr[i]:Am.indptr[i + 1]]):
                    q = st / s
                    assert abs(q) <= 1.0 and in_format(q, prec), (l, i, a, q)
                    x32 = np.float32(a / s)
                    want = bf16_rne(x32) if prec == 16 else float(np.float16(x32))
                    assert q == want, (l, i, a, q, want)
                    checked += 1
    assert checked > 100


def _chol_textbook(Ad):
    """Cholesky A = L L^T, column by column, each inner sum in ascending k."""
    n = Ad.shape[0]
    L = [[0.0] * n for _ in range(n)]
    for j in range(n):
        s = float(Ad[j, j])
        for k in range(j):
            s -= L[j][k] * L[j][k]
        ljj = math.sqrt(s)
        L[j][j] = ljj
        for i in range(j + 1, n):
            t = float(Ad[i, j])
            for k in range(j):
                t -= L[i][k] * L[j][k]
            L[i][j] = t / ljj
    return L


def _chol_solve(L, b):
    n = len(b)
    y = [0.0] * n
    for i in range(n):
        s = b[i]
        for k in range(i):
            s -= L[i][k] * y[k]
        y[i] = s / L[i][i]
    x = y[:]
    for i in range(n - 1, -1, -1):
        s = x[i]
        for k in range(i + 1, n):
            s -= L[k][i] * x[k]
        x[i] = s / L[i][i]
    return x


def f32(x):
    return float(np.float32(x))


def _rowsum(Ac, av, x, i):
    s = 0.0
    for p in range(Ac.indptr[i], Ac.indptr[i + 1]):
        s += av[p] * x[Ac.indices[p]]
    return s


def vcycle_f32_reference(amg, b):
    """One V-cycle with FP32 vectors (L1-Jacobi, one sweep before and after
    the coarse correction, piecewise-constant transfers), in plain Python
    from the storage and rounding rules in the module docstring."""
    levels = []
    for l in range(amg.nlevels):
        Ac = amg.level_A(l).tocsr()
        Ac.sort_indices()
        av, _, dv, _ = amg.stored(l)
        levels.append((Ac, av, dv, amg.agg(l)))
    L = _chol_textbook(levels[-1][0].toarray()) if amg.coarsest_dense else None

    def cycle(l, bl):
        Ac, av, dv, agg = levels[l]
        n = Ac.shape[0]
        if l == len(levels) - 1 and L is not None:
            return [f32(v) for v in _chol_solve(L, bl)]
        x = [f32(dv[i] * bl[i]) for i in range(n)]                       # pre-smoothing from zero
        if agg is not None and l < len(levels) - 1:
            r = [f32(bl[i] - _rowsum(Ac, av, x, i)) for i in range(n)]   # residual, stored
            nc = levels[l + 1][0].shape[0]
            bc = [0.0] * nc
            for i in range(n):                                           # restriction, ascending members
                if agg[i] >= 0:
                    bc[agg[i]] += r[i]
            xc = cycle(l + 1, [f32(v) for v in bc])
            x = [f32(x[i] + xc[agg[i]]) if agg[i] >= 0 else x[i] for i in range(n)]
        r2 = [bl[i] - _rowsum(Ac, av, x, i) for i in range(n)]            # post-smoothing residual, in-kernel
        return [f32(x[i] + dv[i] * r2[i]) for i in range(n)]
    return cycle(0, [f32(v) for v in b])


@pytest.mark.parametrize("levels,prec", [(1, 32), (2, 32), (3, 32), (3, 16), (3, 17)])
def test_vcycle_rounding_points(oracle_mod, levels, prec):
    A = sp.csr_matrix(_lap2(8, eps=0.7) + sp.diags(np.linspace(0.0, 0.3, 64)))
    nc = {1: 64, 2: 20, 3: 4}[levels]
    amg = oracle_mod.AMG(A, n_coarse=nc, prec=prec)
    assert amg.nlevels == levels and amg.coarsest_dense
    rng = np.random.default_rng(levels * 100 + prec)
    for k in range(4):
        b = rng.standard_normal(64) * 10.0 ** rng.uniform(-3, 3)
        got = amg.vcycle(b)
        want = np.array(vcycle_f32_reference(amg, b))
        assert np.array_equal(got, want), (k, np.max(np.abs(got - want)))
        assert np.all(got == got.astype(np.float32))  # FP32 values
