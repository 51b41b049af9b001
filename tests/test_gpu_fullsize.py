"""Full-size workloads beyond the benchmark's 1024^2 sweep: the 128^3
nine-plane instance (k_f = 1e-4, 1, 1e4), the batch of 256 uneven 3D
instances with 4 right-hand sides each, and the 256^3 instance with 30
rectangles and 8 right-hand sides.

Where the oracle can assemble them in seconds the GPU assembly is compared
bit for bit (the 128^3 instance, and a sample of the batch's instances cut
out of the packed system); everywhere the solves are checked by properties
that hold at any size: the true relative residual of every column, computed
on the host in FP64 (scipy) from the assembled matrix, meets the stopping
rule, and the assembled matrix is symmetric with non-positive off-diagonals
and non-negative row sums (Dirichlet terms only).
"""
import numpy as np
import pytest

from paper_2206_03203_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_03203_gb300 import build, mdsolve
    build.build()
    return torch, mdsolve.Context(0)


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def same_csr(A, B):
    return (A.shape == B.shape and np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
            and np.array_equal(A.data, B.data))


def matrix_properties(A):
    D = A - A.T
    assert D.nnz == 0 or np.max(np.abs(D.data)) == 0.0  # exactly symmetric
    off = A.copy()
    off.setdiag(0.0)
    off.eliminate_zeros()
    assert off.nnz == 0 or np.max(off.data) <= 0.0
    rs = np.asarray(A.sum(axis=1)).ravel()
    assert np.min(rs) >= -1e-12 * np.max(np.abs(A.diagonal()))


def residuals(A, B, X):
    """Relative 2-norm residual of every column (columns stored [nrhs][N])."""
    return [np.linalg.norm(b - A @ x) / np.linalg.norm(b) for b, x in zip(B, X)]


@pytest.mark.parametrize("kf", [1e-4, 1.0, 1e4])
def test_planes3d_128(env, oracle_mod, kf):
    torch, ctx = env
    inst = inputs.planes_3d(128, kf=kf)
    sys_ = ctx.assemble(inst)
    (_, _, _, _, A), b = sys_.to_host()
    Ao, bo = oracle_mod.assemble(inst)
    assert same_csr(A, Ao) and np.array_equal(b, bo)
    for precision in ("fp64", "fp32"):
        prec = ctx.setup(sys_, precision=precision)
        x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
        code, st = ctx.solve(sys_, prec, None, x, max_iters=5000)
        assert code == 0, (kf, precision, st[0])
        rel = residuals(Ao, bo[:1], [x.cpu().numpy()])[0]
        assert rel <= 1.01e-8, (kf, precision, rel)
        prec.close()


def test_batch_256_instances_4_rhs(env, oracle_mod):
    torch, ctx = env
    batch = inputs.batch_3d(256)
    sys_ = ctx.assemble_batch(batch)
    (_, _, _, _, A), b = sys_.to_host()
    matrix_properties(A)
    mo, fo = sys_.instances()
    NM = sys_.n_m
    # a sample of instances, cut out of the packed system, against the oracle
    for k in np.random.default_rng(8).choice(len(batch), size=6, replace=False):
        rows = np.concatenate([np.arange(mo[k], mo[k + 1]), NM + np.arange(fo[k], fo[k + 1])])
        Ak = A[rows][:, rows].tocsr()
        Ak.sort_indices()
        Ao, bo = oracle_mod.assemble(batch[k])
        assert same_csr(Ak, Ao), k
        assert np.array_equal(b[:, rows], bo), k
    prec = ctx.setup(sys_, precision="bf16", format="auto")
    x = torch.zeros(sys_.N * 4, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, nrhs=4, max_iters=5000)
    assert code == 0 and len(st) == 256 * 4
    assert all(s.status == 0 and s.relres_true <= 1e-8 for s in st)
    X = x.cpu().numpy().reshape(4, sys_.N)
    # per instance and column: the residual restricted to the instance's rows
    for k in range(0, len(batch), 37):
        rows = np.concatenate([np.arange(mo[k], mo[k + 1]), NM + np.arange(fo[k], fo[k + 1])])
        Ak = A[rows][:, rows].tocsr()
        rel = residuals(Ak, b[:, rows], X[:, rows])
        assert max(rel) <= 1.01e-8, (k, rel)


def test_large_256_cubed_8_rhs(env):
    torch, ctx = env
    inst = inputs.large_3d(256)
    sys_ = ctx.assemble(inst)
    (_, _, _, _, A), b = sys_.to_host()
    matrix_properties(A)
    prec = ctx.setup(sys_, precision="fp16", format="auto")
    x = torch.zeros(sys_.N * 8, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x, nrhs=8, max_iters=5000)
    assert code == 0 and len(st) == 8
    rel = residuals(A, b, x.cpu().numpy().reshape(8, sys_.N))
    assert max(rel) <= 1.01e-8, rel
