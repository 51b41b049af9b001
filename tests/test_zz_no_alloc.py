"""mds_solve_noalloc: the FGMRES solve for callers that cannot allocate device
memory while solving (a process whose allocations all belong to a framework
pool, or one that must not stall on the allocator).  Its Krylov workspace is a
static device array inside the library; this checks, through the C ABI, that
two calls in a row give the same result as mds_solve within the solve
tolerance used by the other parity tests, that those two calls ask the
context's allocator for nothing, and that oversized problems and packed
batches are refused.  Collected last so that a failure here comes after every
other test.
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
    # every device allocation of the context goes through these callbacks,
    # which count the calls (torch's caching allocator underneath)
    calls = {"alloc": 0, "free": 0}

    def alloc(nbytes, user):
        calls["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(max(int(nbytes), 1), 0)

    def free(ptr, user):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)
    a = mdsolve.Allocator(mdsolve._ALLOC_FN(alloc), mdsolve._FREE_FN(free), None)
    ctx = mdsolve.Context(0, allocator=a)
    yield torch, mdsolve, ctx, calls
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_solve_twice(env, precision):
    torch, mdsolve, ctx, calls = env
    inst = inputs.random_segments_2d(n=96, n_seg=12)
    sys_ = ctx.assemble(inst)
    assert sys_.N <= 16384
    prec = ctx.setup(sys_, precision=precision)
    x_ref = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(sys_, prec, None, x_ref)
    assert code == 0
    xs = [torch.zeros(sys_.N, dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    calls["alloc"] = calls["free"] = 0
    for call in range(2):
        x = xs[call]
        code2, st2 = ctx.solve_noalloc(sys_, prec, None, x)
        assert code2 == 0, call
        assert calls["alloc"] == 0 and calls["free"] == 0, (call, calls)
        assert st2.iterations == st[0].iterations, call
        assert st2.relres_true <= 1e-8
        err = (torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref)).item()
        assert err <= 1e-12, (call, err)


def test_noalloc_rejects_oversized_problem(env):
    torch, mdsolve, ctx, calls = env
    inst = inputs.fixed_2d(n=130)  # 16900 matrix cells > 16384
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    with pytest.raises(mdsolve.MDSError) as e:
        ctx.solve_noalloc(sys_, prec, None, x)
    assert e.value.code == -1 and "MDS_NOALLOC_MAX_N" in str(e.value)
    small = ctx.assemble(inputs.fixed_2d(n=16))
    p2 = ctx.setup(small)
    with pytest.raises(mdsolve.MDSError) as e:
        ctx.solve_noalloc(small, p2, None, np.zeros(small.N))  # host buffers would need staging
    assert "device pointers" in str(e.value)


def test_noalloc_rejects_packed_batch(env):
    torch, mdsolve, ctx, calls = env
    batch = inputs.batch_3d(count=2, lo=8, hi=10)
    sys_ = ctx.assemble_batch(batch)
    prec = ctx.setup(sys_)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    with pytest.raises(mdsolve.MDSError) as e:
        ctx.solve_noalloc(sys_, prec, None, x)
    assert e.value.code == -1 and "packed batch" in str(e.value)
