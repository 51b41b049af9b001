"""Asynchronous solves (mds_solve_async / mds_solve_done / mds_solve_wait):
the same result as the blocking call, concurrency across contexts on their
own streams, other calls on a busy context waiting for it, and error paths.
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
    return torch, mdsolve


def make(torch, mdsolve, stream, contrast):
    ctx = mdsolve.Context(0, stream=stream.cuda_stream)
    ctx._stream = stream  # keep the stream object with the context
    inst = inputs.random_segments_2d(n=256, n_seg=20, contrast=contrast)
    sys_ = ctx.assemble(inst)
    prec = ctx.setup(sys_, format="csr")
    return ctx, sys_, prec


def test_async_equals_blocking_on_concurrent_contexts(env):
    torch, mdsolve = env
    streams = [torch.cuda.Stream() for _ in range(3)]
    runs = [make(torch, mdsolve, s, c) for s, c in zip(streams, (1e-4, 1.0, 1e4))]
    ref = []
    for ctx, sys_, prec in runs:
        x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        code, st = ctx.solve(sys_, prec, None, x)
        assert code == 0
        ref.append((x.clone(), st[0].iterations))
    xs = [torch.zeros(sys_.N, dtype=torch.float64, device="cuda") for _, sys_, _ in runs]
    torch.cuda.synchronize()  # the contexts run on their own streams
    for (ctx, sys_, prec), x in zip(runs, xs):
        ctx.solve_async(sys_, prec, None, x)
    for (ctx, sys_, prec), x, (xr, it) in zip(runs, xs, ref):
        code, st = ctx.solve_wait()
        assert code == 0 and st[0].iterations == it and st[0].relres_true <= 1e-8
        torch.cuda.synchronize()
        assert torch.equal(x, xr)


def test_calls_on_a_busy_context_wait(env):
    torch, mdsolve = env
    ctx, sys_, prec = make(torch, mdsolve, torch.cuda.Stream(), 1e2)
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    ctx.solve_async(sys_, prec, None, x)
    ctx.spmv(sys_, x, y)  # joins the solve first, so x is the solution
    assert ctx.solve_done()
    code, st = ctx.solve_wait()
    assert code == 0
    torch.cuda.synchronize()
    (_, _, _, _, A), b = sys_.to_host()
    assert np.allclose(y.cpu().numpy(), A @ x.cpu().numpy(), rtol=1e-13, atol=1e-13)
    assert np.linalg.norm(b[0] - A @ x.cpu().numpy()) <= 1.01e-8 * np.linalg.norm(b[0])


def test_host_buffers_async(env):
    torch, mdsolve = env
    ctx, sys_, prec = make(torch, mdsolve, torch.cuda.Stream(), 1.0)
    xh = np.zeros(sys_.N)
    ctx.solve_async(sys_, prec, None, xh)
    code, st = ctx.solve_wait()
    (_, _, _, _, A), b = sys_.to_host()
    assert code == 0 and np.linalg.norm(b[0] - A @ xh) <= 1.01e-8 * np.linalg.norm(b[0])


def test_async_error_paths(env):
    torch, mdsolve = env
    ctx, sys_, prec = make(torch, mdsolve, torch.cuda.Stream(), 1.0)
    with pytest.raises(mdsolve.MDSError):
        ctx.solve_wait()  # nothing pending
    x = torch.zeros(sys_.N, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    ctx.solve_async(sys_, prec, None, x)
    with pytest.raises(mdsolve.MDSError):
        ctx.solve_async(sys_, prec, None, x)  # the first one was not collected
    code, _ = ctx.solve_wait()
    assert code == 0
    b = torch.full((sys_.N,), float("nan"), dtype=torch.float64, device="cuda")
    x.zero_()
    torch.cuda.synchronize()
    ctx.solve_async(sys_, prec, b, x)
    with pytest.raises(mdsolve.MDSError):
        ctx.solve_wait()
    # the context is usable afterwards
    x.zero_()
    torch.cuda.synchronize()
    code, st = ctx.solve(sys_, prec, None, x)
    assert code == 0 and st[0].relres_true <= 1e-8


def test_torch_caching_allocator(env):
    """A context whose device memory comes from torch's caching allocator
    (mds_allocator): the same solution as with the library's own allocation,
    the memory visible to torch while the objects live, returned after."""
    torch, mdsolve = env
    inst = inputs.random_segments_2d(n=256, n_seg=20, contrast=1e2)
    ref = mdsolve.Context(0)
    s0 = ref.assemble(inst)
    p0 = ref.setup(s0, format="csr")
    x0 = torch.zeros(s0.N, dtype=torch.float64, device="cuda")
    code0, st0 = ref.solve(s0, p0, None, x0)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated(0)
    ctx = mdsolve.Context(0, allocator="torch")
    s = ctx.assemble(inst)
    p = ctx.setup(s, format="csr")
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(s, p, None, x)
    torch.cuda.synchronize()
    held = torch.cuda.memory_allocated(0) - base
    assert code == code0 == 0 and st[0].iterations == st0[0].iterations
    assert torch.equal(x, x0)
    assert held > 8 * s.N * 4  # the blocks and the hierarchy live in torch-managed memory
    p.close()
    s.close()
    ctx.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(0) - base <= 8 * s.N + (1 << 20)  # only x remains


def test_allocator_returning_null_reports_oom(env):
    """A caller allocator that returns NULL makes the call fail with
    MDS_ERR_OOM (-3); the context stays usable for calls that fit."""
    torch, mdsolve = env
    state = {"fail": True}

    def alloc(nbytes, user):
        if state["fail"]:
            return None
        return torch.cuda.caching_allocator_alloc(max(int(nbytes), 1), 0)

    def free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)
    a = mdsolve.Allocator(mdsolve._ALLOC_FN(alloc), mdsolve._FREE_FN(free), None)
    ctx = mdsolve.Context(0, allocator=a)
    with pytest.raises(mdsolve.MDSError) as e:
        ctx.assemble(inputs.fixed_2d(n=8))
    assert e.value.code == -3
    state["fail"] = False
    s = ctx.assemble(inputs.fixed_2d(n=8))
    p = ctx.setup(s)
    x = torch.zeros(s.N, dtype=torch.float64, device="cuda")
    code, st = ctx.solve(s, p, None, x)
    assert code == 0 and st[0].relres_true <= 1e-8
    p.close()
    s.close()
    ctx.close()
