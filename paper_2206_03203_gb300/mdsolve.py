"""Thin ctypes binding of libmdsolve (include/mdsolve.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
PyTorch provides device memory and the CUDA stream.  If the library is
missing this module raises; there is no CPU fallback.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref
from dataclasses import dataclass
from typing import Optional

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libmdsolve.so")

MDS_OK = 0
MDS_WARN_NOT_CONVERGED = 1
PREC = {"fp64": 64, "fp32": 32, "bf16": 16, "fp16": 17}
FORMAT = {"auto": 0, "csr": 1, "sell": 2, "stencil": 3, "stencil-bulk": 4}
FORM = {"auto": 0, "fused": 1, "stored": 2}
PROLONG = {"piecewise": 0, "smoothed": 1}
SMOOTHER = {"l1jacobi": 0, "chebyshev": 1}
KIND = {"lower": 0, "diag": 1, "upper": 2}
KRYLOV = {"fgmres": 0, "pcg": 1, "minres": 2}
KCLASS = {"spmv": 0, "vc_resid": 1, "vc_post": 2, "gs_dot": 3, "gs_axpy": 4, "vcycle": 5, "vc_restrict": 6}


class MDSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mdsolve error {code}: {msg}")
        self.code = code


class Instance(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int), ("km", C.c_void_p), ("n_f", C.c_int64),
                ("fc_axis", C.c_void_p), ("fc_pos", C.c_void_p), ("fc_kf", C.c_void_p), ("fc_a", C.c_void_p),
                ("nrhs", C.c_int), ("pD_left", C.c_void_p), ("pD_right", C.c_void_p), ("on_device", C.c_int),
                ("junction", C.c_int), ("fc_kn", C.c_void_p)]


JUNCTION = {"pairwise": 0, "star": 1, 0: 0, 1: 1}


class Csr(C.Structure):
    _fields_ = [("nrow", C.c_int64), ("ncol", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class TuneCandidate(C.Structure):
    _fields_ = [("smoother", C.c_int), ("sweeps", C.c_int), ("cheb_degree", C.c_int), ("precision", C.c_int),
                ("status", C.c_int), ("iterations", C.c_int), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("n_coarse", C.c_int64)]


# smoother, sweeps, Chebyshev degree, precision[, coarsest size N_c (0: the base options')]
TUNE_DEFAULT = [("l1jacobi", 1, 2, "fp64"), ("l1jacobi", 2, 2, "fp64"), ("chebyshev", 1, 2, "fp64"),
                ("chebyshev", 1, 3, "fp64"), ("l1jacobi", 1, 2, "fp32"), ("l1jacobi", 2, 2, "fp32"),
                ("chebyshev", 1, 2, "fp32"), ("chebyshev", 1, 3, "fp32")]


class SetupOpts(C.Structure):
    _fields_ = [("theta", C.c_double), ("n_coarse", C.c_int64), ("max_levels", C.c_int),
                ("stall_ratio", C.c_double), ("seed", C.c_uint64), ("smoother", C.c_int),
                ("precision", C.c_int), ("lowp_from_level", C.c_int), ("kind", C.c_int), ("format", C.c_int),
                ("sell_c", C.c_int), ("sell_sigma", C.c_int), ("sweeps", C.c_int), ("prolongation", C.c_int),
                ("coarse_tail", C.c_int), ("cheb_degree", C.c_int), ("level_form", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("krylov", C.c_int), ("restart", C.c_int), ("rtol", C.c_double), ("max_iters", C.c_int),
                ("use_precond", C.c_int), ("graphs", C.c_int), ("batched", C.c_int), ("reorth_eta2", C.c_double),
                ("x0_zero", C.c_int)]


class RhsStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("relres_est", C.c_double), ("relres_true", C.c_double)]


_lib = None

# Live handles, closed in dependency order (preconditioners, systems, contexts)
# before interpreter teardown, whatever order the garbage collector would pick.
_live = {0: weakref.WeakSet(), 1: weakref.WeakSet(), 2: weakref.WeakSet()}
_atexit_registered = False


def _close_all():
    for rank in (0, 1, 2):
        for obj in list(_live[rank]):
            try:
                obj.close()
            except Exception:
                pass


def _track(obj, rank):
    global _atexit_registered
    _live[rank].add(obj)
    if not _atexit_registered:
        # registered after torch is imported, so it runs before torch's own exit handlers
        atexit.register(_close_all)
        _atexit_registered = True

# Every entry point of include/mdsolve.h with its ctypes signature.
_SIGS = {
    "mds_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_void_p]),
    "mds_destroy": (C.c_int, [C.c_void_p]),
    "mds_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mds_error_string": (C.c_char_p, [C.c_int]),
    "mds_last_error": (C.c_char_p, [C.c_void_p]),
    "mds_assemble": (C.c_int, [C.c_void_p, C.POINTER(Instance), C.POINTER(C.c_void_p)]),
    "mds_assemble_flux": (C.c_int, [C.c_void_p, C.POINTER(Instance), C.POINTER(C.c_void_p)]),
    "mds_assemble_batch": (C.c_int, [C.c_void_p, C.POINTER(Instance), C.c_int, C.POINTER(C.c_void_p)]),
    "mds_system_instances": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mds_system_from_csr": (C.c_int, [C.c_void_p] + [C.POINTER(Csr)] * 4 + [C.c_void_p, C.POINTER(C.c_void_p)]),
    "mds_system_destroy": (C.c_int, [C.c_void_p]),
    "mds_system_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int64)]),
    "mds_system_view": (C.c_int, [C.c_void_p, C.POINTER(Csr), C.POINTER(C.c_void_p)]),
    "mds_setup_opts_default": (C.c_int, [C.POINTER(SetupOpts)]),
    "mds_setup": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(SetupOpts), C.POINTER(C.c_void_p)]),
    "mds_precond_destroy": (C.c_int, [C.c_void_p]),
    "mds_precond_info": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "mds_precond_level": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(Csr), C.POINTER(C.c_void_p),
                                    C.POINTER(C.c_void_p)]),
    "mds_precond_prolongator": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(Csr)]),
    "mds_precond_level_storage": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int),
                                            C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                            C.POINTER(C.c_void_p), C.POINTER(C.c_int)]),
    "mds_precond_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mds_vcycle": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mds_spmv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mds_solve_opts_default": (C.c_int, [C.POINTER(SolveOpts)]),
    "mds_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                            C.POINTER(SolveOpts), C.POINTER(RhsStats)]),
    "mds_tune": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(SetupOpts), C.POINTER(SolveOpts), C.c_void_p,
                           C.POINTER(TuneCandidate), C.c_int, C.POINTER(C.c_int)]),
    "mds_solve_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                  C.POINTER(SolveOpts)]),
    "mds_solve_done": (C.c_int, [C.c_void_p]),
    "mds_solve_wait": (C.c_int, [C.c_void_p, C.POINTER(RhsStats), C.c_int]),
    "mds_solve_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.POINTER(SolveOpts), C.POINTER(RhsStats)]),
    "mds_timing_enable": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mds_timing_reset": (C.c_int, [C.c_void_p]),
    "mds_timing_query": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mds_timing_sample_every": (C.c_int, [C.c_void_p, C.c_int]),
    "mds_timing_sampled": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mds_memcpy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t]),
    "mds_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
}


def lib():
    """Load libmdsolve.so (built by paper_2206_03203_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmdsolve.so not built ({LIB_PATH}); run paper_2206_03203_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a) -> int:
    """Address of a torch tensor or numpy array (None -> 0)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def setup_opts(**kw) -> SetupOpts:
    o = SetupOpts()
    lib().mds_setup_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "precision":
            v = PREC.get(v, v)
        elif k == "smoother":
            v = SMOOTHER.get(v, v)
        elif k == "kind":
            v = KIND.get(v, v)
        elif k == "format":
            v = FORMAT.get(v, v)
        elif k == "prolongation":
            v = PROLONG.get(v, v)
        elif k == "level_form":
            v = FORM.get(v, v)
        setattr(o, k, v)
    return o


def solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().mds_solve_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "krylov":
            v = KRYLOV.get(v, v)
        setattr(o, k, v)
    return o


@dataclass
class Stats:
    iterations: int
    restarts: int
    status: int
    relres_est: float
    relres_true: float


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", C.c_void_p)]


def torch_allocator(device: int, stream: int) -> Allocator:
    """mds_allocator backed by torch's caching allocator (device memory then
    counts in torch.cuda.memory_allocated and is reused by torch)."""
    import torch

    def alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(max(int(nbytes), 1), device, stream)
        except Exception:  # out of memory: the library reports MDS_ERR_OOM
            return None

    def free(ptr, user):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:  # interpreter shutdown: torch may be gone already
            pass
    return Allocator(_ALLOC_FN(alloc), _FREE_FN(free), None)


def device_arrays(inst) -> dict:
    """Copies of an instance's input arrays in device memory (torch CUDA
    tensors keyed by field name), for assemble / assemble_batch."""
    import torch
    d = dict(km=inst.km, fc_axis=inst.fc_axis, fc_pos=np.ascontiguousarray(inst.fc_pos).reshape(-1),
             fc_kf=inst.fc_kf, fc_a=inst.fc_a, pD_left=inst.pD_left, pD_right=inst.pD_right)
    if getattr(inst, "fc_kn", None) is not None:
        d["fc_kn"] = inst.fc_kn
    return {k: torch.as_tensor(np.ascontiguousarray(v), device="cuda") for k, v in d.items()}


class Context:
    """A library context on one device and stream (torch's current stream by
    default).  allocator="torch" routes every device allocation of the
    library through torch's caching allocator (mds_allocator), an Allocator
    instance through its own callbacks; the default is the library's own
    stream-ordered allocation."""

    def __init__(self, device: int = 0, stream: Optional[int] = None, allocator: Optional[str] = None):
        import torch
        L = lib()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.device = device
        self._alloc = None
        if allocator == "torch":
            self._alloc = torch_allocator(device, stream)  # the callbacks live as long as the context
        elif isinstance(allocator, Allocator):
            self._alloc = allocator
        elif allocator is not None:
            raise ValueError(f"unknown allocator {allocator!r}")
        h = C.c_void_p()
        self._check(L.mds_create(C.byref(h), device, C.c_void_p(stream),
                                 C.byref(self._alloc) if self._alloc is not None else None), ctx=False)
        self.h = h
        _track(self, 2)

    def _check(self, code, ctx=True):
        if code < 0:
            msg = lib().mds_last_error(self.h).decode() if ctx else lib().mds_error_string(code).decode()
            raise MDSError(code, msg)
        return code

    def close(self):
        if getattr(self, "h", None):
            # dependents first
            for rank in (0, 1):
                for obj in list(_live[rank]):
                    if obj.ctx is self:
                        obj.close()
            lib().mds_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: int):
        self._check(lib().mds_set_stream(self.h, C.c_void_p(stream)))

    # ---- problem ----
    def assemble_batch(self, insts, junction=0, device_arrays: Optional[list] = None) -> "System":
        """Pack several instances into one block-diagonal system.  With
        ``device_arrays`` (one dict of torch CUDA tensors per instance, keyed
        by field name) the device copies are read instead of the host arrays."""
        keep, arr = [], (Instance * len(insts))()
        for k, inst in enumerate(insts):
            if device_arrays is None:
                a = dict(km=np.ascontiguousarray(inst.km, dtype=np.float64),
                         fc_axis=np.ascontiguousarray(inst.fc_axis, dtype=np.int32),
                         fc_pos=np.ascontiguousarray(inst.fc_pos, dtype=np.int32).reshape(-1),
                         fc_kf=np.ascontiguousarray(inst.fc_kf, dtype=np.float64),
                         fc_a=np.ascontiguousarray(inst.fc_a, dtype=np.float64),
                         pD_left=np.ascontiguousarray(inst.pD_left, dtype=np.float64),
                         pD_right=np.ascontiguousarray(inst.pD_right, dtype=np.float64))
                if getattr(inst, "fc_kn", None) is not None:
                    a["fc_kn"] = np.ascontiguousarray(inst.fc_kn, dtype=np.float64)
                on_dev = 0
            else:
                a, on_dev = device_arrays[k], 1
            keep.append(a)
            arr[k] = Instance(inst.dim, inst.n, _ptr(a["km"]), inst.n_f, _ptr(a["fc_axis"]), _ptr(a["fc_pos"]),
                              _ptr(a["fc_kf"]), _ptr(a["fc_a"]), inst.nrhs, _ptr(a["pD_left"]), _ptr(a["pD_right"]),
                              on_dev, JUNCTION[junction], _ptr(a.get("fc_kn")))
        h = C.c_void_p()
        self._check(lib().mds_assemble_batch(self.h, arr, len(insts), C.byref(h)))
        return System(self, h)

    def assemble(self, inst, device_arrays: Optional[dict] = None, form: str = "primal",
                 junction=0) -> "System":
        """Assemble an instance (paper_2206_03203_gb300.inputs.Instance).  With
        ``device_arrays`` (torch CUDA tensors keyed by field name) the device
        copies are used instead of the host arrays.  form="flux": the
        paper's partition [pressures of all cells; interface fluxes].
        junction: "pairwise" (0) or "star" (1: star-delta in the primal form,
        intersection cells with their own fluxes in the flux form)."""
        if form not in ("primal", "flux"):
            raise ValueError(f"unknown form {form!r}")
        keep = []
        if device_arrays is None:
            arrs = dict(km=np.ascontiguousarray(inst.km, dtype=np.float64),
                        fc_axis=np.ascontiguousarray(inst.fc_axis, dtype=np.int32),
                        fc_pos=np.ascontiguousarray(inst.fc_pos, dtype=np.int32).reshape(-1),
                        fc_kf=np.ascontiguousarray(inst.fc_kf, dtype=np.float64),
                        fc_a=np.ascontiguousarray(inst.fc_a, dtype=np.float64),
                        pD_left=np.ascontiguousarray(inst.pD_left, dtype=np.float64),
                        pD_right=np.ascontiguousarray(inst.pD_right, dtype=np.float64))
            if getattr(inst, "fc_kn", None) is not None:
                arrs["fc_kn"] = np.ascontiguousarray(inst.fc_kn, dtype=np.float64)
            on_dev = 0
        else:
            arrs = device_arrays
            on_dev = 1
        keep.append(arrs)
        s = Instance(inst.dim, inst.n, _ptr(arrs["km"]), inst.n_f, _ptr(arrs["fc_axis"]), _ptr(arrs["fc_pos"]),
                     _ptr(arrs["fc_kf"]), _ptr(arrs["fc_a"]), inst.nrhs, _ptr(arrs["pD_left"]),
                     _ptr(arrs["pD_right"]), on_dev, JUNCTION[junction], _ptr(arrs.get("fc_kn")))
        h = C.c_void_p()
        fn = lib().mds_assemble_flux if form == "flux" else lib().mds_assemble
        self._check(fn(self.h, C.byref(s), C.byref(h)))
        return System(self, h)

    def system_from_csr(self, blocks, b=None) -> "System":
        """blocks: four (row_ptr, col, val, nrow, ncol) tuples of torch CUDA
        tensors (int32, int32, float64), kept alive by the returned System."""
        cs = [Csr(nr, nc, int(v.numel()), _ptr(rp), _ptr(ci), _ptr(v)) for (rp, ci, v, nr, nc) in blocks]
        h = C.c_void_p()
        self._check(lib().mds_system_from_csr(self.h, *[C.byref(x) for x in cs], C.c_void_p(_ptr(b)), C.byref(h)))
        s = System(self, h)
        s._keep = (blocks, b)
        return s

    def setup(self, sys: "System", **opts) -> "Precond":
        o = setup_opts(**opts)
        h = C.c_void_p()
        self._check(lib().mds_setup(self.h, sys.h, C.byref(o), C.byref(h)))
        return Precond(self, sys, h)

    def solve(self, sys: "System", prec: Optional["Precond"], b=None, x=None, nrhs: int = 1, **opts):
        """Solve on device tensors (or host numpy arrays).  x holds x0 and is
        overwritten (x0_zero=True: the initial guess is zero and x is output
        only).  Returns (status, [Stats])."""
        o = solve_opts(**opts)
        st = (RhsStats * (nrhs * sys.n_inst))()
        code = lib().mds_solve(self.h, sys.h, prec.h if prec is not None else None, C.c_void_p(_ptr(b)),
                               C.c_void_p(_ptr(x)), nrhs, C.byref(o), st)
        self._check(code)
        return code, [Stats(s.iterations, s.restarts, s.status, s.relres_est, s.relres_true) for s in st]

    def tune(self, sys: "System", candidates=None, b=None, base: Optional[dict] = None, **solve_kw):
        """Time set-up + solve for each (smoother, sweeps, cheb_degree,
        precision) candidate; returns (best index or -1, [dict per
        candidate])."""
        cands = candidates or TUNE_DEFAULT
        arr = (TuneCandidate * len(cands))()
        for k, cand in enumerate(cands):
            sm, sw, dg, pr = cand[:4]
            nc = cand[4] if len(cand) > 4 else 0
            arr[k] = TuneCandidate(SMOOTHER.get(sm, sm), sw, dg, PREC.get(pr, pr), 0, 0, 0.0, 0.0, nc)
        so = setup_opts(**(base or {}))
        o = solve_opts(**solve_kw)
        best = C.c_int(-1)
        self._check(lib().mds_tune(self.h, sys.h, C.byref(so), C.byref(o), C.c_void_p(_ptr(b)), arr, len(cands),
                                   C.byref(best)))
        return best.value, [dict(candidate=cands[k], status=a.status, iterations=a.iterations,
                                 setup_ms=a.setup_ms, solve_ms=a.solve_ms) for k, a in enumerate(arr)]

    def solve_async(self, sys: "System", prec: Optional["Precond"], b=None, x=None, nrhs: int = 1, **opts):
        """Start the solve on a library thread and return at once; collect it
        with solve_wait.  b, x, sys and prec must stay alive until then (the
        context keeps references)."""
        o = solve_opts(**opts)
        self._check(lib().mds_solve_async(self.h, sys.h, prec.h if prec is not None else None, C.c_void_p(_ptr(b)),
                                          C.c_void_p(_ptr(x)), nrhs, C.byref(o)))
        self._async = (sys, prec, b, x, nrhs * sys.n_inst)

    def solve_done(self) -> bool:
        return self._check(lib().mds_solve_done(self.h)) == 1

    def solve_wait(self):
        """Wait for the asynchronous solve.  Returns (status, [Stats]) as solve."""
        count = self._async[4] if getattr(self, "_async", None) else 0
        st = (RhsStats * max(count, 1))()
        code = lib().mds_solve_wait(self.h, st, count)
        self._async = None
        self._check(code)
        return code, [Stats(s.iterations, s.restarts, s.status, s.relres_est, s.relres_true) for s in st[:count]]

    def solve_noalloc(self, sys: "System", prec: Optional["Precond"], b=None, x=None, **opts):
        """FGMRES with the library's static workspace (device tensors only,
        n_m + n_f <= 16384).  Returns (status, Stats)."""
        o = solve_opts(**opts)
        st = RhsStats()
        code = lib().mds_solve_noalloc(self.h, sys.h, prec.h if prec is not None else None, C.c_void_p(_ptr(b)),
                                       C.c_void_p(_ptr(x)), C.byref(o), C.byref(st))
        self._check(code)
        return code, Stats(st.iterations, st.restarts, st.status, st.relres_est, st.relres_true)

    def spmv(self, sys, x, y):
        self._check(lib().mds_spmv(self.h, sys.h, C.c_void_p(_ptr(x)), C.c_void_p(_ptr(y))))

    def precond_apply(self, prec, r, z):
        self._check(lib().mds_precond_apply(self.h, prec.h, C.c_void_p(_ptr(r)), C.c_void_p(_ptr(z))))

    def vcycle(self, prec, block, b, x):
        self._check(lib().mds_vcycle(self.h, prec.h, block, C.c_void_p(_ptr(b)), C.c_void_p(_ptr(x))))

    def memcpy(self, dst: int, src: int, nbytes: int):
        self._check(lib().mds_memcpy(self.h, C.c_void_p(dst), C.c_void_p(src), nbytes))

    def to_host(self, ptr: int, count: int, dtype) -> np.ndarray:
        out = np.empty(count, dtype=dtype)
        if count:
            self.memcpy(out.ctypes.data, ptr, out.nbytes)
        return out

    def csr_to_host(self, c: Csr):
        import scipy.sparse as sp
        rp = self.to_host(c.row_ptr, c.nrow + 1, np.int32)
        ci = self.to_host(c.col, c.nnz, np.int32)
        v = self.to_host(c.val, c.nnz, np.float64)
        return sp.csr_matrix((v, ci, rp), shape=(c.nrow, c.ncol))

    # ---- measurement ----
    def timing_enable(self, kclass, on=True):
        k = KCLASS.get(kclass, kclass)
        self._check(lib().mds_timing_enable(self.h, k, 1 if on else 0))

    def timing_reset(self):
        self._check(lib().mds_timing_reset(self.h))

    def timing_query(self, kclass):
        k = KCLASS.get(kclass, kclass)
        n, ms, by, fl = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
        self._check(lib().mds_timing_query(self.h, k, C.byref(n), C.byref(ms), C.byref(by), C.byref(fl)))
        return n.value, ms.value, by.value, fl.value

    def timing_sample_every(self, every: int):
        """Bracket timed classes only in every `every`-th FGMRES restart cycle."""
        self._check(lib().mds_timing_sample_every(self.h, every))

    def timing_sampled(self, kclass):
        """(launches, ms, bytes, flops) of the bracketed launches of a class."""
        k = KCLASS.get(kclass, kclass)
        n, ms, by, fl = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
        self._check(lib().mds_timing_sampled(self.h, k, C.byref(n), C.byref(ms), C.byref(by), C.byref(fl)))
        return n.value, ms.value, by.value, fl.value

    def launch_count(self) -> int:
        n = C.c_int64()
        self._check(lib().mds_launch_count(self.h, C.byref(n)))
        return n.value


class System:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        n_m, n_f, nrhs = C.c_int64(), C.c_int64(), C.c_int()
        nnz = (C.c_int64 * 5)()
        ctx._check(lib().mds_system_info(h, C.byref(n_m), C.byref(n_f), C.byref(nrhs), nnz))
        self.n_m, self.n_f, self.nrhs = n_m.value, n_f.value, nrhs.value
        self.nnz = list(nnz)
        self.N = self.n_m + self.n_f
        ni = C.c_int()
        ctx._check(lib().mds_system_instances(h, C.byref(ni), None, None))
        self.n_inst = ni.value
        _track(self, 1)

    def close(self):
        if getattr(self, "h", None):
            for obj in list(_live[0]):
                if obj.sys is self:
                    obj.close()
            lib().mds_system_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def views(self):
        v = (Csr * 5)()
        b = C.c_void_p()
        self.ctx._check(lib().mds_system_view(self.h, v, C.byref(b)))
        return list(v), b.value

    def to_host(self):
        """(A_mm, A_mf, A_fm, A_ff, A) as scipy CSR and b [nrhs, N] as numpy."""
        v, b = self.views()
        mats = [self.ctx.csr_to_host(x) for x in v]
        bh = self.ctx.to_host(b, self.N * self.nrhs, np.float64).reshape(self.nrhs, self.N)
        return mats, bh

    def instances(self):
        """(m_off, f_off) row offsets of the packed instances."""
        mo = (C.c_int64 * (self.n_inst + 1))()
        fo = (C.c_int64 * (self.n_inst + 1))()
        self.ctx._check(lib().mds_system_instances(self.h, None, mo, fo))
        return list(mo), list(fo)

    def b_ptr(self, k: int = 0) -> int:
        return self.views()[1] + 8 * k * self.N


class Precond:
    def __init__(self, ctx: Context, sys: System, h):
        self.ctx, self.sys, self.h = ctx, sys, h
        _track(self, 0)

    def close(self):
        if getattr(self, "h", None):
            lib().mds_precond_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, block: int):
        nl, dense = C.c_int(), C.c_int()
        ln, lz = (C.c_int64 * 32)(), (C.c_int64 * 32)()
        self.ctx._check(lib().mds_precond_info(self.h, block, C.byref(nl), ln, lz, C.byref(dense)))
        return dict(nlevels=nl.value, n=list(ln)[:nl.value], nnz=list(lz)[:nl.value], dense=dense.value == 1,
                    diagonal=dense.value == 2)

    def prolongator_host(self, block: int, level: int):
        """Smoothed prolongator of a level as scipy CSR (None for injection)."""
        P = Csr()
        self.ctx._check(lib().mds_precond_prolongator(self.h, block, level, C.byref(P)))
        return self.ctx.csr_to_host(P) if P.row_ptr else None

    def level_storage_host(self, block: int, level: int):
        """(value type, stored values in CSR order as float64 or None, row
        scales or None, 1/D1) of a level, as its V-cycle applies them."""
        vt, fmt = C.c_int(), C.c_int()
        vals, rs, dv = C.c_void_p(), C.c_void_p(), C.c_void_p()
        self.ctx._check(lib().mds_precond_level_storage(self.h, block, level, C.byref(vt), C.byref(vals),
                                                        C.byref(rs), C.byref(dv), C.byref(fmt)))

        A, _, _ = self.level_host(block, level)
        n, nnz = A.shape[0], A.nnz
        v = None
        if vals.value:
            if vt.value == 64:
                v = self.ctx.to_host(vals.value, nnz, np.float64)
            elif vt.value == 32:
                v = self.ctx.to_host(vals.value, nnz, np.float32).astype(np.float64)
            elif vt.value == 16:
                u = self.ctx.to_host(vals.value, nnz, np.uint16).astype(np.uint32) << 16
                v = u.view(np.float32).astype(np.float64)
            else:
                v = self.ctx.to_host(vals.value, nnz, np.float16).astype(np.float64)
        r = self.ctx.to_host(rs.value, n, np.float32).astype(np.float64) if rs.value else None
        d = self.ctx.to_host(dv.value, n, np.float64 if vt.value == 64 else np.float32).astype(np.float64)
        return vt.value, v, r, d

    def level_format(self, block: int, level: int) -> str:
        """Storage format the V-cycle reads on a level: csr, sell, stencil or
        stencil-bulk (stencil planes staged by bulk copies)."""
        fmt = C.c_int()
        self.ctx._check(lib().mds_precond_level_storage(self.h, block, level, None, None, None, None, C.byref(fmt)))
        return {1: "csr", 2: "sell", 3: "stencil", 4: "stencil-bulk"}.get(fmt.value, str(fmt.value))

    def level_host(self, block: int, level: int):
        A = Csr()
        agg, roots = C.c_void_p(), C.c_void_p()
        self.ctx._check(lib().mds_precond_level(self.h, block, level, C.byref(A), C.byref(agg), C.byref(roots)))
        M = self.ctx.csr_to_host(A)
        ag = self.ctx.to_host(agg.value, A.nrow, np.int32) if agg.value else None
        ro = self.ctx.to_host(roots.value, A.nrow, np.int8).astype(bool)
        return M, ag, ro
