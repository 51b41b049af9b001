"""Python access to the C oracle: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg and
reference arm of ``bench.py`` may import this package.  The oracle is a plain sequential FP64
implementation of the method of Hu, Keilegavlen & Nordbotten (arXiv:2206.03203)
written independently of the CUDA library (see ``mdoracle.c``).  It never
calls, links or imports the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mdoracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no FMA contraction)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "mdoracle.h"))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _CSR(C.Structure):
    _fields_ = [("nrow", C.c_int64), ("ncol", C.c_int64), ("nnz", C.c_int64),
                ("rp", C.POINTER(C.c_int64)), ("ci", C.POINTER(C.c_int32)),
                ("v", C.POINTER(C.c_double))]


class AMGOpts(C.Structure):
    _fields_ = [("theta", C.c_double), ("n_coarse", C.c_int64), ("max_levels", C.c_int),
                ("stall_ratio", C.c_double), ("seed", C.c_uint64), ("smoother", C.c_int),
                ("prec", C.c_int), ("lowp_from_level", C.c_int), ("sweeps", C.c_int), ("smoothed", C.c_int),
                ("cheb_degree", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("relres_true", C.c_double), ("history_len", C.c_int)]


PREC_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double))

P = C.POINTER
_i32p = P(C.c_int32)
_i64p = P(C.c_int64)
_f64p = P(C.c_double)
_i8p = P(C.c_int8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_csr_new.restype = P(_CSR)
            L.orc_csr_new.argtypes = [C.c_int64, C.c_int64, C.c_int64]
            L.orc_csr_free.argtypes = [P(_CSR)]
            L.orc_assemble.restype = P(_CSR)
            L.orc_assemble.argtypes = [C.c_int, C.c_int, _f64p, C.c_int64, _i32p, _i32p, _f64p,
                                       _f64p, C.c_int, _f64p, _f64p, _f64p]
            L.orc_assemble_flux.restype = P(_CSR)
            L.orc_assemble_flux.argtypes = [C.c_int, C.c_int, _f64p, C.c_int64, _i32p, _i32p, _f64p,
                                       _f64p, C.c_int, _f64p, _f64p, _f64p]
            L.orc_assemble_ex.restype = P(_CSR)
            L.orc_assemble_ex.argtypes = [C.c_int, C.c_int, _f64p, C.c_int64, _i32p, _i32p, _f64p,
                                          _f64p, C.c_int, _f64p, _f64p, C.c_int, C.c_int, _i64p,
                                          P(_f64p), _f64p]
            L.orc_free.argtypes = [C.c_void_p]
            L.orc_split.argtypes = [P(_CSR), C.c_int64] + [P(P(_CSR))] * 4
            L.orc_schur.restype = P(_CSR)
            L.orc_schur.argtypes = [P(_CSR)] * 4
            L.orc_spmv.argtypes = [P(_CSR), _f64p, _f64p]
            L.orc_strength.restype = P(_CSR)
            L.orc_strength.argtypes = [P(_CSR), C.c_double]
            L.orc_mis_key.restype = C.c_uint64
            L.orc_mis_key.argtypes = [C.c_uint64, C.c_int, C.c_int64]
            L.orc_round_lowp.restype = C.c_double
            L.orc_round_lowp.argtypes = [C.c_double, C.c_int]
            L.orc_amg_setup.restype = C.c_void_p
            L.orc_amg_setup.argtypes = [P(_CSR), P(AMGOpts)]
            L.orc_amg_setup_seg.restype = C.c_void_p
            L.orc_amg_setup_seg.argtypes = [P(_CSR), P(AMGOpts), C.c_int, _i64p]
            L.orc_amg_level_seg.argtypes = [C.c_void_p, C.c_int, _i64p]
            L.orc_amg_free.argtypes = [C.c_void_p]
            L.orc_amg_nlevels.restype = C.c_int
            L.orc_amg_nlevels.argtypes = [C.c_void_p]
            L.orc_amg_level_n.restype = C.c_int64
            L.orc_amg_level_n.argtypes = [C.c_void_p, C.c_int]
            L.orc_amg_level_A.restype = P(_CSR)
            L.orc_amg_level_A.argtypes = [C.c_void_p, C.c_int]
            L.orc_amg_level_agg.argtypes = [C.c_void_p, C.c_int, _i32p]
            L.orc_amg_level_roots.argtypes = [C.c_void_p, C.c_int, _i8p]
            L.orc_amg_level_l1.argtypes = [C.c_void_p, C.c_int, _f64p]
            L.orc_amg_level_stored.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p, _f64p]
            L.orc_amg_level_lowp.argtypes = [C.c_void_p, C.c_int]
            L.orc_amg_level_P.restype = P(_CSR)
            L.orc_amg_level_P.argtypes = [C.c_void_p, C.c_int]
            L.orc_amg_coarsest_dense.argtypes = [C.c_void_p]
            L.orc_vcycle.argtypes = [C.c_void_p, _f64p, _f64p]
            L.orc_ml_new.restype = C.c_void_p
            L.orc_ml_new.argtypes = [P(_CSR), C.c_int64, P(AMGOpts), C.c_int]
            L.orc_ml_new_seg.restype = C.c_void_p
            L.orc_ml_new_seg.argtypes = [P(_CSR), C.c_int64, P(AMGOpts), C.c_int, C.c_int, _i64p, _i64p]
            L.orc_ml_free.argtypes = [C.c_void_p]
            L.orc_ml_apply.argtypes = [C.c_void_p, _f64p, _f64p]
            L.orc_ml_amg.restype = C.c_void_p
            L.orc_ml_amg.argtypes = [C.c_void_p, C.c_int]
            L.orc_ml_schur.restype = P(_CSR)
            L.orc_ml_schur.argtypes = [C.c_void_p]
            L.orc_fgmres.argtypes = [P(_CSR), C.c_void_p, C.c_void_p, _f64p, _f64p, C.c_int,
                                     C.c_double, C.c_int, _f64p, P(_Stats)]
            L.orc_pcg.argtypes = [P(_CSR), C.c_void_p, C.c_void_p, _f64p, _f64p, C.c_double,
                                  C.c_int, _f64p, P(_Stats)]
            L.orc_minres.argtypes = [P(_CSR), C.c_void_p, C.c_void_p, _f64p, _f64p, C.c_double,
                                     C.c_int, _f64p, P(_Stats)]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _from_csr(ptr, free=True) -> sp.csr_matrix:
    c = ptr.contents
    n, nnz = c.nrow, c.nnz
    rp = np.ctypeslib.as_array(c.rp, shape=(n + 1,)).copy()
    ci = np.ctypeslib.as_array(c.ci, shape=(max(nnz, 1),))[:nnz].copy()
    v = np.ctypeslib.as_array(c.v, shape=(max(nnz, 1),))[:nnz].copy()
    shape = (n, c.ncol)
    if free:
        lib().orc_csr_free(ptr)
    return sp.csr_matrix((v, ci, rp), shape=shape)


class CSR:
    """An oracle-owned copy of a scipy CSR matrix."""

    def __init__(self, A: sp.csr_matrix):
        A = sp.csr_matrix(A)
        A.sort_indices()
        L = lib()
        self.ptr = L.orc_csr_new(A.shape[0], A.shape[1], A.nnz)
        c = self.ptr.contents
        C.memmove(c.rp, _p(np.ascontiguousarray(A.indptr, dtype=np.int64), _i64p), 8 * (A.shape[0] + 1))
        if A.nnz:
            C.memmove(c.ci, _p(np.ascontiguousarray(A.indices, dtype=np.int32), _i32p), 4 * A.nnz)
            C.memmove(c.v, _p(np.ascontiguousarray(A.data, dtype=np.float64), _f64p), 8 * A.nnz)
        self.shape = A.shape

    def __del__(self):
        try:
            lib().orc_csr_free(self.ptr)
        except Exception:
            pass


def _kn(inst):
    kn = getattr(inst, "fc_kn", None)
    return None if kn is None else np.ascontiguousarray(kn, dtype=np.float64)


def assemble(inst, form="primal", junction=0, with_split=False):
    """Full system (scipy CSR) and right-hand sides [nrhs, N].  form="primal":
    [matrix cells; fracture cells] with the interface flux eliminated;
    form="flux": the paper's partition [all pressures; interface fluxes]
    (N = n_m + 3 n_f with junction 0).  junction=1: junctions of >= 3
    fracture cells are nodes joined by half transmissibilities (star-delta in
    the primal form, intersection cells with their own fluxes in the flux
    form).  with_split=True also returns the size of the first block."""
    if junction or with_split or _kn(inst) is not None:
        return _assemble_ex(inst, form, junction, with_split)
    L = lib()
    N = inst.n_m + inst.n_f if form == "primal" else inst.n_m + 3 * inst.n_f
    b = np.zeros((inst.nrhs, N))
    pos = np.ascontiguousarray(inst.fc_pos, dtype=np.int32).reshape(-1)
    if pos.size == 0:
        pos = np.zeros(3, dtype=np.int32)
    fn = L.orc_assemble if form == "primal" else L.orc_assemble_flux
    ptr = fn(inst.dim, inst.n, _p(inst.km, _f64p), inst.n_f,
                         _p(np.ascontiguousarray(inst.fc_axis, dtype=np.int32), _i32p), _p(pos, _i32p),
                         _p(np.ascontiguousarray(inst.fc_kf), _f64p),
                         _p(np.ascontiguousarray(inst.fc_a), _f64p), inst.nrhs,
                         _p(inst.pD_left, _f64p), _p(inst.pD_right, _f64p), _p(b, _f64p))
    if not ptr:
        raise ValueError("oracle assembly rejected the instance")
    return _from_csr(ptr), b


def _assemble_ex(inst, form, junction, with_split):
    L = lib()
    pos = np.ascontiguousarray(inst.fc_pos, dtype=np.int32).reshape(-1)
    if pos.size == 0:
        pos = np.zeros(3, dtype=np.int32)
    no = C.c_int64()
    bp = _f64p()
    kn = _kn(inst)
    kn_p = _p(kn, _f64p) if kn is not None else None
    ptr = L.orc_assemble_ex(inst.dim, inst.n, _p(inst.km, _f64p), inst.n_f,
                            _p(np.ascontiguousarray(inst.fc_axis, dtype=np.int32), _i32p), _p(pos, _i32p),
                            _p(np.ascontiguousarray(inst.fc_kf), _f64p), _p(np.ascontiguousarray(inst.fc_a), _f64p),
                            inst.nrhs, _p(inst.pD_left, _f64p), _p(inst.pD_right, _f64p), int(form == "flux"),
                            int(junction), C.byref(no), C.byref(bp), kn_p)
    if not ptr:
        raise ValueError("oracle assembly rejected the instance")
    A = _from_csr(ptr)
    nt = A.shape[0]
    b = np.ctypeslib.as_array(bp, shape=(inst.nrhs * nt,)).copy().reshape(inst.nrhs, nt)
    L.orc_free(C.cast(bp, C.c_void_p))
    return (A, b, int(no.value)) if with_split else (A, b)


def split(A, n_m):
    L = lib()
    h = CSR(A)
    outs = [P(_CSR)() for _ in range(4)]
    L.orc_split(h.ptr, n_m, *[C.byref(o) for o in outs])
    return tuple(_from_csr(o) for o in outs)


def schur(Amm, Amf, Afm, Aff):
    """Eq. (7)."""
    hs = [CSR(M) for M in (Amm, Amf, Afm, Aff)]
    ptr = lib().orc_schur(*[h.ptr for h in hs])
    if not ptr:
        raise ValueError("zero diagonal in A_ff")
    return _from_csr(ptr)


def spmv(A, x):
    h = CSR(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(A.shape[0])
    lib().orc_spmv(h.ptr, _p(x, _f64p), _p(y, _f64p))
    return y


def strength(A, theta=0.08):
    h = CSR(A)
    return _from_csr(lib().orc_strength(h.ptr, theta))


def mis_key(seed, level, i):
    return int(lib().orc_mis_key(seed, level, i))


DEFAULT_SEED = 0x2206_0320_3


def amg_opts(theta=None, n_coarse=512, max_levels=25, stall_ratio=0.9, seed=DEFAULT_SEED,
             smoother=0, prec=64, lowp_from_level=1, sweeps=1, smoothed=0, cheb_degree=2) -> AMGOpts:
    """smoother: 0 L1-Jacobi, 1 Chebyshev (degree cheb_degree), 2 Gauss-Seidel.
    theta None: 0.08 for piecewise-constant, 0.04 for smoothed aggregation."""
    if theta is None or theta < 0:
        theta = 0.04 if smoothed else 0.08
    return AMGOpts(theta, n_coarse, max_levels, stall_ratio, seed, smoother, prec, lowp_from_level, sweeps,
                   smoothed, cheb_degree)


def round_lowp(x, prec):
    return float(lib().orc_round_lowp(float(x), prec))


class AMG:
    def __init__(self, A, segments=None, **kw):
        """segments: row offsets [K + 1] of the instances of a packed batch
        (each coarsened as if alone); None for one instance."""
        self.opts = amg_opts(**kw)
        self._A = CSR(A)
        if segments is None:
            self.h = lib().orc_amg_setup(self._A.ptr, C.byref(self.opts))
        else:
            off = np.ascontiguousarray(segments, dtype=np.int64)
            self.h = lib().orc_amg_setup_seg(self._A.ptr, C.byref(self.opts), len(off) - 1, _p(off, _i64p))
        if not self.h:
            raise ValueError("AMG setup failed (coarsest matrix not SPD)")
        self.n = A.shape[0]

    def __del__(self):
        try:
            lib().orc_amg_free(self.h)
        except Exception:
            pass

    @property
    def nlevels(self):
        return lib().orc_amg_nlevels(self.h)

    def level_A(self, l):
        return _from_csr(lib().orc_amg_level_A(self.h, l), free=False)

    def agg(self, l):
        n = lib().orc_amg_level_n(self.h, l)
        out = np.zeros(n, dtype=np.int32)
        if lib().orc_amg_level_agg(self.h, l, _p(out, _i32p)) != 0:
            return None
        return out

    def segments(self, l):
        """Instance segment offsets of level l."""
        out = np.zeros(1025, dtype=np.int64)
        k = lib().orc_amg_level_seg(self.h, l, _p(out, _i64p))
        return out[:k + 1].copy()

    def roots(self, l):
        n = lib().orc_amg_level_n(self.h, l)
        out = np.zeros(n, dtype=np.int8)
        lib().orc_amg_level_roots(self.h, l, _p(out, _i8p))
        return out.astype(bool)

    def l1(self, l):
        n = lib().orc_amg_level_n(self.h, l)
        out = np.zeros(n)
        lib().orc_amg_level_l1(self.h, l, _p(out, _f64p))
        return out

    def stored(self, l):
        """(values in CSR order of level_A(l), row scales, 1/D1) as the
        V-cycle applies them, and the level's low-precision format (16 =
        bf16, 17 = fp16, 0 = none)."""
        A = self.level_A(l)
        av, rs, dv = np.zeros(A.nnz), np.zeros(A.shape[0]), np.zeros(A.shape[0])
        lib().orc_amg_level_stored(self.h, l, _p(av, _f64p), _p(rs, _f64p), _p(dv, _f64p))
        return av, rs, dv, lib().orc_amg_level_lowp(self.h, l)

    def P(self, l):
        ptr = lib().orc_amg_level_P(self.h, l)
        return _from_csr(ptr, free=False) if ptr else None

    @property
    def coarsest_dense(self):
        return lib().orc_amg_coarsest_dense(self.h) == 1

    @property
    def coarsest_diagonal(self):
        """The last level has no couplings and is solved by x = b / a_ii."""
        return lib().orc_amg_coarsest_dense(self.h) == 2

    def vcycle(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n)
        lib().orc_vcycle(self.h, _p(b, _f64p), _p(x, _f64p))
        return x


class _AMGView(AMG):
    def __init__(self, h, n, owner):
        self.h, self.n, self._owner = h, n, owner

    def __del__(self):
        pass


KIND = {"lower": 0, "diag": 1, "upper": 2}


class ML:
    """Block preconditioner of Sec. 3.2: 'lower' = M_L (Alg. 1), 'diag' =
    block diagonal, 'upper' = block upper triangular."""

    def __init__(self, A, n_m, kind="lower", segments=None, **kw):
        """segments: (moff, foff), the matrix-row and fracture-row offsets
        [K + 1] of the instances of a packed batch; None for one instance."""
        self.opts = amg_opts(**kw)
        self._A = CSR(A)
        self.n_m, self.N = n_m, A.shape[0]
        if segments is None:
            self.h = lib().orc_ml_new(self._A.ptr, n_m, C.byref(self.opts), KIND[kind])
        else:
            mo = np.ascontiguousarray(segments[0], dtype=np.int64)
            fo = np.ascontiguousarray(segments[1], dtype=np.int64)
            self.h = lib().orc_ml_new_seg(self._A.ptr, n_m, C.byref(self.opts), KIND[kind], len(mo) - 1,
                                          _p(mo, _i64p), _p(fo, _i64p))
        if not self.h:
            raise ValueError("M_L setup failed")

    def __del__(self):
        try:
            lib().orc_ml_free(self.h)
        except Exception:
            pass

    def apply(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros(self.N)
        lib().orc_ml_apply(self.h, _p(r, _f64p), _p(z, _f64p))
        return z

    def amg(self, block):
        h = lib().orc_ml_amg(self.h, block)
        n = self.n_m if block == 0 else self.N - self.n_m
        return _AMGView(h, n, self) if h else None

    @property
    def schur(self):
        return _from_csr(lib().orc_ml_schur(self.h), free=False)

    @property
    def c_fn(self):
        return C.cast(lib().orc_ml_apply, C.c_void_p)


@dataclass
class Result:
    x: np.ndarray
    iterations: int
    restarts: int
    converged: bool
    relres: float
    history: np.ndarray


def _prec_args(prec, n):
    if prec is None or prec == "identity":
        ctx = np.array([n], dtype=np.int64)
        return C.cast(lib().orc_identity_apply, C.c_void_p), ctx.ctypes.data_as(C.c_void_p), ctx
    if isinstance(prec, ML):
        return prec.c_fn, C.c_void_p(prec.h), None

    def cb(_ctx, r, z):
        rr = np.ctypeslib.as_array(r, shape=(n,))
        zz = np.ctypeslib.as_array(z, shape=(n,))
        zz[:] = prec(rr.copy())
        return 0

    f = PREC_FN(cb)
    return C.cast(f, C.c_void_p), None, f


def fgmres(A, b, prec=None, x0=None, restart=30, rtol=1e-8, maxit=1000, hA=None) -> Result:
    """Right-preconditioned FGMRES(restart); ``prec`` is an ML, 'identity'
    or a Python callable r -> z."""
    n = A.shape[0]
    hA = hA or CSR(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    fn, ctx, keep = _prec_args(prec, n)
    hist = np.zeros(maxit + 2)
    st = _Stats()
    lib().orc_fgmres(hA.ptr, fn, ctx, _p(b, _f64p), _p(x, _f64p), restart, rtol, maxit,
                     _p(hist, _f64p), C.byref(st))
    del keep
    return Result(x, st.iterations, st.restarts, bool(st.converged), st.relres_true,
                  hist[:st.history_len].copy())


def pcg(A, b, prec=None, x0=None, rtol=1e-8, maxit=1000, hA=None) -> Result:
    n = A.shape[0]
    hA = hA or CSR(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    fn, ctx, keep = _prec_args(prec, n)
    hist = np.zeros(maxit + 2)
    st = _Stats()
    lib().orc_pcg(hA.ptr, fn, ctx, _p(b, _f64p), _p(x, _f64p), rtol, maxit, _p(hist, _f64p),
                  C.byref(st))
    del keep
    return Result(x, st.iterations, st.restarts, bool(st.converged), st.relres_true,
                  hist[:st.history_len].copy())


def minres(A, b, prec=None, x0=None, rtol=1e-8, maxit=1000, hA=None) -> Result:
    """Preconditioned MINRES (symmetric A, SPD preconditioner)."""
    n = A.shape[0]
    hA = hA or CSR(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    fn, ctx, keep = _prec_args(prec, n)
    hist = np.zeros(maxit + 2)
    st = _Stats()
    lib().orc_minres(hA.ptr, fn, ctx, _p(b, _f64p), _p(x, _f64p), rtol, maxit, _p(hist, _f64p),
                     C.byref(st))
    del keep
    return Result(x, st.iterations, st.restarts, bool(st.converged), st.relres_true,
                  hist[:st.history_len].copy())


def solve(inst, rhs=0, kind="lower", krylov="fgmres", restart=30, rtol=1e-8, maxit=1000, **kw):
    """Assemble, set up M_L and solve one right-hand side of an instance."""
    A, b = assemble(inst)
    M = ML(A, inst.n_m, kind=kind, **kw)
    if krylov == "pcg":
        return pcg(A, b[rhs], M, rtol=rtol, maxit=maxit), A, b, M
    if krylov == "minres":
        return minres(A, b[rhs], M, rtol=rtol, maxit=maxit), A, b, M
    return fgmres(A, b[rhs], M, restart=restart, rtol=rtol, maxit=maxit), A, b, M
