"""The integer FP64 <-> FP32 conversions of the CUDA kernels (csrc/conv.cuh,
built here for the host) against the host's IEEE 754 conversions: narrowing
rounds to nearest even (ties, binary32 subnormals, overflow to infinity,
signed zeros), widening is exact (subnormals included), NaN stays NaN."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def conv(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("conv") / "libconv.so")
    subprocess.run(["g++", "-O2", "-shared", "-fPIC", "-std=c++17", "-I",
                    os.path.join(ROOT, "paper_2206_03203_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "conv_shim.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)

    def narrow(bits):
        bits = np.ascontiguousarray(bits, dtype=np.uint64)
        res = np.empty(bits.shape, dtype=np.uint32)
        lib.conv_narrow(bits.ctypes.data_as(ctypes.c_void_p), res.ctypes.data_as(ctypes.c_void_p),
                        ctypes.c_long(bits.size))
        return res

    def widen(bits):
        bits = np.ascontiguousarray(bits, dtype=np.uint32)
        res = np.empty(bits.shape, dtype=np.uint64)
        lib.conv_widen(bits.ctypes.data_as(ctypes.c_void_p), res.ctypes.data_as(ctypes.c_void_p),
                       ctypes.c_long(bits.size))
        return res

    return narrow, widen


def check_narrow(narrow, d):
    d = np.asarray(d, dtype=np.float64)
    got = narrow(d.view(np.uint64))
    with np.errstate(over="ignore", invalid="ignore"):
        ref = d.astype(np.float32).view(np.uint32)
    nan = np.isnan(d)
    assert np.all(np.isnan(got[nan].view(np.float32)))
    bad = np.nonzero((got != ref) & ~nan)[0]
    assert bad.size == 0, [(d[i], hex(got[i]), hex(ref[i])) for i in bad[:5]]


def test_narrow_random_encodings(conv):
    narrow, _ = conv
    rng = np.random.default_rng(1)
    check_narrow(narrow, rng.integers(0, 2**64, 2_000_000, dtype=np.uint64).view(np.float64))
    # exponents around the binary32 range (normal, subnormal, overflow)
    e = rng.integers(860, 1160, 2_000_000, dtype=np.uint64)
    m = rng.integers(0, 2**52, 2_000_000, dtype=np.uint64)
    s = rng.integers(0, 2, 2_000_000, dtype=np.uint64)
    check_narrow(narrow, ((s << np.uint64(63)) | (e << np.uint64(52)) | m).view(np.float64))


def test_narrow_ties_and_neighbours(conv):
    narrow, _ = conv
    rng = np.random.default_rng(2)
    f = rng.integers(0, 0x7F7FFFFF, 1_000_000, dtype=np.uint32)  # finite binary32, subnormals included
    lo = f.view(np.float32).astype(np.float64)
    hi = (f + np.uint32(1)).view(np.float32).astype(np.float64)
    mid = (lo + hi) / 2  # exact in binary64: the tie between two neighbours
    for d in (mid, np.nextafter(mid, 0), np.nextafter(mid, np.inf), -mid, lo, -hi):
        check_narrow(narrow, d)


def test_narrow_special_values(conv):
    narrow, _ = conv
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).smallest_subnormal)
    ulp_top = 2.0 ** 104  # spacing of binary32 at its largest binade
    d = [0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, fmax + ulp_top / 2, fmax + ulp_top / 2 - 2.0 ** 75,
         fmax + ulp_top, 2.0 ** 128, 2.0 ** -126, 2.0 ** -126 * (1 - 2.0 ** -24), tiny, tiny / 2, tiny * 0.75,
         tiny / 2 * (1 + 2.0 ** -52), tiny * 1.5, tiny * 2.5, 5e-324, -5e-324, 2.0 ** -1022, 1e-300, 1e300,
         1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -24 + 2.0 ** -52, -1.0 - 2.0 ** -24]
    check_narrow(narrow, np.array(d))


def test_widen_is_exact(conv):
    _, widen = conv
    rng = np.random.default_rng(3)
    sub = np.arange(1, 2**23, dtype=np.uint32)  # every positive binary32 subnormal
    for bits in (rng.integers(0, 2**32, 4_000_000, dtype=np.uint64).astype(np.uint32), sub,
                 sub | np.uint32(0x80000000),
                 np.array([0, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0x7F7FFFFF, 0x00800000],
                          dtype=np.uint32)):
        f = bits.view(np.float32)
        got = widen(bits)
        nan = np.isnan(f)
        assert np.all(np.isnan(got[nan].view(np.float64)))
        with np.errstate(invalid="ignore"):
            ref = f.astype(np.float64).view(np.uint64)
        assert np.array_equal(got[~nan], ref[~nan])
