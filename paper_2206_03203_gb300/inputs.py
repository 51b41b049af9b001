"""Seeded synthetic instances of the mixed-dimensional flow problem.

This module only draws geometry and coefficients; it holds none of the
solver's arithmetic (no transmissibility, no matrix entry, no right-hand side).
Both the CUDA path and the CPU oracle consume its output unchanged.

An instance is a Cartesian grid of n^dim cells on the unit square/cube
(cell size h = 1/n, cell index x-fastest) with

* ``km``      matrix permeability per cell (float64, [n^dim]);
* fracture cells: interior grid faces (codimension-1 objects of Sec. 2.1)
  listed as (normal axis, x, y, z) where the coordinate along the normal axis
  is the face-plane index (1..n-1) and the other coordinates are cell indices;
  each fracture cell carries its tangential permeability ``fc_kf`` and
  aperture ``fc_a``;
* Dirichlet data on the x=0 and x=1 boundary faces, one value per boundary
  face per right-hand side (``pD_left``/``pD_right``, [nrhs, n^(dim-1)],
  face index y-fastest then z); all other boundary faces are no-flow.

Random draws use a counter-based SplitMix64 stream (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the 64-bit
finaliser applied to ``key + (counter+1) * 0x9E3779B97F4A7C15``, with the key
derived from (seed, instance, fracture, field).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from decimal import Decimal, getcontext
from typing import List, Optional

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids for the fields an instance draws
FIELD_KM = 1
FIELD_FRAC = 2
FIELD_GRID = 3
FIELD_RHS = 4


def splitmix64_mix(z):
    """SplitMix64 output finaliser on uint64 (scalar or array), wrapping."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, *ids: int) -> np.uint64:
    """Derive a stream key from a seed and a tuple of stream ids."""
    k = splitmix64_mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    with np.errstate(over="ignore"):
        for i in ids:
            k = splitmix64_mix(k + GOLDEN * np.uint64(i + 1))
    return np.uint64(k)


def draws(key: np.uint64, count: int, start: int = 0) -> np.ndarray:
    """``count`` uint64 draws of the counter-based stream ``key``."""
    c = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64_mix(key + c * GOLDEN)


def to_unit(u64: np.ndarray) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    return (u64 >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class Instance:
    name: str
    dim: int
    n: int
    km: np.ndarray
    fc_axis: np.ndarray
    fc_pos: np.ndarray
    fc_kf: np.ndarray
    fc_a: np.ndarray
    pD_left: np.ndarray
    pD_right: np.ndarray
    meta: dict = field(default_factory=dict)
    # normal permeability per fracture cell (kappa = 2 k_n / a); None: k_n = k_f
    fc_kn: Optional[np.ndarray] = None

    @property
    def n_m(self) -> int:
        return self.n ** self.dim

    @property
    def n_f(self) -> int:
        return int(self.fc_axis.shape[0])

    @property
    def nrhs(self) -> int:
        return int(self.pD_left.shape[0])

    def with_rhs(self, k: int) -> "Instance":
        """The same instance restricted to right-hand side ``k``."""
        return Instance(self.name, self.dim, self.n, self.km, self.fc_axis, self.fc_pos,
                        self.fc_kf, self.fc_a, self.pD_left[k:k + 1].copy(),
                        self.pD_right[k:k + 1].copy(), dict(self.meta), self.fc_kn)


@dataclass
class Rect:
    """An axis-aligned planar fracture on grid faces.

    ``axis`` is the normal axis, ``plane`` the face-plane index (1..n-1),
    ``lo``/``hi`` the half-open cell ranges along the tangential axes in
    ascending axis order (one range in 2D, two in 3D).
    """
    axis: int
    plane: int
    lo: tuple
    hi: tuple
    kf: float
    a: float


def tangential_axes(dim: int, axis: int) -> List[int]:
    return [d for d in range(dim) if d != axis]


def rasterize(dim: int, n: int, rects: List[Rect]):
    """List the fracture cells of ``rects``.

    A face claimed by an earlier fracture is skipped by later ones (overlap
    rule).  Within a fracture the first tangential axis runs fastest.
    """
    axes, pos, kf, ap = [], [], [], []
    claimed = set()
    for r in rects:
        if not (1 <= r.plane <= n - 1):
            raise ValueError("fracture plane must be interior")
        t = tangential_axes(dim, r.axis)
        if dim == 2:
            cells = [(c,) for c in range(r.lo[0], r.hi[0])]
        else:
            cells = [(c0, c1) for c1 in range(r.lo[1], r.hi[1]) for c0 in range(r.lo[0], r.hi[0])]
        for tc in cells:
            p = [0, 0, 0]
            p[r.axis] = r.plane
            for ax, c in zip(t, tc):
                if not (0 <= c < n):
                    raise ValueError("fracture extends outside the grid")
                p[ax] = c
            key = (r.axis, p[0], p[1], p[2])
            if key in claimed:
                continue
            claimed.add(key)
            axes.append(r.axis)
            pos.append(p)
            kf.append(r.kf)
            ap.append(r.a)
    nf = len(axes)
    return (np.asarray(axes, dtype=np.int32).reshape(nf),
            np.asarray(pos, dtype=np.int32).reshape(nf, 3),
            np.asarray(kf, dtype=np.float64).reshape(nf),
            np.asarray(ap, dtype=np.float64).reshape(nf))


# ---------------------------------------------------------------------------
# exp, log and cos from +, -, *, / and exact power-of-two scaling only (Taylor
# and atanh series after an argument reduction), evaluated in a fixed order:
# the generated instances are then bit-identical on every IEEE-754 machine,
# whereas library transcendental functions differ in their last bits between
# platforms.  About 1e-16 relative accuracy is all an input generator needs.
# ---------------------------------------------------------------------------

def _split(x: Decimal):
    """x = hi + lo with hi holding 32 significant bits (hi * k exact for |k| < 2^21)."""
    m, e = math.frexp(float(x))
    hi = math.ldexp(math.floor(m * 2.0 ** 32) / 2.0 ** 32, e)
    return hi, float(x - Decimal(hi))


getcontext().prec = 60
_LN2 = Decimal("0.69314718055994530941723212145817656807550013436025525412068")
_LN10 = Decimal("2.30258509299404568401799145468436420760110148862877297603333")
_PI = Decimal("3.14159265358979323846264338327950288419716939937510582097494")
_LN2_HI, _LN2_LO = _split(_LN2)
_LN10_D = float(_LN10)
_TWO_PI = float(2 * _PI)


def portable_exp(x: np.ndarray) -> np.ndarray:
    """exp(x): x = k ln2 + r, |r| <= ln2 / 2, exp(r) by its Taylor series
    (Horner, 16 terms), times 2^k."""
    x = np.asarray(x, dtype=np.float64)
    k = np.rint(x * (1.0 / float(_LN2)))
    r = (x - k * _LN2_HI) - k * _LN2_LO
    p = np.ones_like(r)
    for n in range(16, 0, -1):
        p = 1.0 + p * (r / n)
    return np.ldexp(p, k.astype(np.int64))


def portable_log(y: np.ndarray) -> np.ndarray:
    """log(y), y > 0: y = m 2^e with m in [sqrt(1/2), sqrt(2)), log m =
    2 atanh(s) with s = (m - 1) / (m + 1), |s| < 0.172 (series to s^27)."""
    y = np.asarray(y, dtype=np.float64)
    m, e = np.frexp(y)
    low = m < 0.70710678118654752440
    m = np.where(low, m * 2.0, m)
    e = np.where(low, e - 1, e).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    t = np.zeros_like(s)
    for q in range(27, 1, -2):
        t = s2 * (1.0 / q + t)
    logm = 2.0 * (s + s * t)
    return e * _LN2_HI + (e * _LN2_LO + logm)


def portable_cos_2pi(u: np.ndarray) -> np.ndarray:
    """cos(2 pi u): reduced by symmetry to x = 2 pi w, w in [0, 1/4], then the
    Taylor series of cos x (14 terms)."""
    u = np.asarray(u, dtype=np.float64)
    w = np.abs(u - np.rint(u))          # [0, 1/2]
    neg = w > 0.25
    w = np.where(neg, 0.5 - w, w)       # cos(2 pi w) = -cos(2 pi (1/2 - w))
    x = w * _TWO_PI
    x2 = x * x
    c = np.ones_like(x)
    for n in range(28, 0, -2):
        c = 1.0 - c * (x2 / (n * (n - 1)))
    return np.where(neg, -c, c)


def lognormal_km(seed: int, inst: int, n_cells: int, sigma: float) -> np.ndarray:
    """k_m = exp(sigma z), z iid N(0,1) per cell by Box-Muller (cosine branch)."""
    if sigma == 0.0:
        return np.ones(n_cells)
    key = stream_key(seed, inst, FIELD_KM)
    d = draws(key, 2 * n_cells)
    u1 = to_unit(d[0::2])
    u2 = to_unit(d[1::2])
    z = np.sqrt(-2.0 * portable_log(1.0 - u1)) * portable_cos_2pi(u2)
    return portable_exp(sigma * z)


def make_instance(name, dim, n, km, rects, pD_left=None, pD_right=None, meta=None) -> Instance:
    ax, pos, kf, ap = rasterize(dim, n, rects)
    nb = n ** (dim - 1)
    if pD_left is None:
        pD_left = np.ones((1, nb))
    if pD_right is None:
        pD_right = np.zeros((1, nb))
    pD_left = np.ascontiguousarray(np.atleast_2d(pD_left), dtype=np.float64)
    pD_right = np.ascontiguousarray(np.atleast_2d(pD_right), dtype=np.float64)
    if pD_left.shape != pD_right.shape or pD_left.shape[1] != nb:
        raise ValueError("Dirichlet arrays must be [nrhs, n^(dim-1)]")
    return Instance(name, dim, n, np.ascontiguousarray(km, dtype=np.float64), ax, pos, kf, ap,
                    pD_left, pD_right, dict(meta or {}))


def snap(c: float, n: int) -> int:
    """Face-plane index of coordinate c: round(c n), kept interior."""
    return int(min(max(int(np.floor(c * n + 0.5)), 1), n - 1))


# ---------------------------------------------------------------------------
# The five workloads (Sec. 4 stands in: the paper's benchmark geometries are
# replaced by seeded Cartesian instances of the same kind).
# ---------------------------------------------------------------------------

def fixed_2d(n: int = 64, kf: float = 1e4, a: float = 1e-4) -> Instance:
    """2D unit square, k_m = 1, four full-length fractures at x = 0.25, 0.75
    and y = 0.3, 0.7; Dirichlet p=1 at x=0 and p=0 at x=1."""
    rects = [Rect(0, snap(0.25, n), (0,), (n,), kf, a),
             Rect(0, snap(0.75, n), (0,), (n,), kf, a),
             Rect(1, snap(0.3, n), (0,), (n,), kf, a),
             Rect(1, snap(0.7, n), (0,), (n,), kf, a)]
    return make_instance(f"2d-{n}-4frac", 2, n, np.ones(n * n), rects,
                         meta={"kf": kf, "a": a})


def random_segments_2d(n: int = 1024, seed: int = 22060302, n_seg: int = 64,
                       contrast: float = 1e4, sigma: float = 1.0, a: float = 1e-4) -> Instance:
    """2D n x n, log-normal k_m, ``n_seg`` axis-aligned segments with length
    fraction U(0.1, 0.6); even-index segments get k_f = contrast, odd ones
    1/contrast."""
    km = lognormal_km(seed, 0, n * n, sigma)
    rects = []
    for f in range(n_seg):
        d = draws(stream_key(seed, 0, FIELD_FRAC, f), 4)
        axis = int(d[0] % np.uint64(2))
        plane = 1 + int(d[1] % np.uint64(n - 1))
        s = 0.1 + 0.5 * float(to_unit(d[2:3])[0])
        cells = max(1, int(np.floor(s * n + 0.5)))
        cells = min(cells, n)
        off = int(d[3] % np.uint64(n - cells + 1))
        kf = contrast if f % 2 == 0 else 1.0 / contrast
        rects.append(Rect(axis, plane, (off,), (off + cells,), kf, a))
    return make_instance(f"2d-{n}-seg{n_seg}-c{contrast:g}", 2, n, km, rects,
                         meta={"seed": seed, "contrast": contrast, "sigma": sigma})


def planes_3d(n: int = 128, kf: float = 1e4, a: float = 1e-3) -> Instance:
    """3D n^3, k_m = 1, nine full fracture planes x, y, z in {0.25, 0.5, 0.75}."""
    rects = []
    for axis in range(3):
        for c in (0.25, 0.5, 0.75):
            rects.append(Rect(axis, snap(c, n), (0, 0), (n, n), kf, a))
    return make_instance(f"3d-{n}-9planes-kf{kf:g}", 3, n, np.ones(n ** 3), rects,
                         meta={"kf": kf, "a": a})


def random_rects_3d(n: int, seed: int, inst: int, n_rect: int, side=(0.2, 0.8),
                    kf: Optional[float] = None, log10kf=(-4.0, 4.0), sigma: float = 1.0,
                    a: float = 1e-4, nrhs: int = 1, random_dirichlet: bool = False) -> Instance:
    """3D n^3 with ``n_rect`` random axis-aligned rectangles (sides U(side)·n
    cells), log-normal k_m; k_f fixed or log10 k_f ~ U(log10kf)."""
    km = lognormal_km(seed, inst, n ** 3, sigma)
    rects = []
    for f in range(n_rect):
        d = draws(stream_key(seed, inst, FIELD_FRAC, f), 8)
        axis = int(d[0] % np.uint64(3))
        plane = 1 + int(d[1] % np.uint64(n - 1))
        lo, hi = [], []
        for t in range(2):
            s = side[0] + (side[1] - side[0]) * float(to_unit(d[2 + t:3 + t])[0])
            cells = min(n, max(1, int(np.floor(s * n + 0.5))))
            off = int(d[4 + t] % np.uint64(n - cells + 1))
            lo.append(off)
            hi.append(off + cells)
        if kf is None:
            e = log10kf[0] + (log10kf[1] - log10kf[0]) * float(to_unit(d[6:7])[0])
            k = float(portable_exp(np.array([e * _LN10_D]))[0])  # 10^e
        else:
            k = kf
        rects.append(Rect(axis, plane, tuple(lo), tuple(hi), k, a))
    nb = n * n
    if random_dirichlet:
        key = stream_key(seed, inst, FIELD_RHS)
        u = to_unit(draws(key, 2 * nrhs * nb)).reshape(nrhs, 2, nb)
        pl, pr = u[:, 0, :].copy(), u[:, 1, :].copy()
    else:
        pl, pr = np.ones((nrhs, nb)), np.zeros((nrhs, nb))
    return make_instance(f"3d-{n}-rect{n_rect}-s{seed}-i{inst}", 3, n, km, rects, pl, pr,
                         meta={"seed": seed, "inst": inst, "sigma": sigma})


def batch_sizes(seed: int, count: int, lo: int = 32, hi: int = 64) -> List[int]:
    """Cube sides n ~ U{lo..hi} for a batch of instances."""
    d = draws(stream_key(seed, 0, FIELD_GRID), count)
    return [lo + int(x % np.uint64(hi - lo + 1)) for x in d]


def batch_instance(i: int, count: int = 256, seed: int = 22060304, nrhs: int = 4, lo: int = 32,
                   hi: int = 64) -> Instance:
    """Instance ``i`` of ``batch_3d(count, seed, nrhs, lo, hi)``, generated alone."""
    n = batch_sizes(seed, count, lo, hi)[i]
    nr = 1 + int(draws(stream_key(seed, i, FIELD_GRID), 1)[0] % np.uint64(12))
    return random_rects_3d(n, seed, i, nr, nrhs=nrhs, random_dirichlet=True)


def batch_3d(count: int = 256, seed: int = 22060304, nrhs: int = 4, lo: int = 32, hi: int = 64):
    """Uneven 3D instances with 1-12 random rectangles each, log10 k_f ~ U(-4, 4),
    log-normal k_m (sigma = 1), ``nrhs`` random-Dirichlet right-hand sides."""
    return [batch_instance(i, count, seed, nrhs, lo, hi) for i in range(count)]


def large_3d(n: int = 256, seed: int = 22060305, nrhs: int = 8) -> Instance:
    """3D n^3, 30 random rectangles, aperture 1e-4, log-normal k_m (sigma = 2),
    k_f = 1e4, ``nrhs`` random-Dirichlet right-hand sides."""
    return random_rects_3d(n, seed, 0, 30, kf=1e4, sigma=2.0, nrhs=nrhs, random_dirichlet=True)


CONTRASTS = [1e-4, 1e-3, 1e-2, 1e-1, 1.0, 1e1, 1e2, 1e3, 1e4]
