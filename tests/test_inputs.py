"""Seeded instance generator: determinism, geometry rules, distributions."""
import os

import numpy as np
import pytest

from paper_2206_03203_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_reference_vector():
    # outputs of the reference SplitMix64 generator from state 0
    vals = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64.txt")) if l.startswith("0x")]
    with np.errstate(over="ignore"):
        got = [int(inputs.splitmix64_mix(inputs.GOLDEN * np.uint64(k))) for k in (1, 2, 3)]
    assert got == vals


def test_draws_match_sequential_generator():
    key = np.uint64(12345)
    d = inputs.draws(key, 5)
    state = int(key)
    for k in range(5):
        state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        z = z ^ (z >> 31)
        assert int(d[k]) == z


def test_fixed_2d_snapping():
    inst = inputs.fixed_2d()
    assert inst.n_f == 256
    planes = sorted({(int(a), int(p[a])) for a, p in zip(inst.fc_axis, inst.fc_pos)})
    assert planes == [(0, 16), (0, 48), (1, 19), (1, 45)]


def test_random_segments_deterministic_and_lognormal():
    a = inputs.random_segments_2d(n=256, n_seg=16)
    b = inputs.random_segments_2d(n=256, n_seg=16)
    assert np.array_equal(a.km, b.km) and np.array_equal(a.fc_pos, b.fc_pos)
    z = np.log(a.km)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
    c = inputs.random_segments_2d(n=256, n_seg=16, seed=7)
    assert not np.array_equal(a.km, c.km)
    # half conducting, half blocking
    assert set(np.unique(a.fc_kf)) <= {1e4, 1e-4}


def test_overlap_rule_first_fracture_claims_face():
    r1 = inputs.Rect(0, 3, (0,), (5,), 10.0, 1e-3)
    r2 = inputs.Rect(0, 3, (2,), (8,), 20.0, 1e-3)
    ax, pos, kf, ap = inputs.rasterize(2, 8, [r1, r2])
    assert len(ax) == 8
    assert np.all(kf[:5] == 10.0) and np.all(kf[5:] == 20.0)
    assert len({tuple(p) for p in pos}) == 8


def test_rasterize_rejects_boundary_plane():
    with pytest.raises(ValueError):
        inputs.rasterize(2, 8, [inputs.Rect(0, 0, (0,), (8,), 1.0, 1.0)])


def test_batch_sizes_range():
    s = inputs.batch_sizes(22060304, 256)
    assert min(s) >= 32 and max(s) <= 64 and len(set(s)) > 10


def test_planes_3d_counts():
    inst = inputs.planes_3d(n=16)
    assert inst.n_f == 9 * 16 * 16
