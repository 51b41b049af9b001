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


def stored_digests():
    return dict(l.split() for l in open(os.path.join(GOLD, "input_digests.txt")) if l.strip() and l[0] != "#")


def test_generated_instances_match_stored_digests():
    """The generator uses no library transcendental function, so its output is
    the same bits on every IEEE-754 machine (the stored digests and iteration
    counts were written on another machine than the GPU tests run on)."""
    import sys
    sys.path.insert(0, GOLD)
    import make_input_digests
    assert make_input_digests.digests() == stored_digests()


def test_portable_elementary_functions():
    rng = np.random.default_rng(0)
    x = rng.uniform(-14.0, 14.0, 100000)
    assert np.max(np.abs(inputs.portable_exp(x) / np.exp(x) - 1.0)) <= 4e-16
    assert inputs.portable_exp(np.array([0.0]))[0] == 1.0
    y = np.concatenate([rng.uniform(0.0, 1.0, 100000), [2.0 ** -53, 0.5, 1.0, 3.0]])
    assert np.max(np.abs(inputs.portable_log(y) - np.log(y))) <= 2e-15
    assert inputs.portable_log(np.array([1.0]))[0] == 0.0
    u = np.concatenate([rng.uniform(0.0, 1.0, 100000), [0.0, 0.25, 0.5, 0.75]])
    assert np.max(np.abs(inputs.portable_cos_2pi(u) - np.cos(2.0 * np.pi * u))) <= 2e-15
