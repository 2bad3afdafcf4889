"""The seeded synthetic workloads that the benchmark and the profile summaries name: sizes, shapes and
the spacing guarantees their docstrings state (placement only; no method arithmetic)."""
import numpy as np

import suspensions


def min_centre_distance(c):
    d2 = np.sum((c[:, None, :] - c[None, :, :]) ** 2, axis=-1)
    np.fill_diagonal(d2, np.inf)
    return float(np.sqrt(d2.min()))


def test_shared_shape_lattice_keeps_its_gap():
    # 1,000 particles of the shared-shape construction: identical (1, 0.5, 0.5) axes, n_phi = 2p, and
    # centres at least 2.6 - 2 x 0.2 apart (bounding spheres of radius 1 keep a gap of 0.2)
    s = suspensions.shared_shape(1000, 6, seed=11)
    assert s.n == 1000
    assert np.all(s.semi_axes == np.array([1.0, 0.5, 0.5]))
    assert np.all(s.p == 6) and np.all(s.nphi == 12)
    assert s.total_nodes == 1000 * 7 * 12
    assert min_centre_distance(s.centres) >= 2.2 - 1e-12
    # uniformly random orientations: unit quaternions, not all equal
    assert np.allclose(np.linalg.norm(s.quats, axis=1), 1.0)
    assert np.ptp(s.quats[:, 0]) > 0.5


def test_s_shared_is_one_shape_at_p16():
    s = suspensions.s_shared()
    assert s.n == 10000 and s.total_nodes == 5_440_000
    assert np.all(s.p == 16) and np.all(s.nphi == 32)
    assert len({tuple(a) for a in s.semi_axes}) == 1


def test_c3_profile_draws_like_the_10000_ellipsoid_workload():
    s = suspensions.c3_profile()
    assert s.n == 2000 and s.total_nodes == 288_000
    assert np.all(s.p == 8) and np.all(s.nphi == 16)
    # triaxial axes in [0.6, 1.4], as the 10,000-ellipsoid draw
    assert s.semi_axes.min() >= 0.6 and s.semi_axes.max() <= 1.4
    r = s.semi_axes.max(axis=1)
    d = np.sqrt(np.sum((s.centres[:, None, :] - s.centres[None, :, :]) ** 2, axis=-1))
    gap = d - r[:, None] - r[None, :]
    np.fill_diagonal(gap, np.inf)
    assert gap.min() >= 0.2 - 1e-9  # bounding-sphere gap of the placement
