"""Pins of the oracle's barycentric Lagrange treecode (oracle/treecode.py), against facts that do not
depend on it: polynomial interpolation is exact on polynomials of the interpolation degree, the
modified charges carry every polynomial moment of the sources up to that degree, the tree's lists
cover every interacting source particle exactly once and keep the own and near particles out of
the approximations, a vanishing opening angle gives back the direct sum, and the approximation error
falls with the degree and stays inside the error model."""
import math

import numpy as np
import pytest

import oracle
import suspensions
from oracle import treecode as tc


def system_of(s):
    return oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats, s.suspension_id)


@pytest.fixture(scope="module")
def cloud():
    """300 ellipsoids at p = 2 (12 nodes each) in the 10% suspension; large enough for accepted cells
    at every degree tested."""
    s = suspensions.random_ellipsoids(300, 2, 4, 0.10, 0.2, seed=11)
    return system_of(s)


@pytest.mark.parametrize("n", [1, 3, 6, 9])
def test_lagrange_basis_reproduces_polynomials(n):
    rng = np.random.default_rng(n)
    lo, hi = -0.7, 2.3
    x = rng.uniform(lo, hi, 200)
    L = tc.lagrange_basis(x, lo, hi, n)
    nodes = 0.5 * (lo + hi) + 0.5 * (hi - lo) * tc.chebyshev_points(n)
    assert np.abs(L.sum(1) - 1.0).max() < 1e-13                        # partition of unity
    for deg in range(n + 1):                                            # exact on degree <= n
        c = rng.normal(size=deg + 1)
        P = np.polynomial.polynomial.polyval
        assert np.abs(L @ P(nodes, c) - P(x, c)).max() < 1e-11 * max(1.0, np.abs(P(x, c)).max())
    # on a node: the unit vector, also for nodes the formula would divide by zero at
    Ln = tc.lagrange_basis(nodes, lo, hi, n)
    assert np.abs(Ln - np.eye(n + 1)).max() < 1e-12
    # one degree too many is not reproduced
    q = np.zeros(n + 2)
    q[-1] = 1.0
    P = np.polynomial.polynomial.polyval
    assert np.abs(L @ P(nodes, q) - P(x, q)).max() > 1e-6


def test_modified_charges_keep_polynomial_moments(cloud):
    """sum_k f(s_k) q_k = sum_s f(y_s) w_s mu_s for every monomial f of degree <= n per axis: this
    pins the charges (transposed or permuted axes, a dropped weight, wrong point order all fail)."""
    s = cloud
    n = 3
    root = tc.build_tree(s, range(len(s.particles)))
    cell = root.children[0]
    x = suspensions.random_density(3, s.total_nodes)
    q = tc.modified_charges(s, cell, n, x)
    g = tc.proxy_points(cell, n)
    y = np.concatenate([s.particles[j].x for j in cell.particles])
    wmu = np.concatenate([s.particles[j].w[:, None] * x[s.sl(j)] for j in cell.particles])
    centre = cell.centre
    for a in range(n + 1):
        for b in range(n + 1):
            for c in range(n + 1):
                f = lambda z: ((z[:, 0] - centre[0]) ** a) * ((z[:, 1] - centre[1]) ** b) * ((z[:, 2] - centre[2]) ** c)
                lhs = f(g) @ q
                rhs = f(y) @ wmu
                assert np.abs(lhs - rhs).max() <= 1e-10 * max(1.0, np.abs(rhs).max()), (a, b, c)
    # degree n + 1 in x is not carried
    f = lambda z: (z[:, 0] - centre[0]) ** (n + 1)
    assert np.abs(f(g) @ q - f(y) @ wmu).max() > 1e-8


def test_cells_bound_their_nodes(cloud):
    s = cloud
    root = tc.build_tree(s, range(len(s.particles)))
    stack = [root]
    while stack:
        cell = stack.pop()
        y = np.concatenate([s.particles[j].x for j in cell.particles])
        assert np.all(y >= cell.lo) and np.all(y <= cell.hi)
        assert np.linalg.norm(y - cell.centre, axis=1).max() <= cell.radius * (1 + 1e-14)
        assert cell.nodes == len(y)
        if cell.children:
            merged = np.sort(np.concatenate([ch.particles for ch in cell.children]))
            assert np.array_equal(merged, cell.particles)
            stack.extend(cell.children)
        else:
            assert len(cell.particles) == 1


@pytest.mark.parametrize("theta,degree", [(0.5, 2), (0.7, 3)])
def test_lists_cover_every_source_once(cloud, theta, degree):
    s = cloud
    t = tc.Treecode(s, theta, degree)
    n = len(s.particles)
    accepted = 0
    for i, (approx, direct) in enumerate(t.lists):
        count = np.zeros(n, int)
        for j in direct:
            count[j] += 1
        for cell in approx:
            accepted += 1
            count[cell.particles] += 1
            assert i not in cell.particles
            assert not any((i, int(j)) in s.near for j in cell.particles)
            assert cell.nodes > (degree + 1) ** 3
        assert np.all(count == 1)
        assert i in direct
    assert accepted > 0
    d, p = t.pair_counts()
    assert p > 0 and d > 0


def test_vanishing_opening_angle_is_the_direct_sum(cloud):
    s = cloud
    t = tc.Treecode(s, 1e-9, 2)
    assert all(len(a) == 0 for a, _ in t.lists)
    x = suspensions.random_density(4, s.total_nodes)
    for kind in ("K", "S"):
        ref = tc.direct_smooth(s, kind, x)
        assert np.abs(t.smooth(kind, x) - ref).max() < 1e-12 * np.abs(ref).max()


def test_error_falls_with_degree_inside_the_model(cloud):
    """The model C(theta) rho^-n holds from degree 2 on (degree 1 exceeds it at theta >= 0.6)."""
    s = cloud
    x = suspensions.random_density(5, s.total_nodes)
    theta = 0.6
    for kind in ("K", "S"):
        ref = tc.direct_smooth(s, kind, x)
        errs = []
        for degree in (2, 3, 4, 5):
            t = tc.Treecode(s, theta, degree)
            assert sum(len(a) for a, _ in t.lists) > 0
            e = np.linalg.norm(t.smooth(kind, x) - ref) / np.linalg.norm(ref)
            errs.append(e)
            assert e <= tc.tree_error_bound(theta, degree), (kind, degree, e)
        assert all(b < a for a, b in zip(errs, errs[1:])), errs


def test_error_bound_values():
    """rho = 1/theta + sqrt(1/theta^2 - 1): theta = 0.5 gives 2 + sqrt(3), theta = 0.6 gives 3."""
    assert abs(tc.tree_error_bound(0.5, 7) - 0.25 * (2 + math.sqrt(3)) ** -7) < 1e-18
    assert abs(tc.tree_error_bound(0.6, 4) - 0.36 / 81) < 1e-15
    assert tc.tree_error_bound(0.5, 8) < tc.tree_error_bound(0.5, 7) < tc.tree_error_bound(0.6, 7)


def test_offdiagonal_with_tree_matches_operator_when_exact(cloud):
    """With no accepted cells, the treecode form of the off-diagonal operator (smooth sum plus the
    near correction) is the oracle's off-diagonal operator."""
    s = cloud
    t = tc.Treecode(s, 1e-9, 2)
    x = suspensions.random_density(6, s.total_nodes)
    nodes = np.arange(0, s.total_nodes, 37)
    full = tc.offdiagonal_with_tree(s, t, "K", x)
    ref = s.apply_rows("K", x, nodes) - np.concatenate(
        [(s.self_block_lab("K", i) @ x[s.sl(i)].reshape(-1)).reshape(-1, 3) for i in range(len(s.particles))])[nodes]
    assert np.abs(full[nodes] - ref).max() < 1e-12 * np.abs(ref).max()


def test_error_model_with_whole_particle_clusters():
    """64 ellipsoids at p = 8 (144 nodes each): at degrees 3 and 4 single particles are approximated,
    the hardest case for the model."""
    s = system_of(suspensions.random_ellipsoids(64, 8, 16, 0.10, 0.2, seed=12))
    x = suspensions.random_density(31, s.total_nodes)
    ref = {k: tc.direct_smooth(s, k, x) for k in "KS"}
    for theta, degree in ((0.5, 3), (0.6, 4), (0.7, 3)):
        t = tc.Treecode(s, theta, degree)
        for k in "KS":
            e = np.linalg.norm(t.smooth(k, x) - ref[k]) / np.linalg.norm(ref[k])
            assert e <= tc.tree_error_bound(theta, degree), (theta, degree, k, e)
