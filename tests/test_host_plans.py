"""Host logic of the library without a GPU: the treecode plan (rbs_treecode_plan) and the near-pair
list (rbs_near_plan), the same host code a context runs, against the oracle's statement of each
(oracle/treecode.py; the near criterion of oracle.System).  Given the same particle centres, radii
and node boxes, the two must build the same trees, interaction lists and near pairs, which exact pair,
cluster and pair-set comparisons check at the sizes of the workloads."""
import numpy as np
import pytest

import oracle
import suspensions
from oracle import treecode as tc


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    return m


def plan_inputs(system):
    parts = system.particles
    nodes = np.array([len(p.w) for p in parts])
    centres = np.array([p.centre for p in parts])
    radius = np.array([p.radius for p in parts])
    box = np.array([np.concatenate(tc.particle_box(p)) for p in parts])
    sid = np.array([p.suspension for p in parts])
    return nodes, centres, radius, box, sid


def check(rbs, system, theta, degree):
    t = tc.Treecode(system, theta, degree)
    direct, proxy = t.pair_counts()
    cells = len({id(c) for a, _ in t.lists for c in a})
    nodes, centres, radius, box, sid = plan_inputs(system)
    plan = rbs.rbs_treecode_plan(nodes, centres, radius, box, sid, theta, degree, system.opt.delta)
    assert (plan["direct_pairs"], plan["proxy_pairs"], plan["cells"]) == (direct, proxy, cells)
    # every interacting pair of nodes is evaluated once, exactly or through a cluster
    total = sum(len(p.w) * sum(len(q.w) for q in system.particles if q.suspension == p.suspension)
                for p in system.particles)
    covered = sum(len(p.w) * (sum(len(system.particles[j].w) for j in d) + sum(c.nodes for c in a))
                  for p, (a, d) in zip(system.particles, t.lists))
    assert covered == total
    assert plan["items"] >= len(system.particles) and plan["segments"] >= len(system.particles)
    assert 0 < plan["tmax"] <= 512
    return plan


@pytest.mark.parametrize("theta,degree", [(0.5, 2), (0.7, 3), (0.3, 2)])
def test_plan_matches_oracle_small(rbs, theta, degree):
    s = suspensions.random_ellipsoids(300, 2, 4, 0.10, 0.2, seed=11)
    system = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats, s.suspension_id)
    plan = check(rbs, system, theta, degree)
    assert plan["proxy_pairs"] > 0


@pytest.mark.parametrize("sizes", [(5, 90, 160), (1, 2, 90), (1,)])
def test_plan_matches_oracle_with_several_suspensions(rbs, sizes):
    """Independent suspensions, including the degenerate ones: a single particle (a one-leaf tree with
    nothing to approximate) and a pair."""
    parts = [suspensions.random_ellipsoids(k, 4, 8, 0.10, 0.2, seed=20 + k) for k in sizes]
    cat = lambda f: np.concatenate([getattr(x, f) for x in parts])
    sid = np.concatenate([np.full(x.n, i) for i, x in enumerate(parts)])
    system = oracle.System(cat("semi_axes"), cat("p"), cat("nphi"), cat("centres"), cat("quats"), sid)
    plan = check(rbs, system, 0.6, 3)
    assert (plan["proxy_pairs"] > 0) == (max(sizes) >= 90)


@pytest.mark.parametrize("theta,degree", [(0.5, 7), (0.4, 12)])
def test_plan_matches_oracle_at_the_1000_ellipsoid_size(rbs, theta, degree):
    """The float32 (0.5, 7) and double-float (0.4, 12) treecodes of the 1,000-ellipsoid workload; the
    pair counts are those the GPU runs reported (2.61e10 and 6.60e10 per apply)."""
    s = suspensions.c2_ellipsoids()
    system = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    plan = check(rbs, system, theta, degree)
    expected = {(0.5, 7): 26121955392, (0.4, 12): 66019686408}[(theta, degree)]
    assert plan["direct_pairs"] + plan["proxy_pairs"] == expected


def test_plan_rejects_bad_arguments(rbs):
    nodes, centres, radius, box = [4], [[0, 0, 0]], [1.0], [[-1, -1, -1, 1, 1, 1]]
    for kw in ({"theta": 1.0}, {"theta": 0.0}, {"degree": 1}, {"degree": 13}, {"sm_count": 0}):
        with pytest.raises(rbs.RbsError):
            rbs.rbs_treecode_plan(nodes, centres, radius, box, **kw)
    with pytest.raises(rbs.RbsError):
        rbs.rbs_treecode_plan([0], centres, radius, box)


def test_near_plan_matches_oracle_near_pairs(rbs):
    """The library's near-pair list (the host code a context runs) equals the oracle's near set on the
    1,000-ellipsoid workload."""
    s = suspensions.c2_ellipsoids()
    system = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    radius = np.array([p.radius for p in system.particles])
    pairs = rbs.rbs_near_plan(s.centres, radius, s.semi_axes.min(1), None, system.opt.delta)
    assert set(map(tuple, pairs.tolist())) == system.near
    assert len(pairs) == len(system.near) > 0


def test_near_plan_on_independent_suspensions(rbs):
    """The 256-suspension workload (25,210 particles): pairs only within a suspension, exactly those
    closer than R_i + R_j + 1 (brute force per suspension)."""
    s = suspensions.c4_batched()
    R = s.semi_axes.max(1)
    pairs = rbs.rbs_near_plan(s.centres, R, s.semi_axes.min(1), s.suspension_id, 1.0)
    got = set(map(tuple, pairs.tolist()))
    want = set()
    for k in np.unique(s.suspension_id):
        idx = np.nonzero(s.suspension_id == k)[0]
        d = np.linalg.norm(s.centres[idx, None, :] - s.centres[None, idx, :], axis=2)
        hit = (d < R[idx, None] + R[None, idx] + 1.0) & ~np.eye(len(idx), dtype=bool)
        want |= {(int(idx[a]), int(idx[b])) for a, b in zip(*np.nonzero(hit))}
    assert got == want and len(got) > 0


def test_near_plan_reports_overlap(rbs):
    centres = np.array([[0.0, 0.0, 0.0], [1.5, 0.0, 0.0], [9.0, 0.0, 0.0]])
    with pytest.raises(rbs.RbsError) as e:
        rbs.rbs_near_plan(centres, [1.0, 1.0, 1.0], [0.8, 0.8, 0.8])
    assert e.value.code == rbs.RBS_EOVERLAP
    # in different suspensions the same centres do not interact
    assert len(rbs.rbs_near_plan(centres, [1.0, 1.0, 1.0], [0.8, 0.8, 0.8], [0, 1, 2])) == 0


@pytest.mark.parametrize("p,nphi", [(2, 4), (5, 10), (8, 16), (10, 22), (12, 24), (16, 32)])
def test_grid_symmetry_tables(rbs, p, nphi):
    """The reflection tables behind the representative-row storage of ellipsoid self blocks, against
    the oracle's grid (Eq. 33): each node is its representative reflected by g_of (sign flips of x, y,
    z per bit), every representative is used, and each irreducible representation's dimension equals
    an independent count over the orbits' stabilisers (computed from the node positions), the eight
    summing to 3 (p + 1) n_phi."""
    from oracle import sphere_grid
    nrep, rep_of, g_of, dims = rbs.rbs_grid_symmetry(p, nphi)
    th, ph, _ = sphere_grid.grid_points(p, nphi)
    s = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    nk = nphi // 4 + 1
    assert nrep == (p // 2 + 1) * nk
    rep_node = (rep_of // nk) * nphi + rep_of % nk
    flips = lambda h: np.array([-1.0 if h & 1 else 1.0, -1.0 if h & 2 else 1.0, -1.0 if h & 4 else 1.0])
    sign = np.array([flips(int(g)) for g in g_of])
    assert np.abs(s[rep_node] * sign - s).max() < 1e-12
    assert set(rep_of.tolist()) == set(range(nrep))
    # independent irrep dimensions: for the orbit of representative r with stabiliser H (the
    # reflections fixing its position), component beta belongs to irrep c when
    # (-1)^popcount(c & h) * (-1)^(bit beta of h) = 1 for every h in H
    want = np.zeros(8, int)
    reps = np.unique(rep_node)
    for t in reps:
        H = [h for h in range(8) if np.abs(s[t] * flips(h) - s[t]).max() < 1e-12]
        for c in range(8):
            for beta in range(3):
                if all((-1) ** (bin(c & h).count("1") + ((h >> beta) & 1)) == 1 for h in H):
                    want[c] += 1
    assert dims.tolist() == want.tolist()
    assert dims.sum() == 3 * (p + 1) * nphi


def test_grid_symmetry_rejects_bad_grids(rbs):
    for p, nphi in ((1, 4), (33, 66), (4, 7), (4, 6)):
        with pytest.raises(rbs.RbsError):
            rbs.rbs_grid_symmetry(p, nphi)


def test_plan_with_mixed_grids(rbs):
    """Particles on different grids (p in {2, 4, 6}, as the batched workload mixes them): ragged node
    counts per particle and per cluster."""
    s = suspensions.random_ellipsoids(200, 2, None, 0.10, 0.2, seed=31)
    rng = np.random.default_rng(31)
    s.p = rng.choice(np.array([2, 4, 6], np.int32), size=s.n).astype(np.int32)
    s.nphi = (2 * s.p).astype(np.int32)
    system = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats, s.suspension_id)
    plan = check(rbs, system, 0.6, 3)
    assert plan["proxy_pairs"] > 0


def test_plan_refuses_more_sources_than_int32(rbs):
    """Source indices are 32-bit: a geometry beyond 2^31 nodes is refused, not wrapped."""
    nodes = [2_000_000_000, 2_000_000_000]
    centres = [[0.0, 0.0, 0.0], [10.0, 0.0, 0.0]]
    box = [[-1, -1, -1, 1, 1, 1], [9, -1, -1, 11, 1, 1]]
    with pytest.raises(rbs.RbsError) as e:
        rbs.rbs_treecode_plan(nodes, centres, [1.0, 1.0], box)
    assert e.value.code == rbs.RBS_ENOMEM
