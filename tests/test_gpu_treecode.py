"""GPU parity of the treecode far field (rbs_options.far_field = RBS_FAR_TREECODE) against the oracle's
statement of the same algorithm (oracle/treecode.py): identical trees and interaction lists (exact
pair and cluster counts), the float32 off-diagonal operators within float32 rounding of the oracle's
treecode and within the error model of the exact operator, and mixed solves that converge to the
exact (direct-sum) answer because the double-float refinement passes stay direct.

Cases: 300 ellipsoids at p = 2 (one work item per particle and source run), and 64 ellipsoids at
p = 8 (source lists split into several runs, whole-particle leaves approximated); the 1,000-ellipsoid
workload at full size with the default parameters.  The double-float passes' treecode
(RBS_FAR_TREECODE_DF) is checked the same way: its lists and operator against the oracle's at a low
degree, and a full-size solve with both treecodes against the exact residual and the all-direct
solve."""
import numpy as np
import pytest

import oracle
import suspensions
from oracle import treecode as tc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    return m


CASES = {
    "cloud300_p2": (lambda: suspensions.random_ellipsoids(300, 2, 4, 0.10, 0.2, seed=11), 0.5, 2),
    "cloud64_p8": (lambda: suspensions.random_ellipsoids(64, 8, 16, 0.10, 0.2, seed=12), 0.7, 3),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, rbs):
    make, theta, degree = CASES[request.param]
    s = make()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats, s.suspension_id)
    tree = tc.Treecode(ref, theta, degree)
    ctx = rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED, far_field=rbs.RBS_FAR_TREECODE,
                      tree_theta=theta, tree_degree=degree)
    ctx.set_suspension(s)
    # the oracle's treecode and exact off-diagonal operators for one seeded density
    x = suspensions.random_density(31, s.total_nodes)
    want, exact = {}, {}
    for kind in ("K", "S"):
        want[kind] = tc.offdiagonal_with_tree(ref, tree, kind, x)
        exact[kind] = want[kind] - tree.smooth(kind, x) + tc.direct_smooth(ref, kind, x)
    yield s, ref, tree, ctx, (x, want, exact)
    ctx.close()


def test_tree_and_lists_match_the_oracle(rbs, case):
    s, ref, tree, ctx, _ = case
    st = rbs.rbs_get_stats(ctx.ctx)
    direct, proxy = tree.pair_counts()
    cells = {id(c) for a, _ in tree.lists for c in a}
    assert proxy > 0
    assert st["tree_proxy_pairs"] == proxy
    assert st["tree_pairs"] == direct + proxy
    assert st["tree_cells"] == len(cells)


@pytest.mark.parametrize("op,kind", [("K_OFF", "K"), ("S_OFF", "S")])
def test_tree_operator_parity(rbs, case, op, kind):
    s, ref, tree, ctx, (x, wants, exacts) = case
    y = rbs.rbs_apply_operator(ctx.ctx, getattr(rbs, "RBS_OP_" + op), rbs.RBS_PREC_MIXED, x)
    want, exact = wants[kind], exacts[kind]
    # float32 rounding of the same sums (compensated tile accumulation)
    assert np.linalg.norm(y - want) <= 2e-6 * np.linalg.norm(want)
    assert np.abs(y - want).max() <= 2e-5 * np.abs(want).max()
    # and the treecode's approximation of the exact smooth sum stays inside the error model
    err = np.linalg.norm(y - exact) / np.linalg.norm(exact)
    assert err <= 1e-5 + tc.tree_error_bound(tree.theta, tree.degree)
    assert err > 1e-7   # the approximation is in use


def test_tree_float64_passes_stay_direct(rbs, case):
    """Double-float applies ignore the treecode: they match the oracle's exact operator."""
    s, ref, tree, ctx, (x, _, exacts) = case
    for op, kind in (("K_OFF", "K"), ("S_OFF", "S")):
        y = rbs.rbs_apply_operator(ctx.ctx, getattr(rbs, "RBS_OP_" + op), rbs.RBS_PREC_DF, x)
        assert np.abs(y - exacts[kind]).max() <= 1e-11 * np.abs(exacts[kind]).max()


def test_tree_mixed_solve_matches_direct_mixed_solve(rbs, case):
    s, ref, tree, ctx, _ = case
    v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-10, want_density=True)
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED) as d:
        d.set_suspension(s)
        v0, om0, mu0, its0 = rbs.rbs_mobility_solve(d.ctx, s.F, s.T, 1e-12, want_density=True)
    V, V0 = np.concatenate([v, om]), np.concatenate([v0, om0])
    assert np.linalg.norm(V - V0) <= 1e-8 * np.linalg.norm(V0)
    assert np.linalg.norm(mu - mu0) <= 1e-7 * np.linalg.norm(mu0)


def test_tree_solve_on_the_eight_spheres_matches_lu(rbs):
    """The 8-sphere case against the oracle's dense LU solution, with the treecode approximating some
    pairs (degree 2: 27 proxy points per cluster of 144 nodes)."""
    s = suspensions.c1_spheres()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    tree = tc.Treecode(ref, 0.5, 2)
    assert tree.pair_counts()[1] > 0
    vr, omr, mur, _, _ = ref.solve(s.F, s.T, method="lu")
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED, far_field=rbs.RBS_FAR_TREECODE, tree_theta=0.5,
                     tree_degree=2) as ctx:
        ctx.set_suspension(s)
        st = rbs.rbs_get_stats(ctx.ctx)
        assert st["tree_proxy_pairs"] == tree.pair_counts()[1]
        v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-11, want_density=True)
    V, Vr = np.concatenate([v, om]), np.concatenate([vr, omr])
    assert np.linalg.norm(V - Vr) <= 1e-9 * np.linalg.norm(Vr)


def test_tree_rejects_bad_parameters(rbs):
    for kw in ({"far_field": 3}, {"tree_theta": 0.0}, {"tree_theta": 1.0}, {"tree_degree": 1},
               {"tree_degree": 11}, {"tree_df_theta": 1.0}, {"tree_df_degree": 13}):
        with pytest.raises(rbs.RbsError):
            rbs.rbs_create(device=0, **kw)


@pytest.mark.slow
def test_c2_tree_mixed_solve_residual_rows(rbs):
    """The 1,000-ellipsoid workload at full size with the default treecode (theta 0.5, degree 7): the
    operator at sampled rows within the error model, and the solve's true residual at sampled rows
    below the tolerance."""
    s = suspensions.c2_ellipsoids()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    rng = np.random.default_rng(8)
    rows = np.array(sorted(set(rng.choice(s.total_nodes, 6, replace=False)) | {0, s.total_nodes - 1}))
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED, far_field=rbs.RBS_FAR_TREECODE) as ctx:
        ctx.set_suspension(s)
        st = rbs.rbs_get_stats(ctx.ctx)
        assert 0 < st["tree_pairs"] < st["far_pairs"]
        x = suspensions.random_density(33, s.total_nodes)
        y = rbs.rbs_apply_operator(ctx.ctx, rbs.RBS_OP_A, rbs.RBS_PREC_MIXED, x)
        yr = ref.apply_rows("K", x, rows, half=0.5, with_L=True)
        assert np.abs(y[rows] - yr).max() < (1e-5 + tc.tree_error_bound(0.5, 7)) * np.abs(yr).max()
        v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-10, want_density=True)
    rho = ref.incident_density(s.F, s.T)
    b_rows = -ref.apply_rows("K", rho, rows, half=0.5)
    r_rows = b_rows - ref.apply_rows("K", mu, rows, half=0.5, with_L=True)
    assert np.abs(r_rows).max() < 1e-8 * np.abs(b_rows).max()


def test_df_tree_lists_and_operator_match_the_oracle(rbs):
    """The double-float passes' treecode (far_field = RBS_FAR_TREECODE_DF) on 64 ellipsoids at p = 8,
    at theta 0.5 and degree 3 so that single particles are approximated: identical lists, and the
    double-float traction operator equal to the oracle's treecode operator to double-float rounding
    (the cluster charges are formed in float64 on both sides)."""
    s = suspensions.random_ellipsoids(64, 8, 16, 0.10, 0.2, seed=12)
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats, s.suspension_id)
    tree = tc.Treecode(ref, 0.5, 3)
    direct, proxy = tree.pair_counts()
    x = suspensions.random_density(34, s.total_nodes)
    want = tc.offdiagonal_with_tree(ref, tree, "K", x)
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED, far_field=rbs.RBS_FAR_TREECODE_DF, tree_df_theta=0.5,
                     tree_df_degree=3) as ctx:
        ctx.set_suspension(s)
        st = rbs.rbs_get_stats(ctx.ctx)
        assert st["tree_df_proxy_pairs"] == proxy > 0
        assert st["tree_df_pairs"] == direct + proxy
        assert st["tree_df_cells"] == len({id(c) for a, _ in tree.lists for c in a})
        y = rbs.rbs_apply_operator(ctx.ctx, rbs.RBS_OP_K_OFF, rbs.RBS_PREC_DF, x)
    assert np.abs(y - want).max() <= 1e-11 * np.abs(want).max()


@pytest.mark.slow
def test_c2_df_tree_solve(rbs):
    """The 1,000-ellipsoid workload with treecodes in both the float32 and the double-float passes at
    their defaults (theta 0.4, degree 12 for the latter): the solve's true residual at sampled rows
    stays below the tolerance, and its velocities agree with the all-direct mixed solve to 1e-8."""
    s = suspensions.c2_ellipsoids()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    rng = np.random.default_rng(9)
    rows = np.array(sorted(set(rng.choice(s.total_nodes, 6, replace=False)) | {0, s.total_nodes - 1}))
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED, far_field=rbs.RBS_FAR_TREECODE_DF) as ctx:
        ctx.set_suspension(s)
        st = rbs.rbs_get_stats(ctx.ctx)
        assert 0 < st["tree_df_pairs"] < st["far_pairs"]
        v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-10, want_density=True)
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED) as d:
        d.set_suspension(s)
        v0, om0, _, _ = rbs.rbs_mobility_solve(d.ctx, s.F, s.T, 1e-12)
    V, V0 = np.concatenate([v, om]), np.concatenate([v0, om0])
    assert np.linalg.norm(V - V0) <= 1e-8 * np.linalg.norm(V0)
    rho = ref.incident_density(s.F, s.T)
    b_rows = -ref.apply_rows("K", rho, rows, half=0.5)
    r_rows = b_rows - ref.apply_rows("K", mu, rows, half=0.5, with_L=True)
    assert np.abs(r_rows).max() < 1e-8 * np.abs(b_rows).max()
