"""Parity of the contact force algorithm (Section 3.4, rbs_options.contact_gap) with the oracle: the
contacts found, their points and forces, the corrected velocities and density; the no-slip condition
at contact; two equal spheres pushed together stay at rest under time stepping.  Tolerances (relative
L2): float64 velocities 1e-10, density 1e-9, contact forces 1e-8 (the 3 n_c x 3 n_c contact system
amplifies the solves' 1e-12 error by its condition number), mixed-precision velocities 1e-7."""
import numpy as np
import pytest

from oracle import contact as oc
from test_gpu_parity import rel
from test_oracle_contact import three_ellipsoids, two_spheres

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    import torch
    assert torch.cuda.is_available()
    return m


def geometry_of(s):
    axes = np.array([pt.body.axes for pt in s.particles])
    cen = np.array([pt.centre for pt in s.particles])
    return axes, cen


@pytest.mark.parametrize("prec,tol_v", [("FP64", 1e-10), ("MIXED", 1e-7)])
def test_contact_solve_matches_oracle(rbs, prec, tol_v):
    s, rng = three_ellipsoids()
    q = np.random.default_rng(5).normal(size=(3, 4))  # the orientations three_ellipsoids drew
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    F, T = rng.normal(size=(2, 3, 3))
    vr, omr, mur, cts, Fcr = oc.solve_with_contacts(s, F, T, 0.1)
    axes, cen = geometry_of(s)
    with rbs.Context(device=0, precision=getattr(rbs, "RBS_PREC_" + prec), contact_gap=0.1) as ctx:
        ctx.set_geometry(axes, 6, 12, cen, q)
        v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, F, T, 1e-13 if prec == "FP64" else 1e-11,
                                                want_density=True)
        pairs, points, forces = rbs.rbs_get_contacts(ctx.ctx)
        assert rbs.rbs_get_stats(ctx.ctx)["n_contacts"] == len(cts)
    assert [tuple(p) for p in pairs] == [(i, j) for i, j, _ in cts]
    assert np.abs(points - np.array([x for _, _, x in cts])).max() < 1e-12
    assert rel(forces, Fcr) < (1e-8 if prec == "FP64" else 1e-6)
    assert rel(np.concatenate([v, om]), np.concatenate([vr, omr])) < tol_v
    if prec == "FP64":
        assert rel(mu, mur) < 1e-9
    V = np.concatenate([v, om], 1).reshape(-1)
    assert np.abs(oc.velocity_difference_map(s, cts) @ V).max() < 1e-9 * np.abs(V).max()


def test_equal_spheres_pushed_together_stay_at_rest(rbs):
    F = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    T = np.zeros((2, 3))
    cen = np.array([[0.0, 0.0, 0.0], [2.03, 0.0, 0.0]])
    quats = np.tile([1.0, 0, 0, 0], (2, 1))
    with rbs.Context(device=0, contact_gap=0.05) as ctx:
        ctx.set_geometry([[1, 1, 1]] * 2, 6, 12, cen, quats)
        v, om, _, _ = rbs.rbs_mobility_solve(ctx.ctx, F, T, 1e-13)
        assert np.abs(v).max() < 1e-10 and np.abs(om).max() < 1e-10
        rbs.rbs_advance(ctx.ctx, F, T, 0.1, 3, rbs.RBS_RK4, 1e-12)
        c_end, _ = rbs.rbs_get_state(ctx.ctx, 2)
    assert np.abs(c_end - cen).max() < 1e-9
    with rbs.Context(device=0) as ctx:  # without contact handling they approach
        ctx.set_geometry([[1, 1, 1]] * 2, 6, 12, cen, quats)
        rbs.rbs_advance(ctx.ctx, F, T, 0.1, 3, rbs.RBS_RK4, 1e-12)
        c_free, _ = rbs.rbs_get_state(ctx.ctx, 2)
    assert c_free[1, 0] - c_free[0, 0] < 2.03 - 1e-4


def test_no_contact_beyond_the_gap(rbs):
    s = two_spheres(0.2)
    F = np.array([[1.0, 0.3, 0], [-1.0, 0, 0.2]])
    T = np.array([[0.1, 0, 0], [0, 0.2, 0]])
    cen = np.array([pt.centre for pt in s.particles])
    with rbs.Context(device=0, contact_gap=0.1) as a, rbs.Context(device=0) as b:
        a.set_geometry([[1, 1, 1]] * 2, 6, 12, cen, np.tile([1.0, 0, 0, 0], (2, 1)))
        b.set_geometry([[1, 1, 1]] * 2, 6, 12, cen, np.tile([1.0, 0, 0, 0], (2, 1)))
        va, oa, _, _ = rbs.rbs_mobility_solve(a.ctx, F, T, 1e-13)
        vb, ob, _, _ = rbs.rbs_mobility_solve(b.ctx, F, T, 1e-13)
        assert rbs.rbs_get_stats(a.ctx)["n_contacts"] == 0
    assert np.array_equal(va, vb) and np.array_equal(oa, ob)
