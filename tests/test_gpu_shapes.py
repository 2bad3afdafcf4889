"""Parity of the CUDA path with the float64 oracle for general coefficient surfaces (Section 3,
Eqs. 31, 35-37): nodes, normals and weights, every operator, and the solves.  Tolerances as for the
ellipsoid parity tests (relative L2): float64 operators 1e-12, float64 solve 1e-11, double-float
operators 1e-11, float32 operators 2e-5, mixed solve 1e-8."""
import numpy as np
import pytest

import oracle
import suspensions
from oracle import shapes as shp
from shape_inputs import star_shape
from test_gpu_parity import oracle_op, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    import torch
    assert torch.cuda.is_available()
    return m


def shape_system():
    """Five particles on three input surfaces (two star shapes and an ellipsoid written as degree-1
    coefficients), p in {5, 6}, n_phi in {10, 12, 14}; spacing 3 along a bent line, so neighbours are
    near (R ~ 1.3) and 5 * 84-ish nodes leave a ragged tail of the 128-node tiles."""
    shapes = [star_shape(1), star_shape(2), shp.sh_coefficients_of_ellipsoid((1.1, 0.9, 0.75))]
    shape_of = np.array([0, 1, 2, 0, 1], np.int32)
    p = np.array([6, 5, 6, 5, 6], np.int32)
    nphi = np.array([12, 10, 14, 12, 12], np.int32)
    centres = np.array([[0, 0, 0], [3.0, 0.3, 0.1], [5.8, 1.2, -0.4], [8.6, 2.0, 0.5], [11.5, 2.2, 0.0]])
    rng = np.random.default_rng(11)
    q = rng.normal(size=(5, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    F = rng.normal(size=(5, 3))
    T = rng.normal(size=(5, 3))
    return shapes, shape_of, p, nphi, centres, q, F, T


@pytest.fixture(scope="module")
def shaped(rbs):
    shapes, shape_of, p, nphi, centres, q, F, T = shape_system()
    ref = oracle.System(None, p, nphi, centres, q, shapes=shapes, shape_of=shape_of)
    ctx = rbs.Context(device=0).set_shapes(shapes, shape_of, p, nphi, centres, q)
    assert len(ref.near) > 0 and ref.total_nodes % 128 != 0
    yield (shapes, shape_of, p, nphi, centres, q, F, T), ref, ctx
    ctx.close()


def test_surface_matches_oracle(rbs, shaped):
    _, ref, ctx = shaped
    x, nrm, w = rbs.rbs_get_surface(ctx.ctx)
    xr = np.concatenate([pt.x for pt in ref.particles])
    nr = np.concatenate([pt.normal for pt in ref.particles])
    wr = np.concatenate([pt.w for pt in ref.particles])
    assert np.abs(x - xr).max() < 1e-13 and np.abs(nrm - nr).max() < 1e-12
    assert np.abs(w - wr).max() < 1e-13
    st = rbs.rbs_get_stats(ctx.ctx)
    assert st["near_pairs"] == len(ref.near) and st["total_nodes"] == ref.total_nodes
    assert st["n_shapes"] == len(ref._bodies)


@pytest.mark.parametrize("name", ["K_SELF", "S_SELF", "K_OFF", "S_OFF", "A", "S"])
def test_float64_operators_match_oracle(rbs, shaped, name):
    _, ref, ctx = shaped
    x = suspensions.random_density(8, ref.total_nodes)
    y = rbs.rbs_apply_operator(ctx.ctx, getattr(rbs, "RBS_OP_" + name), rbs.RBS_PREC_FP64, x)
    assert rel(y, oracle_op(ref, name, x)) < 1e-12


@pytest.mark.parametrize("name", ["A", "K_OFF", "S_OFF"])
def test_reduced_precision_operators(rbs, shaped, name):
    _, ref, ctx = shaped
    x = suspensions.random_density(9, ref.total_nodes)
    yr = oracle_op(ref, name, x)
    op = getattr(rbs, "RBS_OP_" + name)
    assert rel(rbs.rbs_apply_operator(ctx.ctx, op, rbs.RBS_PREC_DF, x), yr) < 1e-11
    assert rel(rbs.rbs_apply_operator(ctx.ctx, op, rbs.RBS_PREC_MIXED, x), yr) < 2e-5


def test_solves_match_oracle(rbs, shaped):
    (shapes, shape_of, p, nphi, centres, q, F, T), ref, ctx = shaped
    vr, omr, mur, _, _ = ref.solve(F, T)
    v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, F, T, 1e-13, want_density=True)
    assert rel(np.concatenate([v, om]), np.concatenate([vr, omr])) < 1e-11
    assert rel(mu, mur) < 1e-10
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED) as mctx:
        mctx.set_shapes(shapes, shape_of, p, nphi, centres, q)
        v, om, _, _ = rbs.rbs_mobility_solve(mctx.ctx, F, T, 1e-10)
    assert rel(np.concatenate([v, om]), np.concatenate([vr, omr])) < 1e-8


def test_coefficient_ellipsoid_matches_the_analytic_path(rbs):
    """Three ellipsoids given both ways; the pair distances (2.6 and >= 6) sit far from the near
    threshold R_i + R_j + 1 under either bounding radius (largest semi-axis, or largest node distance)."""
    axes = np.array([[1.1, 0.9, 0.75], [0.8, 1.0, 0.7], [1.1, 0.9, 0.75]])
    centres = np.array([[0, 0, 0], [2.6, 0, 0], [2.0, 6.0, 0.5]])
    rng = np.random.default_rng(4)
    q = rng.normal(size=(3, 4))
    F, T = rng.normal(size=(2, 3, 3))
    shapes = [shp.sh_coefficients_of_ellipsoid(a) for a in axes[:2]]
    with rbs.Context(device=0) as a, rbs.Context(device=0) as b:
        a.set_geometry(axes, 6, 14, centres, q)
        b.set_shapes(shapes, [0, 1, 0], 6, 14, centres, q)
        assert rbs.rbs_get_stats(a.ctx)["near_pairs"] == rbs.rbs_get_stats(b.ctx)["near_pairs"] == 2
        xa, na, wa = rbs.rbs_get_surface(a.ctx)
        xb, nb, wb = rbs.rbs_get_surface(b.ctx)
        assert np.abs(xa - xb).max() < 1e-13 and np.abs(na - nb).max() < 1e-13 and np.abs(wa - wb).max() < 1e-13
        va, oa, _, _ = rbs.rbs_mobility_solve(a.ctx, F, T, 1e-13)
        vb, ob, _, _ = rbs.rbs_mobility_solve(b.ctx, F, T, 1e-13)
    assert rel(np.concatenate([vb, ob]), np.concatenate([va, oa])) < 1e-12


def test_invalid_coefficient_surfaces_are_rejected(rbs):
    coef, pg = star_shape(3)
    with rbs.Context(device=0) as ctx:
        for shapes, shape_of in (([(-coef, pg)], [0]),                   # inward parametrisation
                                 ([(np.zeros((3, 4)), 1)], [0]),         # degenerate (J = 0)
                                 ([(coef, pg)], [1])):                   # shape index out of range
            with pytest.raises(rbs.RbsError) as e:
                ctx.set_shapes(shapes, shape_of, 6, 12, [[0, 0, 0]], [[1, 0, 0, 0]])
            assert e.value.code == rbs.RBS_EINVAL
        ctx.set_shapes([(coef, pg)], [0], 6, 12, [[0, 0, 0]], [[1, 0, 0, 0]])
        v, om, _, _ = rbs.rbs_mobility_solve(ctx.ctx, np.ones((1, 3)), np.zeros((1, 3)), 1e-10)
        assert np.all(np.isfinite(v)) and np.all(np.isfinite(om))
