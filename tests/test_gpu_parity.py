"""Parity of the CUDA path (through the C ABI) with the float64 oracle on identical seeded inputs.

Tolerances (relative L2 over the stacked outputs):
* float64 operators: 1e-12 (both sides evaluate the same sums in float64; only the summation order
  differs, so the gap is a few hundred units in the last place);
* float64 solve, (v, omega): 1e-11;
* double-float operator (float64-class steps of the mixed solve): 1e-11 (double-float carries about
  44 bits per operation; tiles of 128 terms are summed in double-float, then in float64);
* float32 operator (inner-solve arithmetic): 2e-5 (float32 unit roundoff 6e-8 per pair, rsqrtf within
  2 ulp, blocks rounded to float32, sums of up to 10^5 terms with per-tile compensation);
* mixed-precision solve, (v, omega): 1e-8.
"""
import math

import numpy as np
import pytest

import oracle
import suspensions

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    import torch
    assert torch.cuda.is_available()
    return m


def mixed_system():
    """7 ellipsoids, p in {4, 5, 6}, n_phi = 2p or 2p + 2, near pairs present, 502 nodes (a ragged
    tail of the 128-node tiles)."""
    s = suspensions.random_ellipsoids(7, 4, None, 0.12, 0.2, seed=21)
    s.p = np.array([4, 6, 5, 6, 4, 5, 6], np.int32)
    s.nphi = np.array([8, 14, 10, 12, 10, 12, 14], np.int32)
    return s


@pytest.fixture(scope="module")
def small(rbs):
    s = mixed_system()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    ctx = rbs.Context(device=0).set_suspension(s)
    assert len(ref.near) > 0 and s.total_nodes % 128 != 0
    yield s, ref, ctx
    ctx.close()


def test_surface_matches_oracle(rbs, small):
    s, ref, ctx = small
    x, nrm, w = rbs.rbs_get_surface(ctx.ctx)
    xr = np.concatenate([p.x for p in ref.particles])
    nr = np.concatenate([p.normal for p in ref.particles])
    wr = np.concatenate([p.w for p in ref.particles])
    assert np.abs(x - xr).max() < 1e-13 and np.abs(nrm - nr).max() < 1e-13
    assert np.abs(w - wr).max() < 1e-14
    st = rbs.rbs_get_stats(ctx.ctx)
    assert st["near_pairs"] == len(ref.near) and st["total_nodes"] == s.total_nodes


def test_incident_density_and_rigid_velocities(rbs, small):
    s, ref, ctx = small
    rho = rbs.rbs_incident_density(ctx.ctx, s.F, s.T)
    assert rel(rho, ref.incident_density(s.F, s.T)) < 1e-13
    u = suspensions.random_density(5, s.total_nodes)
    v, om = rbs.rbs_rigid_velocities(ctx.ctx, u, s.n)
    vr, omr = ref.rigid_velocities(u)
    assert rel(v, vr) < 1e-13 and rel(om, omr) < 1e-13


OPS = {
    "K_SELF": ("K", 0.0, False, "self"),
    "S_SELF": ("S", 0.0, False, "self"),
    "K_OFF": ("K", 0.0, False, "off"),
    "S_OFF": ("S", 0.0, False, "off"),
    "A": ("K", 0.5, True, "all"),
    "HALF_K": ("K", 0.5, False, "all"),
    "S": ("S", 0.0, False, "all"),
}


def oracle_op(ref, name, x):
    kind, half, with_L, part = OPS[name]
    if part == "all":
        return ref.apply(kind, x, half=half, with_L=with_L)
    y = np.zeros_like(x)
    for i, pi in enumerate(ref.particles):
        si = ref.sl(i)
        if part == "self":
            y[si] = (ref.self_block_lab(kind, i) @ x[si].reshape(-1)).reshape(-1, 3)
        else:
            for j, pj in enumerate(ref.particles):
                if j != i and oracle.operators.interacts(pi, pj):
                    y[si] += np.einsum("tkms,sm->tk", ref.pair_block(kind, i, j), x[ref.sl(j)])
    return y


@pytest.mark.parametrize("name", list(OPS))
def test_float64_operators_match_oracle(rbs, small, name):
    s, ref, ctx = small
    x = suspensions.random_density(1, s.total_nodes)
    y = rbs.rbs_apply_operator(ctx.ctx, getattr(rbs, "RBS_OP_" + name), rbs.RBS_PREC_FP64, x)
    assert rel(y, oracle_op(ref, name, x)) < 1e-12


def test_projection_operator_matches_oracle(rbs, small):
    s, ref, ctx = small
    x = suspensions.random_density(2, s.total_nodes)
    y = rbs.rbs_apply_operator(ctx.ctx, rbs.RBS_OP_L, rbs.RBS_PREC_FP64, x)
    yr = np.zeros_like(x)
    for i, p in enumerate(ref.particles):
        yr[ref.sl(i)] = np.einsum("tkms,sm->tk", oracle.operators.projection_block(p), x[ref.sl(i)])
    assert rel(y, yr) < 1e-13


@pytest.mark.parametrize("name", ["A", "K_OFF", "S_OFF", "HALF_K", "S"])
def test_double_float_operators_match_oracle(rbs, small, name):
    s, ref, ctx = small
    x = suspensions.random_density(6, s.total_nodes)
    y = rbs.rbs_apply_operator(ctx.ctx, getattr(rbs, "RBS_OP_" + name), rbs.RBS_PREC_DF, x)
    assert rel(y, oracle_op(ref, name, x)) < 1e-11


@pytest.mark.parametrize("name", ["A", "K_OFF", "S_OFF", "HALF_K"])
def test_float32_operators_within_float32_bound(rbs, small, name):
    s, ref, ctx = small
    x = suspensions.random_density(3, s.total_nodes)
    y = rbs.rbs_apply_operator(ctx.ctx, getattr(rbs, "RBS_OP_" + name), rbs.RBS_PREC_MIXED, x)
    assert rel(y, oracle_op(ref, name, x)) < 2e-5


def test_float64_solve_matches_oracle_lu(rbs, small):
    s, ref, ctx = small
    v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-13, want_density=True)
    vr, omr, mur, _, _ = ref.solve(s.F, s.T)
    assert rel(np.concatenate([v, om]), np.concatenate([vr, omr])) < 1e-11
    assert rel(mu, mur) < 1e-10
    assert 0 < its < 40


@pytest.mark.parametrize("refine", ["DF", "FP64"])
def test_mixed_solve_matches_oracle(rbs, small, refine):
    s, ref, _ = small
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED,
                     refine_precision=getattr(rbs, "RBS_PREC_" + refine)) as ctx:
        ctx.set_suspension(s)
        v, om, _, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-10)
        st = rbs.rbs_get_stats(ctx.ctx)
    vr, omr, *_ = ref.solve(s.F, s.T)
    assert rel(np.concatenate([v, om]), np.concatenate([vr, omr])) < 1e-8
    assert st["refinements"] >= 1 and st["residual"] <= 1e-10


def test_mixed_solve_at_tight_tolerance(rbs, small):
    """At tol 1e-12 the refinement takes float64-class passes (fused traction + Stokeslet) until the
    residual is small enough for float32 updates; the answer meets the oracle's LU at the double-float
    level, and a previous-solution warm start reaches the same answer."""
    s, ref, _ = small
    vr, omr, *_ = ref.solve(s.F, s.T)
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED, warm_start=rbs.RBS_WARM_PREVIOUS) as ctx:
        ctx.set_suspension(s)
        v, om, _, _ = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-12)
        st = rbs.rbs_get_stats(ctx.ctx)
        assert st["residual"] <= 1e-12 and st["kernel_count"][rbs.RBS_KC_PAIR_KSDF] >= 1
        assert rel(np.concatenate([v, om]), np.concatenate([vr, omr])) < 1e-10
        v2, om2, _, its2 = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-12)
    assert rel(np.concatenate([v2, om2]), np.concatenate([vr, omr])) < 1e-10


def test_unpreconditioned_solve_agrees(rbs, small):
    s, ref, _ = small
    with rbs.Context(device=0, preconditioner=0) as ctx:
        ctx.set_suspension(s)
        v, om, _, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-13)
    vr, omr, *_ = ref.solve(s.F, s.T)
    assert rel(np.concatenate([v, om]), np.concatenate([vr, omr])) < 1e-11


def test_c1_spheres_float64_solve(rbs):
    """The 8-sphere workload (p = 8, 3,456 unknowns) against the oracle's dense LU."""
    s = suspensions.c1_spheres()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    vr, omr, *_ = ref.solve(s.F, s.T)
    with rbs.Context(device=0) as ctx:
        ctx.set_suspension(s)
        v, om, _, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-12)
    assert rel(np.concatenate([v, om]), np.concatenate([vr, omr])) < 1e-11


def test_single_sphere_stokes_law_on_gpu(rbs):
    F = np.array([[0.3, -1.2, 0.8]])
    T = np.array([[1.1, 0.4, -0.6]])
    a = 1.3
    with rbs.Context(device=0) as ctx:
        ctx.set_geometry([[a, a, a]], 8, 16, [[2.0, -1.0, 0.5]], [[0.9, 0.1, -0.3, 0.2]])
        v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, F, T, 1e-12, want_density=True)
    assert np.allclose(v, F / (6 * math.pi * a), atol=1e-14, rtol=0)
    assert np.allclose(om, T / (8 * math.pi * a ** 3), atol=1e-14, rtol=0)


def test_separate_suspensions_do_not_interact(rbs):
    s = mixed_system()
    sid = np.array([0, 0, 0, 1, 1, 1, 1], np.int32)
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats, suspension_id=sid)
    vr, omr, *_ = ref.solve(s.F, s.T)
    with rbs.Context(device=0) as ctx:
        ctx.set_geometry(s.semi_axes, s.p, s.nphi, s.centres, s.quats, sid)
        v, om, _, _ = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-13)
    assert rel(np.concatenate([v, om]), np.concatenate([vr, omr])) < 1e-11


def test_error_statuses(rbs):
    with rbs.Context(device=0) as ctx:
        with pytest.raises(rbs.RbsError) as e:
            rbs.rbs_mobility_solve(ctx.ctx, np.zeros((1, 3)), np.zeros((1, 3)), 1e-8)
        assert e.value.code == rbs.RBS_ESTATE
        with pytest.raises(rbs.RbsError) as e:
            ctx.set_geometry([[1, 1, 1], [1, 1, 1]], 4, 8, [[0, 0, 0], [1.0, 0, 0]], [[1, 0, 0, 0]] * 2)
        assert e.value.code == rbs.RBS_EOVERLAP
        with pytest.raises(rbs.RbsError) as e:
            ctx.set_geometry([[1, 1, 1]], 1, 2, [[0, 0, 0]], [[1, 0, 0, 0]])
        assert e.value.code == rbs.RBS_EINVAL
        ctx.set_geometry([[1, 1, 1]], 4, 8, [[0, 0, 0]], [[1, 0, 0, 0]])
        with pytest.raises(rbs.RbsError) as e:
            rbs.rbs_mobility_solve(ctx.ctx, np.full((1, 3), np.nan), np.zeros((1, 3)), 1e-8)
        assert e.value.code == rbs.RBS_EINVAL
        # the context stays usable after the errors
        v, om, _, _ = rbs.rbs_mobility_solve(ctx.ctx, np.ones((1, 3)), np.zeros((1, 3)), 1e-10)
        assert np.allclose(v, 1 / (6 * math.pi))


def test_device_pointer_entry_points(rbs, small):
    import torch
    s, ref, ctx = small
    F = torch.tensor(s.F, device="cuda")
    T = torch.tensor(s.T, device="cuda")
    v = torch.zeros_like(F)
    om = torch.zeros_like(F)
    rbs.rbs_mobility_solve_device(ctx.ctx, F, T, 1e-13, v, om)
    vh, omh, _, _ = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-13)
    assert np.allclose(v.cpu().numpy(), vh, atol=1e-15) and np.allclose(om.cpu().numpy(), omh, atol=1e-15)
    x = torch.tensor(suspensions.random_density(4, s.total_nodes), device="cuda")
    y = torch.zeros_like(x)
    rbs.rbs_apply_operator_device(ctx.ctx, rbs.RBS_OP_A, rbs.RBS_PREC_FP64, x, y)
    assert rel(y.cpu().numpy(), oracle_op(ref, "A", x.cpu().numpy())) < 1e-12


@pytest.mark.parametrize("variant", [1, 2, 4, 9, 10, 12])
def test_every_pair_kernel_variant_matches_oracle(rbs, variant):
    """The autotuner picks among 1, 2 and 4 targets per thread, and for float32 also among the packed
    kernels (9, 10, 12: two sources per instruction); each variant is held to the same bounds."""
    s = mixed_system()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    x = suspensions.random_density(7, s.total_nodes)
    with rbs.Context(device=0, pair_variant=variant) as ctx:
        ctx.set_suspension(s)
        for name in ("K_OFF", "S_OFF"):
            y_ref = oracle_op(ref, name, x)
            op = getattr(rbs, "RBS_OP_" + name)
            assert rel(rbs.rbs_apply_operator(ctx.ctx, op, rbs.RBS_PREC_MIXED, x), y_ref) < 2e-5
            assert rel(rbs.rbs_apply_operator(ctx.ctx, op, rbs.RBS_PREC_DF, x), y_ref) < 1e-11
