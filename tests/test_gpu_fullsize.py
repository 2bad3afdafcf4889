"""Parity at the full sizes of the workloads, in the launch configuration bench.py times (persistent
grids, autotuned kernel variants): the GPU applies each operator to a seeded density over all
312,000 (or 495,616) nodes and the oracle recomputes sampled rows one at a time, each over every
source particle (smooth, upsampled-near and singular-rule parts).  Tolerances as in
test_gpu_parity.py: float64 1e-12, double-float 1e-11, float32 2e-5 (relative to the largest sampled
row); the mixed solve is checked through its residual at sampled rows and its constraints."""
import numpy as np
import pytest

import oracle
import suspensions

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    return m


def sample_nodes(s, count, seed):
    """Seeded nodes spread over the particle list, first and last node of the system included."""
    rng = np.random.default_rng(seed)
    pick = list(rng.choice(s.total_nodes, size=count - 2, replace=False))
    return np.array(sorted(set(pick + [0, s.total_nodes - 1])))


@pytest.fixture(scope="module")
def c2(rbs):
    s = suspensions.c2_ellipsoids()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    ctx = rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED)
    ctx.set_suspension(s)
    yield s, ref, ctx
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("DF", 1e-11), ("MIXED", 2e-5)])
@pytest.mark.parametrize("op,kind,half,with_L", [("A", "K", 0.5, True), ("S", "S", 0.0, False)])
def test_c2_operators_at_sampled_rows(rbs, c2, prec, tol, op, kind, half, with_L):
    s, ref, ctx = c2
    x = suspensions.random_density(21, s.total_nodes)
    y = rbs.rbs_apply_operator(ctx.ctx, getattr(rbs, "RBS_OP_" + op), getattr(rbs, "RBS_PREC_" + prec), x)
    rows = sample_nodes(s, 6, 5)
    yr = ref.apply_rows(kind, x, rows, half=half, with_L=with_L)
    assert np.abs(y[rows] - yr).max() < tol * np.abs(yr).max()


def test_c2_float64_operator_at_sampled_rows(rbs, c2):
    s, ref, ctx = c2
    x = suspensions.random_density(22, s.total_nodes)
    y = rbs.rbs_apply_operator(ctx.ctx, rbs.RBS_OP_HALF_K, rbs.RBS_PREC_FP64, x)
    rows = sample_nodes(s, 4, 6)
    yr = ref.apply_rows("K", x, rows, half=0.5)
    assert np.abs(y[rows] - yr).max() < 1e-12 * np.abs(yr).max()


def test_c2_mixed_solve_residual_rows_and_constraints(rbs, c2):
    s, ref, ctx = c2
    v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-10, want_density=True)
    rows = sample_nodes(s, 6, 7)
    rho = ref.incident_density(s.F, s.T)
    b_rows = -ref.apply_rows("K", rho, rows, half=0.5)
    r_rows = b_rows - ref.apply_rows("K", mu, rows, half=0.5, with_L=True)
    assert np.abs(r_rows).max() < 1e-8 * np.abs(b_rows).max()
    # Eq. 20 for the solution, particle by particle
    x, nrm, w = rbs.rbs_get_surface(ctx.ctx)
    for i in (0, 499, 999):
        sl = ref.sl(i)
        pt = ref.particles[i]
        assert np.abs((w[sl, None] * mu[sl]).sum(0)).max() < 1e-6 * np.abs(w[sl, None] * mu[sl]).sum()
        assert np.abs((w[sl, None] * np.cross(pt.r, mu[sl])).sum(0)).max() < 1e-5 * np.abs(mu[sl]).sum() * pt.area


def test_c5_operator_at_sampled_rows(rbs):
    """The 2,048-ellipsoid sedimentation workload at full size (495,616 nodes), double-float."""
    s = suspensions.c5_sedimenting()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    x = suspensions.random_density(23, s.total_nodes)
    with rbs.Context(device=0) as ctx:
        ctx.set_suspension(s)
        y = rbs.rbs_apply_operator(ctx.ctx, rbs.RBS_OP_A, rbs.RBS_PREC_DF, x)
    rows = sample_nodes(s, 4, 8)
    yr = ref.apply_rows("K", x, rows, half=0.5, with_L=True)
    assert np.abs(y[rows] - yr).max() < 1e-11 * np.abs(yr).max()


def test_c3_operator_and_mixed_solve(rbs):
    """The 10,000-ellipsoid workload at full size (1,440,000 nodes, p = 8): the double-float operator
    at sampled rows against the oracle, then mixed solves at 1e-8 and 1e-10 whose (v, omega) agree to
    1e-8 and whose residual at sampled rows, recomputed by the oracle, meets the tolerance."""
    s = suspensions.c3_ellipsoids()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    x = suspensions.random_density(31, s.total_nodes)
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED) as ctx:
        ctx.set_suspension(s)
        y = rbs.rbs_apply_operator(ctx.ctx, rbs.RBS_OP_A, rbs.RBS_PREC_DF, x)
        rows = sample_nodes(s, 4, 9)
        yr = ref.apply_rows("K", x, rows, half=0.5, with_L=True)
        assert np.abs(y[rows] - yr).max() < 1e-11 * np.abs(yr).max()
        v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-8, want_density=True)
        v2, om2, _, _ = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-10)
    V, V2 = np.concatenate([v, om], 1), np.concatenate([v2, om2], 1)
    assert np.linalg.norm(V - V2) < 1e-8 * np.linalg.norm(V2)
    rows = sample_nodes(s, 4, 10)
    rho = ref.incident_density(s.F, s.T)
    b_rows = -ref.apply_rows("K", rho, rows, half=0.5)
    r_rows = b_rows - ref.apply_rows("K", mu, rows, half=0.5, with_L=True)
    assert np.abs(r_rows).max() < 1e-7 * np.abs(b_rows).max()


def test_c4_batched_suspensions(rbs):
    """256 independent suspensions of 4-512 ellipsoids with p in {6, 8, 12, 16} (25,210 particles,
    6.77M nodes) in one context: the double-float operator at sampled rows against the oracle (which
    keeps the suspensions apart), then mixed solves at 1e-8 and 1e-10 whose (v, omega) agree to 1e-8.
    Every suspension converges on its own right-hand side: the library reports each suspension's
    iterations and relative residual (all within 1e-8); the oracle recomputes, for every suspension,
    its residual at two sampled rows against 1e-8 of that suspension's ||b_s|| (estimated from its
    sampled rows of b), and for the three smallest suspensions the whole residual against ||b_s||."""
    s = suspensions.c4_batched()
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats, suspension_id=s.suspension_id)
    x = suspensions.random_density(41, s.total_nodes)
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED) as ctx:
        ctx.set_suspension(s)
        assert rbs.rbs_get_stats(ctx.ctx)["near_pairs"] == len(ref.near)
        y = rbs.rbs_apply_operator(ctx.ctx, rbs.RBS_OP_A, rbs.RBS_PREC_DF, x)
        rows = sample_nodes(s, 6, 11)
        yr = ref.apply_rows("K", x, rows, half=0.5, with_L=True)
        assert np.abs(y[rows] - yr).max() < 1e-11 * np.abs(yr).max()
        v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-8, want_density=True, per_suspension=True)
        its_s, res_s = rbs.rbs_get_suspension_results(ctx.ctx)
        v2, om2, _, _ = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-10)
    V, V2 = np.concatenate([v, om], 1), np.concatenate([v2, om2], 1)
    assert np.linalg.norm(V - V2) < 1e-8 * np.linalg.norm(V2)
    S = int(s.suspension_id.max()) + 1
    assert its.shape == (S,) and (its > 0).all() and (its == its_s).all()
    assert (res_s <= 1e-8).all()
    rho = ref.incident_density(s.F, s.T)
    # node ranges of the suspensions
    npp = s.nodes_per_particle
    node_off = np.concatenate([[0], np.cumsum(npp)])
    first = np.searchsorted(s.suspension_id, np.arange(S), side="left")
    last = np.searchsorted(s.suspension_id, np.arange(S), side="right")
    counts = last - first
    rng = np.random.default_rng(13)
    for q in range(S):
        a, b = node_off[first[q]], node_off[last[q]]
        rows = np.sort(rng.choice(np.arange(a, b), size=2, replace=False))
        b_rows = -ref.apply_rows("K", rho, rows, half=0.5)
        r_rows = b_rows - ref.apply_rows("K", mu, rows, half=0.5, with_L=True)
        bnorm_est = np.sqrt(3 * (b - a) * np.mean(b_rows ** 2))  # ||b_s||_2 from the rows' mean square
        assert np.abs(r_rows).max() < 1e-8 * bnorm_est, (q, counts[q])
    for q in np.argsort(counts, kind="stable")[:3]:
        a, b = node_off[first[q]], node_off[last[q]]
        rows = np.arange(a, b)
        b_rows = -ref.apply_rows("K", rho, rows, half=0.5)
        r_rows = b_rows - ref.apply_rows("K", mu, rows, half=0.5, with_L=True)
        assert np.linalg.norm(r_rows) <= 1.2e-8 * np.linalg.norm(b_rows), (q, counts[q])
