"""Batched suspensions converge one by one.

Particles of different suspensions do not interact, so each suspension of a batch is its own linear
system (Eq. 25).  The library's GMRES keeps one Krylov recursion per suspension and stops each on its
own residual; these tests check that every suspension meets the tolerance on its own right-hand side,
whatever the size or the force scale of the others, against the oracle's dense LU of that suspension
alone.  They also check that the captured CUDA-graph GMRES (a conditional loop that runs a restart
cycle on the device) and the host-driven GMRES agree, and that the per-suspension iteration counts
and residuals come back through the C ABI.
"""
import numpy as np
import pytest

import oracle
import suspensions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    return m


def small_batch():
    """Three suspensions of 2, 5 and 9 ellipsoids at p = 6, each placed on its own (seeds 51-53); the
    forces and torques of the first are scaled by 1e-6, so its right-hand side is negligible in the
    norm of the whole batch."""
    parts = [suspensions.random_ellipsoids(k, 6, 12, 0.08, 0.2, seed=50 + q) for q, k in enumerate((2, 5, 9), 1)]
    parts[0].F = parts[0].F * 1e-6
    parts[0].T = parts[0].T * 1e-6
    for q, s in enumerate(parts):
        s.suspension_id[:] = q
    cat = lambda f: np.concatenate([getattr(x, f) for x in parts])
    whole = suspensions.Suspension(cat("semi_axes"), cat("p"), cat("nphi"), cat("centres"), cat("quats"), cat("F"),
                                   cat("T"), cat("suspension_id"), "batch_2_5_9")
    return whole, parts


@pytest.fixture(scope="module")
def batch():
    whole, parts = small_batch()
    refs = []
    for s in parts:
        sys_ = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
        v, om, _, _, _ = sys_.solve(s.F, s.T, method="lu")
        refs.append(np.concatenate([v, om], 1))
    return whole, parts, refs


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("graphs", [1, 0])
@pytest.mark.parametrize("prec,tol,bound", [("FP64", 1e-12, 1e-10), ("MIXED", 1e-10, 1e-8)])
def test_each_suspension_meets_its_own_tolerance(rbs, batch, prec, tol, bound, graphs):
    whole, parts, refs = batch
    with rbs.Context(device=0, precision=getattr(rbs, "RBS_PREC_" + prec), graphs=graphs) as ctx:
        ctx.set_suspension(whole)
        assert rbs.rbs_suspension_count(ctx.ctx) == 3
        v, om, _, its = rbs.rbs_mobility_solve(ctx.ctx, whole.F, whole.T, tol, per_suspension=True)
        its2, res = rbs.rbs_get_suspension_results(ctx.ctx)
        st = rbs.rbs_get_stats(ctx.ctx)
    assert its.shape == (3,) and (its > 0).all() and (its == its2).all()
    assert (res <= tol).all(), res
    assert st["iterations"] == its.max()
    V = np.concatenate([v, om], 1)
    first = 0
    for s, ref in zip(parts, refs):
        assert rel(V[first:first + s.n], ref) < bound
        first += s.n
    if graphs:
        assert st["kernel_count"][rbs.RBS_KC_GMRES_GRAPH] > 0  # the captured cycle ran


def test_graph_and_host_driven_gmres_agree(rbs, batch):
    """The same kernels launched from the host or replayed from the captured graph: the same answer."""
    whole, _, _ = batch
    out = []
    for graphs in (1, 0):
        with rbs.Context(device=0, precision=rbs.RBS_PREC_FP64, graphs=graphs) as ctx:
            ctx.set_suspension(whole)
            for k in range(2):  # the second solve replays the graph captured during the first
                v, om, mu, its = rbs.rbs_mobility_solve(ctx.ctx, whole.F, whole.T, 1e-12, want_density=True,
                                                        per_suspension=True)
            out.append((np.concatenate([v, om], 1), mu, its))
    assert rel(out[0][0], out[1][0]) < 1e-12
    assert rel(out[0][1], out[1][1]) < 1e-11
    assert (out[0][2] == out[1][2]).all()


def test_one_suspension_batch_matches_single_context(rbs):
    """A batch whose suspensions are copies of one suspension at far-apart places gives each copy the
    single-suspension answer and the same iteration count."""
    s = suspensions.random_ellipsoids(6, 6, 12, 0.08, 0.2, seed=61)
    with rbs.Context(device=0, precision=rbs.RBS_PREC_FP64) as ctx:
        ctx.set_suspension(s)
        v1, om1, _, its1 = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-12)
    k = 3
    cen = np.concatenate([s.centres + 1000.0 * q for q in range(k)])
    sid = np.repeat(np.arange(k, dtype=np.int32), s.n)
    with rbs.Context(device=0, precision=rbs.RBS_PREC_FP64) as ctx:
        ctx.set_geometry(np.tile(s.semi_axes, (k, 1)), np.tile(s.p, k), np.tile(s.nphi, k), cen,
                         np.tile(s.quats, (k, 1)), sid)
        v, om, _, its = rbs.rbs_mobility_solve(ctx.ctx, np.tile(s.F, (k, 1)), np.tile(s.T, (k, 1)), 1e-12,
                                               per_suspension=True)
    V1 = np.concatenate([v1, om1], 1)
    V = np.concatenate([v, om], 1)
    for q in range(k):
        assert rel(V[q * s.n:(q + 1) * s.n], V1) < 1e-11
    # the copies' pair sums are split differently over the GPU, so rounding may differ slightly
    assert (np.abs(its - its1) <= 1).all()
