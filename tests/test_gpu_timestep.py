"""Parity of rbs_advance (Section 3.3 rigid-body time stepping on the GPU) with the oracle's stepper
on identical inputs.  Tolerances: float64 path 1e-10 on centres and quaternions after several steps
(each stage's velocities agree to ~1e-12 and errors grow mildly over the steps); mixed path 1e-8."""
import math

import numpy as np
import pytest

import oracle.timestep as ots
import suspensions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    return m


def three_ellipsoids():
    s = suspensions.random_ellipsoids(3, 5, 10, 0.06, 0.4, seed=51)
    s.F = np.array([[0.0, 0.0, -1.0], [0.3, 0.0, -1.0], [0.0, -0.2, -0.8]])
    s.T = np.array([[0.2, 0.0, 0.0], [0.0, 0.1, 0.0], [0.0, 0.0, -0.3]])
    return s


@pytest.mark.parametrize("scheme,steps", [("rk4", 3), ("trapezoid", 2), ("euler", 2)])
def test_advance_matches_oracle_float64(rbs, scheme, steps):
    s = three_ellipsoids()
    dt = 0.25
    c_ref, q_ref = ots.advance(s.semi_axes, s.p, s.nphi, s.centres, s.quats, s.F, s.T, dt, steps, scheme)
    code = {"rk4": rbs.RBS_RK4, "trapezoid": rbs.RBS_RK_TRAPEZOID, "euler": rbs.RBS_RK_EULER}[scheme]
    with rbs.Context(device=0) as ctx:
        ctx.set_suspension(s)
        its = rbs.rbs_advance(ctx.ctx, s.F, s.T, dt, steps, code, 1e-13)
        c, q = rbs.rbs_get_state(ctx.ctx, s.n)
    assert its > 0
    assert np.abs(c - c_ref).max() < 1e-10
    assert np.abs(q - q_ref).max() < 1e-10
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-14)


def test_advance_mixed_precision_matches_oracle(rbs):
    s = three_ellipsoids()
    c_ref, q_ref = ots.advance(s.semi_axes, s.p, s.nphi, s.centres, s.quats, s.F, s.T, 0.25, 2, "rk4")
    with rbs.Context(device=0, precision=rbs.RBS_PREC_MIXED) as ctx:
        ctx.set_suspension(s)
        rbs.rbs_advance(ctx.ctx, s.F, s.T, 0.25, 2, rbs.RBS_RK4, 1e-11)
        c, q = rbs.rbs_get_state(ctx.ctx, s.n)
    assert np.abs(c - c_ref).max() < 1e-8 and np.abs(q - q_ref).max() < 1e-8


def test_single_sphere_moves_exactly_on_gpu(rbs):
    a = 1.2
    F = np.array([[0.4, -0.2, 0.9]])
    T = np.array([[0.0, 0.0, 3.0]])
    with rbs.Context(device=0) as ctx:
        ctx.set_geometry([[a, a, a]], 6, 12, [[0.0, 0.0, 0.0]], [[1.0, 0, 0, 0]])
        rbs.rbs_advance(ctx.ctx, F, T, 0.1, 10, rbs.RBS_RK4, 1e-12)
        c, q = rbs.rbs_get_state(ctx.ctx, 1)
    assert np.allclose(c, F / (6 * math.pi * a), atol=1e-13)
    wz = 3.0 / (8 * math.pi * a ** 3)
    assert np.abs(q - np.array([[math.cos(wz / 2), 0, 0, math.sin(wz / 2)]])).max() < 1e-9
