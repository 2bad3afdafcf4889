"""Parity of the magnetostatic coupling (Section 4.1.3) with the oracle: the Laplace operators K^L and
S^L on scalar node fields (smooth, near and singular rules), the single-layer density q, and the net
magnetic forces and torques; the sphere's closed form and the ellipsoid's demagnetisation torque on the
GPU; and one Euler step of two paramagnetic spheres against the oracle.  Tolerances: operators 1e-11
(relative L2; the smooth sums run in double-float arithmetic), q and the forces 1e-10 (GMRES to
1e-13)."""
import math

import numpy as np
import pytest

import oracle
from oracle import magnetic as om
from test_gpu_parity import rel
from test_oracle_magnetic import three_ellipsoids

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    import torch
    assert torch.cuda.is_available()
    return m


@pytest.fixture(scope="module")
def trio(rbs):
    axes, cen, q = three_ellipsoids()
    s = oracle.System(axes, 6, 12, cen, q)
    assert len(s.near) > 0
    ctx = rbs.Context(device=0).set_geometry(axes, 6, 12, cen, q)
    yield s, om.Magnetic(s), ctx
    ctx.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_laplace_operators_match_oracle(rbs, trio, kind):
    s, m, ctx = trio
    x = np.random.default_rng(3).normal(size=s.total_nodes)
    y = rbs.rbs_apply_laplace(ctx.ctx, kind, x)
    assert rel(y, m.assemble("KS"[kind]) @ x) < 1e-11


def test_magnetic_forces_match_oracle(rbs, trio):
    s, m, ctx = trio
    H0 = np.array([0.2, 0.7, -0.4])
    Fr, Tr, qr = m.forces(H0, 3.0)
    F, T, q, its = rbs.rbs_magnetic_forces(ctx.ctx, H0, 3.0, 1e-13, len(s.particles), s.total_nodes)
    assert rel(q, qr) < 1e-10
    assert rel(np.concatenate([F, T]), np.concatenate([Fr, Tr])) < 1e-10
    assert 0 < its < 60


def test_sphere_and_ellipsoid_closed_forms(rbs):
    H0 = np.array([0.3, -0.5, 0.8])
    mr = 2.0
    beta = (mr - 1) / (mr + 2)
    with rbs.Context(device=0) as ctx:
        ctx.set_geometry([[1, 1, 1]], 8, 16, [[0.5, -0.2, 0.1]], [[0.9, 0.1, 0.3, -0.2]])
        F, T, q, _ = rbs.rbs_magnetic_forces(ctx.ctx, H0, mr, 1e-13, 1, 9 * 16)
        _, n, _ = rbs.rbs_get_surface(ctx.ctx)
    assert np.abs(q - 3 * beta * n @ H0).max() < 1e-12
    assert np.abs(F).max() < 1e-12 and np.abs(T).max() < 1e-12
    axes = (1.3, 0.8, 0.6)
    with rbs.Context(device=0) as ctx:
        ctx.set_geometry([axes], 12, 24, [[0, 0, 0]], [[1, 0, 0, 0]])
        F, T, _, _ = rbs.rbs_magnetic_forces(ctx.ctx, H0, mr, 1e-13, 1)
    chi = mr - 1
    M = chi * H0 / (1 + chi * om.demagnetization_factors(axes))
    Tc = 4.0 / 3.0 * math.pi * np.prod(axes) * np.cross(M, H0)
    assert np.abs(T[0] - Tc).max() < 1e-5 * np.abs(Tc).max() and np.abs(F).max() < 1e-11


def test_euler_step_of_paramagnetic_spheres(rbs):
    """Two spheres along the field attract; one explicit Euler step with magnetic forces added to the
    applied ones matches the oracle's forces, mobility solve and update."""
    H0 = np.array([0.0, 0.0, 2.0])
    mr, dt = 2.0, 0.1
    cen = np.array([[0.0, 0.0, 0.0], [0.3, 0.0, 3.0]])
    quats = np.tile([1.0, 0, 0, 0], (2, 1))
    s = oracle.System([[1, 1, 1]] * 2, 6, 12, cen, quats)
    Fm, Tm, _ = om.Magnetic(s).forces(H0, mr)
    v, om_, *_ = s.solve(Fm, Tm)
    with rbs.Context(device=0, magnetic_field=(0.0, 0.0, 2.0), mu_ratio=mr) as ctx:
        ctx.set_geometry([[1, 1, 1]] * 2, 6, 12, cen, quats)
        rbs.rbs_advance(ctx.ctx, np.zeros((2, 3)), np.zeros((2, 3)), dt, 1, rbs.RBS_RK_EULER, 1e-13)
        c1, _ = rbs.rbs_get_state(ctx.ctx, 2)
    assert np.abs(c1 - (cen + dt * v)).max() < 1e-10 * np.abs(dt * v).max() + 1e-14
    assert (c1[1, 2] - c1[0, 2]) < 3.0  # attraction along the field
