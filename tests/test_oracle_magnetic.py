"""Pins of the magnetostatic coupling in the oracle (Section 4.1.3): a sphere in a uniform field
(q = 3 beta H0 . n and the exterior field (1 - beta) H0 + 3 beta (H0 . n) n, beta = (mu - mu0) /
(mu + 2 mu0), no net force or torque), an ellipsoid's torque against the demagnetisation-factor closed
form, two spheres attracting along the field and repelling across it and approaching the point-dipole
force law as they separate, zero net charge on every surface and zero total force, covariance under a
rigid motion of the whole configuration with the field, and no field perturbation when mu = mu0."""
import math

import numpy as np

import oracle
from oracle import magnetic as om
from oracle.timestep import quat_mul


def test_sphere_in_a_uniform_field():
    H0 = np.array([0.3, -0.5, 0.8])
    mr = 2.0
    beta = (mr - 1) / (mr + 2)
    s = oracle.System([[1, 1, 1]], 8, 16, [[0.5, -0.2, 0.1]], [[0.9, 0.1, 0.3, -0.2]])
    m = om.Magnetic(s)
    F, T, q = m.forces(H0, mr)
    n = s.particles[0].normal
    assert np.abs(q - 3 * beta * n @ H0).max() < 1e-13
    H = m.surface_field(H0, q)
    assert np.abs(H - ((1 - beta) * H0 + 3 * beta * (n @ H0)[:, None] * n)).max() < 1e-12
    assert np.abs(F).max() < 1e-13 and np.abs(T).max() < 1e-13


def test_demagnetisation_factors():
    assert np.allclose(om.demagnetization_factors((1.0, 1.0, 1.0)), 1.0 / 3.0, atol=1e-12)
    N = om.demagnetization_factors((1.3, 0.8, 0.6))
    assert abs(N.sum() - 1.0) < 1e-12 and N[0] < N[1] < N[2]


def test_ellipsoid_torque_matches_the_closed_form():
    """A linear magnetic ellipsoid in a uniform field: M_i = chi H0_i / (1 + chi N_i) in the body frame,
    torque mu0 V M x H0, no net force."""
    axes = (1.3, 0.8, 0.6)
    H0 = np.array([0.3, -0.5, 0.8])
    mr = 2.0
    chi = mr - 1.0
    s = oracle.System([axes], 12, 24, [[0, 0, 0]], [[1, 0, 0, 0]])
    F, T, q = om.Magnetic(s).forces(H0, mr)
    M = chi * H0 / (1 + chi * om.demagnetization_factors(axes))
    Tc = 4.0 / 3.0 * math.pi * np.prod(axes) * np.cross(M, H0)
    assert np.abs(T[0] - Tc).max() < 1e-5 * np.abs(Tc).max()
    assert np.abs(F).max() < 1e-12


def test_two_spheres_approach_the_dipole_law():
    mr = 2.0
    beta = (mr - 1) / (mr + 2)
    m = 4 * math.pi * beta
    H0 = np.array([0.0, 0.0, 1.0])
    dev = {}
    for d in (4.0, 10.0):
        for along in (True, False):
            c2 = [0, 0, d] if along else [d, 0, 0]
            s = oracle.System([[1, 1, 1]] * 2, 8, 16, [[0, 0, 0], c2], [[1, 0, 0, 0]] * 2)
            F, _, _ = om.Magnetic(s).forces(H0, mr)
            assert np.abs(F.sum(0)).max() < 1e-12
            if along:
                f, law = F[1, 2], -3 * m * m / (2 * math.pi * d ** 4)      # attraction along the field
            else:
                f, law = F[1, 0], 3 * m * m / (4 * math.pi * d ** 4)       # repulsion across it
            assert np.sign(f) == np.sign(law)
            dev[(d, along)] = abs(f / law - 1)
    for along in (True, False):
        assert dev[(10.0, along)] < 0.1 * dev[(4.0, along)] and dev[(10.0, along)] < 2e-3


def three_ellipsoids():
    rng = np.random.default_rng(8)
    q = rng.normal(size=(3, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    axes = np.array([[1.1, 0.7, 0.8], [0.9, 0.8, 0.6], [0.8, 0.75, 0.7]])
    cen = np.array([[0.0, 0.0, 0.0], [2.4, 0.5, -0.3], [0.4, 2.5, 0.9]])
    return axes, cen, q


def test_charge_neutrality_balance_and_covariance():
    axes, cen, q = three_ellipsoids()
    H0 = np.array([0.2, 0.7, -0.4])
    s = oracle.System(axes, 6, 12, cen, q)
    F, T, qq = om.Magnetic(s).forces(H0, 3.0)
    # both hold exactly for the continuous problem (Gauss's theorem; Newton's third law) and to the
    # quadrature error of the neighbours' near fields here (p = 6)
    for i, pt in enumerate(s.particles):
        assert abs(pt.w @ qq[s.sl(i)]) < 1e-4 * (pt.w @ np.abs(qq[s.sl(i)]))
    assert np.abs(F.sum(0)).max() < 1e-3 * np.abs(F).max()
    Qq = np.array([0.6, -0.2, 0.7, 0.33])
    Qq /= np.linalg.norm(Qq)
    Q = oracle.quat_to_rot(Qq)
    s2 = oracle.System(axes, 6, 12, cen @ Q.T + 0.7, quat_mul(np.tile(Qq, (3, 1)), q))
    F2, T2, _ = om.Magnetic(s2).forces(Q @ H0, 3.0)
    assert np.allclose(F2, F @ Q.T, atol=1e-12) and np.allclose(T2, T @ Q.T, atol=1e-12)


def test_no_perturbation_when_permeabilities_match():
    axes, cen, q = three_ellipsoids()
    s = oracle.System(axes, 6, 12, cen, q)
    F, T, qq = om.Magnetic(s).forces([0.2, 0.7, -0.4], 1.0)
    assert np.abs(qq).max() == 0.0 and np.abs(F).max() < 1e-14 and np.abs(T).max() < 1e-14
