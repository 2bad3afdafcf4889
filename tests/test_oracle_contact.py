"""Pins of the contact force algorithm in the oracle (Section 3.4): the maps C and D are each
other's transpose (written independently), contact forces exert no net force or torque on a pair,
the symmetric part of D M C is positive definite (D M C itself is symmetric only up to the
discretisation's reciprocity error, which near contact is about 10% at p = 6 and 1% at p = 10), the
corrected velocities satisfy the no-slip condition at every contact and equal the mobility of the
total forces, two equal spheres pushed together along their line of centres come to rest, and
particles farther apart than the gap are left alone."""
import numpy as np

import oracle
from oracle import contact as oc


def two_spheres(gap, p=6):
    cen = np.array([[0.0, 0.0, 0.0], [2.0 + gap, 0.0, 0.0]])
    return oracle.System([[1, 1, 1]] * 2, p, 2 * p, cen, np.tile([1.0, 0, 0, 0], (2, 1)))


def three_ellipsoids(p=6):
    """Ellipsoids 0 and 1 nearly touch (a contact at gap 0.1); ellipsoid 2 is near but not in contact."""
    rng = np.random.default_rng(5)
    q = rng.normal(size=(3, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    axes = np.array([[1.0, 0.7, 0.8], [0.9, 0.8, 0.6], [0.8, 0.8, 0.7]])
    cen = np.array([[0.0, 0.0, 0.0], [1.62, 0.35, -0.2], [0.3, 2.2, 0.4]])
    return oracle.System(axes, p, 2 * p, cen, q), rng


def test_maps_are_transposes_and_balance():
    s, _ = three_ellipsoids()
    cts = oc.find_contacts(s, 0.1)
    assert len(cts) >= 1
    C = oc.contact_map(s, cts)
    D = oc.velocity_difference_map(s, cts)
    assert np.abs(D - C.T).max() < 1e-15
    cen = np.array([pt.centre for pt in s.particles])
    for col in range(C.shape[1]):
        FT = C[:, col].reshape(-1, 6)
        assert np.abs(FT[:, :3].sum(0)).max() < 1e-14                          # no net force
        torque = FT[:, 3:] + np.cross(cen, FT[:, :3])                          # about the origin
        assert np.abs(torque.sum(0)).max() < 1e-13                              # no net torque


def test_contact_system_is_spd_and_enforces_no_slip():
    s, rng = three_ellipsoids()
    F, T = rng.normal(size=(2, 3, 3))
    v, om, mu, cts, Fc = oc.solve_with_contacts(s, F, T, 0.1)
    assert [(i, j) for i, j, _ in cts] == [(0, 1)]
    C = oc.contact_map(s, cts)
    M = s.mobility_matrix()
    DMC = C.T @ M @ C
    assert np.linalg.eigvalsh(0.5 * (DMC + DMC.T)).min() > 0
    V = np.concatenate([v, om], 1).reshape(-1)
    assert np.abs(oc.velocity_difference_map(s, cts) @ V).max() < 1e-12 * np.abs(V).max()
    # the corrected motion is the mobility of the total forces F + C F_c
    FT = np.concatenate([F, T], 1).reshape(-1) + C @ Fc.reshape(-1)
    assert np.allclose(V, M @ FT, atol=1e-12)


def test_equal_spheres_pushed_together_come_to_rest():
    s = two_spheres(0.03)
    F = np.array([[1.0, 0, 0], [-1.0, 0, 0]])
    v0, om0, *_ = s.solve(F, np.zeros((2, 3)))
    assert v0[0, 0] > 1e-3                                                     # they would approach
    v, om, mu, cts, Fc = oc.solve_with_contacts(s, F, np.zeros((2, 3)), 0.05)
    assert len(cts) == 1 and np.allclose(cts[0][2], [1.015, 0, 0], atol=1e-14)
    assert np.abs(v).max() < 1e-12 and np.abs(om).max() < 1e-12
    assert np.allclose(Fc[0], [-1.0, 0, 0], atol=1e-10)                        # the contact force cancels F


def test_no_contact_beyond_the_gap():
    s = two_spheres(0.2)
    F = np.array([[1.0, 0.3, 0], [-1.0, 0, 0.2]])
    T = np.array([[0.1, 0, 0], [0, 0.2, 0]])
    v, om, mu, cts, Fc = oc.solve_with_contacts(s, F, T, 0.1)
    v0, om0, mu0, _, _ = s.solve(F, T)
    assert cts == [] and np.array_equal(v, v0) and np.array_equal(mu, mu0)

