"""Pins of general coefficient surfaces in the oracle (Section 3, Eqs. 31, 36, 37): an ellipsoid given
by its degree-1 coefficients reproduces the analytic ellipsoid path, a non-ellipsoidal shape obeys the
identities of the formulation (divergence theorem, Eq. 14, Eq. 17, Eq. 20, reciprocity, rigid-motion
covariance), and its mobility converges spectrally in p."""
import numpy as np
import pytest

import oracle
from oracle import shapes as shp
from oracle.geometry import body_surface_sh
from oracle.timestep import quat_mul
from shape_inputs import star_shape


def _peanut(pg=4, seed=0):
    return star_shape(seed, pg)


def test_coefficient_ellipsoid_reproduces_the_analytic_one():
    axes = (1.3, 0.7, 0.9)
    coef, pg = shp.sh_coefficients_of_ellipsoid(axes)
    F = np.array([[0.4, -0.3, 1.0]])
    T = np.array([[0.2, 0.5, -0.1]])
    q = [[0.9, 0.2, -0.3, 0.1]]
    a = oracle.System([axes], 8, 16, [[1, 2, 3]], q)
    b = oracle.System(None, 8, 16, [[1, 2, 3]], q, shapes=[(coef, pg)], shape_of=[0])
    va, oa, ma, _, _ = a.solve(F, T)
    vb, ob, mb, _, _ = b.solve(F, T)
    assert np.abs(va - vb).max() < 1e-13 and np.abs(oa - ob).max() < 1e-13 and np.abs(ma - mb).max() < 1e-12


def test_surface_identities_of_a_general_shape():
    coef, pg = _peanut()
    b = body_surface_sh(coef, pg, 16, 32, 32)
    assert np.allclose((b.w[:, None] * b.normal).sum(0), 0.0, atol=1e-12)
    assert np.allclose((b.w[:, None] * b.x).sum(0), 0.0, atol=1e-12)       # centred at the area centroid
    assert np.allclose(np.linalg.norm(b.normal, axis=1), 1.0, atol=1e-14)
    vol16 = (b.w * np.einsum("ij,ij->i", b.x, b.normal)).sum() / 3
    b32 = body_surface_sh(coef, pg, 32, 64, 32)
    vol32 = (b32.w * np.einsum("ij,ij->i", b32.x, b32.normal)).sum() / 3
    assert abs(vol16 - vol32) < 1e-10 * vol32
    # the evaluator agrees with the grid nodes and normals
    s = np.stack([np.sin(b.theta) * np.cos(b.phi), np.sin(b.theta) * np.sin(b.phi), np.cos(b.theta)], 1)
    x, J, n = b.shape.evaluate(s)
    assert np.abs(x - b.x).max() < 1e-13 and np.abs(n - b.normal).max() < 1e-12
    assert np.allclose(J * np.sin(b.theta), b.W, rtol=1e-12)


@pytest.mark.slow
def test_formulation_identities_on_general_shapes():
    c1, pg = _peanut(seed=1)
    c2, _ = _peanut(seed=2)
    s = oracle.System(None, 8, 16, [[0, 0, 0], [3.0, 0.4, 0.2]], [[1, 0, 0, 0], [0.8, 0.3, -0.2, 0.46]],
                      shapes=[(c1, pg), (c2, pg)], shape_of=[0, 1])
    rng = np.random.default_rng(3)
    F, T = rng.normal(size=(2, 3)), rng.normal(size=(2, 3))
    rho = s.incident_density(F, T)
    # a smooth density: rho plus a low-degree field of the body-frame coordinates
    mu_s = rho + np.concatenate([0.3 * pt.r[:, [1, 2, 0]] ** 2 for pt in s.particles])
    y = s.apply("K", mu_s, half=0.5)
    for i, pt in enumerate(s.particles):
        sl = s.sl(i)
        assert np.allclose((pt.w[:, None] * rho[sl]).sum(0), F[i], atol=1e-12)                  # Eq. 17
        assert np.allclose((pt.w[:, None] * np.cross(pt.r, rho[sl])).sum(0), T[i], atol=1e-12)
        scale = np.abs(pt.w[:, None] * mu_s[sl]).sum()
        assert np.abs((pt.w[:, None] * y[sl]).sum(0)).max() < 1e-4 * scale                       # Eq. 14
    M = s.mobility_matrix()
    assert np.abs(M - M.T).max() < 1e-4 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    # rigid-motion covariance
    Qq = np.array([0.6, -0.2, 0.7, 0.33])
    Qq /= np.linalg.norm(Qq)
    Q = oracle.quat_to_rot(Qq)
    cen = np.array([[0, 0, 0], [3.0, 0.4, 0.2]])
    qs = np.array([[1, 0, 0, 0], [0.8, 0.3, -0.2, 0.46]])
    s2 = oracle.System(None, 8, 16, cen @ Q.T + 1.0, quat_mul(np.tile(Qq, (2, 1)), qs),
                       shapes=[(c1, pg), (c2, pg)], shape_of=[0, 1])
    v0, o0, *_ = s.solve(F, T)
    v1, o1, *_ = s2.solve(F @ Q.T, T @ Q.T)
    assert np.allclose(v1, v0 @ Q.T, atol=1e-12) and np.allclose(o1, o0 @ Q.T, atol=1e-12)


@pytest.mark.slow
def test_general_shape_mobility_converges_spectrally():
    coef, pg = _peanut(seed=4)
    F = np.array([[0.3, -0.2, 1.0]])
    T = np.array([[0.5, 0.1, -0.4]])
    res = []
    for p in (6, 10, 16):
        s = oracle.System(None, p, 2 * p, [[0, 0, 0]], [[1, 0, 0, 0]], shapes=[(coef, pg)], shape_of=[0])
        v, om, *_ = s.solve(F, T)
        res.append(np.concatenate([v.ravel(), om.ravel()]))
    e1 = np.abs(res[0] - res[2]).max()
    e2 = np.abs(res[1] - res[2]).max()
    assert e2 < 0.05 * e1 and e2 < 1e-5
