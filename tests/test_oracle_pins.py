"""Pins of the float64 oracle against facts fixed outside it: library quadrature and special
functions, closed forms (Stokes' law for a sphere, the Oberbeck / Jeffery resistance of an ellipsoid,
the single-layer and traction operators of a sphere on uniform and rotational data), exact identities
of the formulation (Eqs. 14, 17, 20), symmetry and definiteness of the mobility matrix, exact rigid
motion covariance, spectral convergence, and the far-field two-sphere interaction."""
import math

import numpy as np
import pytest
import scipy.special as sps
from scipy.integrate import quad

import oracle
from oracle import operators as ops
from oracle import sphere_grid as sg
from oracle.geometry import body_surface, ellipsoid_jacobian, quat_to_rot


def random_rotation(seed):
    q = np.random.default_rng(seed).normal(size=4)
    return q / np.linalg.norm(q)


# -------------------------------------------------------------------------------- grid, transforms

@pytest.mark.parametrize("n", [1, 2, 5, 9, 13, 25, 33])
def test_gauss_legendre_matches_library_and_is_exact(n):
    t, lam = sg.gauss_legendre(n)
    tr, lr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(t, tr, atol=1e-14) and np.allclose(lam, lr, atol=1e-14)
    for deg in range(2 * n):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.sum(lam * t ** deg) - exact) < 1e-13


def test_normalised_legendre_matches_scipy():
    p = 12
    t = np.linspace(-0.97, 0.99, 11)
    P = sg.legendre_normalized(p, t)
    for n in range(p + 1):
        for m in range(n + 1):
            ref = sps.lpmv(m, n, t) * (-1.0) ** m  # drop the Condon-Shortley sign
            ref *= math.sqrt((2 * n + 1) / (4 * math.pi) * math.factorial(n - m) / math.factorial(n + m))
            assert np.allclose(P[n, m], ref, rtol=1e-11, atol=1e-13), (n, m)


@pytest.mark.parametrize("p,nphi", [(4, 8), (6, 14), (8, 16), (10, 22)])
def test_transform_is_exact_on_retained_space(p, nphi):
    """Analysis after synthesis is the identity (the grid rule integrates products exactly), and
    interpolation reproduces retained-space functions at arbitrary points."""
    th, ph, _ = sg.grid_points(p, nphi)
    Y = sg.real_sh(p, sg.mmax_for(nphi), th, ph)
    An = sg.analysis_matrix(p, nphi)
    assert np.allclose(An @ Y.T, np.eye(Y.shape[0]), atol=1e-12)
    rng = np.random.default_rng(0)
    coef = rng.normal(size=Y.shape[0])
    pts_th = np.arccos(rng.uniform(-1, 1, 40))
    pts_ph = rng.uniform(0, 2 * math.pi, 40)
    f_grid = coef @ Y
    f_pts = coef @ sg.real_sh(p, sg.mmax_for(nphi), pts_th, pts_ph)
    assert np.allclose(sg.interpolation_matrix(p, nphi, pts_th, pts_ph) @ f_grid, f_pts, atol=1e-12)


# -------------------------------------------------------------------------------- geometry

def ellipsoid_area(a, b, c):
    """Closed form (Legendre incomplete elliptic integrals), a >= b >= c."""
    a, b, c = sorted((a, b, c), reverse=True)
    if a == c:
        return 4 * math.pi * a * a
    phi = math.acos(c / a)
    m = (a * a * (b * b - c * c)) / (b * b * (a * a - c * c))
    return 2 * math.pi * c * c + 2 * math.pi * a * b / math.sin(phi) * (
        sps.ellipeinc(phi, m) * math.sin(phi) ** 2 + sps.ellipkinc(phi, m) * math.cos(phi) ** 2)


def test_sphere_area_and_moment_exact():
    a = 1.3
    b = body_surface([a, a, a], 6, 12)
    assert abs(b.area - 4 * math.pi * a * a) < 1e-12
    tau = oracle.System([[a, a, a]], 6, 12, [[0, 0, 0]], [[1, 0, 0, 0]]).particles[0].tau
    assert np.allclose(tau, 8 * math.pi * a ** 4 / 3 * np.eye(3), atol=1e-12)


def test_ellipsoid_area_converges_spectrally():
    axes = (1.4, 0.9, 0.6)
    exact = ellipsoid_area(*axes)
    errs = [abs(body_surface(axes, p, 2 * p).area - exact) for p in (4, 8, 16, 32)]
    assert errs[3] < 1e-12 and errs[1] < errs[0] * 1e-2 and errs[2] < errs[1] * 1e-3


def test_normals_weights_and_area_element():
    axes = np.array([1.2, 0.7, 0.9])
    b = body_surface(axes, 10, 22)
    assert np.allclose(np.linalg.norm(b.normal, axis=1), 1.0, atol=1e-14)
    # divergence theorem: the closed surface integral of n vanishes; the centroid is the centre
    assert np.allclose((b.w[:, None] * b.normal).sum(0), 0.0, atol=1e-13)
    assert np.allclose((b.w[:, None] * b.x).sum(0), 0.0, atol=1e-13)
    # W of Eq. 36 equals (area per solid angle) x sin(theta); normal is the gradient direction
    s = b.x / axes[None, :]
    assert np.allclose(b.W, ellipsoid_jacobian(axes, s) * np.sin(b.theta), rtol=1e-13)
    g = b.x / axes[None, :] ** 2
    assert np.allclose(b.normal, g / np.linalg.norm(g, axis=1, keepdims=True), atol=1e-14)
    # volume by the divergence theorem: (1/3) int x . n dS = 4 pi abc / 3
    vol = (b.w * np.einsum("ij,ij->i", b.x, b.normal)).sum() / 3
    assert abs(vol - 4 * math.pi * axes.prod() / 3) < 1e-9


def test_quaternion_rotation_is_orthonormal_and_matches_axis_angle():
    q = random_rotation(3)
    R = quat_to_rot(q)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-15) and abs(np.linalg.det(R) - 1) < 1e-14
    ang = 0.7
    axis = np.array([1.0, 2.0, -0.5]) / np.linalg.norm([1.0, 2.0, -0.5])
    qa = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    Rod = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
    assert np.allclose(quat_to_rot(qa), Rod, atol=1e-15)


def test_incident_density_reproduces_force_and_torque():
    """Eq. 17: the discrete rho of Eq. 19 carries exactly F_i and T_i."""
    rng = np.random.default_rng(1)
    s = oracle.System([[1.2, 0.7, 0.9], [0.8, 0.8, 1.3]], [6, 8], [12, 18],
                      [[0, 0, 0], [4, 1, 0]], [random_rotation(1), random_rotation(2)])
    F, T = rng.normal(size=(2, 3)), rng.normal(size=(2, 3))
    rho = s.incident_density(F, T)
    for i, pt in enumerate(s.particles):
        r = rho[s.sl(i)]
        assert np.allclose((pt.w[:, None] * r).sum(0), F[i], atol=1e-13)
        assert np.allclose((pt.w[:, None] * np.cross(pt.r, r)).sum(0), T[i], atol=1e-13)


# -------------------------------------------------------------------------------- operators

def test_sphere_self_operators_on_rigid_tractions():
    """Closed forms on a sphere of radius a: S[c] = (2a/3) c and K[c] = -c/2 for a constant c
    (the traction of translation), S[w x n] = (a/3) w x n and K[w x n] = -(w x n)/2 (rotation);
    so 1/2 I + K annihilates rigid-motion tractions."""
    a, p = 1.5, 8
    body = body_surface([a, a, a], p, 2 * p)
    S = ops.self_block("S", body, 2 * p)
    K = ops.self_block("K", body, 2 * p)
    c = np.array([0.3, -1.1, 0.7])
    const = np.tile(c, (len(body.w), 1)).reshape(-1)
    rot = np.cross(c[None, :], body.normal).reshape(-1)
    assert np.allclose(S @ const, 2 * a / 3 * const, atol=1e-12)
    assert np.allclose(K @ const, -0.5 * const, atol=1e-12)
    assert np.allclose(S @ rot, a / 3 * rot, atol=1e-12)
    assert np.allclose(K @ rot, -0.5 * rot, atol=1e-12)


@pytest.mark.slow
def test_interior_traction_has_no_net_force_or_torque():
    """Eq. 14: for any mu the interior traction 1/2 mu + K mu integrates to zero force and torque on
    each particle (self, near and far blocks alike), to discretisation error."""
    s = oracle.System([[1.2, 0.7, 0.9], [0.8, 0.8, 1.3], [1.0, 0.6, 0.6]], 10, 20,
                      [[0, 0, 0], [2.9, 0.3, 0.1], [9, 0, 0]],
                      [random_rotation(4), random_rotation(5), random_rotation(6)])
    assert (0, 1) in s.near and (0, 2) not in s.near
    ths = np.repeat(sg.grid_angles(10, 20)[0], 20)
    phs = np.tile(sg.grid_angles(10, 20)[1], 11)
    # a smooth density: low-degree harmonics per component
    mu = np.concatenate([np.stack([np.cos(ths) + 0.3 * np.sin(ths) * np.cos(phs + i),
                                   np.sin(ths) * np.sin(2 * phs), 0.5 + np.cos(ths) ** 2 * (i + 1)], 1)
                         for i in range(3)])
    y = s.apply("K", mu, half=0.5)
    for i, pt in enumerate(s.particles):
        f = y[s.sl(i)]
        scale = np.abs(pt.w[:, None] * mu[s.sl(i)]).sum()
        assert np.abs((pt.w[:, None] * f).sum(0)).max() < 1e-6 * scale
        assert np.abs((pt.w[:, None] * np.cross(pt.r, f)).sum(0)).max() < 1e-6 * scale


def test_self_rule_converges_in_rule_order():
    body = body_surface([1.3, 0.7, 0.9], 8, 16)
    t = [0, 40, 77, 143]
    for kind in ("S", "K"):
        ref = ops.self_rows(kind, body, t, 48)
        e16 = np.abs(ops.self_rows(kind, body, t, 16) - ref).max() / np.abs(ref).max()
        e24 = np.abs(ops.self_rows(kind, body, t, 24) - ref).max() / np.abs(ref).max()
        assert e16 < 1e-5 and e24 < 1e-8 and e24 < e16 * 1e-2, kind


def test_near_rule_converges_with_upsampling():
    s = oracle.System([[1.2, 0.7, 0.9], [0.8, 0.8, 1.3]], 8, 16, [[0, 0, 0], [2.6, 0.2, 0.1]],
                      [random_rotation(7), random_rotation(8)])
    pi, pj = s.particles
    b2 = ops.near_block("K", pi, pj, 16)
    b4 = ops.near_block("K", pi, pj, 32)
    b8 = ops.near_block("K", pi, pj, 48)
    e2 = np.abs(b2 - b8).max()
    e4 = np.abs(b4 - b8).max()
    assert e4 < e2 * 0.1 and e4 < 1e-4 * np.abs(b8).max()


def test_self_block_rotation_covariance():
    """Eq. 38: the singular rule computed on the rotated surface equals R A R^T."""
    body = body_surface([1.3, 0.7, 0.9], 6, 12)
    A = ops.self_block("K", body, 12)
    R = quat_to_rot(random_rotation(9))
    Ar = ops.rotate_block(A, R)
    # apply to a field: rotating the field, applying, rotating back equals applying A directly
    f = np.random.default_rng(2).normal(size=(len(body.w), 3))
    lhs = (Ar @ (f @ R.T).reshape(-1)).reshape(-1, 3) @ R
    assert np.allclose(lhs, (A @ f.reshape(-1)).reshape(-1, 3), atol=1e-13)


# -------------------------------------------------------------------------------- the whole solve

@pytest.mark.parametrize("a", [1.0, 0.7])
def test_single_sphere_stokes_law(a):
    """v = F / (6 pi mu a), omega = T / (8 pi mu a^3), and mu = 0."""
    s = oracle.System([[a, a, a]], 8, 16, [[1, 2, 3]], [random_rotation(11)])
    F = np.array([[1.0, -0.5, 0.3]])
    T = np.array([[0.2, 0.7, -1.1]])
    v, om, mu, _, _ = s.solve(F, T)
    assert np.allclose(v, F / (6 * math.pi * a), atol=1e-14)
    assert np.allclose(om, T / (8 * math.pi * a ** 3), atol=1e-14)
    assert np.abs(mu).max() < 1e-13


def oberbeck(axes):
    """Translational and rotational mobilities of an ellipsoid along / about its axes (Oberbeck,
    Jeffery; e.g. Kim & Karrila, Microhydrodynamics, ch. 3), mu = 1."""
    a = np.asarray(axes, float)
    D = lambda l: math.sqrt((a[0] ** 2 + l) * (a[1] ** 2 + l) * (a[2] ** 2 + l))
    chi = quad(lambda l: 1 / D(l), 0, np.inf, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    al = [quad(lambda l, s=s: 1 / ((s * s + l) * D(l)), 0, np.inf, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
          for s in a]
    mt = [(chi + a[i] ** 2 * al[i]) / (16 * math.pi) for i in range(3)]
    mr = []
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        mr.append(3 * (a[j] ** 2 * al[j] + a[k] ** 2 * al[k]) / (16 * math.pi * (a[j] ** 2 + a[k] ** 2)))
    return np.array(mt), np.array(mr)


@pytest.mark.slow
def test_single_ellipsoid_matches_oberbeck_jeffery_and_converges():
    axes = np.array([1.0, 0.8, 0.6])
    mt, mr = oberbeck(axes)
    R = quat_to_rot(random_rotation(12))
    errs = []
    for p in (6, 12):
        s = oracle.System([axes], p, 2 * p, [[0.5, -1, 2]], [random_rotation(12)])
        A = s.assemble("K", half=0.5, with_L=True)
        err = 0.0
        for e in range(3):
            for kind in ("F", "T"):
                F = np.zeros((1, 3))
                T = np.zeros((1, 3))
                (F if kind == "F" else T)[0] = R[:, e]        # along the e-th body axis, lab frame
                rho = s.incident_density(F, T)
                mu = np.linalg.solve(A, s.rhs(rho).reshape(-1)).reshape(-1, 3)
                v, om = s.rigid_velocities(s.apply("S", rho + mu))
                got = v[0] if kind == "F" else om[0]
                want = (mt if kind == "F" else mr)[e] * R[:, e]
                err = max(err, np.abs(got - want).max())
        errs.append(err)
    assert errs[1] < 1e-8 and errs[1] < errs[0] * 1e-2


@pytest.mark.slow
def test_solution_satisfies_constraints_and_lu_equals_gmres():
    """Eq. 20 (integral mu = 0, integral r x mu = 0 per particle) holds for the solution of Eq. 25, and
    the dense and iterative solves agree."""
    s = oracle.System([[1.2, 0.7, 0.9], [0.8, 0.8, 1.3], [1.0, 0.6, 0.6]], 8, 16,
                      [[0, 0, 0], [2.9, 0.3, 0.1], [0.5, 3.4, -0.8]],
                      [random_rotation(13), random_rotation(14), random_rotation(15)])
    rng = np.random.default_rng(3)
    F, T = rng.normal(size=(3, 3)), rng.normal(size=(3, 3))
    v1, o1, mu1, _, _ = s.solve(F, T, method="lu")
    v2, o2, mu2, _, its = s.solve(F, T, method="gmres", tol=1e-13)
    assert np.allclose(mu1, mu2, atol=1e-11) and np.allclose(v1, v2, atol=1e-12) and its > 0
    for i, pt in enumerate(s.particles):
        m = mu1[s.sl(i)]
        assert np.abs((pt.w[:, None] * m).sum(0)).max() < 1e-6
        assert np.abs((pt.w[:, None] * np.cross(pt.r, m)).sum(0)).max() < 1e-6


@pytest.mark.slow
def test_mobility_matrix_symmetric_positive_definite():
    """Lorentz reciprocity and dissipation: M = M^T > 0, to discretisation error."""
    s = oracle.System([[1.2, 0.7, 0.9], [0.8, 0.8, 1.3]], 8, 16, [[0, 0, 0], [2.8, 0.6, -0.2]],
                      [random_rotation(16), random_rotation(17)])
    M = s.mobility_matrix()
    assert np.abs(M - M.T).max() < 1e-6 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_rigid_motion_covariance_is_exact():
    """A global rotation Q and shift of the whole configuration rotates (v, omega) by Q exactly, and
    relabelling the particles permutes them."""
    axes = [[1.2, 0.7, 0.9], [0.8, 0.8, 1.3]]
    cen = np.array([[0, 0, 0], [3.0, 0.4, 0.2]])
    qs = [random_rotation(18), random_rotation(19)]
    F = np.array([[1.0, 0.2, -0.3], [0.1, -0.7, 0.4]])
    T = np.array([[0.3, 0.1, 0.2], [-0.2, 0.5, 0.1]])
    s0 = oracle.System(axes, 6, 12, cen, qs)
    v0, o0, *_ = s0.solve(F, T)
    Qq = random_rotation(20)
    Q = quat_to_rot(Qq)

    def qmul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])

    s1 = oracle.System(axes, 6, 12, cen @ Q.T + np.array([5.0, -2, 1]), [qmul(Qq, q) for q in qs])
    v1, o1, *_ = s1.solve(F @ Q.T, T @ Q.T)
    assert np.allclose(v1, v0 @ Q.T, atol=1e-13) and np.allclose(o1, o0 @ Q.T, atol=1e-13)
    s2 = oracle.System(axes[::-1], 6, 12, cen[::-1], qs[::-1])
    v2, o2, *_ = s2.solve(F[::-1], T[::-1])
    assert np.allclose(v2, v0[::-1], atol=1e-13) and np.allclose(o2, o0[::-1], atol=1e-13)


@pytest.mark.slow
def test_two_distant_spheres_approach_rotne_prager():
    """The pair mobility of two unit spheres tends to the Rotne-Prager-Yamakawa tensor
    (1 / 8 pi d) [(1 + 2/(3 d^2)) I + (1 - 2 / d^2) dd], with an error falling like d^-4."""
    devs = []
    for d in (6.0, 12.0):
        s = oracle.System([[1, 1, 1], [1, 1, 1]], 6, 12, [[0, 0, 0], [d, 0, 0]], [[1, 0, 0, 0]] * 2)
        F = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, 0.0]])
        v, *_ = s.solve(F, np.zeros((2, 3)))
        dh = np.array([1.0, 0, 0])
        rpy = ((1 + 2 / (3 * d * d)) * np.eye(3) + (1 - 2 / d ** 2) * np.outer(dh, dh)) / (8 * math.pi * d)
        devs.append(np.abs(v[0] - rpy @ F[1]).max() / np.abs(rpy @ F[1]).max())
    assert devs[1] < devs[0] / 8 and devs[1] < 1e-3


def test_near_list_follows_the_stated_criterion():
    s = oracle.System([[1.0, 0.5, 0.5], [1.4, 1.0, 1.0], [1, 1, 1]], 4, 8,
                      [[0, 0, 0], [3.39, 0, 0], [0, 0, 3.6]], [[1, 0, 0, 0]] * 3)
    # |c0 - c1| = 3.39 < 1 + 1.4 + 1 ; |c0 - c2| = 3.6 > 1 + 1 + 1 ; |c1 - c2| = 4.96 > 3.4
    assert s.near == {(0, 1), (1, 0)}
