"""Oracle: particle surfaces, quadrature weights and moments (Section 3, Eqs. 31-37; Section 2.2,
Eq. 18; Section 3.3, Eq. 40).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Surfaces are ellipsoids with semi-axes (a, b, c) in the body frame, x_b = (a sin t cos f,
b sin t sin f, c cos t), whose coordinate functions are spherical harmonics of degree 1 (so the
spectral derivatives of Eq. 37 are the analytic ones used below), or general coefficient surfaces
(oracle/shapes.py).  The lab frame is x = c_i + R(q_i) x_b (Eq. 40 with the body frame as reference);
the centroid x^c_i of Eq. 18 is the ellipsoid centre, or the area centroid of a coefficient surface.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .sphere_grid import grid_angles


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of a unit quaternion q = (w, x, y, z) (normalised here); shape (..., 3, 3)."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


@dataclasses.dataclass
class BodySurface:
    """One particle surface on its (p + 1) x n_phi grid, in its body frame."""
    axes: np.ndarray     # (3,) semi-axes of an ellipsoid; for a coefficient shape its bounding radius x3
    p: int
    nphi: int
    x: np.ndarray        # (N_p, 3) nodes
    normal: np.ndarray   # (N_p, 3) outward unit normals
    w: np.ndarray        # (N_p,) quadrature weights of Eq. 35
    W: np.ndarray        # (N_p,) area element of Eq. 36
    theta: np.ndarray    # (N_p,) parameter angles of the nodes
    phi: np.ndarray
    shape: object = None  # SHShape for coefficient surfaces, None for ellipsoids
    radius: float = 0.0   # bounding radius for the near criterion

    @property
    def area(self) -> float:
        return float(self.w.sum())

    def point(self, s):
        return ellipsoid_point(self.axes, s) if self.shape is None else self.shape.point(s)

    def jacobian(self, s):
        return ellipsoid_jacobian(self.axes, s) if self.shape is None else self.shape.jacobian(s)

    def normal_at(self, s):
        return ellipsoid_normal(self.axes, s) if self.shape is None else self.shape.normal(s)


def ellipsoid_point(axes: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Body-frame surface point x_b = diag(a, b, c) s of the parameter-sphere point s (unit vector)."""
    return s * np.asarray(axes)[None, :]


def ellipsoid_jacobian(axes: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Area of the surface per unit solid angle of the parameter sphere at s, i.e. W / sin(theta)
    of Eq. 36; for x = D s it is |cof(D) s| = |(bc s_x, ac s_y, ab s_z)|.  Defined at the poles too."""
    a, b, c = axes
    return np.sqrt((b * c * s[..., 0]) ** 2 + (a * c * s[..., 1]) ** 2 + (a * b * s[..., 2]) ** 2)


def ellipsoid_normal(axes: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Outward unit normal at x = D s: proportional to D^{-1} s."""
    g = s / np.asarray(axes)[None, :]
    return g / np.linalg.norm(g, axis=-1, keepdims=True)


def body_surface(axes, p: int, nphi: int) -> BodySurface:
    """Nodes (Eq. 33), tangent vectors (analytic = spectral, Eq. 37), area element W (Eq. 36),
    normal x_theta x x_phi / W and weights w_jk = 2 pi lambda_j W_jk / (n_phi sin theta_j) (Eq. 35)."""
    axes = np.asarray(axes, dtype=np.float64)
    a, b, c = axes
    theta, phi, _, lam = grid_angles(p, nphi)
    th = np.repeat(theta, nphi)
    ph = np.tile(phi, p + 1)
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    x = np.stack([a * st * cp, b * st * sp, c * ct], axis=1)
    x_th = np.stack([a * ct * cp, b * ct * sp, -c * st], axis=1)
    x_ph = np.stack([-a * st * sp, b * st * cp, np.zeros_like(st)], axis=1)
    E = np.einsum("ij,ij->i", x_th, x_th)
    G = np.einsum("ij,ij->i", x_ph, x_ph)
    Fm = np.einsum("ij,ij->i", x_th, x_ph)
    W = np.sqrt(E * G - Fm * Fm)
    normal = np.cross(x_th, x_ph) / W[:, None]
    w = 2.0 * math.pi * np.repeat(lam, nphi) * W / (nphi * st)
    return BodySurface(axes, p, nphi, x, normal, w, W, th, ph, None, float(np.max(axes)))


def body_surface_sh(coef, pg: int, p: int, nphi: int, p_up: int) -> BodySurface:
    """A coefficient surface (Eq. 31) on its grid: tangents by spectral differentiation (Eq. 37), W of
    Eq. 36, weights of Eq. 35; the body frame is moved to the area centroid, and the bounding radius is
    the largest centroid distance over the nodes of the order-p_up grid."""
    from .shapes import SHShape, basis_with_derivatives
    from .sphere_grid import grid_points
    shape = SHShape(coef, pg)
    theta, phi, _, lam = grid_angles(p, nphi)
    th = np.repeat(theta, nphi)
    ph = np.tile(phi, p + 1)
    Y, Yt, Yp = basis_with_derivatives(pg, th, ph)
    x = (shape.coef @ Y).T
    x_th = (shape.coef @ Yt).T
    x_ph = (shape.coef @ Yp).T * np.sin(th)[:, None]
    E = np.einsum("ij,ij->i", x_th, x_th)
    G = np.einsum("ij,ij->i", x_ph, x_ph)
    Fm = np.einsum("ij,ij->i", x_th, x_ph)
    W = np.sqrt(E * G - Fm * Fm)
    normal = np.cross(x_th, x_ph) / W[:, None]
    w = 2.0 * math.pi * np.repeat(lam, nphi) * W / (nphi * np.sin(th))
    centroid = (w[:, None] * x).sum(0) / w.sum()
    shape.shift = centroid
    x = x - centroid
    nphi_up = nphi + 2 * (p_up - p)
    thu, phu, _ = grid_points(p_up, nphi_up)
    su = np.stack([np.sin(thu) * np.cos(phu), np.sin(thu) * np.sin(phu), np.cos(thu)], axis=1)
    radius = float(np.linalg.norm(shape.point(su), axis=1).max())
    return BodySurface(np.full(3, radius), p, nphi, x, normal, w, W, th, ph, shape, radius)


def moment_tensor(r: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Eq. 18: tau = sum_s w_s (|r_s|^2 I - r_s r_s^T), r measured from the centroid."""
    rr = np.einsum("s,s->", w, np.einsum("si,si->s", r, r))
    return rr * np.eye(3) - np.einsum("s,si,sj->ij", w, r, r)


@dataclasses.dataclass
class Particle:
    """One particle in the lab frame."""
    index: int
    body: BodySurface
    centre: np.ndarray   # (3,)
    R: np.ndarray        # (3, 3)
    x: np.ndarray        # (N_p, 3) lab-frame nodes
    normal: np.ndarray   # (N_p, 3)
    w: np.ndarray        # (N_p,)
    r: np.ndarray        # (N_p, 3) x - centre
    area: float
    tau: np.ndarray      # (3, 3)
    suspension: int
    radius: float        # bounding radius of the near criterion
    offset: int          # first global node index


def place(body: BodySurface, centre, R, index: int, suspension: int, offset: int) -> Particle:
    """Lab-frame copy of a body surface: x = c + R x_b, n = R n_b (Eq. 40)."""
    centre = np.asarray(centre, dtype=np.float64)
    r = body.x @ R.T
    x = r + centre[None, :]
    normal = body.normal @ R.T
    return Particle(index, body, centre, R, x, normal, body.w.copy(), r, float(body.w.sum()),
                    moment_tensor(r, body.w), suspension, float(body.radius), offset)
