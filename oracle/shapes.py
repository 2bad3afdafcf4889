"""Oracle: general genus-0 particle surfaces given by spherical-harmonic coefficients (Section 3,
Eqs. 31, 36, 37): x(theta, phi) = sum c_nm Y_nm(theta, phi), tangents by spectral differentiation,
W of Eq. 36, weights of Eq. 35.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Coefficient order (shared with the CUDA path): real orthonormal harmonics without the
Condon-Shortley sign, m = 0..p_g, n = m..p_g, the cos term then (m > 0) the sin term; a shape is a
(3, (p_g + 1)^2) array of x, y, z coefficients.  The body frame is centred at the surface's area
centroid on the particle's own grid (the x^c of Eq. 18), and the bounding radius used by the near
criterion is the largest distance from it over the nodes of the upsampled grid.

Derivatives are formed from regular expressions at every parameter point, poles included:
dPbar_n^m/dtheta = (sqrt((n+m)(n-m+1)) Pbar_n^{m-1} - sqrt((n+m+1)(n-m)) Pbar_n^{m+1}) / 2 for m >= 1,
dPbar_n^0/dtheta = -sqrt(n (n+1)) Pbar_n^1, and Pbar_n^m / sin(theta) (m >= 1) by the same n-recurrence
started from sin^(m-1)(theta); so x_phi / sin(theta) and J = W / sin(theta) = |x_theta x x_phi / sin(theta)|
are evaluated without dividing by sin(theta).
"""
from __future__ import annotations

import math

import numpy as np

from .sphere_grid import legendre_normalized


def n_coef(pg: int) -> int:
    return (pg + 1) ** 2


def _legendre_over_sin(p: int, t: np.ndarray) -> np.ndarray:
    """Q[n, m] = Pbar_n^m(t) / sin(theta) for 1 <= m <= n <= p (zero for m = 0)."""
    s = np.sqrt(np.maximum(0.0, 1.0 - t * t))
    Q = np.zeros((p + 1, p + 1) + t.shape)
    pmm = np.full(t.shape, 1.0 / math.sqrt(4.0 * math.pi))   # Pbar_0^0
    qmm = None
    for m in range(1, p + 1):
        # Pbar_m^m = sqrt((2m+1)/(2m)) s Pbar_{m-1}^{m-1}; Q_m^m = sqrt((2m+1)/(2m)) Pbar_{m-1}^{m-1}
        qmm = math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * pmm
        pmm = qmm * s
        Q[m, m] = qmm
        if m + 1 <= p:
            Q[m + 1, m] = math.sqrt(2.0 * m + 3.0) * t * qmm
        for n in range(m + 2, p + 1):
            a = math.sqrt((4.0 * n * n - 1.0) / (n * n - m * m))
            b = math.sqrt(((n - 1.0) ** 2 - m * m) / (4.0 * (n - 1.0) ** 2 - 1.0))
            Q[n, m] = a * (t * Q[n - 1, m] - b * Q[n - 2, m])
    return Q


def basis_with_derivatives(pg: int, theta: np.ndarray, phi: np.ndarray):
    """Y, dY/dtheta and (dY/dphi) / sin(theta) in the shared coefficient order; each (n_coef, n_pts)."""
    t = np.cos(theta)
    P = legendre_normalized(pg, t)
    Q = _legendre_over_sin(pg, t)

    def dP(n, m):
        if m == 0:
            return -math.sqrt(n * (n + 1.0)) * P[n, 1] if n >= 1 else np.zeros_like(t)
        up = math.sqrt((n + m + 1.0) * (n - m)) * P[n, m + 1] if m + 1 <= n else 0.0
        return 0.5 * (math.sqrt((n + m) * (n - m + 1.0)) * P[n, m - 1] - up)

    Y, Yt, Yp = [], [], []
    r2 = math.sqrt(2.0)
    for m in range(0, pg + 1):
        for n in range(m, pg + 1):
            if m == 0:
                Y.append(P[n, 0])
                Yt.append(dP(n, 0))
                Yp.append(np.zeros_like(t))
            else:
                c, s = np.cos(m * phi), np.sin(m * phi)
                Y.append(r2 * P[n, m] * c)
                Yt.append(r2 * dP(n, m) * c)
                Yp.append(-r2 * m * Q[n, m] * s)
                Y.append(r2 * P[n, m] * s)
                Yt.append(r2 * dP(n, m) * s)
                Yp.append(r2 * m * Q[n, m] * c)
    return np.array(Y), np.array(Yt), np.array(Yp)


class SHShape:
    """A surface given by coefficients; evaluates points, area per solid angle and normals."""

    def __init__(self, coef: np.ndarray, pg: int, shift=None):
        self.coef = np.asarray(coef, float).reshape(3, n_coef(pg))
        self.pg = pg
        self.shift = np.zeros(3) if shift is None else np.asarray(shift, float)

    def evaluate(self, s: np.ndarray):
        """Point, J = |x_theta x x_phi| / sin(theta) and unit normal at parameter-sphere points s."""
        s = np.asarray(s, float)
        theta = np.arccos(np.clip(s[..., 2], -1.0, 1.0))
        phi = np.arctan2(s[..., 1], s[..., 0])
        Y, Yt, Yp = basis_with_derivatives(self.pg, theta.ravel(), phi.ravel())
        x = (self.coef @ Y).T - self.shift
        xt = (self.coef @ Yt).T
        xp = (self.coef @ Yp).T
        cr = np.cross(xt, xp)
        J = np.linalg.norm(cr, axis=1)
        return x.reshape(s.shape), J.reshape(s.shape[:-1]), (cr / J[:, None]).reshape(s.shape)

    def point(self, s):
        return self.evaluate(s)[0]

    def jacobian(self, s):
        return self.evaluate(s)[1]

    def normal(self, s):
        return self.evaluate(s)[2]


def sh_coefficients_of_ellipsoid(axes) -> tuple[np.ndarray, int]:
    """The ellipsoid x = (a s_x, b s_y, c s_z) as degree-1 coefficients in the shared order:
    s_z = sqrt(4 pi / 3) Y_10, s_x = sqrt(4 pi / 3) Y_11(cos), s_y = sqrt(4 pi / 3) Y_11(sin)."""
    a, b, c = axes
    k = math.sqrt(4.0 * math.pi / 3.0)
    coef = np.zeros((3, 4))
    # order: (n=0,m=0), (n=1,m=0), (n=1,m=1,cos), (n=1,m=1,sin)
    coef[0, 2] = a * k
    coef[1, 3] = b * k
    coef[2, 1] = c * k
    return coef, 1
