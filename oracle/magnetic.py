"""Oracle: magnetostatic coupling of paramagnetic particles (Section 4.1.3, magnetorheological flow).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The field outside the particles is H = -grad phi with phi = -H0 . x + S^L[q] (S^L the Laplace single
layer, G(x, y) = 1 / (4 pi |x - y|)); the jump conditions across each surface lead to the second-kind
equation (1/2 I + eta K^L) q = eta H0 . n, eta = (mu - mu0) / (mu + mu0), K^L the normal derivative of
S^L at the target, kernel -(r . n_x) / (4 pi |r|^3), r = x - y.  The discretisation reuses the
mobility solve's: the same grids and weights, the smooth rule for far pairs, upsampled sources for
near pairs, and the rotated-pole singular rule (scalar kernels) for each particle's own surface.

Readings (the paper leaves them open):
* the surface field is the fluid-side limit: tangential part -grad_s phi by spectral differentiation
  of phi on each particle's grid (Eq. 37), normal part H0 . n + q / 2 - K^L[q] (the exterior jump);
* the Maxwell traction on a particle is the fluid-side stress mu0 [(H . n) H - |H|^2 n / 2] with
  mu0 = 1 (forces scale with mu0 |H0|^2);
* the coupling to the mobility problem goes through each particle's net magnetic force and torque
  (the rigid velocities depend on the densities only through them).
"""
from __future__ import annotations

import math

import numpy as np

from . import operators as ops
from .shapes import basis_with_derivatives
from .sphere_grid import angles_of, grid_angles, interpolation_matrix, mmax_for

FOUR_PI = 4.0 * math.pi


def laplace_kernel(kind: str, r: np.ndarray, n_t: np.ndarray) -> np.ndarray:
    """'S': 1 / (4 pi |r|); 'K': -(r . n_t) / (4 pi |r|^3)."""
    d = np.linalg.norm(r, axis=-1)
    if kind == "S":
        return 1.0 / (FOUR_PI * d)
    if kind == "K":
        return -np.einsum("...i,...i->...", r, n_t) / (FOUR_PI * d ** 3)
    raise ValueError(kind)


def self_block_scalar(kind: str, body, p_s: int) -> np.ndarray:
    """Body-frame scalar self block (N_p x N_p) by the rotated-pole rule, as ops.self_rows."""
    s0, wgt = ops.rotated_rule(p_s)
    n = len(body.w)
    out = np.zeros((n, n))
    for t in range(n):
        s = s0 @ ops.pole_rotation(body.theta[t], body.phi[t]).T
        y = body.point(s)
        J = body.jacobian(s)
        k = laplace_kernel(kind, body.x[t][None, :] - y, body.normal[t][None, :])
        th, ph = angles_of(s)
        out[t] = (wgt * J * k) @ interpolation_matrix(body.p, body.nphi, th, ph)
    return out


class Magnetic:
    """The Laplace operators of a System's particles, the solution q and the surface field."""

    def __init__(self, system):
        self.s = system
        self._self: dict[tuple, np.ndarray] = {}

    def self_block(self, kind: str, i: int) -> np.ndarray:
        key = (kind,) + self.s.body_key(i)
        if key not in self._self:
            b = self.s.particles[i].body
            self._self[key] = self_block_scalar(kind, b, self.s.opt.p_self_factor * b.p)
        return self._self[key]

    def assemble(self, kind: str, half: float = 0.0) -> np.ndarray:
        """half I + the scalar operator, N x N (self blocks are rotation invariant)."""
        s = self.s
        N = s.total_nodes
        A = half * np.eye(N)
        for i, pi in enumerate(s.particles):
            si = s.sl(i)
            A[si, si] += self.self_block(kind, i)
            for j, pj in enumerate(s.particles):
                if j == i or not ops.interacts(pi, pj):
                    continue
                sj = s.sl(j)
                if (i, j) in s.near:
                    yu, wu, U = ops.upsampled_source(pj, s.p_up(j))
                    k = laplace_kernel(kind, pi.x[:, None, :] - yu[None, :, :], pi.normal[:, None, :])
                    A[si, sj] += (k * wu[None, :]) @ U
                else:
                    k = laplace_kernel(kind, pi.x[:, None, :] - pj.x[None, :, :], pi.normal[:, None, :])
                    A[si, sj] += k * pj.w[None, :]
        return A

    def solve(self, H0, mu_ratio: float):
        """q of (1/2 I + eta K^L) q = eta H0 . n."""
        eta = (mu_ratio - 1.0) / (mu_ratio + 1.0)
        n = np.concatenate([pt.normal for pt in self.s.particles])
        b = eta * (n @ np.asarray(H0, float))
        A = 0.5 * np.eye(len(b)) + eta * self.assemble("K")
        return np.linalg.solve(A, b)

    def surface_field(self, H0, q: np.ndarray) -> np.ndarray:
        """H on the fluid side at every node (total_nodes x 3)."""
        s = self.s
        H0 = np.asarray(H0, float)
        x = np.concatenate([pt.x for pt in s.particles])
        n = np.concatenate([pt.normal for pt in s.particles])
        phi = -(x @ H0) + self.assemble("S") @ q
        Hn = n @ H0 + 0.5 * q - self.assemble("K") @ q
        H = np.zeros_like(x)
        for i, pt in enumerate(s.particles):
            si = s.sl(i)
            g = surface_gradient(pt, phi[si])
            H[si] = -g + Hn[si][:, None] * pt.normal   # g lies in the tangent plane
        return H

    def forces(self, H0, mu_ratio: float):
        """Net magnetic force and torque on every particle (n x 3 each), and q."""
        q = self.solve(H0, mu_ratio)
        H = self.surface_field(H0, q)
        n = np.concatenate([pt.normal for pt in self.s.particles])
        f = np.einsum("ij,ij->i", H, n)[:, None] * H - 0.5 * np.einsum("ij,ij->i", H, H)[:, None] * n
        F = np.zeros((len(self.s.particles), 3))
        T = np.zeros_like(F)
        for i, pt in enumerate(self.s.particles):
            si = self.s.sl(i)
            F[i] = (pt.w[:, None] * f[si]).sum(0)
            T[i] = (pt.w[:, None] * np.cross(pt.r, f[si])).sum(0)
        return F, T, q


def surface_gradient(particle, f: np.ndarray) -> np.ndarray:
    """Tangential gradient of a grid function on one particle (lab frame), by spectral
    differentiation: coefficients on the retained space (n <= p, m <= m_max) by the grid quadrature,
    then d/dtheta and (d/dphi) / sin(theta) of the expansion at the nodes, combined with the surface
    tangents a = x_theta and b = x_phi / sin(theta):
    grad f = [((b.b) f_t - (a.b) f_p) a + ((a.a) f_p - (a.b) f_t) b] / ((a.a)(b.b) - (a.b)^2),
    f_t = df/dtheta, f_p = (df/dphi) / sin(theta)."""
    body = particle.body
    p, nphi = body.p, body.nphi
    th, ph = body.theta, body.phi
    _, _, _, lam = grid_angles(p, nphi)
    qw = np.repeat(lam, nphi) * (2.0 * math.pi / nphi)
    Y, Yt, Yp = basis_with_derivatives(p, th, ph)
    keep = []
    mmax = mmax_for(nphi)
    for m in range(0, p + 1):
        for _n in range(m, p + 1):
            keep.extend([m <= mmax] * (1 if m == 0 else 2))
    keep = np.array(keep)
    Y, Yt, Yp = Y[keep], Yt[keep], Yp[keep]
    coef = Y @ (qw * f)
    ft = Yt.T @ coef
    fp = Yp.T @ coef
    a, b = body_tangents(body)
    a = a @ particle.R.T
    b = b @ particle.R.T
    aa = np.einsum("ij,ij->i", a, a)
    bb = np.einsum("ij,ij->i", b, b)
    ab = np.einsum("ij,ij->i", a, b)
    det = aa * bb - ab * ab
    return (((bb * ft - ab * fp) / det)[:, None] * a + ((aa * fp - ab * ft) / det)[:, None] * b)


def body_tangents(body):
    """x_theta and x_phi / sin(theta) at the body's nodes (body frame)."""
    th, ph = body.theta, body.phi
    if body.shape is None:
        D = np.asarray(body.axes)
        a = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], 1) * D[None, :]
        b = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], 1) * D[None, :]
        return a, b
    _, Yt, Yp = basis_with_derivatives(body.shape.pg, th, ph)
    return (body.shape.coef @ Yt).T, (body.shape.coef @ Yp).T


def demagnetization_factors(axes) -> np.ndarray:
    """N_i = (abc / 2) int_0^inf dl / ((a_i^2 + l) sqrt((a^2 + l)(b^2 + l)(c^2 + l))) (sum = 1); the
    substitution l = t / (1 - t) maps the integral to [0, 1)."""
    from scipy.integrate import quad
    a, b, c = axes
    out = []
    for ai in axes:
        def f(t):
            lam = t / (1.0 - t)
            return 1.0 / ((ai * ai + lam) * math.sqrt((a * a + lam) * (b * b + lam) * (c * c + lam))) / (1.0 - t) ** 2
        out.append(0.5 * a * b * c * quad(f, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13, limit=400)[0])
    return np.array(out)
