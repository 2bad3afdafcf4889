"""Oracle: the discretised layer potentials S and K and the operator L (Sections 2.1-2.3 and 3-3.1;
Eqs. 10-13, 22-26, 34-35, 38).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Every operator is a sum over (target node t, source particle j) of 3 x 3 blocks:
* j on another particle, not near (smooth rule, Eq. 35): k(x_t - y_s) w_s at the base grid nodes;
* j on another particle, near: the source density is upsampled to a finer grid of order p_up
  (Section 3: "upsample the boundary data") and the smooth rule is applied on that grid;
* j the target's own particle: the rotated-pole singular rule described below, computed once per
  body shape in the body frame and rotated, A_lab = R A_body R^T (Eq. 38).
Particles with different suspension ids do not interact.

Readings of the paper used here (each a named option with this default):
* K_ij of Eq. 22 integrates over the source surface Gamma_j (the printed Gamma_i is a typo).
* Near pairs: particles i != j with |c_i - c_j| < R_i + R_j + delta, R the bounding radius (the
  largest semi-axis of an ellipsoid, the largest node distance on the upsampled grid otherwise),
  delta = 1; sources upsampled to p_up = 2p with n_phi_up = n_phi + 2 (p_up - p).
* Singular rule (Section 3 defers to a rule that is not reproduced in the paper): rotate the
  parameter sphere so that the target sits at the north pole, theta' = 0; integrate over the rotated
  sphere with Gauss-Legendre in theta' on [0, pi] (p_s + 1 points, the sin(theta') of the solid
  angle cancels the 1/r singularity) and the trapezoidal rule in phi' (2 p_s + 2 points); the density
  at the rotated points comes from the spherical-harmonic expansion of the grid values.  The rotation
  taking the pole to the target at parameter angles (theta_t, phi_t) is R_z(phi_t) R_y(theta_t).
  Default p_s = 2p.
"""
from __future__ import annotations

import math

import numpy as np

from .sphere_grid import angles_of, gauss_legendre, grid_points, interpolation_matrix

FOUR_PI = 4.0 * math.pi
EIGHT_PI = 8.0 * math.pi


# ---------------------------------------------------------------------------------------------
# Kernels

def stokeslet(r: np.ndarray) -> np.ndarray:
    """Eq. 10: G(x, y) = (1 / 8 pi) (I / |r| + r r^T / |r|^3), r = x - y.  Shape (..., 3, 3)."""
    d = np.linalg.norm(r, axis=-1)
    out = np.einsum("...i,...j->...ij", r, r) / (d ** 3)[..., None, None]
    out = out + np.eye(3) / d[..., None, None]
    return out / EIGHT_PI


def traction(r: np.ndarray, n_t: np.ndarray) -> np.ndarray:
    """Eqs. 13 and 22: the 3 x 3 matrix M with (K rho)_k = n_l T_klm rho_m = M_km rho_m,
    M = -(3 / 4 pi) (r . n_t) r r^T / |r|^5, r = x - y, n_t the normal at the target."""
    d = np.linalg.norm(r, axis=-1)
    rn = np.einsum("...i,...i->...", r, n_t)
    out = np.einsum("...i,...j->...ij", r, r) * (rn / d ** 5)[..., None, None]
    return -3.0 / FOUR_PI * out


def kernel_matrix(kind: str, r: np.ndarray, n_t: np.ndarray) -> np.ndarray:
    if kind == "K":
        return traction(r, n_t)
    if kind == "S":
        return stokeslet(r)
    raise ValueError(kind)


# ---------------------------------------------------------------------------------------------
# Singular self rule (body frame)

def rotated_rule(p_s: int):
    """Points and weights of the rotated-pole rule around the north pole: theta' = pi (u + 1) / 2 over
    the (p_s + 1)-point Gauss-Legendre nodes u, phi' = 2 pi b / (2 p_s + 2); the weight includes the
    sin(theta') of the solid angle.  Returns (s' (M, 3), weights (M,))."""
    u, lam = gauss_legendre(p_s + 1)
    th = 0.5 * math.pi * (u + 1.0)
    wth = 0.5 * math.pi * lam
    nb = 2 * p_s + 2
    ph = 2.0 * math.pi * np.arange(nb) / nb
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    s = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], axis=-1).reshape(-1, 3)
    wgt = (wth[:, None] * np.sin(TH) * (2.0 * math.pi / nb)).reshape(-1)
    return s, wgt


def pole_rotation(theta_t: float, phi_t: float) -> np.ndarray:
    """R_z(phi_t) R_y(theta_t): takes the north pole to the parameter point (theta_t, phi_t)."""
    ct, st, cp, sp = math.cos(theta_t), math.sin(theta_t), math.cos(phi_t), math.sin(phi_t)
    Ry = np.array([[ct, 0.0, st], [0.0, 1.0, 0.0], [-st, 0.0, ct]])
    Rz = np.array([[cp, -sp, 0.0], [sp, cp, 0.0], [0.0, 0.0, 1.0]])
    return Rz @ Ry


def self_rows(kind: str, body, targets, p_s: int) -> np.ndarray:
    """Rows of the body-frame self block for the given target nodes: shape (len(targets), 3, 3, N_p),
    entry [t, k, m, s] = sum over rotated points a of
        weight_a J(s'_a) kernel(x_t - x(s'_a))_km Interp(s'_a)_s,
    with J the area per unit solid angle (W / sin theta of Eq. 36)."""
    s0, wgt = rotated_rule(p_s)
    out = np.zeros((len(targets), 3, 3, len(body.w)))
    for row, t in enumerate(targets):
        s = s0 @ pole_rotation(body.theta[t], body.phi[t]).T
        y = body.point(s)
        J = body.jacobian(s)
        kern = kernel_matrix(kind, body.x[t][None, :] - y, body.normal[t][None, :])
        th, ph = angles_of(s)
        interp = interpolation_matrix(body.p, body.nphi, th, ph)
        out[row] = np.einsum("a,akm,as->kms", wgt * J, kern, interp)
    return out


def self_block(kind: str, body, p_s: int) -> np.ndarray:
    """Whole body-frame self block (3 N_p x 3 N_p), index 3 * node + component."""
    rows = self_rows(kind, body, range(len(body.w)), p_s)
    n = len(body.w)
    return rows.transpose(0, 1, 3, 2).reshape(3 * n, 3 * n)


def rotate_block(block: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Eq. 38: every 3 x 3 sub-block B -> R B R^T."""
    nt, ns = block.shape[0] // 3, block.shape[1] // 3
    b = block.reshape(nt, 3, ns, 3)
    return np.einsum("ik,tkSl,jl->tiSj", R, b, R).reshape(3 * nt, 3 * ns)


# ---------------------------------------------------------------------------------------------
# Near-singular rule: upsampled sources

def upsampled_source(particle, p_up: int):
    """Nodes, weights and interpolation matrix of a source particle on its order-p_up grid
    (n_phi_up = n_phi + 2 (p_up - p)), in the lab frame."""
    body = particle.body
    nphi_up = body.nphi + 2 * (p_up - body.p)
    th, ph, q = grid_points(p_up, nphi_up)
    s = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], axis=1)
    xb = body.point(s)
    w = q * body.jacobian(s)
    U = interpolation_matrix(body.p, body.nphi, th, ph)
    return xb @ particle.R.T + particle.centre[None, :], w, U


def is_near(pi, pj, delta: float) -> bool:
    return bool(np.linalg.norm(pi.centre - pj.centre) < pi.radius + pj.radius + delta)


def interacts(pi, pj) -> bool:
    return pi.index != pj.index and pi.suspension == pj.suspension


def far_block(kind: str, pt, ps, targets=None) -> np.ndarray:
    """Smooth-rule block: [t, k, m, s] = kernel(x_t - y_s)_km w_s, base grid of the source."""
    tg = slice(None) if targets is None else targets
    r = pt.x[tg][:, None, :] - ps.x[None, :, :]
    kern = kernel_matrix(kind, r, pt.normal[tg][:, None, :])
    return np.einsum("tskm,s->tkms", kern, ps.w)


def near_block(kind: str, pt, ps, p_up: int, targets=None) -> np.ndarray:
    """Upsampled block: [t, k, m, s] = sum_u kernel(x_t - y_u)_km w_u U_us."""
    tg = slice(None) if targets is None else targets
    yu, wu, U = upsampled_source(ps, p_up)
    r = pt.x[tg][:, None, :] - yu[None, :, :]
    kern = kernel_matrix(kind, r, pt.normal[tg][:, None, :])
    return np.einsum("tukm,u,us->tkms", kern, wu, U)


def projection_block(pt, targets=None) -> np.ndarray:
    """Eq. 26, L_i[mu](x_t) = sum_s w_s mu_s + (sum_s w_s r_s x mu_s) x r_t, as a block
    [t, k, m, s] = w_s (I - [r_t]_x [r_s]_x)_km, with [a]_x b = a x b."""
    tg = slice(None) if targets is None else targets

    def cross_mat(a):
        z = np.zeros(a.shape[:-1])
        return np.stack([np.stack([z, -a[..., 2], a[..., 1]], -1),
                         np.stack([a[..., 2], z, -a[..., 0]], -1),
                         np.stack([-a[..., 1], a[..., 0], z], -1)], -2)

    ct = cross_mat(pt.r[tg])             # (T, 3, 3)
    cs = cross_mat(pt.r)                 # (S, 3, 3)
    prod = np.einsum("tka,sam->tskm", ct, cs)
    blk = np.eye(3)[None, None] - prod
    return np.einsum("tskm,s->tkms", blk, pt.w)
