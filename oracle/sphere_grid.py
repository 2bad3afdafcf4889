"""Oracle: the parametric grid and the spherical-harmonic transforms (Section 3, Eqs. 31-35).

TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline leg of the benchmark may
import anything under oracle/.  Plain numpy, float64, written for reading rather than speed.

Readings of the paper used here:
* The azimuthal point count n_phi is a per-particle parameter; Eq. 33 prints 2p + 2 while the system
  sizes of Section 4.2 imply 2p.  Both are supported.
* The transforms keep degrees 0 <= n <= p and orders |m| <= m_max = floor((n_phi - 1) / 2), in the
  real orthonormal basis; on a grid of n_phi = 2p points the orders +-p cannot be told apart, so they
  are dropped.  Coefficients are taken by Gauss-Legendre x trapezoid projection, which is exact on
  that space, and "interpolation" means analysis on the grid followed by synthesis anywhere.
"""
from __future__ import annotations

import math

import numpy as np


def gauss_legendre(n: int) -> tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre rule on [-1, 1] (the t_j and lambda_j of Eqs. 33-35), by the
    Golub-Welsch method: the nodes are the eigenvalues of the Jacobi matrix of the Legendre
    three-term recurrence, the weights twice the squared first components of its eigenvectors."""
    if n == 1:
        return np.zeros(1), np.full(1, 2.0)
    k = np.arange(1, n, dtype=np.float64)
    beta = k / np.sqrt(4.0 * k * k - 1.0)
    jac = np.diag(beta, 1) + np.diag(beta, -1)
    t, vec = np.linalg.eigh(jac)
    lam = 2.0 * vec[0, :] ** 2
    return t, lam


def grid_angles(p: int, nphi: int):
    """Eq. 33: theta_j = arccos(t_j) over the p + 1 Gauss-Legendre nodes (t ascending) and
    phi_k = 2 pi k / n_phi.  Returns (theta, phi, t, lambda)."""
    t, lam = gauss_legendre(p + 1)
    theta = np.arccos(t)
    phi = 2.0 * math.pi * np.arange(nphi) / nphi
    return theta, phi, t, lam


def grid_points(p: int, nphi: int):
    """Flattened grid, node index = j * n_phi + k.  Returns theta, phi (each (N,)) and the
    unit-sphere quadrature weight (2 pi / n_phi) lambda_j of every node."""
    theta, phi, _, lam = grid_angles(p, nphi)
    th = np.repeat(theta, nphi)
    ph = np.tile(phi, p + 1)
    q = np.repeat(lam, nphi) * (2.0 * math.pi / nphi)
    return th, ph, q


def legendre_normalized(p: int, t: np.ndarray) -> np.ndarray:
    """Pbar[n, m] = sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!) P_n^m(t) for 0 <= m <= n <= p (the
    normalisation of Eq. 32, without the Condon-Shortley sign), by the standard stable recurrences
    in n at fixed m.  Shape (p+1, p+1) + t.shape; entries with m > n are zero."""
    t = np.asarray(t, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - t * t))
    P = np.zeros((p + 1, p + 1) + t.shape)
    P[0, 0] = 1.0 / math.sqrt(4.0 * math.pi)
    for m in range(1, p + 1):
        P[m, m] = math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * P[m - 1, m - 1]
    for m in range(0, p):
        P[m + 1, m] = math.sqrt(2.0 * m + 3.0) * t * P[m, m]
    for m in range(0, p + 1):
        for n in range(m + 2, p + 1):
            a = math.sqrt((4.0 * n * n - 1.0) / (n * n - m * m))
            b = math.sqrt(((n - 1.0) ** 2 - m * m) / (4.0 * (n - 1.0) ** 2 - 1.0))
            P[n, m] = a * (t * P[n - 1, m] - b * P[n - 2, m])
    return P


def sh_index(p: int, mmax: int) -> list[tuple[int, int]]:
    """The retained (n, m) pairs: 0 <= n <= p, |m| <= min(n, m_max)."""
    return [(n, m) for n in range(p + 1) for m in range(-min(n, mmax), min(n, mmax) + 1)]


def mmax_for(nphi: int) -> int:
    return (nphi - 1) // 2


def real_sh(p: int, mmax: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics of Eq. 32 (cos(m phi), sin(|m| phi) in place of
    e^{i m phi}, times sqrt 2 for m != 0) at the given points.  Shape (n_basis, n_points)."""
    P = legendre_normalized(p, np.cos(theta))
    rows = []
    for n, m in sh_index(p, mmax):
        if m == 0:
            rows.append(P[n, 0])
        elif m > 0:
            rows.append(math.sqrt(2.0) * P[n, m] * np.cos(m * phi))
        else:
            rows.append(math.sqrt(2.0) * P[n, -m] * np.sin(-m * phi))
    return np.array(rows)


def analysis_matrix(p: int, nphi: int) -> np.ndarray:
    """Forward transform on the grid (Section 3): coefficient = sum over nodes of Y(node) f(node)
    (2 pi / n_phi) lambda_j.  Shape (n_basis, N_p)."""
    th, ph, q = grid_points(p, nphi)
    return real_sh(p, mmax_for(nphi), th, ph) * q[None, :]


def interpolation_matrix(p: int, nphi: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Values at arbitrary parameter points of the spherical-harmonic expansion of grid data:
    synthesis after analysis.  Shape (n_points, N_p)."""
    Y = real_sh(p, mmax_for(nphi), np.asarray(theta, float), np.asarray(phi, float))
    return Y.T @ analysis_matrix(p, nphi)


def angles_of(s: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Polar and azimuthal angle of unit vectors s (..., 3)."""
    theta = np.arccos(np.clip(s[..., 2], -1.0, 1.0))
    phi = np.arctan2(s[..., 1], s[..., 0])
    return theta, phi
