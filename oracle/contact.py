"""Oracle: the contact force algorithm (Section 3.4; Algorithm 1, the contact branch).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For every pair of surfaces in contact at a point x*, a contact force f acts on the first surface and
-f on the second, and the rigid-body velocities of the two surfaces must agree at x* (no slip).
With C the map from the contact forces to the particles' forces and torques and D the map from the
particles' velocities to the velocity differences at the contact points, the contact forces solve
(D M C) F_c = -D V_0, with M the mobility matrix; the matrix D M C is built from 3 n_c mobility
solves, one per column of C.  Then V = V_0 + (M C) F_c, and the densities are updated the same way.

Readings (the paper does not fix them):
* two particles of one suspension are in contact when the smallest distance between the nodes of
  their upsampled grids (order p_up, as for the near rule) is below a gap threshold; the contact
  point x* is the midpoint of that closest node pair (ties: the first pair in node order);
* D is the transpose of C: for particles i, j with arms r_i = x* - c_i, r_j = x* - c_j,
  C puts (f, r_i x f) on i and (-f, -r_j x f) on j, and D V = v_i + w_i x r_i - v_j - w_j x r_j.
"""
from __future__ import annotations

import numpy as np

from .operators import interacts, is_near, upsampled_source


def find_contacts(system, gap: float):
    """Contacts (i, j, x*) with i < j, in ascending (i, j) order."""
    out = []
    parts = system.particles
    p_up = system.opt.p_up_factor
    for i, pi in enumerate(parts):
        for j in range(i + 1, len(parts)):
            pj = parts[j]
            if not interacts(pi, pj) or not is_near(pi, pj, system.opt.delta):
                continue
            xi, _, _ = upsampled_source(pi, p_up * pi.body.p)
            xj, _, _ = upsampled_source(pj, p_up * pj.body.p)
            d2 = ((xi[:, None, :] - xj[None, :, :]) ** 2).sum(-1)
            k = int(np.argmin(d2))
            a, b = divmod(k, xj.shape[0])
            if np.sqrt(d2[a, b]) < gap:
                out.append((i, j, 0.5 * (xi[a] + xj[b])))
    return out


def contact_map(system, contacts) -> np.ndarray:
    """C: (6 n) x (3 n_c); column 3 k + c is the force/torque vector of a unit force along axis c at
    contact k (f on the first particle, -f on the second)."""
    n = len(system.particles)
    C = np.zeros((6 * n, 3 * len(contacts)))
    for k, (i, j, xs) in enumerate(contacts):
        ri = xs - system.particles[i].centre
        rj = xs - system.particles[j].centre
        for c in range(3):
            f = np.zeros(3)
            f[c] = 1.0
            C[6 * i:6 * i + 3, 3 * k + c] += f
            C[6 * i + 3:6 * i + 6, 3 * k + c] += np.cross(ri, f)
            C[6 * j:6 * j + 3, 3 * k + c] -= f
            C[6 * j + 3:6 * j + 6, 3 * k + c] -= np.cross(rj, f)
    return C


def velocity_difference_map(system, contacts) -> np.ndarray:
    """D: (3 n_c) x (6 n); (D V) at contact k is v_i + w_i x r_i - v_j - w_j x r_j, written out
    directly from the no-slip condition (not as the transpose of C)."""
    n = len(system.particles)
    D = np.zeros((3 * len(contacts), 6 * n))

    def cross_matrix(a):
        return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])

    for k, (i, j, xs) in enumerate(contacts):
        ri = xs - system.particles[i].centre
        rj = xs - system.particles[j].centre
        # w x r = -[r]_x w
        D[3 * k:3 * k + 3, 6 * i:6 * i + 3] += np.eye(3)
        D[3 * k:3 * k + 3, 6 * i + 3:6 * i + 6] -= cross_matrix(ri)
        D[3 * k:3 * k + 3, 6 * j:6 * j + 3] -= np.eye(3)
        D[3 * k:3 * k + 3, 6 * j + 3:6 * j + 6] += cross_matrix(rj)
    return D


def solve_with_contacts(system, F, T, gap: float):
    """Algorithm 1 lines 3-9 for one configuration: the mobility solve, contact detection, the
    contact forces from D M C and the corrected velocities and density.  Returns
    (v, omega, mu, contacts, F_c)."""
    n = len(system.particles)
    v0, om0, mu0, _, _ = system.solve(F, T)
    contacts = find_contacts(system, gap)
    if not contacts:
        return v0, om0, mu0, contacts, np.zeros((0, 3))
    C = contact_map(system, contacts)
    D = velocity_difference_map(system, contacts)
    V0 = np.concatenate([v0, om0], axis=1).reshape(-1)
    MC = np.zeros((6 * n, C.shape[1]))
    mus = []
    for col in range(C.shape[1]):
        FT = C[:, col].reshape(n, 6)
        vk, omk, muk, _, _ = system.solve(FT[:, :3], FT[:, 3:])
        MC[:, col] = np.concatenate([vk, omk], axis=1).reshape(-1)
        mus.append(muk)
    Fc = np.linalg.solve(D @ MC, -D @ V0)
    V = (V0 + MC @ Fc).reshape(n, 6)
    mu = mu0 + sum(f * m for f, m in zip(Fc, mus))
    return V[:, :3], V[:, 3:], mu, contacts, Fc.reshape(-1, 3)
