"""Oracle: the discrete mobility solve (Sections 2.2-2.3, 3 and Algorithm 1; Eqs. 18-19, 24-26, 41-42).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Steps, in the order of the method's three-step summary at the start of Section 3:
1. incident density rho (Eq. 19);
2. the scattered density mu from (1/2 I + K + L) mu = -(1/2 I + K) rho (Eq. 25), by dense LU on
   small systems or by GMRES on the same operator applied block by block;
3. u = S[rho + mu] on the surface, then v_i (Eq. 41) and omega_i (Eq. 42).
Vectors over the surface are (total_nodes, 3) arrays, particle-major, node index j * n_phi + k.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import operators as ops
from .geometry import body_surface, body_surface_sh, place, quat_to_rot


@dataclasses.dataclass
class Options:
    delta: float = 1.0          # near criterion margin
    p_up_factor: int = 2        # near sources upsampled to p_up = factor * p
    p_self_factor: int = 2      # singular rule order p_s = factor * p
    viscosity: float = 1.0      # mu of Eq. 2; velocities scale as 1 / mu


class System:
    """Geometry plus the pieces of the discrete operators.  Self blocks are built once per distinct
    (semi-axes, p, n_phi) in the body frame and rotated per particle (Eq. 38)."""

    def __init__(self, semi_axes, p, nphi, centres, quats, suspension_id=None, options: Options | None = None,
                 shapes=None, shape_of=None):
        """Ellipsoids by semi_axes (n x 3), or coefficient surfaces: shapes = list of (coef, p_g) and
        shape_of[i] the shape of particle i (semi_axes is then ignored and may be None)."""
        self.opt = options or Options()
        if shapes is not None:
            n = len(shape_of)
            semi_axes = np.zeros((n, 3))
        else:
            semi_axes = np.asarray(semi_axes, np.float64).reshape(-1, 3)
            n = semi_axes.shape[0]
        p = np.broadcast_to(np.asarray(p, np.int64), (n,))
        nphi = np.broadcast_to(np.asarray(nphi, np.int64), (n,))
        centres = np.asarray(centres, np.float64).reshape(n, 3)
        quats = np.asarray(quats, np.float64).reshape(n, 4)
        sid = np.zeros(n, np.int64) if suspension_id is None else np.asarray(suspension_id, np.int64)
        self._bodies: dict[tuple, object] = {}
        self._self_cache: dict[tuple, np.ndarray] = {}
        self.particles = []
        offset = 0
        for i in range(n):
            if shapes is not None:
                key = ("sh", int(shape_of[i]), int(p[i]), int(nphi[i]))
                if key not in self._bodies:
                    coef, pg = shapes[int(shape_of[i])]
                    self._bodies[key] = body_surface_sh(coef, pg, int(p[i]), int(nphi[i]),
                                                        self.opt.p_up_factor * int(p[i]))
            else:
                key = (tuple(semi_axes[i]), int(p[i]), int(nphi[i]))
                if key not in self._bodies:
                    self._bodies[key] = body_surface(semi_axes[i], int(p[i]), int(nphi[i]))
            body = self._bodies[key]
            self.particles.append(place(body, centres[i], quat_to_rot(quats[i]), i, int(sid[i]), offset))
            offset += len(body.w)
        self.total_nodes = offset
        # near pairs: same suspension, i != j, |c_i - c_j| < R_i + R_j + delta (ops.is_near), tested
        # for all pairs with array arithmetic in row blocks
        cen = np.array([pt.centre for pt in self.particles])
        rad = np.array([pt.radius for pt in self.particles])
        self.near = set()
        for i0 in range(0, n, 1024):
            i1 = min(n, i0 + 1024)
            dist = np.linalg.norm(cen[i0:i1, None, :] - cen[None, :, :], axis=2)
            hit = (dist < rad[i0:i1, None] + rad[None, :] + self.opt.delta) & (sid[i0:i1, None] == sid[None, :])
            for a, b in zip(*np.nonzero(hit)):
                if i0 + a != b:
                    self.near.add((int(i0 + a), int(b)))

    # -- helpers -------------------------------------------------------------------------------
    def sl(self, i: int) -> slice:
        pt = self.particles[i]
        return slice(pt.offset, pt.offset + len(pt.w))

    def body_key(self, i: int):
        b = self.particles[i].body
        return (id(b), b.p, b.nphi)

    def self_block_body(self, kind: str, i: int) -> np.ndarray:
        key = (kind,) + self.body_key(i)
        if key not in self._self_cache:
            b = self.particles[i].body
            self._self_cache[key] = ops.self_block(kind, b, self.opt.p_self_factor * b.p)
        return self._self_cache[key]

    def self_block_lab(self, kind: str, i: int) -> np.ndarray:
        return ops.rotate_block(self.self_block_body(kind, i), self.particles[i].R)

    def p_up(self, j: int) -> int:
        return self.opt.p_up_factor * self.particles[j].body.p

    def pair_block(self, kind: str, i: int, j: int, targets=None) -> np.ndarray:
        """[t, k, m, s] block of target particle i and source particle j != i (far or near)."""
        pi, pj = self.particles[i], self.particles[j]
        if (i, j) in self.near:
            return ops.near_block(kind, pi, pj, self.p_up(j), targets)
        return ops.far_block(kind, pi, pj, targets)

    # -- dense assembly (small systems) --------------------------------------------------------
    def assemble(self, kind: str, half: float = 0.0, with_L: bool = False) -> np.ndarray:
        """Dense matrix of half * I + kind-operator (+ L), 3N x 3N, index 3 * node + component."""
        N3 = 3 * self.total_nodes
        A = np.zeros((N3, N3))
        for i, pi in enumerate(self.particles):
            ri = slice(3 * pi.offset, 3 * (pi.offset + len(pi.w)))
            for j, pj in enumerate(self.particles):
                rj = slice(3 * pj.offset, 3 * (pj.offset + len(pj.w)))
                if i == j:
                    blk = self.self_block_lab(kind, i)
                    if with_L:
                        blk = blk + _flat(ops.projection_block(pi))
                    A[ri, rj] = blk
                elif ops.interacts(pi, pj):
                    A[ri, rj] = _flat(self.pair_block(kind, i, j))
        A[np.diag_indices(N3)] += half
        return A

    # -- matrix-free application ----------------------------------------------------------------
    def apply(self, kind: str, x: np.ndarray, half: float = 0.0, with_L: bool = False) -> np.ndarray:
        """(half * I + kind-operator (+ L)) x for a surface field x (total_nodes, 3)."""
        x = np.asarray(x, np.float64).reshape(self.total_nodes, 3)
        y = half * x.copy()
        for i, pi in enumerate(self.particles):
            si = self.sl(i)
            acc = (self.self_block_lab(kind, i) @ x[si].reshape(-1)).reshape(-1, 3)
            if with_L:
                acc += np.einsum("tkms,sm->tk", ops.projection_block(pi), x[si])
            for j, pj in enumerate(self.particles):
                if j != i and ops.interacts(pi, pj):
                    acc += np.einsum("tkms,sm->tk", self.pair_block(kind, i, j), x[self.sl(j)])
            y[si] += acc
        return y

    def apply_rows(self, kind: str, x: np.ndarray, nodes, half: float = 0.0, with_L: bool = False) -> np.ndarray:
        """The same operator at selected global nodes only, computing just those rows (works at any
        system size: O(total_nodes) per row plus one singular-rule row)."""
        x = np.asarray(x, np.float64).reshape(self.total_nodes, 3)
        nodes = np.asarray(nodes)
        owner = np.searchsorted([pt.offset for pt in self.particles], nodes, side="right") - 1
        out = np.zeros((len(nodes), 3))
        for row, (g, i) in enumerate(zip(nodes, owner)):
            pi = self.particles[i]
            t = int(g - pi.offset)
            b = pi.body
            srow = ops.self_rows(kind, b, [t], self.opt.p_self_factor * b.p)[0]      # (3, 3, S) body
            srow = np.einsum("ik,kms,jm->ijs", pi.R, srow, pi.R)
            acc = half * x[g] + np.einsum("kms,sm->k", srow, x[self.sl(i)])
            if with_L:
                acc += np.einsum("tkms,sm->k", ops.projection_block(pi, [t]), x[self.sl(i)])
            for j, pj in enumerate(self.particles):
                if j != i and ops.interacts(pi, pj):
                    acc += np.einsum("tkms,sm->k", self.pair_block(kind, i, j, [t]), x[self.sl(j)])
            out[row] = acc
        return out

    # -- the method ---------------------------------------------------------------------------
    def incident_density(self, F, T) -> np.ndarray:
        """Eq. 19: rho_t = F_i / |Gamma_i| + (tau_i^{-1} T_i) x (x_t - x^c_i)."""
        F = np.asarray(F, np.float64).reshape(-1, 3)
        T = np.asarray(T, np.float64).reshape(-1, 3)
        rho = np.zeros((self.total_nodes, 3))
        for i, pt in enumerate(self.particles):
            a = np.linalg.solve(pt.tau, T[i])
            rho[self.sl(i)] = F[i][None, :] / pt.area + np.cross(a[None, :], pt.r)
        return rho

    def rhs(self, rho: np.ndarray) -> np.ndarray:
        """Right-hand side of Eq. 25: -(1/2 I + K) rho."""
        return -self.apply("K", rho, half=0.5)

    def rigid_velocities(self, u: np.ndarray):
        """Eqs. 41-42: v_i = (1 / |Gamma_i|) sum w u, omega_i = tau_i^{-1} sum w (x - x^c_i) x u."""
        u = np.asarray(u).reshape(self.total_nodes, 3)
        n = len(self.particles)
        v = np.zeros((n, 3))
        om = np.zeros((n, 3))
        for i, pt in enumerate(self.particles):
            ui = u[self.sl(i)]
            v[i] = (pt.w[:, None] * ui).sum(0) / pt.area
            om[i] = np.linalg.solve(pt.tau, (pt.w[:, None] * np.cross(pt.r, ui)).sum(0))
        return v / self.opt.viscosity, om / self.opt.viscosity

    def solve(self, F, T, method: str = "lu", tol: float = 1e-13, restart: int = 200, maxiter: int = 2000):
        """Algorithm 1, lines 3-5, without contact: returns v, omega, mu, rho, iterations."""
        rho = self.incident_density(F, T)
        b = self.rhs(rho)
        if method == "lu":
            A = self.assemble("K", half=0.5, with_L=True)
            mu = np.linalg.solve(A, b.reshape(-1)).reshape(-1, 3)
            its = 0
        else:
            mu, its, _ = gmres(lambda z: self.apply("K", z.reshape(-1, 3), half=0.5, with_L=True).reshape(-1),
                               b.reshape(-1), tol, restart, maxiter)
            mu = mu.reshape(-1, 3)
        u = self.apply("S", rho + mu)
        v, om = self.rigid_velocities(u)
        return v, om, mu, rho, its

    def mobility_matrix(self) -> np.ndarray:
        """The 6n x 6n matrix M of Eq. 1, V = M F with V = (v_1, omega_1, ...), F = (F_1, T_1, ...),
        one dense solve per column."""
        n = len(self.particles)
        A = self.assemble("K", half=0.5, with_L=True)
        lu_solve = _lu(A)
        M = np.zeros((6 * n, 6 * n))
        for col in range(6 * n):
            F = np.zeros((n, 3))
            T = np.zeros((n, 3))
            (F if col % 6 < 3 else T)[col // 6, col % 3] = 1.0
            rho = self.incident_density(F, T)
            mu = lu_solve(self.rhs(rho).reshape(-1)).reshape(-1, 3)
            v, om = self.rigid_velocities(self.apply("S", rho + mu))
            M[:, col] = np.concatenate([v, om], axis=1).reshape(-1)
        return M


def _flat(blk: np.ndarray) -> np.ndarray:
    nt, _, _, ns = blk.shape
    return blk.transpose(0, 1, 3, 2).reshape(3 * nt, 3 * ns)


def _lu(A: np.ndarray):
    import scipy.linalg as sla
    fac = sla.lu_factor(A)
    return lambda b: sla.lu_solve(fac, b)


def gmres(apply, b: np.ndarray, tol: float, restart: int, maxiter: int, x0=None):
    """Restarted GMRES (Section 3.2), modified Gram-Schmidt with one reorthogonalisation pass,
    Givens rotations; stops when ||b - A x|| <= tol ||b||.  Returns (x, iterations, residual)."""
    n = b.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    its = 0
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm or its >= maxiter:
            return x, its, beta / bnorm
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(restart):
            w = apply(V[k])
            for _ in range(2):
                for i in range(k + 1):
                    h = V[i] @ w
                    H[i, k] += h
                    w = w - h * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                a, c = H[i, k], H[i + 1, k]
                H[i, k] = cs[i] * a + sn[i] * c
                H[i + 1, k] = -sn[i] * a + cs[i] * c
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            its += 1
            k_done = k + 1
            if abs(g[k + 1]) <= tol * bnorm or its >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + V[:k_done].T @ y
