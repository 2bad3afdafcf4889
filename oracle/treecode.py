"""Oracle: a barycentric Lagrange treecode for the smooth pair sums (the far field of Section 3.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The smooth rule (Eq. 35) sums kernel(x_t - y_s) w_s mu_s over the nodes s of every other particle
of the suspension.  Section 3.1 evaluates these sums with a fast multipole method; this module
states the hierarchical approximation that the CUDA path can use for its float32 inner applies
instead: the barycentric Lagrange treecode (Wang, Krasny and Tlupova, 2020), which interpolates the
kernel in the source variable on a tensor Chebyshev grid of each well-separated cluster.  Its steps,
for one suspension:

1. Tree.  An octree over the particle centres: a cell holding more than one particle splits at the
   midpoint of its centres' bounding box, a particle going to the octant given by the three
   comparisons c > midpoint; children are kept in octant order 0..7 (x the low bit), each listing
   its particles in ascending index order.  Every cell has
   * a box: the union of its particles' node bounding boxes (so it holds every source node),
   * a centre: the midpoint of that box,
   * a radius r = max_j (|c_j - centre| + R_j), R_j the particle's bounding radius (so every node of
     the cell lies within r of the centre),
   * a node count.
2. Interaction lists.  The targets of each particle i form one batch, with the batch's own leaf
   cell giving its centre and radius.  A depth-first traversal from the root (children in order)
   accepts a cell C for approximation when
       r_B + r_C < theta * d,   d >= r_B + r_C + delta   and   (n + 1)^3 < nodes(C),
   d the distance between the centres, delta the near margin; otherwise it descends, and a leaf
   that is not accepted is evaluated directly.  A well-separated cell can hold neither particle i
   nor a particle near it (the second condition), so the self and near rules are untouched.
3. Modified charges.  For an accepted cell with box [lo, hi] and Chebyshev points of the second kind
   s_k = mid + half cos(k pi / n), k = 0..n, per axis, the charge of proxy point (a, b, c) is
       q_abc = sum_{s in C} L_a(y_s,x) L_b(y_s,y) L_c(y_s,z) w_s mu_s,
   L the barycentric Lagrange basis of those points (weights (-1)^k, halved at both ends).
4. Evaluation.  y_t = sum over direct particles j != i of kernel(x_t - y_s) w_s mu_s
                    + sum over accepted cells of sum_k kernel(x_t - s_k) q_k.

When the kernel is a polynomial of degree <= n in each coordinate of the source, step 3-4 is
exact; otherwise its error decays like rho^-n, rho = 1/theta + sqrt(1/theta^2 - 1) the Bernstein
ellipse parameter of the interpolation interval seen from the nearest accepted target.  The
bound used by the CUDA path's refinement logic is C(theta) rho^-n, relative (see tree_error_bound);
it is an empirical model, checked against this module for degrees 2 to 6 and theta 0.5 to 0.7.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import operators as ops


def chebyshev_points(n: int) -> np.ndarray:
    """cos(k pi / n), k = 0..n (Chebyshev points of the second kind on [-1, 1], descending)."""
    return np.cos(np.arange(n + 1) * math.pi / n)


def barycentric_weights(n: int) -> np.ndarray:
    """Barycentric weights of the second-kind Chebyshev points: (-1)^k, halved at k = 0 and n."""
    w = (-1.0) ** np.arange(n + 1)
    w[0] *= 0.5
    w[-1] *= 0.5
    return w


def lagrange_basis(x: np.ndarray, lo: float, hi: float, n: int) -> np.ndarray:
    """L_k(x) for the n + 1 Chebyshev points of [lo, hi]: shape (len(x), n + 1).  A point on a node
    gets the unit vector of that node."""
    x = np.asarray(x, np.float64)
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    u = (x - mid) / half if half > 0 else np.zeros_like(x)
    s = chebyshev_points(n)
    w = barycentric_weights(n)
    diff = u[:, None] - s[None, :]
    hit = diff == 0.0
    diff[hit] = 1.0
    t = w[None, :] / diff
    L = t / t.sum(axis=1, keepdims=True)
    rows = hit.any(axis=1)
    L[rows] = hit[rows].astype(np.float64)
    return L


def tree_error_bound(theta: float, degree: int) -> float:
    """C(theta) rho^-n, rho = 1/theta + sqrt(1/theta^2 - 1), C = 0.25 max(1, (theta / 0.5)^2): the
    relative error the CUDA path assumes for a treecode apply when deciding whether a correction may
    be applied in float32.  An empirical model: the measured constant err * rho^n stays below 0.12 at
    theta = 0.5, 0.26 at 0.6 and 0.4 at 0.7 on the suspensions of the tests."""
    a = 1.0 / theta
    return 0.25 * max(1.0, (theta / 0.5) ** 2) * (a + math.sqrt(a * a - 1.0)) ** (-degree)


@dataclasses.dataclass
class Cell:
    particles: np.ndarray      # ascending particle indices
    lo: np.ndarray             # (3,) box of the particles' nodes
    hi: np.ndarray
    centre: np.ndarray
    radius: float
    nodes: int
    children: list


def particle_box(pt) -> tuple[np.ndarray, np.ndarray]:
    """Bounding box of one particle's nodes (lab frame)."""
    return pt.x.min(axis=0), pt.x.max(axis=0)


def build_tree(system, members) -> Cell:
    """Step 1 for the particles `members` (one suspension), returning the root."""
    parts = system.particles
    members = np.asarray(members, np.int64)

    def make(idx: np.ndarray, depth: int) -> Cell:
        boxes = [particle_box(parts[j]) for j in idx]
        lo = np.min([b[0] for b in boxes], axis=0)
        hi = np.max([b[1] for b in boxes], axis=0)
        centre = 0.5 * (lo + hi)
        radius = max(float(np.linalg.norm(parts[j].centre - centre)) + parts[j].radius for j in idx)
        nodes = int(sum(len(parts[j].w) for j in idx))
        cell = Cell(idx, lo, hi, centre, radius, nodes, [])
        if len(idx) > 1 and depth < 64:
            c = np.array([parts[j].centre for j in idx])
            mid = 0.5 * (c.min(axis=0) + c.max(axis=0))
            octant = (c[:, 0] > mid[0]).astype(int) + 2 * (c[:, 1] > mid[1]) + 4 * (c[:, 2] > mid[2])
            groups = [idx[octant == k] for k in range(8) if np.any(octant == k)]
            if len(groups) > 1:
                cell.children = [make(g, depth + 1) for g in groups]
        return cell

    return make(np.sort(members), 0)


def leaf_of(root: Cell, i: int) -> Cell:
    """The leaf cell holding particle i."""
    cell = root
    while cell.children:
        cell = next(ch for ch in cell.children if i in ch.particles)
    return cell


def interaction_lists(root: Cell, batch: Cell, theta: float, degree: int, delta: float):
    """Step 2 for one target batch: (accepted cells, directly evaluated particles), both in
    depth-first order."""
    approx, direct = [], []
    nprox = (degree + 1) ** 3

    def visit(cell: Cell):
        d = float(np.linalg.norm(batch.centre - cell.centre))
        rr = batch.radius + cell.radius
        if rr < theta * d and d >= rr + delta and nprox < cell.nodes:
            approx.append(cell)
        elif cell.children:
            for ch in cell.children:
                visit(ch)
        else:
            direct.extend(int(j) for j in cell.particles)

    visit(root)
    return approx, direct


def proxy_points(cell: Cell, degree: int) -> np.ndarray:
    """The (n + 1)^3 tensor Chebyshev points of a cell's box, index a (n+1)^2 + b (n+1) + c for the
    x, y, z point indices a, b, c."""
    s = chebyshev_points(degree)
    ax = [0.5 * (cell.lo[d] + cell.hi[d]) + 0.5 * (cell.hi[d] - cell.lo[d]) * s for d in range(3)]
    g = np.stack(np.meshgrid(ax[0], ax[1], ax[2], indexing="ij"), axis=-1)
    return g.reshape(-1, 3)


def modified_charges(system, cell: Cell, degree: int, x: np.ndarray) -> np.ndarray:
    """Step 3: q_abc = sum_s L_a L_b L_c w_s mu_s over the cell's nodes, shape ((n+1)^3, 3), ordered
    like proxy_points."""
    ys, qs = [], []
    for j in cell.particles:
        pt = system.particles[j]
        ys.append(pt.x)
        qs.append(pt.w[:, None] * x[system.sl(j)])
    y = np.concatenate(ys)
    q = np.concatenate(qs)
    L = [lagrange_basis(y[:, d], cell.lo[d], cell.hi[d], degree) for d in range(3)]
    return np.einsum("sa,sb,sc,sk->abck", L[0], L[1], L[2], q).reshape(-1, 3)


class Treecode:
    """Steps 1-4 over a System: trees per suspension and lists per target particle."""

    def __init__(self, system, theta: float = 0.5, degree: int = 7):
        self.s = system
        self.theta = float(theta)
        self.degree = int(degree)
        parts = system.particles
        sids = sorted({pt.suspension for pt in parts})
        self.roots = {}
        for sid in sids:
            self.roots[sid] = build_tree(system, [pt.index for pt in parts if pt.suspension == sid])
        self.lists = []
        for pt in parts:
            root = self.roots[pt.suspension]
            batch = leaf_of(root, pt.index)
            self.lists.append(interaction_lists(root, batch, self.theta, self.degree, system.opt.delta))

    def pair_counts(self) -> tuple[int, int]:
        """(direct node pairs, proxy pairs) of one apply: targets x sources, the own particle's nodes
        counted among the direct sources (the kernels visit and mask them)."""
        direct = proxy = 0
        nprox = (self.degree + 1) ** 3
        for pt, (approx, dlist) in zip(self.s.particles, self.lists):
            nt = len(pt.w)
            direct += nt * sum(len(self.s.particles[j].w) for j in dlist)
            proxy += nt * nprox * len(approx)
        return direct, proxy

    def smooth(self, kind: str, x: np.ndarray) -> np.ndarray:
        """Step 4: the treecode's smooth pair sum (no self, no near correction), (total_nodes, 3)."""
        s = self.s
        x = np.asarray(x, np.float64).reshape(s.total_nodes, 3)
        charges = {}
        y = np.zeros_like(x)
        for i, (approx, dlist) in enumerate(self.lists):
            pt = s.particles[i]
            acc = np.zeros((len(pt.w), 3))
            for j in dlist:
                if j != i:
                    acc += np.einsum("tkms,sm->tk", ops.far_block(kind, pt, s.particles[j]), x[s.sl(j)])
            for cell in approx:
                key = id(cell)
                if key not in charges:
                    charges[key] = (proxy_points(cell, self.degree), modified_charges(s, cell, self.degree, x))
                g, q = charges[key]
                kern = ops.kernel_matrix(kind, pt.x[:, None, :] - g[None, :, :], pt.normal[:, None, :])
                acc += np.einsum("tgkm,gm->tk", kern, q)
            y[s.sl(i)] = acc
        return y


def direct_smooth(system, kind: str, x: np.ndarray) -> np.ndarray:
    """The exact smooth pair sum the treecode approximates: sum over every other particle of the
    suspension of the base-grid rule, near particles included."""
    x = np.asarray(x, np.float64).reshape(system.total_nodes, 3)
    y = np.zeros_like(x)
    for i, pi in enumerate(system.particles):
        for j, pj in enumerate(system.particles):
            if ops.interacts(pi, pj):
                y[system.sl(i)] += np.einsum("tkms,sm->tk", ops.far_block(kind, pi, pj), x[system.sl(j)])
    return y


def offdiagonal_with_tree(system, tree: Treecode, kind: str, x: np.ndarray) -> np.ndarray:
    """The off-diagonal operator as the CUDA path forms it with the treecode: the treecode's smooth
    sum plus the near correction (upsampled rule minus the base-grid rule for near pairs)."""
    x = np.asarray(x, np.float64).reshape(system.total_nodes, 3)
    y = tree.smooth(kind, x)
    for (i, j) in system.near:
        pi, pj = system.particles[i], system.particles[j]
        blk = ops.near_block(kind, pi, pj, system.p_up(j)) - ops.far_block(kind, pi, pj)
        y[system.sl(i)] += np.einsum("tkms,sm->tk", blk, x[system.sl(j)])
    return y
