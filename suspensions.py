"""Seeded synthetic suspensions of rigid ellipsoids: the inputs shared by the CUDA path and the oracle.

This module only draws random numbers and places particles; it holds none of the boundary-integral
arithmetic.  Every suspension is a set of ellipsoids given by their semi-axes (a, b, c), the
spherical-harmonic order p and azimuthal point count n_phi of their surface grid, centres,
orientations (unit quaternions, scalar first) and the applied forces F and torques T (Section 2,
Eqs. 1-5: forces and torques in, velocities out).

Placement is random sequential addition inside a cube, with a minimum gap between the bounding
spheres of the particles (radius = largest semi-axis), so the true surface gap is never below it.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Suspension:
    semi_axes: np.ndarray       # (n, 3) float64
    p: np.ndarray               # (n,) int32, spherical-harmonic order per particle
    nphi: np.ndarray            # (n,) int32, azimuthal points per particle
    centres: np.ndarray         # (n, 3) float64
    quats: np.ndarray           # (n, 4) float64, unit quaternions (w, x, y, z)
    F: np.ndarray               # (n, 3) float64
    T: np.ndarray               # (n, 3) float64
    suspension_id: np.ndarray   # (n,) int32, particles interact only within one suspension
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.semi_axes.shape[0])

    @property
    def nodes_per_particle(self) -> np.ndarray:
        return (self.p + 1) * self.nphi

    @property
    def total_nodes(self) -> int:
        return int(self.nodes_per_particle.sum())


def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed rotations: a normalised 4-D Gaussian, sign fixed so that w >= 0."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return q


def place_rsa(rng: np.random.Generator, radii: np.ndarray, lo: float, hi: float, gap: float,
              max_attempts: int = 50_000_000) -> np.ndarray:
    """Random sequential addition of spheres of the given radii, centres uniform in [lo, hi]^3,
    keeping |c_i - c_j| >= r_i + r_j + gap.  Particles are inserted in the order given; candidates
    are drawn in batches whose size doubles after each batch with no admissible point."""
    n = len(radii)
    if n == 0:
        return np.zeros((0, 3))
    rmax = float(radii.max())
    ncell = max(1, int(math.floor((hi - lo) / (2.0 * rmax + gap))))
    cell = (hi - lo) / ncell
    # a cell of side >= 2 rmax + gap holds at most a handful of bounding spheres
    cap = 16
    table = -np.ones((ncell + 2, ncell + 2, ncell + 2, cap), dtype=np.int64)
    fill = np.zeros((ncell + 2, ncell + 2, ncell + 2), dtype=np.int64)
    offs = np.array([(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)])
    centres = np.zeros((n, 3))
    rad_pad = np.append(radii, 0.0)          # index -1 -> padding entry
    cen_pad = np.zeros((n + 1, 3))
    attempts = 0
    for i in range(n):
        batch = 4
        while True:
            cand = rng.uniform(lo, hi, size=(batch, 3))
            attempts += batch
            ci = np.minimum(((cand - lo) / cell).astype(np.int64), ncell - 1) + 1
            nc = ci[:, None, :] + offs[None, :, :]                       # (B, 27, 3)
            idx = table[nc[..., 0], nc[..., 1], nc[..., 2]].reshape(batch, -1)  # (B, 27*cap)
            d = np.linalg.norm(cand[:, None, :] - cen_pad[idx], axis=2)
            need = radii[i] + rad_pad[idx] + gap
            ok = np.all((idx < 0) | (d >= need), axis=1)
            good = np.flatnonzero(ok)
            if len(good):
                c = cand[good[0]]
                k = np.minimum(((c - lo) / cell).astype(np.int64), ncell - 1) + 1
                if fill[k[0], k[1], k[2]] >= cap:
                    raise RuntimeError("cell capacity exceeded in random sequential addition")
                table[k[0], k[1], k[2], fill[k[0], k[1], k[2]]] = i
                fill[k[0], k[1], k[2]] += 1
                centres[i] = c
                cen_pad[i] = c
                break
            if attempts > max_attempts:
                raise RuntimeError(f"random sequential addition stalled at particle {i} of {n}")
            batch = min(batch * 2, 8192)
    return centres


def cube_side(n: int, mean_volume: float, volume_fraction: float) -> float:
    """Side of the cube that holds n particles of the given mean volume at the volume fraction."""
    return (n * mean_volume / volume_fraction) ** (1.0 / 3.0)


def random_ellipsoids(n: int, p: int | np.ndarray, nphi: int | np.ndarray | None, volume_fraction: float,
                      gap: float, seed: int, axes_lo: float = 0.6, axes_hi: float = 1.4,
                      name: str = "") -> Suspension:
    """n triaxial ellipsoids, semi-axes i.i.d. U[axes_lo, axes_hi], uniformly random orientation,
    centres uniform in a cube sized for the volume fraction (mean volume (4 pi / 3) E[abc] with
    E[abc] = ((lo + hi) / 2)^3), bounding-sphere gap `gap`; F, T ~ N(0, 1) per component."""
    rng = np.random.default_rng(seed)
    axes = rng.uniform(axes_lo, axes_hi, size=(n, 3))
    quats = random_quaternions(rng, n)
    mean_abc = ((axes_lo + axes_hi) / 2.0) ** 3
    L = cube_side(n, 4.0 * math.pi / 3.0 * mean_abc, volume_fraction)
    radii = axes.max(axis=1)
    centres = place_rsa(rng, radii, -L / 2, L / 2, gap)
    F = rng.normal(size=(n, 3))
    T = rng.normal(size=(n, 3))
    p_arr = np.broadcast_to(np.asarray(p, dtype=np.int32), (n,)).copy()
    if nphi is None:
        nphi_arr = 2 * p_arr
    else:
        nphi_arr = np.broadcast_to(np.asarray(nphi, dtype=np.int32), (n,)).copy()
    return Suspension(axes, p_arr, nphi_arr, centres, quats, F, T, np.zeros(n, np.int32), name)


def spheres_in_box(n: int, radius: float, half_width: float, gap: float, p: int, nphi: int,
                   seed: int, name: str = "") -> Suspension:
    """n equal spheres, centres uniform in [-half_width, half_width]^3 with surface gap >= gap."""
    rng = np.random.default_rng(seed)
    centres = place_rsa(rng, np.full(n, radius), -half_width, half_width, gap)
    F = rng.normal(size=(n, 3))
    T = rng.normal(size=(n, 3))
    quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    return Suspension(np.full((n, 3), radius), np.full(n, p, np.int32), np.full(n, nphi, np.int32),
                      centres, quats, F, T, np.zeros(n, np.int32), name)


def sphere_lattice(nz: int, p: int, spacing: float = 5.0, radius: float = 1.0) -> Suspension:
    """The 2 x 2 x nz lattice of spheres with the given centre spacing used in the paper's scaling
    runs (Section 4.2, Tables 1-2), sedimenting under F = (0, 0, -1), T = 0."""
    idx = np.array([(i, j, k) for k in range(nz) for j in range(2) for i in range(2)], dtype=np.float64)
    centres = idx * spacing
    centres -= centres.mean(axis=0)
    n = len(centres)
    F = np.tile([0.0, 0.0, -1.0], (n, 1))
    return Suspension(np.full((n, 3), radius), np.full(n, p, np.int32), np.full(n, 2 * p, np.int32),
                      centres, np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), F, np.zeros((n, 3)),
                      np.zeros(n, np.int32), f"lattice_2x2x{nz}_p{p}")


def forces(seed: int, n: int, draw: int) -> tuple[np.ndarray, np.ndarray]:
    """The draw-th seeded (F, T) pair, F, T ~ N(0, 1) per component."""
    rng = np.random.default_rng([seed, 1000 + draw])
    return rng.normal(size=(n, 3)), rng.normal(size=(n, 3))


def random_density(seed: int, total_nodes: int) -> np.ndarray:
    """A seeded N(0, 1) surface vector field, (total_nodes, 3)."""
    return np.random.default_rng([seed, 7]).normal(size=(total_nodes, 3))


# ----------------------------------------------------------------------------------------------
# The five workloads (sizes and distributions as stated beside each).

def c1_spheres() -> Suspension:
    """8 unit spheres, centres uniform in [-6, 6]^3 (seed 0) with surface gap >= 0.5; p = 8 on a
    9 x 16 grid (144 nodes per sphere, 3,456 unknowns); F, T ~ N(0, 1)."""
    return spheres_in_box(8, 1.0, 6.0, 0.5, 8, 16, seed=0, name="c1_8_spheres_p8")


def c2_ellipsoids() -> Suspension:
    """1,000 ellipsoids, semi-axes U[0.6, 1.4], random orientation, ~10% volume fraction, gap 0.2,
    p = 12 on a 13 x 24 grid (312 nodes per particle, 936,000 unknowns); seed 1."""
    return random_ellipsoids(1000, 12, 24, 0.10, 0.2, seed=1, name="c2_1000_ellipsoids_p12")


def c3_ellipsoids() -> Suspension:
    """10,000 ellipsoids, ~15% volume fraction, gap 0.2, p = 8 on a 9 x 16 grid (1.44M nodes); seed 2."""
    return random_ellipsoids(10000, 8, 16, 0.15, 0.2, seed=2, name="c3_10000_ellipsoids_p8")


def c4_batched(max_suspensions: int = 256) -> Suspension:
    """256 independent suspensions, particle counts floor(exp U[ln 4, ln 513)), per-particle p drawn
    from {6, 8, 12, 16} with n_phi = 2p, each at ~10% volume fraction with gap 0.2; seed 3."""
    rng = np.random.default_rng(3)
    counts = np.floor(np.exp(rng.uniform(math.log(4), math.log(513), size=max_suspensions))).astype(int)
    parts = []
    for s, ns in enumerate(counts):
        sub = random_ellipsoids(int(ns), 8, None, 0.10, 0.2, seed=int(rng.integers(1 << 31)))
        sub.p = rng.choice(np.array([6, 8, 12, 16], np.int32), size=int(ns)).astype(np.int32)
        sub.nphi = (2 * sub.p).astype(np.int32)
        sub.suspension_id[:] = s
        parts.append(sub)
    cat = lambda f: np.concatenate([getattr(x, f) for x in parts])
    return Suspension(cat("semi_axes"), cat("p"), cat("nphi"), cat("centres"), cat("quats"), cat("F"),
                      cat("T"), cat("suspension_id"), "c4_batched_256")


def c5_sedimenting() -> Suspension:
    """2,048 ellipsoids, ~10% volume fraction, gap 0.2, p = 10 on an 11 x 22 grid (242 nodes per
    particle); sedimenting under F = (0, 0, -1), T = 0; seed 4."""
    s = random_ellipsoids(2048, 10, 22, 0.10, 0.2, seed=4, name="c5_2048_ellipsoids_p10")
    s.F = np.tile([0.0, 0.0, -1.0], (s.n, 1))
    s.T = np.zeros((s.n, 3))
    return s


def profile_ellipsoids() -> Suspension:
    """400 ellipsoids drawn like the 1,000-ellipsoid workload but at p = 8 (57,600 nodes, ~10% volume
    fraction, gap 0.2; seed 1): a case of the same kernels small enough for hardware-counter captures
    (about 2 GB on the device) that still fills every SM."""
    return random_ellipsoids(400, 8, 16, 0.10, 0.2, seed=1, name="profile_400_ellipsoids_p8")


def c3_profile() -> Suspension:
    """2,000 ellipsoids drawn like the 10,000-ellipsoid workload (~15% volume fraction, gap 0.2, p = 8
    on a 9 x 16 grid, 288,000 nodes; seed 2): a case of the same treecode kernels small enough for
    hardware-counter captures (pair sums of well under a second per launch)."""
    return random_ellipsoids(2000, 8, 16, 0.15, 0.2, seed=2, name="c3_profile_2000_ellipsoids_p8")


def shared_shape(n: int, p: int, seed: int, spacing: float = 2.6, jitter: float = 0.2,
                 axes=(1.0, 0.5, 0.5), name: str = "") -> Suspension:
    """n identical ellipsoids (semi-axes (1, 0.5, 0.5) by default, the shape of the paper's ellipsoid
    lattices, Section 4.2) on a cubic lattice of the given spacing, centres perturbed uniformly by up
    to `jitter` per axis and uniformly random orientations (seeded); n_phi = 2p; F, T ~ N(0, 1).  With
    the default spacing and jitter the bounding spheres keep a gap of at least 0.2."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil(n ** (1.0 / 3.0) - 1e-9))
    g = np.arange(m) * spacing
    cen = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)[:n]
    cen = cen - cen.mean(axis=0) + rng.uniform(-jitter, jitter, size=(n, 3))
    quats = random_quaternions(rng, n)
    F = rng.normal(size=(n, 3))
    T = rng.normal(size=(n, 3))
    return Suspension(np.tile(np.asarray(axes, np.float64), (n, 1)), np.full(n, p, np.int32),
                      np.full(n, 2 * p, np.int32), cen, quats, F, T, np.zeros(n, np.int32), name)


def s_shared() -> Suspension:
    """10,000 identical (1, 0.5, 0.5) ellipsoids on a perturbed cubic lattice (spacing 2.6, jitter 0.2,
    random orientations; seed 5) at p = 16 on a 17 x 32 grid (544 nodes per particle, 5.44M nodes): every
    particle shares one self block of 1,632 x 1,632, so the block applications form a GEMM."""
    return shared_shape(10000, 16, seed=5, name="s_shared_10000_ellipsoids_p16")


def c5_small() -> Suspension:
    """The sedimenting-ellipsoid workload at 256 particles (same distributions as the 2,048-particle
    one: p = 10 on an 11 x 22 grid, ~10% volume fraction, gap 0.2, F = (0, 0, -1), T = 0; seed 4),
    small enough to time tens of RK4 steps."""
    s = random_ellipsoids(256, 10, 22, 0.10, 0.2, seed=4, name="c5_256_ellipsoids_p10")
    s.F = np.tile([0.0, 0.0, -1.0], (s.n, 1))
    s.T = np.zeros((s.n, 3))
    return s


WORKLOADS = {
    "c1": c1_spheres,
    "profile": profile_ellipsoids,
    "c2": c2_ellipsoids,
    "c3": c3_ellipsoids,
    "c3_profile": c3_profile,
    "s_shared": s_shared,
    "c4": c4_batched,
    "c5": c5_sedimenting,
    "c5_small": c5_small,
}
