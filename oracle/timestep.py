"""Oracle: rigid-body time stepping (Section 3.3, Eqs. 40 and 43; Algorithm 1 without contact).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Each particle's state is its centre c_i and unit quaternion q_i (scalar first); the body-frame surface
never changes (Eq. 40), so the discrete self blocks rotate with R(q_i) (Eq. 38).  The ODEs of Eq. 43
are dc/dt = v and dR/dt = M(omega) R, written for the quaternion as dq/dt = 1/2 (0, omega) q (Hamilton
product).  Explicit Runge-Kutta schemes: forward Euler, the trapezoidal rule (Heun) and classical RK4;
the quaternion is renormalised after each step.  Forces and torques are held fixed over the run.
"""
from __future__ import annotations

import numpy as np

from .system import Options, System


def quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Hamilton product of quaternions (w, x, y, z), row-wise."""
    w1, x1, y1, z1 = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    w2, x2, y2, z2 = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=-1)


def rates(semi_axes, p, nphi, centres, quats, F, T, options=None, suspension_id=None):
    """(dc/dt, dq/dt) of every particle: one mobility solve (dense LU) at the given configuration."""
    s = System(semi_axes, p, nphi, centres, quats, suspension_id, options or Options())
    v, om, *_ = s.solve(F, T)
    q = np.asarray(quats, float)
    qdot = 0.5 * quat_mul(np.concatenate([np.zeros((len(om), 1)), om], axis=1), q)
    return v, qdot


SCHEMES = {
    "euler": ([[]], [1.0]),
    "trapezoid": ([[], [1.0]], [0.5, 0.5]),
    "rk4": ([[], [0.5], [0.0, 0.5], [0.0, 0.0, 1.0]], [1 / 6, 1 / 3, 1 / 3, 1 / 6]),
}


def advance(semi_axes, p, nphi, centres, quats, F, T, dt: float, steps: int, scheme: str = "rk4",
            options=None, suspension_id=None):
    """Explicit Runge-Kutta steps of the rigid-body ODEs; returns the final (centres, quats)."""
    A, b = SCHEMES[scheme]
    c = np.array(centres, float)
    q = np.array(quats, float)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    for _ in range(steps):
        kc, kq = [], []
        for stage in range(len(b)):
            cs = c + dt * sum(a * k for a, k in zip(A[stage], kc)) if stage else c
            qs = q + dt * sum(a * k for a, k in zip(A[stage], kq)) if stage else q
            dc, dq = rates(semi_axes, p, nphi, cs, qs, F, T, options, suspension_id)
            kc.append(dc)
            kq.append(dq)
        c = c + dt * sum(bi * k for bi, k in zip(b, kc))
        q = q + dt * sum(bi * k for bi, k in zip(b, kq))
        q /= np.linalg.norm(q, axis=1, keepdims=True)
    return c, q
