"""Oracle: the learned GMRES warm start (an addition to the method: the paper's GMRES of Section 3.2
starts from zero; any initial guess leaves the converged solution unchanged, only the iteration count
moves).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definitions shared with the CUDA path (stated here, implemented independently there):

* Features of particle i, 128 float values: F_i and T_i in the body frame (R_i^T F_i, R_i^T T_i), its
  semi-axes, then for each of its 16 nearest neighbours j (same suspension; by centre distance,
  ascending, ties to the lower index) the body-frame offset R_i^T (c_j - c_i) and the relative
  rotation conj(q_i) q_j as a quaternion with non-negative scalar part; absent neighbours and the
  tail (entries 121-127) are zero.
* Target of particle i: the real spherical-harmonic coefficients of its body-frame density
  R_i^T mu on its own grid, component-major [x | y | z], each in the order m = 0..m_max,
  n = m..p, cos then (m > 0) sin, with the orthonormal basis of Eq. 32 (no Condon-Shortley sign).
* Network: y = W3 g(W2 g(W1 x + b1) + b2) + b3, widths 128 -> 256 -> 256 -> 3 n_basis, g the GELU
  (tanh form); loss = mean squared error over particles and outputs.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import quat_to_rot
from .sphere_grid import analysis_matrix, legendre_normalized, mmax_for, real_sh

N_NEIGH = 16
N_FEAT = 128
HIDDEN = 256


def quat_conj_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """conj(a) * b for unit quaternions (w, x, y, z)."""
    w1, x1, y1, z1 = a[0], -a[1], -a[2], -a[3]
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def neighbours(centres: np.ndarray, suspension_id=None, k: int = N_NEIGH) -> list[list[int]]:
    """The k nearest other particles of each particle (same suspension), by brute force."""
    c = np.asarray(centres, float)
    n = len(c)
    sid = np.zeros(n, int) if suspension_id is None else np.asarray(suspension_id)
    out = []
    for i in range(n):
        d = np.linalg.norm(c - c[i], axis=1)
        cand = [j for j in range(n) if j != i and sid[j] == sid[i]]
        cand.sort(key=lambda j: (d[j], j))
        out.append(cand[:k])
    return out


def features(semi_axes, centres, quats, F, T, suspension_id=None) -> np.ndarray:
    """(n, 128) feature rows as defined in the module docstring."""
    axes = np.asarray(semi_axes, float).reshape(-1, 3)
    c = np.asarray(centres, float).reshape(-1, 3)
    q = np.asarray(quats, float).reshape(-1, 4)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    F = np.asarray(F, float).reshape(-1, 3)
    T = np.asarray(T, float).reshape(-1, 3)
    n = len(c)
    nb = neighbours(c, suspension_id)
    X = np.zeros((n, N_FEAT))
    for i in range(n):
        R = quat_to_rot(q[i])
        X[i, 0:3] = R.T @ F[i]
        X[i, 3:6] = R.T @ T[i]
        X[i, 6:9] = axes[i]
        for k, j in enumerate(nb[i]):
            rq = quat_conj_mul(q[i], q[j])
            if rq[0] < 0:
                rq = -rq
            X[i, 9 + 7 * k: 12 + 7 * k] = R.T @ (c[j] - c[i])
            X[i, 12 + 7 * k: 16 + 7 * k] = rq
    return X


def basis_permutation(p: int, nphi: int) -> np.ndarray:
    """Index into the oracle's real_sh rows (n-major) of each coefficient in the shared m-major order."""
    mmax = mmax_for(nphi)
    own = [(n, m) for n in range(p + 1) for m in range(-min(n, mmax), min(n, mmax) + 1)]
    pos = {nm: k for k, nm in enumerate(own)}
    order = []
    for m in range(0, mmax + 1):
        for n in range(m, p + 1):
            order.append(pos[(n, m)])
            if m > 0:
                order.append(pos[(n, -m)])
    return np.array(order)


def target_coefficients(system, mu: np.ndarray) -> np.ndarray:
    """(n, 3 n_basis) body-frame spherical-harmonic coefficients of mu per particle."""
    rows = []
    for i, pt in enumerate(system.particles):
        b = pt.body
        An = analysis_matrix(b.p, b.nphi)[basis_permutation(b.p, b.nphi)]
        mub = mu[system.sl(i)] @ pt.R          # rows: R^T mu_t
        rows.append((An @ mub).T.reshape(-1))  # [x | y | z]
    return np.array(rows)


def synthesize(system, coef: np.ndarray) -> np.ndarray:
    """Lab-frame surface density from per-particle body-frame coefficients (inverse of the above)."""
    out = np.zeros((system.total_nodes, 3))
    for i, pt in enumerate(system.particles):
        b = pt.body
        Y = real_sh(b.p, mmax_for(b.nphi), b.theta, b.phi)[basis_permutation(b.p, b.nphi)]
        nb = Y.shape[0]
        cb = coef[i].reshape(3, nb)
        out[system.sl(i)] = (cb @ Y).T @ pt.R.T
    return out


# ------------------------------------------------------------------------------------------- MLP

GELU_C = math.sqrt(2.0 / math.pi)


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(GELU_C * (x + 0.044715 * x ** 3)))


def gelu_grad(x):
    u = GELU_C * (x + 0.044715 * x ** 3)
    t = np.tanh(u)
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_C * (1.0 + 3 * 0.044715 * x * x)


def init_params(n_out: int, seed: int = 0):
    """He-style initial weights (the seeded draw both sides may load)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(size=(N_FEAT, HIDDEN)) * math.sqrt(2.0 / N_FEAT)
    W2 = rng.normal(size=(HIDDEN, HIDDEN)) * math.sqrt(2.0 / HIDDEN)
    W3 = rng.normal(size=(HIDDEN, n_out)) * math.sqrt(1.0 / HIDDEN)
    return {"W1": W1, "b1": np.zeros(HIDDEN), "W2": W2, "b2": np.zeros(HIDDEN), "W3": W3, "b3": np.zeros(n_out)}


def forward(params, X):
    """Returns the output and the cache of pre-activations."""
    z1 = X @ params["W1"] + params["b1"]
    h1 = gelu(z1)
    z2 = h1 @ params["W2"] + params["b2"]
    h2 = gelu(z2)
    y = h2 @ params["W3"] + params["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_and_grads(params, X, Y):
    """Mean squared error over all entries and its gradients (reverse-mode, written out)."""
    y, (X, z1, h1, z2, h2) = forward(params, X)
    diff = y - Y
    L = float(np.mean(diff ** 2))
    dy = 2.0 * diff / diff.size
    g = {"W3": h2.T @ dy, "b3": dy.sum(0)}
    dh2 = dy @ params["W3"].T
    dz2 = dh2 * gelu_grad(z2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ params["W2"].T
    dz1 = dh1 * gelu_grad(z1)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return L, g


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) in place; state holds m, v and the step count."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = b1 * m + (1 - b1) * grads[k]
        v[...] = b2 * v + (1 - b2) * grads[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        params[k] -= lr * mh / (np.sqrt(vh) + eps)
