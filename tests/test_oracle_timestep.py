"""Pins of the oracle's rigid-body time stepping (Section 3.3, Eqs. 40 and 43): the exact motion of a
single sphere under constant force and torque, and the convergence orders of the explicit schemes the
paper uses (forward Euler 1, trapezoidal 2, RK4 4; Tables 4-5 report about 2 and 4 per halving of dt)."""
import math

import numpy as np
import pytest

from oracle import timestep


def test_single_sphere_moves_exactly():
    a = 1.2
    F = np.array([[0.4, -0.2, 0.9]])
    T = np.array([[0.0, 0.0, 3.0]])
    q0 = np.array([[1.0, 0.0, 0.0, 0.0]])
    t_end = 1.0
    c, q = timestep.advance([[a, a, a]], 4, 8, [[0.0, 0.0, 0.0]], q0, F, T, 0.1, 10, "rk4")
    assert np.allclose(c, F * t_end / (6 * math.pi * a), atol=1e-13)
    wz = 3.0 / (8 * math.pi * a ** 3)
    q_exact = np.array([[math.cos(wz * t_end / 2), 0.0, 0.0, math.sin(wz * t_end / 2)]])
    assert np.abs(q - q_exact).max() < 1e-9


@pytest.mark.slow
@pytest.mark.parametrize("scheme,order", [("euler", 1), ("trapezoid", 2), ("rk4", 4)])
def test_scheme_orders_on_two_ellipsoids(scheme, order):
    axes = [[1.0, 0.6, 0.5], [0.8, 0.8, 0.5]]
    cen = [[0.0, 0.0, 0.0], [2.6, 0.3, 0.2]]
    qs = [[0.9, 0.1, 0.3, -0.2], [0.7, -0.4, 0.2, 0.5]]
    F = np.array([[0.0, 0.0, -1.0], [0.5, 0.0, -1.0]])
    T = np.array([[0.3, 0.0, 0.0], [0.0, -0.4, 0.2]])
    t_end = 0.8
    res = []
    for m in (2, 4, 8, 16):
        c, q = timestep.advance(axes, 4, 8, cen, qs, F, T, t_end / m, m, scheme)
        res.append(np.concatenate([c.ravel(), q.ravel()]))
    e1 = np.abs(res[1] - res[0]).max()
    e2 = np.abs(res[2] - res[1]).max()
    e3 = np.abs(res[3] - res[2]).max()
    rate = math.log2(e2 / e3)
    assert abs(rate - order) < 0.35 and e3 < e1
