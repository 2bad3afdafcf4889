"""Seeded coefficient surfaces for the tests of general particle shapes (Section 3, Eq. 31).

`star_shape` is a smooth star-shaped genus-0 surface: the ellipsoid (1.2, 0.8, 0.7) scaled radially by
1 + 0.08 (random degree-2 and degree-3 harmonics), x = r(s) D s.  Its coordinate functions have degree
<= 4, so their coefficients in the library's basis order are taken exactly by a Gauss-Legendre x
trapezoid projection on a (5 x 10) grid.  Returns (coef (3, 25), 4)."""
import math

import numpy as np

from oracle import shapes as shp


def star_shape(seed=0, pg=4, axes=(1.2, 0.8, 0.7), amplitude=0.08):
    rng = np.random.default_rng(seed)
    amp = amplitude * rng.normal(size=shp.n_coef(3))
    amp[:4] = 0.0                       # no degree-0 or degree-1 part in the radial factor
    nth, nph = pg + 1, 2 * pg + 2
    t, lam = np.polynomial.legendre.leggauss(nth)
    th = np.repeat(np.arccos(t), nph)
    ph = np.tile(2 * math.pi * np.arange(nph) / nph, nth)
    q = np.repeat(lam, nph) * 2 * math.pi / nph
    s = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)
    Y3, _, _ = shp.basis_with_derivatives(3, th, ph)
    r = 1.0 + amp @ Y3
    x = r[:, None] * s * np.asarray(axes, float)[None, :]
    Y, _, _ = shp.basis_with_derivatives(pg, th, ph)
    return ((Y * q[None, :]) @ x).T.copy(), pg
