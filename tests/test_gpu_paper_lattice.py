"""GMRES iteration counts on the paper's lattice set-up (tests/golden/paper_gmres_iterations.json),
a soft pin of the preconditioned second-kind system: the paper reports 4-5 iterations to 1e-6 for
sphere lattices and 5-6 for ellipsoid lattices (Section 4.2)."""
import json
import os

import numpy as np
import pytest

import suspensions

pytestmark = pytest.mark.gpu
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_gmres_iterations.json")))


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    return m


@pytest.mark.parametrize("nz,p", [(8, 8), (16, 8), (8, 16)])
def test_sphere_lattice_iterations(rbs, nz, p):
    s = suspensions.sphere_lattice(nz, p)
    lo, hi = GOLDEN["reported_iterations"]["unit_spheres"]
    with rbs.Context(device=0) as ctx:
        ctx.set_suspension(s)
        _, _, _, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-6)
    assert lo - 2 <= its <= hi + 2, its


@pytest.mark.parametrize("axes", [(1.0, 0.5, 0.5), (1.0, 1.0, 0.5)])
def test_ellipsoid_lattice_iterations(rbs, axes):
    s = suspensions.sphere_lattice(8, 8)
    s.semi_axes = np.tile(axes, (s.n, 1))
    lo, hi = GOLDEN["reported_iterations"]["ellipsoids_1_05_05_and_1_1_05"]
    with rbs.Context(device=0) as ctx:
        ctx.set_suspension(s)
        _, _, _, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-6)
    assert lo - 2 <= its <= hi + 2, its
