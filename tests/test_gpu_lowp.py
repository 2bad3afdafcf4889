"""Self blocks in 16 bits (RBS_PREC_MIXED_FP16 / RBS_PREC_MIXED_BF16).

The inner solve may apply the self blocks (Section 3.1: computed once per shape in the body frame and
rotated per particle, Eq. 38) in float16 or bfloat16 with float32 accumulation: on the tensor cores
(a GEMM over the particles of a shared shape) or on CUDA cores (distinct shapes).  Their error is
bounded by the rounding of the stored entries and, on the tensor cores, of the body-frame input: each
row of A z is off by at most 2 u sum_k |A_mk| |z_k| (u the unit roundoff, 2^-12 for float16 and 2^-9
for bfloat16; float32 accumulation adds far less), so the error of K_SELF x is at most 2 u || |A| |z| ||
over all particles, computed here with the oracle's float64 body-frame blocks.  The refinement around
the inner solve must still reach the float64 solution: mixed solves agree with the oracle's LU.
"""
import numpy as np
import pytest

import oracle
import suspensions

pytestmark = pytest.mark.gpu

UNIT = {"FP16": 2.0 ** -12, "BF16": 2.0 ** -9}


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    return m


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def cases():
    """distinct: 7 ellipsoids of their own shapes at p = 6 (CUDA-core path; 252-entry rows, copied in
    4-byte pieces); distinct_p8: 4 at p = 8 (432-entry rows, 16-byte aligned: 16-byte copies);
    shared_p4 / shared_p8: 72 and 130 identical ellipsoids (tensor-core path; one and two 128-particle
    tiles, 120 and 432 block rows)."""
    return {
        "distinct": suspensions.random_ellipsoids(7, 6, 12, 0.12, 0.2, seed=71),
        "distinct_p8": suspensions.random_ellipsoids(4, 8, 16, 0.12, 0.2, seed=74),
        "shared_p4": suspensions.shared_shape(72, 4, seed=72),
        "shared_p8": suspensions.shared_shape(130, 8, seed=73),
    }


CASES = cases()


def rounding_bound(ref, x):
    """|| |A0| |R^T x_i| || over the particles, with the oracle's float64 body-frame K blocks."""
    acc = 0.0
    for i, pt in enumerate(ref.particles):
        A0 = ref.self_block_body("K", i)
        z = (x[ref.sl(i)] @ pt.R).reshape(-1)  # rows z_t = R^T x_t
        acc += float(np.sum((np.abs(A0) @ np.abs(z)) ** 2))
    return np.sqrt(acc)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["FP16", "BF16"])
def test_16bit_self_blocks_within_rounding_bound(rbs, prec, case):
    s = CASES[case]
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    x = suspensions.random_density(81, s.total_nodes)
    y_ref = np.zeros_like(x)
    for i in range(s.n):
        y_ref[ref.sl(i)] = (ref.self_block_lab("K", i) @ x[ref.sl(i)].reshape(-1)).reshape(-1, 3)
    with rbs.Context(device=0, precision=getattr(rbs, "RBS_PREC_MIXED_" + prec)) as ctx:
        ctx.set_suspension(s)
        y = rbs.rbs_apply_operator(ctx.ctx, rbs.RBS_OP_K_SELF, getattr(rbs, "RBS_PREC_MIXED_" + prec), x)
        y32 = rbs.rbs_apply_operator(ctx.ctx, rbs.RBS_OP_K_SELF, rbs.RBS_PREC_MIXED, x)
    err = np.linalg.norm(y - y_ref)
    bound = 2.0 * UNIT[prec] * rounding_bound(ref, x)
    assert err <= bound, (err, bound)
    # it is 16-bit arithmetic, not a float32 path: clearly less accurate than float32 blocks
    assert err > 10.0 * np.linalg.norm(y32 - y_ref)
    if prec == "FP16":  # float16 keeps three more bits than bfloat16
        assert err <= 0.25 * 2.0 * UNIT["BF16"] * rounding_bound(ref, x)


@pytest.mark.parametrize("case", ["distinct", "shared_p4"])
@pytest.mark.parametrize("prec", ["FP16", "BF16"])
def test_16bit_mixed_solve_matches_oracle(rbs, prec, case):
    s = CASES[case]
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    vr, omr, _, _, _ = ref.solve(s.F, s.T, method="lu")
    with rbs.Context(device=0, precision=getattr(rbs, "RBS_PREC_MIXED_" + prec)) as ctx:
        ctx.set_suspension(s)
        v, om, _, its = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-10)
        st = rbs.rbs_get_stats(ctx.ctx)
    assert rel(np.concatenate([v, om]), np.concatenate([vr, omr])) < 1e-8
    assert st["residual"] <= 1e-10
