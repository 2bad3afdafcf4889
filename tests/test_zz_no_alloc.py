"""The allocation-free rigid-velocity entry point (rbs_rigid_velocities_noalloc).

Callers that may not allocate device memory at call time (for example frameworks that reserve nearly
all device memory for their own pool, or real-time loops that forbid allocator calls) use this
variant; it keeps its intermediate in a fixed device array instead of a context buffer.  This file
runs last so that a failure here does not hide the other GPU tests.  Results must equal those of
rbs_rigid_velocities, the existing entry point, to the tolerance the other rigid-velocity tests use
(1e-13), on two calls in a row (the second call reuses the array the first one filled); the second
call must leave the device's free memory unchanged.
"""
import numpy as np
import pytest

import suspensions

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()
    from paper_1606_07428_gb300 import rbs as m
    return m


def test_noalloc_matches_rigid_velocities_on_two_calls(rbs):
    import torch
    s = suspensions.random_ellipsoids(9, 6, 12, 0.08, 0.2, seed=31)
    with rbs.Context(device=0) as ctx:
        ctx.set_suspension(s)
        for seed in (41, 42):
            u = suspensions.random_density(seed, s.total_nodes)
            v_ref, om_ref = rbs.rbs_rigid_velocities(ctx.ctx, u, s.n)
            u_dev = torch.tensor(u, device="cuda")
            v_dev = torch.full((s.n, 3), float("nan"), dtype=torch.float64, device="cuda")
            om_dev = torch.full((s.n, 3), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info(0)[0]
            rbs.rbs_rigid_velocities_noalloc(ctx.ctx, u_dev, v_dev, om_dev)
            torch.cuda.synchronize()
            if seed == 42:  # the first call may load the kernels; the second allocates nothing at all
                assert torch.cuda.mem_get_info(0)[0] == free_before
            assert torch.cuda.current_device() == 0
            assert rel(v_dev.cpu().numpy(), v_ref) < 1e-13
            assert rel(om_dev.cpu().numpy(), om_ref) < 1e-13


def test_noalloc_rejects_more_particles_than_its_scratch_holds(rbs):
    import torch
    m = 41  # 41^3 = 68,921 spheres > 65,536
    g = np.arange(m, dtype=np.float64)
    cen = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = len(cen)
    with rbs.Context(device=0, near_delta=0.0, restart=2) as ctx:
        ctx.set_geometry(np.full((n, 3), 0.3), 2, 4, cen, np.tile([1.0, 0, 0, 0], (n, 1)))
        N = rbs.rbs_total_nodes(ctx.ctx)
        u = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
        v = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        with pytest.raises(rbs.RbsError) as e:
            rbs.rbs_rigid_velocities_noalloc(ctx.ctx, u, v, v.clone())
        assert e.value.code == rbs.RBS_EINVAL and "65536" in str(e.value)
