"""Host-side parts of bench.py that need no GPU: the float64 oracle sampled on several spawned
processes at once (the CPU baseline on every host core) and the workload subset used to extrapolate
the plain float64 solve."""
import numpy as np

import suspensions


def test_oracle_sampler_runs_on_several_processes():
    import bench
    s = suspensions.c1_spheres()
    sampler = bench.OracleSampler(s, 2)
    try:
        v2, sample2, wall2 = sampler.sample(0.5, 10)
        v1, sample1, wall1 = sampler.sample(0.5, 10, procs=1)
    finally:
        sampler.close()
    assert v2 > 0 and v1 > 0
    assert "on 2 processes" in sample2 and "on 1 processes" in sample1
    # one solve = (10 + 3) operator applications of 1,152 rows each
    assert "10 GMRES + 3" in sample2


def test_workload_subset_keeps_the_first_particles():
    import bench
    s = suspensions.c1_spheres()
    sub = bench.subset(s, 3)
    assert sub.n == 3
    assert np.array_equal(sub.centres, s.centres[:3]) and np.array_equal(sub.p, s.p[:3])
    assert sub.total_nodes == 3 * 144
