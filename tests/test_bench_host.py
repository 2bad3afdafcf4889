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


def test_roofline_fractions_reproduce_by_hand():
    """The fractions of the bench line follow from the algorithmic work: 57 flops per fused
    double-float pair and 29 per float32 traction pair against 152 x 128 x 2 x f, bytes of stored
    float32 block entries against the HBM copy bandwidth, 16 flops per stored float64 block entry
    against 152 x 2 x 2 x f."""
    import bench
    f_mhz, hbm = 2070.0, 6786.2
    fp32 = 152 * 128 * 2 * f_mhz * 1e6
    kernels = {
        # per-launch figures of the 10,000-ellipsoid bench line: 5.48e11 pairs in 5,062 ms
        "pair_both_df": {"ms": 5062.29, "launches": 1, "units": 5.47688915712e11},
        "pair_traction_f32": {"ms": 192.05, "launches": 1, "units": 2.02985445888e11},
        "particle_blocks": {"ms": 0.3512, "launches": 1, "units": 1.296e9},
        "gmres_graph": {"ms": 4195.9, "launches": 2, "units": 21.0},
    }
    roof = bench.kernel_rooflines(kernels, f_mhz, hbm)
    df = roof["pair_both_df"]
    assert abs(df["frac"] - 57 * 5.47688915712e11 / 5.06229 / fp32) < 1e-9
    assert 0.07 < df["frac"] < 0.085  # 6.17 TFLOP/s of 80.5
    assert abs(df["issue_efficiency"] - 248 * 5.47688915712e11 / 5.06229 / (152 * 128 * f_mhz * 1e6)) < 1e-9
    assert abs(roof["pair_traction_f32"]["frac"] - 29 * 2.02985445888e11 / 0.19205 / fp32) < 1e-9
    blk = roof["particle_blocks"]
    assert blk["bound"] == "hbm" and abs(blk["frac"] - 1.296e9 / 0.3512e-3 / 1e9 / hbm) < 1e-12
    assert 0.5 < blk["frac"] < 0.6
    assert abs(roof["gmres_graph"]["ms_per_step"] - 4195.9 / 21.0) < 1e-9
    # five solves' float64 block launches of that bench line: 15 applies of the K blocks (10,000
    # particles x 75 stored rows x 432 float64 entries each) and 5 of the L term alone (no entries)
    e = {"ms": 77.0766, "launches": 20, "units": 15 * 10000 * 75 * 432 * 8.0}
    f64 = bench.block_f64_roofline(e, f_mhz)
    assert abs(f64["frac"] - 16 * 15 * 3.24e8 / 77.0766e-3 / (152 * 2 * 2 * f_mhz * 1e6)) < 1e-9
    assert f64["bound"] == "fp64" and 0.75 < f64["frac"] < 0.85
    assert abs(f64["ms_per_launch"] - 77.0766 / 20) < 1e-12
