"""Benchmark of the rigid-particle mobility solve on GB300.

One step = one complete mobility solve (forces and torques in, velocities out) of the chosen
arithmetic (float32 inner GMRES with float64 refinement, double-float right-hand side, residuals and
velocity) on a fixed suspension, for a fresh seeded (F, T) draw resident in device memory.  The
default workload is the metric's: 10,000 triaxial ellipsoids at p = 8 (1.44M nodes, 4.32M unknowns,
~15% volume fraction), at the largest GMRES tolerance in {1e-8, 1e-9, 1e-10} whose (v, omega) error
against a 1e-12 solve is <= 1e-8 (in practice 1e-8), with treecodes for the float32 inner applies and
the double-float passes.

The JSON line carries: device-timed solves/s (value), the same through the host-buffer C ABI call
(e2e), the plain float64 solve rate extrapolated from timed float64 operator applications, the error of
the chosen path against a 1e-12 solve, Stokeslet and traction pair rates, the dominant kernel's
roofline (its algorithmic flops over its device time from the library's CUDA events on its stream,
against the float32 FMA peak at the sampled clock), SM clocks sampled during the timed region, and the
float64 CPU oracle timed on a bounded sample on every host core and on one (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload c3]
Under torchrun each rank solves its own draws on its own GPU (independent replicas, weak scaling);
rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import suspensions  # noqa: E402

METRIC = "mobility solves/s at 1e-8 rel. error (chosen vs plain FP64); Stokeslet Gpair/s"
SMS = 152
L2_BYTES = 129 * 2 ** 20
FP64_DFMA_PER_CLK_SM = 2     # float64 FMA lanes per SM per clock (measured 1.19 TFLOP/s at 2.07 GHz)
FP32_LANES_PER_SM = 128
# algorithmic work per node pair (minimal float32 flops with FMA = 2): traction 29 (20 FMA-pipe
# instructions + 1 MUFU), Stokeslet 28 (18 + 1 MUFU); the fused double-float pass evaluates both (57);
# float64 operations per pair (the float64 reciprocal square root counted as 7): traction 27, Stokeslet 25
FLOPS_PER_PAIR = {"traction": 29.0, "stokeslet": 28.0, "both": 57.0}
FP64_OPS_PER_PAIR = {"traction": 27.0, "stokeslet": 25.0}
# DRAM bytes per launch from ncu captures of the direct kernels on the 400-ellipsoid profiling case
# (57,600 nodes), scaled by node count to the benchmarked case: the pair kernels read their inputs
# once (sources are re-read from L2), so traffic grows with N, not with the N^2 pairs
NCU_TRAFFIC = {"pair_traction_df": (6.404864e6, 57600), "pair_traction_f32": (4.872192e6, 57600),
               "pair_both_df": (8.511744e6, 57600)}
# float32-pipe operations per pair the double-float kernels issue, counted from the source of
# pair2_df (separation 24, r^2 28, reciprocal square root 8, r . density 28, powers 8, then the
# traction tail 76, the Stokeslet tail 76, or both tails sharing 1/r^5 and r . n: 152): the issue
# efficiency of a double-float kernel is measured against this count, its roofline against the flops
DF_INSTR_PER_PAIR = {"traction": 172.0, "stokeslet": 172.0, "both": 248.0}
# DRAM bytes per launch of the fused double-float treecode kernel from an ncu capture on the
# 2,000-ellipsoid profiling case (288,000 nodes; 83.27 MB read + 6.95 MB written, theta 0.45, degree 11,
# one target per thread), scaled by node count like the direct kernels' figures
TREE_DF_TRAFFIC = (9.0224640e7, 288000)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(suspensions.WORKLOADS))
    ap.add_argument("--tol", type=float, default=None,
                    help="GMRES tolerance; default: the largest of 1e-8, 1e-9, 1e-10 whose (v, omega) error "
                         "against a 1e-12 reference solve is <= 1e-8")
    ap.add_argument("--no-error-check", action="store_true",
                    help="skip the 1e-12 reference solve (and so error_vs_reference), for launch-list captures "
                         "whose kernel shares should be the timed solves'; needs --tol")
    ap.add_argument("--fp64-steps", type=int, default=0, help="timed plain float64 solves (0: extrapolate)")
    ap.add_argument("--fp64-subset", type=int, default=1500,
                    help="particles of the workload whose float64 operator applications are timed to extrapolate "
                         "the plain float64 solve when --fp64-steps is 0 (0 skips)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle CPU sample")
    ap.add_argument("--cpu-procs", type=int, default=0, help="oracle sample processes (0: every host core)")
    ap.add_argument("--pair-variant", type=int, default=0,
                    help="pair-kernel variant (rbs_options.pair_variant); 0 lets the library's autotuner choose")
    ap.add_argument("--far-field", default="tree-df", choices=["direct", "tree", "tree-df"],
                    help="direct sums over all node pairs; tree: the treecode for the float32 inner applies "
                         "(double-float passes stay direct); tree-df: treecodes for both "
                         "(rbs_options.far_field)")
    ap.add_argument("--tree-df-theta", type=float, default=0.45,
                    help="opening angle of the double-float passes' treecode (rbs_options.tree_df_theta) with "
                         "--far-field tree-df")
    ap.add_argument("--tree-df-degree", type=int, default=11,
                    help="its interpolation degree (rbs_options.tree_df_degree).  Relative error of the far "
                         "traction sum on the 10,000-ellipsoid geometry (float64 treecode against the exact "
                         "sum at six particles) and pairs per apply: theta 0.45 / degree 11: 1.0e-9, 5.5e11; "
                         "0.45 / 12: 1.6e-10, 6.6e11; 0.4 / 10: 1.2e-9, 5.6e11; 0.5 / 12: 3.0e-9, 5.5e11; "
                         "0.5 / 11: 1.1e-8, 4.5e11")
    ap.add_argument("--experiment", default=None, choices=[None, "warmstart", "magnetic", "selfgemm"],
                    help="warmstart: learned vs previous-step vs zero initial guesses in RK4 sedimentation; "
                         "magnetic: time steps of paramagnetic spheres in a uniform field (each prints its own "
                         "JSON line; the default run is the benchmark above)")
    ap.add_argument("--solves", type=int, default=1,
                    help="selfgemm experiment: mobility solves per arithmetic after the operator timings (0 skips)")
    ap.add_argument("--warm-modes", default="ZERO,PREVIOUS,LEARNED,LEARNED_DELTA",
                    help="warmstart experiment: initial guesses compared (RBS_WARM_* names)")
    ap.add_argument("--train-steps", type=int, default=10)
    ap.add_argument("--eval-steps", type=int, default=10)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--dt", type=float, default=0.05)
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------- ranks

def reduce_max(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (one all-reduce; identity on one rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time (weak scaling of replicas)."""
    return units_per_rank * world / (max_ms / 1e3)


# ---------------------------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = [r for r in csv.reader(open(self.file.name)) if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------- CPU oracle

_ORACLE = None


def _oracle_worker_init(arrays):
    """Worker set-up (spawned process, one thread): the oracle's system for the workload's arrays."""
    global _ORACLE
    import oracle
    semi_axes, p, nphi, centres, quats, sid = arrays
    _ORACLE = (oracle.System(semi_axes, p, nphi, centres, quats, sid), int((p + 1) @ nphi))


def _oracle_rows(args):
    """Rows of the float64 system operator (1/2 I + K + L) at seeded random nodes for budget seconds:
    returns (rows, seconds)."""
    seed, budget = args
    ref, total = _ORACLE
    mu = suspensions.random_density(9, total)
    rng = np.random.default_rng([seed, 11])
    rows = 0
    t0 = time.perf_counter()
    while True:
        ref.apply_rows("K", mu, [int(rng.integers(total))], half=0.5, with_L=True)
        rows += 1
        el = time.perf_counter() - t0
        if el > budget or rows >= 4096:
            return rows, el


class OracleSampler:
    """The float64 oracle timed on a bounded sample of the workload: rows of the system operator at
    random nodes, each computed in full (every source particle, the near upsampling and a singular-rule
    row), on `procs` spawned single-threaded processes at once (all host cores by default).  One solve
    is extrapolated as (iterations + 3) operator applications."""

    def __init__(self, susp, procs: int):
        import multiprocessing as mp
        self.susp = susp
        self.procs = procs
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        arrays = (susp.semi_axes, susp.p, susp.nphi, susp.centres, susp.quats, susp.suspension_id)
        t0 = time.perf_counter()
        self.pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_worker_init, initargs=(arrays,))
        self.pool.map(_oracle_rows, [(k, 0.0) for k in range(procs)])  # every worker has built its system
        self.setup_s = time.perf_counter() - t0
        self.draw = 0

    def sample(self, budget_s: float, iterations: int, procs: int | None = None):
        procs = procs or self.procs
        t0 = time.perf_counter()
        out = self.pool.map(_oracle_rows, [(1000 * self.draw + k, budget_s) for k in range(procs)], chunksize=1)
        wall = time.perf_counter() - t0
        self.draw += 1
        rows = sum(r for r, _ in out)
        per_row = wall / rows  # wall time per row with `procs` processes at work
        solve_s = per_row * self.susp.total_nodes * (iterations + 3)
        sample = (f"{rows} rows of the float64 operator at random nodes of the {self.susp.name} workload on "
                  f"{procs} processes ({wall:.1f} s wall, {per_row * 1e3:.1f} ms per row aggregate; oracle "
                  f"set-up {self.setup_s:.1f} s excluded); one solve extrapolated as {iterations} GMRES + 3 "
                  f"operator applications")
        return 1.0 / solve_s, sample, wall

    def close(self):
        self.pool.terminate()
        self.pool.join()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    susp = suspensions.WORKLOADS[args.workload]()
    iters = 21  # the chosen path's GMRES iterations at this workload (its bench line reports them)
    procs = args.cpu_procs or host_cores()
    sampler = OracleSampler(susp, procs)
    per_step = max(2.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    vals = []
    sample = ""
    for k in range(args.warmup + args.steps):
        v, sample, _ = sampler.sample(per_step, iters)
        if k >= args.warmup:
            vals.append(v)
    sampler.close()
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": susp.name, "n_particles": susp.n, "p": int(susp.p[0]), "nodes": susp.total_nodes,
                       "unknowns": 3 * susp.total_nodes, "tol": args.tol or 1e-8},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": procs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------- our arm

def pair_kind(name: str) -> str:
    return "traction" if "traction" in name else ("both" if "both" in name else "stokeslet")


def kernel_rooflines(kernels, f_mhz, hbm_gbs):
    """Achieved rate of every timed kernel class against the roofline that bounds it: the float32 FMA
    peak (algorithmic flops per pair) for float32 and double-float pair sums, with the issue efficiency
    of the double-float kernels beside it; the float64 FMA rate for float64 pair sums; HBM bandwidth
    for the particle-block kernel (bytes of block entries)."""
    f = f_mhz * 1e6
    fp32 = SMS * FP32_LANES_PER_SM * 2 * f
    out = {}
    for name, e in kernels.items():
        if e["ms"] <= 0 or not e["launches"]:
            continue
        rate = e["units"] / (e["ms"] / 1e3)
        row = {"ms_per_launch": e["ms"] / e["launches"]}
        if name.startswith("pair_"):
            kind = pair_kind(name)
            row["achieved_gpair_s"] = rate / 1e9
            if name.endswith("_f32") or name.endswith("_df"):
                tf = rate * FLOPS_PER_PAIR[kind]
                row.update({"achieved_tflops": tf / 1e12, "peak_tflops": fp32 / 1e12, "frac": tf / fp32,
                            "bound": "alu"})
                if name.endswith("_df"):
                    row["issue_efficiency"] = rate * DF_INSTR_PER_PAIR[kind] / (SMS * FP32_LANES_PER_SM * f)
            else:
                peak = SMS * FP64_DFMA_PER_CLK_SM * f / FP64_OPS_PER_PAIR[kind]
                row.update({"peak_gpair_s": peak / 1e9, "frac": rate / peak, "bound": "alu"})
        elif name == "particle_blocks":
            row.update({"achieved_gb_s": rate / 1e9, "peak_gb_s": hbm_gbs, "frac": rate / 1e9 / hbm_gbs,
                        "bound": "hbm"})
        elif name == "gmres_graph":
            row = {"ms_per_launch": e["ms"] / e["launches"], "arnoldi_steps": e["units"],
                   "ms_per_step": e["ms"] / max(1.0, e["units"])}
        else:
            row["achieved_gpair_s"] = rate / 1e9
        out[name] = row
    return out


def block_f64_roofline(e, f_mhz):
    """The particle-block kernel's float64 launches (RBS_KC_BLOCKS_F64; units = bytes of float64 entries)
    against the float64 FMA peak: each stored entry is multiplied with the input of all 8 reflections,
    16 flops per entry."""
    flops = 16.0 * e["units"] / 8.0
    fp64 = SMS * FP64_DFMA_PER_CLK_SM * 2 * f_mhz * 1e6
    rate = flops / (e["ms"] / 1e3)
    return {"ms_per_launch": e["ms"] / e["launches"], "launches": e["launches"], "achieved_tflops": rate / 1e12,
            "peak_tflops": fp64 / 1e12, "frac": rate / fp64, "bound": "fp64",
            "basis": "float64 block applies of the double-float passes (with the L-only applies): 16 flops per "
                     "stored entry against 152 SMs x 2 float64 FMA per clock"}


def kernel_table(stats):
    from paper_1606_07428_gb300 import rbs
    out = {}
    for k, name in enumerate(rbs.KERNEL_CLASSES):
        if stats["kernel_count"][k]:
            out[name] = {"ms": stats["kernel_ms"][k], "launches": stats["kernel_count"][k],
                         "units": stats["kernel_units"][k]}
    return out


def subset(susp, count: int):
    """The first `count` particles of a suspension (the same draws, placed first)."""
    k = min(count, susp.n)
    return suspensions.Suspension(susp.semi_axes[:k], susp.p[:k], susp.nphi[:k], susp.centres[:k], susp.quats[:k],
                                  susp.F[:k], susp.T[:k], susp.suspension_id[:k], f"{susp.name}_first{k}")


def plain_fp64_extrapolated(rbs, susp, args, iterations, stream, local):
    """The plain float64 solve (float64 everything, same preconditioner, zero start) extrapolated from
    timed float64 operator applications on the first fp64_subset particles of the workload: the
    per-pair rates of the float64 traction and Stokeslet sums and the per-unit times of the particle
    blocks and the near correction, scaled to the workload's pairs, nodes and near units; one solve =
    (iterations + 3) applications of A plus one of S."""
    import torch
    sub = subset(susp, args.fp64_subset)
    with rbs.Context(device=local, precision=rbs.RBS_PREC_FP64, timing=1, stream=stream.cuda_stream) as c64:
        c64.set_suspension(sub)
        x = torch.tensor(suspensions.random_density(5, sub.total_nodes), device="cuda")
        y = torch.zeros_like(x)
        rbs.rbs_apply_operator_device(c64.ctx, rbs.RBS_OP_A, rbs.RBS_PREC_FP64, x, y)  # warm
        rbs.rbs_reset_stats(c64.ctx)
        for op in (rbs.RBS_OP_A, rbs.RBS_OP_S):
            rbs.rbs_apply_operator_device(c64.ctx, op, rbs.RBS_PREC_FP64, x, y)
        torch.cuda.synchronize()
        st = rbs.rbs_get_stats(c64.ctx)
    return kernel_table(st), sub, st


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1606_07428_gb300 import rbs

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    susp = suspensions.WORKLOADS[args.workload]()
    n = susp.n
    stream = torch.cuda.current_stream()
    far = {"direct": rbs.RBS_FAR_DIRECT, "tree": rbs.RBS_FAR_TREECODE, "tree-df": rbs.RBS_FAR_TREECODE_DF}[args.far_field]
    ctx = rbs.Context(device=local, precision=rbs.RBS_PREC_MIXED, timing=1, stream=stream.cuda_stream,
                      pair_variant=args.pair_variant, far_field=far, tree_df_theta=args.tree_df_theta,
                      tree_df_degree=args.tree_df_degree)
    ctx.set_suspension(susp)
    st0 = rbs.rbs_get_stats(ctx.ctx)
    setup_ms = st0["setup_ms"]
    tree_info = None
    if far != rbs.RBS_FAR_DIRECT:
        opts = rbs.rbs_default_options()
        tree_info = {"theta": opts.tree_theta, "degree": opts.tree_degree, "cells": st0["tree_cells"],
                     "pairs_per_apply": st0["tree_pairs"], "proxy_pairs_per_apply": st0["tree_proxy_pairs"],
                     "direct_pairs_per_apply": st0["far_pairs"],
                     "reduction": st0["far_pairs"] / max(1, st0["tree_pairs"])}
        if far == rbs.RBS_FAR_TREECODE_DF:
            tree_info["double_float"] = {"theta": args.tree_df_theta, "degree": args.tree_df_degree,
                                         "cells": st0["tree_df_cells"], "pairs_per_apply": st0["tree_df_pairs"],
                                         "proxy_pairs_per_apply": st0["tree_df_proxy_pairs"],
                                         "reduction": st0["far_pairs"] / max(1, st0["tree_df_pairs"])}

    draws = [suspensions.forces(100 + rank, n, k) for k in range(args.warmup + args.steps)]
    F_dev = torch.tensor(np.stack([d[0] for d in draws]), device="cuda")
    T_dev = torch.tensor(np.stack([d[1] for d in draws]), device="cuda")
    v_dev = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    om_dev = torch.zeros_like(v_dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    # tolerance at 1e-8 relative error: reference = the same discrete system solved to 1e-12 (its residual
    # verified in double-float), then the largest candidate tolerance meeting the error bound
    F0 = draws[args.warmup][0]
    T0 = draws[args.warmup][1]
    if args.no_error_check and not args.tol:
        raise SystemExit("--no-error-check needs --tol")
    if args.no_error_check:
        pass
    elif far == rbs.RBS_FAR_TREECODE_DF:
        # the double-float passes approximate the far field too: the reference stays direct
        with rbs.Context(device=local, precision=rbs.RBS_PREC_MIXED, stream=stream.cuda_stream) as ref_ctx:
            ref_ctx.set_suspension(susp)
            v_ref, om_ref, _, _ = rbs.rbs_mobility_solve(ref_ctx.ctx, F0, T0, 1e-12)
    else:
        v_ref, om_ref, _, _ = rbs.rbs_mobility_solve(ctx.ctx, F0, T0, 1e-12)
    V_ref = None if args.no_error_check else np.concatenate([v_ref, om_ref], 1)

    def error_of(v, om):
        if V_ref is None:
            return None
        return float(np.linalg.norm(np.concatenate([v, om], 1) - V_ref) / np.linalg.norm(V_ref))

    tol_trials = {}
    for cand in ([args.tol] if args.tol else [1e-8, 1e-9, 1e-10]):
        v_c, om_c, _, _ = rbs.rbs_mobility_solve(ctx.ctx, F0, T0, cand)
        tol_trials[cand] = error_of(v_c, om_c)
        args.tol = cand
        if tol_trials[cand] is None or tol_trials[cand] <= 1e-8:
            break
    err = tol_trials[args.tol]

    for k in range(args.warmup):
        rbs.rbs_mobility_solve_device(ctx.ctx, F_dev[k], T_dev[k], args.tol, v_dev, om_dev)
    barrier()
    rbs.rbs_reset_stats(ctx.ctx)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    iters = []
    barrier()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))                      # L2 flush between timed solves
            starts[k].record(stream)
            its = rbs.rbs_mobility_solve_device(ctx.ctx, F_dev[args.warmup + k], T_dev[args.warmup + k], args.tol,
                                                v_dev, om_dev)
            ends[k].record(stream)
            iters.append(its)
        torch.cuda.synchronize()
    times = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    total_ms = sum(times)
    stats = rbs.rbs_get_stats(ctx.ctx)
    refinements = stats["refinements"]
    total_ms = reduce_max(total_ms, world, "cuda")
    value = whole_job_rate(args.steps, world, total_ms)
    kernels = kernel_table(stats)
    launches = stats["launches"]
    clocks = clk.summary()
    mean_iters = float(np.mean(iters)) if iters else 0.0

    # end to end through the host-buffer entry point (pinned host arrays, copies inside the timing)
    e2e = None
    if args.e2e_steps > 0:
        Fh = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        Th = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        vh = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        omh = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        its_h = np.zeros(max(1, rbs.rbs_suspension_count(ctx.ctx)), np.int32)
        lib = rbs.load()
        barrier()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            Fh[:] = draws[(args.warmup + k) % len(draws)][0]
            Th[:] = draws[(args.warmup + k) % len(draws)][1]
            rc = lib.rbs_mobility_solve(ctx.ctx, Fh.ctypes.data, Th.ctypes.data, args.tol, vh.ctypes.data,
                                        omh.ctypes.data, None, its_h.ctypes.data)
            if rc != 0:
                raise RuntimeError(rbs.rbs_last_error(ctx.ctx))
        el = reduce_max(time.perf_counter() - t0, world, "cuda")
        e2e = {"value": whole_job_rate(args.e2e_steps, world, el * 1e3), "unit": "solves/s",
               "h2d_bytes_per_step": 2 * 3 * 8 * n, "d2h_bytes_per_step": 2 * 3 * 8 * n}

    # per-kernel rates outside the solve (the inner solve's kernels run inside the captured GMRES graph,
    # which is timed as one unit): one apply of each operator in each arithmetic, timed by class
    x_dev = torch.tensor(suspensions.random_density(3, susp.total_nodes), device="cuda")
    y_dev = torch.zeros_like(x_dev)
    rbs.rbs_reset_stats(ctx.ctx)
    for op, prec in ((rbs.RBS_OP_A, rbs.RBS_PREC_MIXED), (rbs.RBS_OP_S_OFF, rbs.RBS_PREC_MIXED),
                     (rbs.RBS_OP_S_OFF, rbs.RBS_PREC_DF)):
        rbs.rbs_apply_operator_device(ctx.ctx, op, prec, x_dev, y_dev)
    op_kernels = kernel_table(rbs.rbs_get_stats(ctx.ctx))

    # the plain float64 path at the same tolerance: timed solves, or extrapolated from a subset
    plain = None
    if args.fp64_steps > 0:
        with rbs.Context(device=local, precision=rbs.RBS_PREC_FP64, timing=1, stream=stream.cuda_stream) as c64:
            c64.set_suspension(susp)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.fp64_steps):
                its64 = rbs.rbs_mobility_solve_device(c64.ctx, F_dev[args.warmup + k], T_dev[args.warmup + k],
                                                      args.tol, v_dev, om_dev)
                if k == 0:
                    v64 = v_dev.cpu().numpy().copy()
                    om64 = om_dev.cpu().numpy().copy()
            e1.record(stream)
            torch.cuda.synchronize()
            ms64 = e0.elapsed_time(e1) / args.fp64_steps
        plain = {"solves_per_s": 1e3 / ms64, "ms_per_solve": ms64, "steps": args.fp64_steps, "tol": args.tol,
                 "gmres_iterations": its64, "error_vs_reference": error_of(v64, om64), "basis": "timed"}
    elif args.fp64_subset > 0 and world == 1:
        tab, sub, st_sub = plain_fp64_extrapolated(rbs, susp, args, mean_iters, stream, local)

        def per_unit(name):
            e = tab.get(name)
            return (e["ms"] / e["units"]) if e and e["units"] > 0 else 0.0

        near_sub = tab.get("near_correction", {"ms": 0.0, "launches": 1})
        # the workload's units per application: far pairs, stored block bytes (float64 = twice the
        # float32 bytes the mixed path reads), near pair-nodes
        far_full = st0["far_pairs"]
        t_K = per_unit("pair_traction_f64") * far_full
        t_S = per_unit("pair_stokeslet_f64") * far_full
        blocks_per_node = (tab["particle_blocks"]["ms"] / tab["particle_blocks"]["launches"]) / sub.total_nodes \
            if "particle_blocks" in tab else 0.0
        t_blocks = blocks_per_node * susp.total_nodes
        t_near = (near_sub["ms"] / max(1, near_sub["launches"])) * (st0["near_pairs"] / max(1, st_sub["near_pairs"]))
        t_A = t_K + 2 * t_blocks + t_near  # preconditioner + system blocks, pairs, near
        its64 = max(1, int(round(mean_iters)))
        ms64 = (its64 + 3) * t_A + t_S + t_blocks + t_near
        plain = {"solves_per_s": 1e3 / ms64, "ms_per_solve": ms64, "tol": args.tol, "gmres_iterations": its64,
                 "basis": (f"extrapolated: float64 operator applications timed on the first {sub.n} particles "
                           f"({sub.total_nodes} nodes) of the workload, scaled to its {far_full:.4g} far pairs, "
                           f"{susp.total_nodes} nodes and {st0['near_pairs']} near pairs; one solve = "
                           f"(iterations + 3) applications of A plus one of S, iterations taken from the chosen path"),
                 "subset_kernels": tab,
                 "traction_f64_gpair_s": (1.0 / per_unit("pair_traction_f64") / 1e6) if per_unit("pair_traction_f64") else None,
                 "stokeslet_f64_gpair_s": (1.0 / per_unit("pair_stokeslet_f64") / 1e6) if per_unit("pair_stokeslet_f64") else None}

    # pair rates and the roofline of the dominant kernel of the chosen path
    f_mhz = clocks.get("sm_mhz") or 2070.0
    fp32_peak_tflops = SMS * FP32_LANES_PER_SM * 2 * f_mhz * 1e6 / 1e12
    fp64_peak_tflops = SMS * FP64_DFMA_PER_CLK_SM * 2 * f_mhz * 1e6 / 1e12

    def rate(tab, name):
        e = tab.get(name)
        return None if not e or e["ms"] <= 0 else e["units"] / (e["ms"] / 1e3) / 1e9

    gpairs = {"stokeslet_f32": rate(op_kernels, "pair_stokeslet_f32"),
              "stokeslet_df": rate(op_kernels, "pair_stokeslet_df"),
              "traction_f32": rate(op_kernels, "pair_traction_f32"),
              "traction_and_stokeslet_df": rate(kernels, "pair_both_df")}
    if plain and "traction_f64_gpair_s" in plain:
        gpairs["traction_f64_plain"] = plain["traction_f64_gpair_s"]
        gpairs["stokeslet_f64_plain"] = plain["stokeslet_f64_gpair_s"]
    timed = {k: v for k, v in kernels.items() if k != "gmres_graph"}
    dom = max(timed.items(), key=lambda kv: kv[1]["ms"])
    name, e = dom
    per_launch_ms = e["ms"] / e["launches"]
    units_per_launch = e["units"] / e["launches"]
    if name.startswith("pair_") and not name.endswith("f64"):
        kind = pair_kind(name)
        pairs_s = units_per_launch / (per_launch_ms / 1e3)
        achieved = pairs_s * FLOPS_PER_PAIR[kind] / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak_tflops, "traffic": None, "kernel": name,
                "peak_basis": f"float32 FMA peak derived from the unit counts: {SMS} SMs x 128 lanes x 2 flop x "
                              f"{f_mhz:.0f} MHz (median SM clock sampled under load); not in MEASURED_PEAKS.json",
                "achieved_basis": f"{FLOPS_PER_PAIR[kind]:.0f} algorithmic flops per evaluated pair "
                                  f"x {units_per_launch:.4g} pairs per launch / CUDA-event time per launch",
                "gpair_s": pairs_s / 1e9}
        if name.endswith("_df"):
            roof["issue_efficiency"] = pairs_s * DF_INSTR_PER_PAIR[kind] / (SMS * FP32_LANES_PER_SM * f_mhz * 1e6)
            roof["issue_basis"] = (f"{DF_INSTR_PER_PAIR[kind]:.0f} float32 operations the double-float kernel issues "
                                   f"per pair against {SMS} SMs x 128 lanes x {f_mhz:.0f} MHz")
    elif name.startswith("pair_"):
        kind = pair_kind(name)
        achieved = units_per_launch * FP64_OPS_PER_PAIR[kind] * 2 / (per_launch_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak_tflops, "traffic": None, "kernel": name,
                "peak_basis": f"float64 FMA: {SMS} SMs x 2 lanes x 2 flop x {f_mhz:.0f} MHz"}
    else:
        peaks = {}
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        except Exception:
            pass
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        achieved = units_per_launch / (per_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "kernel": name,
                "peak_basis": "of measured copy bandwidth" if peaks else "of fallback 6.8 TB/s"}
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0))
    except Exception:
        hbm_peak = 6800.0
    # the block kernel with float32 entries (HBM-bound) and with float64 entries (float64-pipe-bound)
    rooflines = kernel_rooflines({**op_kernels, **{k: v for k, v in kernels.items() if k != "particle_blocks"}},
                                 f_mhz, hbm_peak)
    if "particle_blocks_f64" in kernels and kernels["particle_blocks_f64"]["ms"] > 0:
        rooflines["particle_blocks_f64"] = block_f64_roofline(kernels["particle_blocks_f64"], f_mhz)
    # the captured counters belong to the direct kernels (and the double-float treecode kernel, captured
    # on its own profiling case): a treecode kernel without a capture has none
    tree_df_class = name.endswith("_df") and far == rbs.RBS_FAR_TREECODE_DF
    treecode_class = (name.endswith("_f32") and far != rbs.RBS_FAR_DIRECT)
    if tree_df_class and TREE_DF_TRAFFIC is not None:
        bytes_, nodes_ = TREE_DF_TRAFFIC
        roof["traffic"] = bytes_ * susp.total_nodes / nodes_
        roof["traffic_basis"] = ("ncu dram read+write of the double-float treecode kernel on the 2,000-ellipsoid "
                                 "profiling case, scaled by node count")
    elif name in NCU_TRAFFIC and not treecode_class and not tree_df_class:
        bytes_, nodes_ = NCU_TRAFFIC[name]
        roof["traffic"] = bytes_ * susp.total_nodes / nodes_
        roof["traffic_basis"] = "ncu dram read+write of the 400-ellipsoid capture, scaled by node count"
    else:
        roof["traffic_basis"] = "null: no dram counters captured for this kernel"
    roof["ms_per_launch"] = per_launch_ms
    roof["share_of_step"] = e["ms"] / total_ms if world == 1 else None

    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        procs = args.cpu_procs or host_cores()
        sampler = OracleSampler(susp, procs)
        its_c = max(1, int(round(mean_iters)))
        cpu_val, sample, _ = sampler.sample(args.cpu_seconds, its_c)
        one_val, one_sample, _ = sampler.sample(max(3.0, args.cpu_seconds / 2), its_c, procs=1)
        sampler.close()
        cpu = {"value": cpu_val, "unit": "solves/s", "cores": procs, "kind": "oracle", "sample": sample,
               "single_core": {"value": one_val, "unit": "solves/s", "cores": 1, "sample": one_sample}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": susp.name, "n_particles": n, "p": int(susp.p[0]), "nodes": susp.total_nodes,
                       "unknowns": 3 * susp.total_nodes, "tol": args.tol, "precision": "mixed",
                       "far_field": {"direct": "direct sums",
                                     "tree": "treecode for the float32 inner applies, direct double-float passes",
                                     "tree-df": "treecodes for the float32 applies and the double-float passes"}[
                                         args.far_field],
                       "preconditioner": "block-diagonal", "gmres": "per-suspension, graph-captured Arnoldi cycle",
                       "gmres_iterations": iters, "refinements_last": refinements, "setup_ms": setup_ms,
                       "l2": "flushed before every timed solve (258 MB write); working set > L2",
                       "parallelism": f"replicas x{world}"},
            "error_vs_reference": err,
            "tolerance_trials": {f"{k:.0e}": v for k, v in tol_trials.items()},
            "plain_fp64": plain,
            "speedup_vs_plain_fp64": (value / world) / plain["solves_per_s"] if plain else None,
            "gpair_per_s": gpairs,
            "kernels": kernels,
            "operator_kernels": op_kernels,
            "pair_variant": dict(zip(["traction_f32", "stokeslet_f32", "traction_df", "stokeslet_df",
                                      "traction_and_stokeslet_df"], stats.get("pair_variant", []))),
            "treecode": tree_info,
            "roofline": roof,
            "kernel_rooflines": rooflines,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": launches,
            "gpu_launches_per_step": launches / max(1, args.steps),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_warmstart_experiment(args):
    """RK4 sedimentation (Algorithm 1 without contact) of the workload: train the warm-start network on
    the densities of the first train_steps steps (solved with the previous-stage guess), then run
    eval_steps more steps from the same configuration with zero, previous-stage and learned initial
    guesses, and report GMRES iterations per solve and solves/s for each."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    susp = suspensions.WORKLOADS[args.workload]()
    tol = args.tol or 1e-8
    prec = rbs.RBS_PREC_MIXED
    far = {"direct": rbs.RBS_FAR_DIRECT, "tree": rbs.RBS_FAR_TREECODE, "tree-df": rbs.RBS_FAR_TREECODE_DF}[args.far_field]
    with rbs.Context(device=0, precision=prec, warm_start=rbs.RBS_WARM_PREVIOUS, warm_record=1,
                     stream=stream.cuda_stream, far_field=far) as ctx:
        ctx.set_suspension(susp)
        t0 = time.perf_counter()
        its_train = rbs.rbs_advance(ctx.ctx, susp.F, susp.T, args.dt, args.train_steps, rbs.RBS_RK4, tol)
        t_train_solves = time.perf_counter() - t0
        t0 = time.perf_counter()
        loss_first = rbs.rbs_warmstart_train(ctx.ctx, 1, batch=256, lr=1e-3, seed=1)
        loss = rbs.rbs_warmstart_train(ctx.ctx, args.epochs - 1, batch=256, lr=1e-3, seed=1)
        t_train = time.perf_counter() - t0
        params, scale = rbs.rbs_warmstart_weights(ctx.ctx)
        cen, quat = rbs.rbs_get_state(ctx.ctx, susp.n)
    out = {}
    finals = {}
    for mode in args.warm_modes.split(","):
        with rbs.Context(device=0, precision=prec, warm_start=getattr(rbs, "RBS_WARM_" + mode),
                         stream=stream.cuda_stream, far_field=far) as ctx:
            ctx.set_geometry(susp.semi_axes, susp.p, susp.nphi, cen, quat)
            if mode.startswith("LEARNED"):
                rbs.rbs_warmstart_weights(ctx.ctx, params, scale=scale)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            its = rbs.rbs_advance(ctx.ctx, susp.F, susp.T, args.dt, args.eval_steps, rbs.RBS_RK4, tol)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            solves = 4 * args.eval_steps
            c_end, _ = rbs.rbs_get_state(ctx.ctx, susp.n)
            finals[mode] = c_end
            out[mode.lower()] = {"gmres_iterations_per_solve": its / solves, "solves_per_s": solves / (ms / 1e3),
                                 "ms": ms}
    base = "ZERO" if "ZERO" in finals else "PREVIOUS"
    drift = {m: float(np.abs(finals[m] - finals[base]).max()) for m in finals}
    line = {"experiment": "learned warm start in RK4 sedimentation", "workload": susp.name, "n_particles": susp.n,
            "nodes": susp.total_nodes, "precision": "mixed", "far_field": args.far_field, "tol": tol, "dt": args.dt,
            "train_steps": args.train_steps, "train_samples": 4 * args.train_steps * susp.n,
            "train_iterations_per_solve": its_train / (4 * args.train_steps),
            "train_solve_seconds": t_train_solves, "epochs": args.epochs, "train_seconds": t_train,
            "loss_first_epoch": loss_first, "loss_last_epoch": loss, "eval_steps": args.eval_steps,
            "results": out, f"max_centre_difference_vs_{base.lower()}_start": drift}
    print(json.dumps(line), flush=True)


def run_selfgemm_experiment(args):
    """Self blocks on the tensor cores (the workload's particles share one shape, so their block
    applications form a GEMM): for float32 blocks (CUDA cores) and for float16 and bfloat16 blocks
    (tcgen05 GEMM), times `--warmup` + `--steps` applications of each arithmetic's K self-block
    operator (the GEMM kernel alone by its CUDA events: TFLOP/s against the measured bf16 peak), then,
    unless --solves is 0, one mobility solve per arithmetic at the chosen tolerance with its GMRES
    iterations, refinements and double-float passes, and its (v, omega) error against the float32-block
    solve at 1e-10."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    susp = suspensions.WORKLOADS[args.workload]()
    tol = args.tol or 1e-8
    far = {"direct": rbs.RBS_FAR_DIRECT, "tree": rbs.RBS_FAR_TREECODE, "tree-df": rbs.RBS_FAR_TREECODE_DF}[args.far_field]
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        bf16_peak = float(peaks["bf16_tflops"])
        peak_basis = "of measured (MEASURED_PEAKS.json bf16_tflops, burst; float16 has the same dense rate)"
    except Exception:
        bf16_peak, peak_basis = 1900.0, "of fallback 1.9 PFLOP/s"
    x_dev = torch.tensor(suspensions.random_density(3, susp.total_nodes), device="cuda")
    y_dev = torch.zeros_like(x_dev)
    out = {}
    V_ref = None
    for name in ("MIXED", "MIXED_FP16", "MIXED_BF16"):
        prec = getattr(rbs, "RBS_PREC_" + name)
        with rbs.Context(device=0, precision=prec, timing=1, stream=stream.cuda_stream, far_field=far) as ctx:
            ctx.set_suspension(susp)
            setup_ms = rbs.rbs_get_stats(ctx.ctx)["setup_ms"]
            for k in range(args.warmup):
                rbs.rbs_apply_operator_device(ctx.ctx, rbs.RBS_OP_K_SELF, prec, x_dev, y_dev)
            torch.cuda.synchronize()
            rbs.rbs_reset_stats(ctx.ctx)
            for k in range(max(1, args.steps)):
                rbs.rbs_apply_operator_device(ctx.ctx, rbs.RBS_OP_K_SELF, prec, x_dev, y_dev)
            torch.cuda.synchronize()
            tab = kernel_table(rbs.rbs_get_stats(ctx.ctx))
            row = {"setup_ms": setup_ms, "self_apply_kernels": tab}
            if "self_gemm" in tab:
                e = tab["self_gemm"]
                tf = e["units"] / (e["ms"] / 1e3) / 1e12
                row["self_gemm"] = {"ms_per_launch": e["ms"] / e["launches"], "tflops": tf, "peak_tflops": bf16_peak,
                                    "frac": tf / bf16_peak, "peak_basis": peak_basis,
                                    "flops_per_launch": e["units"] / e["launches"]}
            if "particle_blocks" in tab:
                e = tab["particle_blocks"]
                row["block_apply_ms"] = e["ms"] / e["launches"]
            if args.solves > 0:
                if V_ref is None and name == "MIXED":
                    v0, om0, _, _ = rbs.rbs_mobility_solve(ctx.ctx, susp.F, susp.T, 1e-10)
                    V_ref = np.concatenate([v0, om0], 1)
                rbs.rbs_reset_stats(ctx.ctx)
                t0 = time.perf_counter()
                v, om, _, its = rbs.rbs_mobility_solve(ctx.ctx, susp.F, susp.T, tol)
                el = time.perf_counter() - t0
                st = rbs.rbs_get_stats(ctx.ctx)
                tabs = kernel_table(st)
                df_passes = sum(tabs[k]["launches"] for k in ("pair_both_df",) if k in tabs)
                row.update({"solve_s": el, "gmres_iterations": its, "refinements": st["refinements"],
                            "double_float_passes": df_passes,
                            "error_vs_float32_blocks_1e-10": float(np.linalg.norm(np.concatenate([v, om], 1) - V_ref) /
                                                                   np.linalg.norm(V_ref))})
            out[name.lower()] = row
    line = {"experiment": "self blocks on the tensor cores (shared shape)", "workload": susp.name,
            "n_particles": susp.n, "p": int(susp.p[0]), "nodes": susp.total_nodes, "tol": tol,
            "far_field": args.far_field, "results": out}
    print(json.dumps(line), flush=True)


def run_magnetic_experiment(args):
    """The magnetorheological set-up of the paper's Fig. 1 (Section 4.1.3): 512 unit spheres at p = 8
    on a perturbed 8 x 8 x 8 cubic lattice (spacing 3, seeded perturbation 0.2) in the field
    H0 = (10 / sqrt 3) (1, -1, -1) with mu / mu0 = 2, 294,912 unknowns (3 Stokes + 1 Laplace per node).
    Times RK4 steps (each stage: magnetic forces, then the mobility solve) in float64 and mixed
    precision, and reports the parts."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs
    torch.cuda.set_device(0)
    rng = np.random.default_rng(6)
    g = np.arange(8) * 3.0
    cen = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    cen = cen - cen.mean(0) + rng.uniform(-0.2, 0.2, size=cen.shape)
    n = len(cen)
    quats = np.tile([1.0, 0, 0, 0], (n, 1))
    H0 = 10.0 / math.sqrt(3.0) * np.array([1.0, -1.0, -1.0])
    tol = args.tol or 1e-8
    out = {}
    for prec in ("FP64", "MIXED"):
        far = rbs.RBS_FAR_DIRECT
        if prec == "MIXED":
            far = {"direct": rbs.RBS_FAR_DIRECT, "tree": rbs.RBS_FAR_TREECODE,
                   "tree-df": rbs.RBS_FAR_TREECODE_DF}[args.far_field]
        with rbs.Context(device=0, precision=getattr(rbs, "RBS_PREC_" + prec), magnetic_field=tuple(H0),
                         mu_ratio=2.0, timing=1, far_field=far) as ctx:
            ctx.set_geometry(np.ones((n, 3)), 8, 16, cen, quats)
            t0 = time.perf_counter()
            F, T, q, its_m = rbs.rbs_magnetic_forces(ctx.ctx, H0, 2.0, tol, n, 9 * 16 * n)
            t_mag_first = time.perf_counter() - t0
            t0 = time.perf_counter()
            F, T, q, its_m = rbs.rbs_magnetic_forces(ctx.ctx, H0, 2.0, tol, n, 9 * 16 * n)
            t_mag = time.perf_counter() - t0
            t0 = time.perf_counter()
            v, om, _, its_s = rbs.rbs_mobility_solve(ctx.ctx, F, T, tol)
            t_solve = time.perf_counter() - t0
            t0 = time.perf_counter()
            steps = max(1, args.steps // 5)
            its_adv = rbs.rbs_advance(ctx.ctx, np.zeros((n, 3)), np.zeros((n, 3)), 0.01, steps, rbs.RBS_RK4, tol)
            t_step = (time.perf_counter() - t0) / steps
            out[prec.lower()] = {"magnetic_forces_s": t_mag, "magnetic_first_call_s": t_mag_first,
                                 "laplace_gmres_iterations": its_m, "mobility_solve_s": t_solve,
                                 "mobility_gmres_iterations": its_s, "rk4_step_s": t_step, "rk4_steps": steps,
                                 "max_force": float(np.abs(F).max())}
    line = {"experiment": "magnetorheological spheres (Fig. 1 set-up)", "n_particles": n, "p": 8,
            "unknowns": 4 * 9 * 16 * n, "tol": tol, "H0": H0.tolist(), "mu_ratio": 2.0,
            "far_field": f"{args.far_field} (mixed-precision stages)", "results": out,
            "paper_context": "about 5 minutes per time step on one Xeon E5-2690 v2 node with FMM (Fig. 1 caption)"}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.experiment == "warmstart":
        run_warmstart_experiment(args)
        return
    if args.experiment == "magnetic":
        run_magnetic_experiment(args)
        return
    if args.experiment == "selfgemm":
        run_selfgemm_experiment(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
