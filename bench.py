#!/usr/bin/env python
"""Benchmark: sparse LU factor + solve over the irregular block grid.

Workload: 3-D 7-point nonsymmetric convection-diffusion operator on a 40^3
grid (n = 64,000) in nested-dissection order, 4 right-hand sides, FP64,
irregular blocking (Algorithm 3, S = 1000, step 2; the block-size bound
max_num and the sparse/dense threshold picked by the autotuner), seeded
synthetic data.  One step = value scatter + numerical factorization
(GETRF / GESSM / TSTRF / SSSSM per level) + forward/backward solve of the 4
right-hand sides.  The factors (42.6 M values, 340 MB) exceed the 126 MB L2,
so no flush is needed between steps.

Metric: GFLOP/s of factor + solve, with the algorithmic flop count
sum_k (l_k + 2 l_k u_k) of the filled pattern plus 2 nnz(L+U) per
right-hand side for the solve; higher is better.  Extra legs in the same
run: FP32 factors + FP64 refinement to backward error <= 1e-14, the same
code with regular 128-row blocking (FP64 and FP32), 256 batched grids
replayed from a CUDA graph against a per-matrix loop, the 48 x 48 grid
(irregular against regular 64), autograd forward + backward on the 32^3
parameterised operator, and the n = 200,000 bordered circuit matrix (FP32 +
refinement against FP64; --no-circuit skips it).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own replica (the factorization of one
matrix is not sharded); value = all ranks' flops / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD = "grid7cd_40"
METRIC = ("factor+solve GFLOP/s (FP64, irregular blocks, 40^3 7-point "
          "convection-diffusion, n=64000, 4 RHS, backward error <= 1e-14)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP32+IR / regular / e2e / CPU legs")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="precision of the timed leg (fp32: FP32 factors + FP64 "
                         "refinement); the headline metric is fp64, fp32 serves "
                         "profiling captures of the FP32 kernels")
    ap.add_argument("--no-circuit", action="store_true",
                    help="skip the n = 200,000 circuit leg (about 2 minutes)")
    ap.add_argument("--reference-grid", type=int, default=40,
                    help="grid edge of the reference arm's oracle runs (40: the "
                         "benchmark's input; smaller only for quick checks of "
                         "the line's shape)")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["grid7cd_40", "grid7cd_32", "grid7cd_24"],
                    help="40^3 is the benchmark; the smaller grids of the same "
                         "family serve profiling captures")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(ms, world, device="cpu"):
    """Step time of the whole job: the maximum over ranks (all-reduce MAX on
    the current process group; the value itself at world size 1)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(flops_per_rank, ms, world):
    """Whole-job throughput: every rank factors its own replica (weak
    scaling), so the job does world x flops_per_rank in the slowest rank's
    time."""
    return world * flops_per_rank / (ms * 1e-3) / 1e9


def step_flops(plan, nrhs):
    return plan.info["flops"] + 2 * plan.info["nnz_lu"] * nrhs


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 8:
                self.rows.append(f)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def timed(torch, fn, steps, warmup, barrier=None, nvtx=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if nvtx:                      # lets an ncu launch list select these steps
        torch.cuda.nvtx.range_push(nvtx)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    if nvtx:
        torch.cuda.nvtx.range_pop()
    if barrier:
        barrier()
    return e0.elapsed_time(e1) / steps


def fp64_peak_tflops(torch):
    """cuBLAS DGEMM rate measured live (the FP64 ceiling of this GPU)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2 * n ** 3 / (best * 1e-3) / 1e12


def measured_peak(key, fallback):
    """A figure of MEASURED_PEAKS.json (driver-written), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, ValueError, KeyError):
        return fallback


def recorded_traffic(kernel, workload, launches):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.txt: kernel, workload, source digest, bytes per step),
    or None when there is none for this kernel and workload or the kernel
    sources changed since the counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path) or launches <= 0:
        return None
    h = hashlib.sha1()
    for f in ("factor.cu", "device_common.cuh", "slu_internal.hpp"):
        with open(os.path.join(ROOT, "paper_2512_04389_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    digest = h.hexdigest()[:12]
    with open(path) as fh:
        for line in fh:
            f = line.split()
            if len(f) == 4 and f[0] == kernel and f[1] == workload and f[2] == digest:
                return float(f[3]) / launches
    return None


def host_cpu():
    """Model name and logical core count of the host."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": model, "nproc": os.cpu_count()}


def oracle_step(m):
    """One oracle factor + solve of grid7_cd(m) (4 RHS): (seconds, flops).
    Module level so that spawned worker processes can run it."""
    from oracle import lu as OL
    s = workloads.grid7_cd(m)
    t = time.perf_counter()
    F = OL.lu(s.n, s.colptr, s.rowidx, s.values)
    OL.solve(F, s.rhs)
    dt = time.perf_counter() - t
    return dt, OL.flops(F) + 2 * (len(F["Li"]) + len(F["Ui"])) * s.nrhs


def cpu_oracle_leg(m=40):
    """The oracle as it stands on the benchmark's own input (grid7_cd(40),
    full size, seed 0, 4 RHS): one factor + solve on one host core."""
    dt, fl = oracle_step(m)
    return {"value": fl / dt / 1e9, "unit": "GFLOP/s", "cores": 1,
            "kind": "oracle", "host": host_cpu(),
            "sample": f"grid7cd_{m} at full size (n={m ** 3}, 4 RHS): one "
                      f"factor+solve, {dt:.1f} s on 1 host core"}


def batch_leg(torch, S, dev, args):
    """256 independent 2-D 5-point matrices (k ~ U{16..96}), FP32 factors +
    FP64 refinement on 1 RHS each: one batch plan (per-member irregular
    blocking, levels merged, factorization replayed from a CUDA graph)
    against a loop of per-matrix factor + solve calls."""
    from paper_2512_04389_b300.tune import tune, candidates
    ms = workloads.batch_grid5(count=256, seed=0)
    ns, cps, ris = [m.n for m in ms], [m.colptr for m in ms], [m.rowidx for m in ms]
    vb = dev(np.concatenate([m.values for m in ms]))
    bb = dev(np.concatenate([m.rhs[:, 0] for m in ms]))
    # the irregular and the regular blocking each tuned on the batch plan
    best_i, _ = tune(ns, cps, ris, vb, bb, precision="fp32")
    best_r, _ = tune(ns, cps, ris, vb, bb, precision="fp32",
                     cands=candidates("regular_sizes"))
    PB = S.Plan(ns, cps, ris, precision="fp32", **best_i)
    FB = S.Factor(PB, vb)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        FB.set_graph(True)

        def step_b():
            FB.refactor(vb)
            FB.solve(bb)
        msb = timed(torch, step_b, args.steps, 2)
        _, ib = FB.solve(bb, info=True)
        FB.set_graph(False)
    # the level walk of all members as one persistent launch (the tuned
    # blocking with every block dense, which the persistent kernel needs)
    pers = dict(best_i, dense_threshold=0.0)
    PP = S.Plan(ns, cps, ris, precision="fp32", **pers)
    FP = S.Factor(PP, vb)
    with torch.cuda.stream(st):
        FP.set_graph(True)

        def step_pl():
            FP.refactor(vb)
            FP.solve(bb)
        msp_levels = timed(torch, step_pl, args.steps, 2)
        FP.set_persistent(True)
        l0 = FP.stats()["launches"]
        FP.refactor(vb)
        torch.cuda.synchronize()
        pl_launches = FP.stats()["launches"] - l0
        msp = timed(torch, step_pl, args.steps, 2)
        FP.set_graph(False)
    FP.set_persistent(False)
    del FP, PP
    # the same batch with the tuned regular blocking of every member
    PR = S.Plan(ns, cps, ris, precision="fp32", **best_r)
    FR = S.Factor(PR, vb)
    with torch.cuda.stream(st):
        FR.set_graph(True)

        def step_r():
            FR.refactor(vb)
            FR.solve(bb)
        msr = timed(torch, step_r, args.steps, 2)
        FR.set_graph(False)
    del FR, PR
    PS = S.Plan([m.n for m in ms], [m.colptr for m in ms],
                [m.rowidx for m in ms], precision="fp32", dense_threshold=0.0,
                blocking="regular_select")
    FS = S.Factor(PS, vb)
    with torch.cuda.stream(st):
        FS.set_graph(True)

        def step_s():
            FS.refactor(vb)
            FS.solve(bb)
        mss = timed(torch, step_s, args.steps, 2)
        FS.set_graph(False)
    del FS, PS
    plans = [S.Plan(m.n, m.colptr, m.rowidx, precision="fp32", **best_i)
             for m in ms]
    vs = [dev(m.values) for m in ms]
    rs = [dev(m.rhs[:, 0]) for m in ms]
    fs = [S.Factor(p, v) for p, v in zip(plans, vs)]

    def step_l():
        for f, v, r in zip(fs, vs, rs):
            f.refactor(v)
            f.solve(r)
    msl = timed(torch, step_l, max(1, args.steps // 2), 1)
    fl = sum(p.info["flops"] + 2 * p.info["nnz_lu"] for p in plans)
    return {"ms_per_step": msb, "gflops": fl / (msb * 1e-3) / 1e9,
            "loop_ms_per_step": msl, "speedup_vs_loop": msl / msb,
            "tuned": best_i, "regular_tuned": best_r,
            "persistent": {"options": pers, "graph_ms_per_step": msp,
                           "per_level_graph_ms_per_step": msp_levels,
                           "factor_launches": pl_launches},
            "regular_tuned_graph_ms_per_step": msr, "irregular_speedup": msr / msb,
            "regular_select_graph_ms_per_step": mss,
            "backward_error_max_member": ib["backward_error"],
            "ir_iterations": ib["iterations"], "levels": PB.info["nlevels"],
            "n_total": PB.info["n"]}


def run_legs(extras, legs, *leg_args):
    """Run the extra legs in order, each into extras[name]; a leg that
    raises is recorded as {"error": ...} (traceback on stderr) and the rest
    still run, so the headline line is always printed."""
    import traceback
    for name, fn in legs:
        try:
            extras[name] = fn(*leg_args)
        except Exception as e:  # noqa: BLE001
            traceback.print_exc()
            extras[name] = {"error": f"{type(e).__name__}: {e}"}


def small_grid_leg(torch, S, dev, args):
    """48 x 48 5-point grid (n = 2304), FP64, irregular blocking against
    regular 64 x 64 blocking in the same code, 1 RHS."""
    from paper_2512_04389_b300.tune import tune
    s = workloads.grid5(48)
    v, r = dev(s.values), dev(s.rhs)
    out = {}
    from paper_2512_04389_b300.tune import candidates
    for name, opts in (("irregular", {}),
                       ("regular64", dict(blocking="regular", regular_block=64)),
                       ("regular_select", dict(blocking="regular_select")),
                       ("regular_tuned", None)):
        if opts is None:           # block size and threshold both searched
            best, _ = tune(s.n, s.colptr, s.rowidx, v, r, precision="fp64",
                           cands=candidates("regular_sizes", s.n))
            opts = {}
        else:
            best, _ = tune(s.n, s.colptr, s.rowidx, v, r, precision="fp64", **opts)
        P = S.Plan(s.n, s.colptr, s.rowidx, **opts, **best)
        F = S.Factor(P, v)

        def step():
            F.refactor(v)
            F.solve(r)
        ms = timed(torch, step, args.steps, 3)
        out[name] = {"ms_per_step": ms, "tuned": best,
                     "blocks_1d": P.info["nblocks_1d"], "levels": P.info["nlevels"],
                     "gflops": step_flops(P, s.nrhs) / (ms * 1e-3) / 1e9}
    return out


def circuit_leg(torch, S, dev, args):
    """Bordered circuit matrix, n = 200,000 (4,000 border rows), 8 RHS:
    FP32 factors + FP64 refinement to backward error <= 1e-14 against the
    plain FP64 factorization, and the FP32 leg with regular 128-row
    blocking.  The options are the best of one-off sweeps on B300 (tuning
    here would repeat the 2-4 s analysis per candidate): sparse/dense
    threshold 0.02 for FP32 and 0.05 for FP64; FP32 irregular blocking with
    S = n / 128 samples (tile-aligned spacing), max_num 1, and both FP32
    legs with one TF32 pass on the tensor cores (the border is a dense
    contraction).  One timed factor + solve each."""
    s = workloads.circuit_bbd()
    v, r = dev(s.values), dev(s.rhs)
    out = {"n": s.n, "nnz_a": s.nnz}
    for leg, prec, extra in (("fp32", "fp32",
                              dict(sample_points=2000, b_min=128, max_num=1, tc_passes=1)),
                             ("fp64", "fp64", {}),
                             ("fp32_regular128", "fp32",
                              dict(blocking="regular", regular_block=128, tc_passes=1))):
        t0 = time.perf_counter()
        thr = 0.02 if prec == "fp32" else 0.05
        P = S.Plan(s.n, s.colptr, s.rowidx, precision=prec, dense_threshold=thr,
                   device=True, **extra)
        ana = time.perf_counter() - t0
        if leg == "fp32":           # the host analysis of the same plan, once
            t0 = time.perf_counter()
            PH = S.Plan(s.n, s.colptr, s.rowidx, precision=prec, dense_threshold=thr,
                        **extra)
            out["analysis"] = {"device_s": ana, "device_phase_ms": P.info["phase_ms"],
                               "host_s": time.perf_counter() - t0,
                               "host_phase_ms": PH.info["phase_ms"],
                               "same_plan": PH.digest() == P.digest()}
            del PH
        F = S.Factor(P, v)

        def step():
            F.refactor(v)
            F.solve(r)
        ms = timed(torch, step, 1, 1)
        _, info = F.solve(r, info=True)
        out[leg] = {"ms_per_step": ms, "analyze_s": ana, "dense_threshold": thr,
                     "gflops": step_flops(P, s.nrhs) / (ms * 1e-3) / 1e9,
                     "backward_error": info["backward_error"],
                     "ir_iterations": info["iterations"],
                     "nnz_lu": P.info["nnz_lu"], "flops_factor": P.info["flops"],
                     "levels": P.info["nlevels"]}
        del F, P
        torch.cuda.empty_cache()
    out["irregular_speedup_fp32"] = (out["fp32_regular128"]["ms_per_step"] /
                                     out["fp32"]["ms_per_step"])
    return out


def autograd_leg(torch, S, dev, args):
    """x = A(theta)^{-1} b on the parameterised 32^3 operator (n = 32,768),
    FP64: forward solve plus backward (transposed solve through the stored
    factors and the gradient gather), loss 1/2 ||x||^2."""
    from paper_2512_04389_b300.autograd import lu_solve
    from paper_2512_04389_b300.tune import tune, candidates
    s = workloads.grid7_theta(32)
    v0, b0 = dev(s.values), dev(s.rhs[:, 0])
    best_i, _ = tune(s.n, s.colptr, s.rowidx, v0, b0, precision="fp64")
    best_r, _ = tune(s.n, s.colptr, s.rowidx, v0, b0, precision="fp64",
                     cands=candidates("regular_sizes", s.n))
    P = S.Plan(s.n, s.colptr, s.rowidx, **best_i)

    PR = S.Plan(s.n, s.colptr, s.rowidx, **best_r)

    def run(plan):
        def step():
            vv = v0.clone().requires_grad_(True)
            bb = b0.clone().requires_grad_(True)
            x = lu_solve(vv, bb, plan)
            (0.5 * (x * x).sum()).backward()
        return timed(torch, step, args.steps, 2)
    PSel = S.Plan(s.n, s.colptr, s.rowidx, dense_threshold=0.0,
                  blocking="regular_select")
    ms = run(P)
    msr = run(PR)
    mss = run(PSel)
    return {"ms_per_step": ms, "n": s.n, "nnz_a": s.nnz,
            "tuned": best_i, "regular_tuned": best_r,
            "regular_tuned_ms_per_step": msr, "irregular_speedup": msr / ms,
            "regular_select_ms_per_step": mss,
            "regular_select_block": PSel.info["regular_block"],
            "what": "factor + solve forward, transposed solve + gradient gather backward"}


def reference_workers(steps):
    """Worker processes for the reference arm: one per timed step, at most
    one per host core and 16, and about 2 GB of host memory each (one
    full-size oracle factorization holds under 1 GB)."""
    try:
        with open("/proc/meminfo") as f:
            avail = next(int(l.split()[1]) for l in f if l.startswith("MemAvailable"))
        by_mem = max(1, avail // (2 * 1024 * 1024))
    except (OSError, StopIteration, ValueError):
        by_mem = 4
    return max(1, min(steps, os.cpu_count() or 1, 16, by_mem))


def run_reference(args):
    """The oracle as it stands on the benchmark's own input: every step is
    one full-size factor + solve of grid7_cd(40).  The steps run as
    independent processes spread over the host's cores (the oracle itself
    is sequential), so value = steps x flops / wall time of the timed
    steps.  Warm-up: untimed oracle runs of grid7_cd(12) that start the
    workers and load the oracle's library."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import multiprocessing as mp
    m = args.reference_grid
    wl = f"grid7cd_{m}"
    cores = reference_workers(args.steps)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(oracle_step, [12] * max(args.warmup, cores), chunksize=1)
        t0 = time.perf_counter()
        res = pool.map(oracle_step, [m] * args.steps, chunksize=1)
        wall = time.perf_counter() - t0
    fl = res[0][1]
    ms = 1e3 * wall / args.steps
    v = args.steps * fl / wall / 1e9
    per = sorted(r[0] for r in res)
    sample = (f"each step: one oracle factor+solve of {wl} at full size "
              f"(n={m ** 3}, 4 RHS); {args.steps} steps as independent "
              f"processes on {cores} host cores, {wall:.1f} s wall, "
              f"{per[len(per) // 2]:.1f} s median per step")
    cfg = {"workload": wl, "n": m ** 3, "nrhs": 4,
           "host_cores": os.cpu_count(), "workers": cores}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": cores,
                         "kind": "oracle", "sample": sample, "host": host_cpu()},
        "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    barrier = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        barrier = dist.barrier
    from paper_2512_04389_b300 import slu as S
    from paper_2512_04389_b300.tune import tune

    s = workloads.grid7_cd(int(args.workload.split("_")[1]))
    dev = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float64,
                                    device="cuda")
    vals_d, rhs_d = dev(s.values), dev(s.rhs)
    # sparse/dense switch picked by the autotuner (cached per pattern)
    best64, tun64 = tune(s.n, s.colptr, s.rowidx, vals_d, rhs_d,
                         precision=args.precision)
    # the plan from the device analysis (symbolic factorization and
    # Algorithms 2 / 3 on the GPU); the host analysis gives the same plan
    plan = S.Plan(s.n, s.colptr, s.rowidx, precision=args.precision, device=True, **best64)
    host_plan = S.Plan(s.n, s.colptr, s.rowidx, precision=args.precision, **best64)
    assert host_plan.digest() == plan.digest()
    analysis = {"device_ms": plan.info["analyze_ms"],
                "device_phase_ms": plan.info["phase_ms"],
                "host_ms": host_plan.info["analyze_ms"],
                "host_phase_ms": host_plan.info["phase_ms"]}
    del host_plan
    fl = step_flops(plan, s.nrhs)
    # the step runs on a created stream: the level walk is replayed from the
    # CUDA graph recorded at the first refactor (slu_set_graph; the solves
    # are always replayed from theirs)
    step_stream = torch.cuda.Stream()
    torch.cuda.set_stream(step_stream)
    F = S.Factor(plan, vals_d)
    F.set_graph(True)

    def step():
        F.refactor(vals_d)
        F.solve(rhs_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = F.stats()["launches"]
    with Clocks(local) as clk:
        ms = timed(torch, step, args.steps, 0, barrier, nvtx="bench_step")
    launches = (F.stats()["launches"] - l0) // max(1, args.steps)
    # the same step with the level walk launched kernel by kernel
    F.set_graph(False)
    ms_direct = timed(torch, step, args.steps, 1)
    F.set_graph(True)
    ms = max_over_ranks(ms, world, device="cuda")
    value = job_gflops(fl, ms, world)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    X, sinfo = F.solve(rhs_d, info=True)
    ms_factor = timed(torch, lambda: F.refactor(vals_d), args.steps, 1)
    ms_solve = timed(torch, lambda: F.solve(rhs_d), args.steps, 1)
    metric = METRIC if args.precision == "fp64" else METRIC.replace(
        "FP64,", "FP32 factors + FP64 refinement,")
    out = {"metric": metric, "value": value, "unit": "GFLOP/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "n": s.n, "nrhs": s.nrhs,
                      "nnz_a": s.nnz, "nnz_lu": plan.info["nnz_lu"],
                      "flops_factor": plan.info["flops"],
                      "blocks_1d": plan.info["nblocks_1d"],
                      "levels": plan.info["nlevels"],
                      "analyze_ms": plan.info["analyze_ms"], "analysis": analysis,
                      "factor_ms": ms_factor, "solve_ms": ms_solve,
                      "launch": "level walk replayed from a CUDA graph",
                      "ms_per_step_kernel_by_kernel": ms_direct,
                      "tuned": best64, "tuning_ms": tun64,
                      "backward_error": sinfo["backward_error"],
                      "l2": "no flush: factors (340 MB) exceed L2",
                      "parallelism": f"replicas x{world}"},
           "gpu_launches": int(launches),
           "clocks": clk.summary()}

    # per-kernel-class times by CUDA events over the same number of steps
    # (kernel by kernel: a replayed graph records no per-launch events)
    F.set_graph(False)
    F.set_profiling(True)
    for _ in range(args.steps):
        step()
    st = F.stats()
    F.set_profiling(False)
    F.set_graph(True)
    # the paper's three classes; the explicit diagonal inverses are part of
    # how GESSM / TSTRF run here, so their time counts under the panel
    fcls = plan.flops_by_class()
    cls_ms = {k: v / args.steps for k, v in st["ms"].items()}
    cls_ms["panel"] += cls_ms.pop("inv")
    dom = max(("getrf", "panel", "ssssm"), key=lambda k: cls_ms[k])
    names = {"getrf": "k_getrf_dense", "panel": "k_inv+k_panel_inv",
             "ssssm": "k_ssssm_gemm" if args.precision == "fp64" else "k_ssssm_tc"}
    if args.precision == "fp64":
        peak, bound = fp64_peak_tflops(torch), "alu"
        peak_src = ("cuBLAS DGEMM 4096^3 measured live in this run (FP64 has no "
                    "driver-measured peak; nominal 1.25 TFLOP/s)")
    elif dom == "ssssm":
        # TF32 tensor peak = measured BF16 peak x nominal TF32/BF16 ratio
        # (1.1 / 2.25); the tile runs 3 TF32 MMAs per useful product
        peak, bound = measured_peak("bf16_tflops", 1800.0) * 1.1 / 2.25, "tensor"
        peak_src = "MEASURED_PEAKS.json bf16_tflops x 1.1/2.25 (TF32), 3 MMAs per product"
    else:
        peak, bound = 148 * 128 * 2 * 2.032e9 / 1e12, "alu"
        peak_src = "FP32 FMA: 148 SMs x 128 lanes x 2 flop x 2.032 GHz"
    ach = fcls[dom] / (cls_ms[dom] * 1e-3) / 1e12
    calls = {k: v // args.steps for k, v in st["calls"].items()}
    calls["panel"] += calls.pop("inv")
    out["roofline"] = {
        "kernel": names[dom], "bound": bound, "achieved": ach, "peak": peak,
        "unit": "TFLOP/s", "frac": ach / peak,
        "traffic": recorded_traffic(names[dom], args.workload, calls[dom]),
        "peak_source": peak_src,
        "frac_by_class": {k: fcls[k] / (cls_ms[k] * 1e-3) / 1e12 / peak
                          for k in ("getrf", "panel", "ssssm") if cls_ms[k] > 0},
        "ms_per_step_by_class": cls_ms,
        "flops_per_step_by_class": fcls,
        "launches_per_step_by_class": calls}

    if not args.no_extras:
        extras = {}
        # FP32 factors + FP64 refinement
        best32, tun32 = tune(s.n, s.colptr, s.rowidx, vals_d, rhs_d,
                             precision="fp32")
        p32 = S.Plan(s.n, s.colptr, s.rowidx, precision="fp32", **best32)
        F32 = S.Factor(p32, vals_d)

        def step32():
            F32.refactor(vals_d)
            F32.solve(rhs_d)
        ms32 = timed(torch, step32, args.steps, 2)
        _, i32 = F32.solve(rhs_d, info=True)
        extras["fp32_ir"] = {"ms_per_step": ms32, "tuned": best32,
                             "gflops": fl / (ms32 * 1e-3) / 1e9,
                             "backward_error": i32["backward_error"],
                             "ir_iterations": i32["iterations"]}
        del F32
        # regular blocking, same code
        bestr, _ = tune(s.n, s.colptr, s.rowidx, vals_d, rhs_d,
                        precision="fp64", blocking="regular", regular_block=128)
        preg = S.Plan(s.n, s.colptr, s.rowidx, blocking="regular",
                      regular_block=128, **bestr)
        Freg = S.Factor(preg, vals_d)

        def stepreg():
            Freg.refactor(vals_d)
            Freg.solve(rhs_d)
        msr = timed(torch, stepreg, args.steps, 2)
        extras["regular128_fp64"] = {"ms_per_step": msr, "tuned": bestr,
                                     "gflops": fl / (msr * 1e-3) / 1e9,
                                     "levels": preg.info["nlevels"]}
        del Freg
        # the regular blocking tuned over block size and threshold (as many
        # candidates as the irregular search), FP64 and FP32 + refinement;
        # these legs launch kernel by kernel, so the FP64 ratios are taken
        # against the irregular step launched the same way
        from paper_2512_04389_b300.tune import candidates
        for prec in ("fp64", "fp32"):
            bt, tt = tune(s.n, s.colptr, s.rowidx, vals_d, rhs_d, precision=prec,
                          cands=candidates("regular_sizes", s.n))
            pt = S.Plan(s.n, s.colptr, s.rowidx, precision=prec, **bt)
            Ft = S.Factor(pt, vals_d)

            def stept():
                Ft.refactor(vals_d)
                Ft.solve(rhs_d)
            mst = timed(torch, stept, args.steps, 2)
            extras[f"regular_tuned_{prec}"] = {
                "ms_per_step": mst, "tuned": bt, "gflops": fl / (mst * 1e-3) / 1e9,
                "levels": pt.info["nlevels"], "tuning_ms": tt,
                "irregular_speedup": mst / (ms_direct if prec == "fp64" else ms32)}
            del Ft, pt
            # the regular-size selection policy (no timing runs): its size
            # and threshold 0, the tuned choice on these grids
            ps_ = S.Plan(s.n, s.colptr, s.rowidx, precision=prec,
                         blocking="regular_select", dense_threshold=0.0)
            Fs = S.Factor(ps_, vals_d)

            def steps_():
                Fs.refactor(vals_d)
                Fs.solve(rhs_d)
            mss = timed(torch, steps_, args.steps, 2)
            extras[f"regular_select_{prec}"] = {
                "ms_per_step": mss, "regular_block": ps_.info["regular_block"],
                "gflops": fl / (mss * 1e-3) / 1e9,
                "irregular_speedup": mss / (ms_direct if prec == "fp64" else ms32)}
            del Fs, ps_
        bestr32, _ = tune(s.n, s.colptr, s.rowidx, vals_d, rhs_d,
                          precision="fp32", blocking="regular", regular_block=128)
        preg32 = S.Plan(s.n, s.colptr, s.rowidx, blocking="regular",
                        regular_block=128, precision="fp32", **bestr32)
        Freg32 = S.Factor(preg32, vals_d)

        def stepreg32():
            Freg32.refactor(vals_d)
            Freg32.solve(rhs_d)
        msr32 = timed(torch, stepreg32, args.steps, 2)
        extras["regular128_fp32_ir"] = {"ms_per_step": msr32, "tuned": bestr32,
                                        "gflops": fl / (msr32 * 1e-3) / 1e9}
        del Freg32
        legs = [("batch_256_grid5", batch_leg), ("grid5_48", small_grid_leg),
                ("autograd_theta_32", autograd_leg)]
        if not args.no_circuit:
            legs.append(("circuit_200k", circuit_leg))
        run_legs(extras, legs, torch, S, dev, args)
        out["extras"] = extras
        # end to end through the public API with host buffers
        vals_h = torch.from_numpy(np.ascontiguousarray(s.values)).pin_memory()
        rhs_h = torch.from_numpy(np.ascontiguousarray(s.rhs.T)).pin_memory()
        x_h = torch.empty((s.nrhs, s.n), dtype=torch.float64).pin_memory()
        rhs_dt = torch.empty((s.nrhs, s.n), dtype=torch.float64, device="cuda")

        def step_e2e():
            vals_d.copy_(vals_h, non_blocking=True)
            rhs_dt.copy_(rhs_h, non_blocking=True)
            F.refactor(vals_d)
            X = F.solve(rhs_dt.t())
            x_h.copy_(X.t(), non_blocking=True)
        mse = timed(torch, step_e2e, args.steps, 1)
        out["e2e"] = {"value": fl / (mse * 1e-3) / 1e9, "unit": "GFLOP/s",
                      "ms_per_step": mse,
                      "h2d_bytes_per_step": 8 * (s.nnz + s.n * s.nrhs),
                      "d2h_bytes_per_step": 8 * s.n * s.nrhs}
        out["cpu_baseline"] = cpu_oracle_leg()
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
