"""Benchmark of the FP64 GKS S2O4 step (hybrid DF + WENO-AO reconstruction) on GB300.

Default workload: the seeded four-quadrant Riemann problem on a 400 x 400 mesh of [0,1]^2,
GKS flux, time limiter on, outflow boundaries, CFL 0.5 (seed 3; seed 2 draws a near-vacuum
rarefaction on which the scheme loses positivity at step 12, on the GPU and the oracle alike).  One benchmark "step" is one
full S2O4 step of Algorithm 1 (CFL dt, ghost fill, two stages of sweeps + update), i.e. two
cell-stage updates per cell.  Metric: FP64 cell-stage updates per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank advances its own replica of the
workload (independent problems, weak scaling); the timed region is bracketed by a barrier and
a device synchronisation and the maximum time over ranks is used.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "cell-stage/s"
SEED = 3
BENCH_N = 400          # mesh side of the benchmark workload; --n other than this is a scan, not the benchmark


def metric_name(n: int) -> str:
    return "FP64 cell-stage updates/s (GKS S2O4 step, four-quadrant %dx%d)" % (n, n)


def workload_name(n: int) -> str:
    return "quadrants_%dx%d_gks_seed%d" % (n, n, SEED)

# FP64 roofline denominator of this GPU: 152 SMs x 2 FP64 FMA units per SM per clock x 2 flops
# x 2070 MHz maximum SM clock = 1258.6 GFLOP/s (the recipe's nominal 1.25 TFLOP/s FP64 rate).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070

# Per-unit counts of the Gauss-point flux kernel (FP64 flops = 2*DFMA + DADD + DMUL per Gauss point,
# FP64-pipe instructions per Gauss point, DRAM bytes per launch at 400 x 400) are read from the
# machine-readable line of the committed ncu summary of that kernel, which also records a hash of
# the kernel sources it was measured on; the counts are used only while that hash matches.
FLUX_PROFILE = os.path.join(ROOT, "profiles", "k_flux_gks_counts.txt")


def profile_counts(path: str = FLUX_PROFILE):
    """(counts, reason): the machine-readable `counts:` line of a kernel's ncu summary, a JSON object
    with flops_per_unit, fp64_inst_per_unit, traffic_bytes_per_launch (at the benchmark size) and
    source_hash; counts is None with the reason when the file or line is missing or the forward
    kernels' sources have changed since the capture."""
    from paper_2402_10914_gb300 import build
    try:
        lines = [l for l in open(path) if l.startswith("counts:")]
    except OSError:
        return None, "no profile summary"
    if not lines:
        return None, "no counts line in the profile summary"
    c = json.loads(lines[-1][len("counts:"):])
    if c.get("source_hash") != build.kernel_source_hash():
        return None, "kernel sources changed since the ncu capture"
    return c, None
# steps of the oracle's timed sample (about 0.9 s each at 400 x 400 on 16 Arm cores)
CPU_SAMPLE_STEPS = 12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=400, help="mesh side of the four-quadrant workload")
    p.add_argument("--workload", default="quadrants",
                   choices=["quadrants", "batch", "adjoint", "blast", "robustness", "resolution"],
                   help="quadrants: the 400x400 GKS step (default); batch: the 64-problem uneven batch; "
                        "adjoint: gradient / forward time on the 256x256 vortex, 100 steps; "
                        "blast: the 1e6 pressure-ratio blast run to its end time; "
                        "robustness: maximum Mach numbers of the 123 problem and the hurricane-like flow; "
                        "resolution: the planar-shock (500^2) and planar-contact (800^2) Riemann problems")
    p.add_argument("--blast-n", type=int, default=2048, help="mesh side of the blast workload")
    p.add_argument("--blast-t", type=float, default=0.01, help="end time of the blast workload")
    p.add_argument("--no-adjoint", action="store_true", help="leave the adjoint summary out of the default line")
    p.add_argument("--no-batch", action="store_true", help="leave the 64-problem batch summary out of the default line")
    p.add_argument("--adj-n", type=int, default=256, help="mesh side of the adjoint workload")
    p.add_argument("--adj-steps", type=int, default=100, help="S2O4 steps of the adjoint workload")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def max_over_ranks(x: float, ws: int) -> float:
    """The maximum of x over all ranks (x itself on one rank).  NCCL reduces a device tensor, gloo
    (the CPU test backend) a host one."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, ws: int, max_ms: float) -> float:
    """Whole-job throughput of ws independent replicas (weak scaling): every rank processes the
    same units, and the job takes as long as its slowest rank."""
    return units_per_rank * ws / (max_ms * 1e-3)


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("DFGKS_BENCH_GLOO") is None else "gloo")
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def bench_ours(args, ws, rank, local):
    import torch
    from paper_2402_10914_gb300 import inputs as I
    from paper_2402_10914_gb300.solver import Solver

    torch.cuda.set_device(local)
    w = I.quadrants(args.n, seed=SEED)
    s = w.settings
    cells = s.nx * s.ny
    sol = Solver(s)
    sol.set_ic(w.W0)
    stream = sol.stream
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")   # 256 MiB > 129 MB L2
    # warm-up steps (untimed)
    sol.step(args.warmup)
    sol.set_timing(True)
    sol.timing(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))                     # evict the previous step's working set from L2
        starts[k].record(stream)
        done, _ = sol.step(1)
        ends[k].record(stream)
        assert done == 1
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, ws)
    timing = sol.timing()
    sol.set_timing(False)
    launches = sum(v["launches"] for v in timing.values())
    value = replica_throughput(2.0 * cells * args.steps, ws, total_ms)

    # roofline of the dominant kernel (the Gauss-point flux kernel)
    share = {k: v["ms"] for k, v in timing.items()}
    dominant = max(share, key=share.get)
    fl = timing["flux"]
    avg_flux_ms = fl["ms"] / max(fl["timed"], 1)
    # one flux launch per stage covers the Gauss points of both directions (fused x/y sweeps)
    gps_per_launch = 2.0 * ((s.nx + 1) * s.ny + (s.ny + 1) * s.nx)
    counts, why = profile_counts()
    traffic = counts.get("traffic_bytes_per_launch") if counts and args.n == BENCH_N else None
    roof = {"kernel": "k_flux_xy<GKS> (Gauss-point flux, x and y faces)", "bound": "alu", "unit": "GFLOP/s",
            "peak": round(FP64_PEAK_GFLOPS, 1), "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz",
            "avg_launch_ms": avg_flux_ms, "launches_timed": fl["timed"], "traffic": traffic,
            "traffic_unit": "B per launch (ncu dram read+write)",
            "kernel_time_share": {k: round(v / max(sum(share.values()), 1e-30), 4) for k, v in share.items()},
            "dominant_kernel_class": dominant,
            "counts_source": os.path.relpath(FLUX_PROFILE, ROOT) if counts else why}
    if counts:
        fpu = float(counts["flops_per_unit"])
        achieved = fpu * gps_per_launch / (avg_flux_ms * 1e-3) / 1e9
        roof.update({"achieved": round(achieved, 2), "frac": round(achieved / FP64_PEAK_GFLOPS, 4),
                     "flops_per_unit": fpu, "unit_of_work": "Gauss point",
                     "units_per_launch": gps_per_launch})
        if counts.get("fp64_inst_per_unit"):
            issue = float(counts["fp64_inst_per_unit"]) * gps_per_launch / (avg_flux_ms * 1e-3)
            roof["fp64_issue_frac"] = round(issue / (FP64_PEAK_GFLOPS / 2.0 * 1e9), 4)
        if traffic is not None:
            roof["dram_gbs"] = round(traffic / (avg_flux_ms * 1e-3) / 1e9, 1)
    else:
        roof.update({"achieved": None, "frac": None})
    # FP64 probe as a cross-check of the denominator
    try:
        import ctypes
        from paper_2402_10914_gb300 import _lib
        g, ms = ctypes.c_double(), ctypes.c_double()
        if _lib.lib().dfgks_probe_fp64(4000, ctypes.byref(g), ctypes.byref(ms)) == 0:
            roof["fp64_probe_gflops"] = round(g.value, 1)
    except Exception:
        pass

    # end to end through the C ABI with host buffers: H2D of the step's inputs from pinned memory,
    # the step, D2H of the result, every step
    e2e = None
    if not args.no_e2e:
        Wh = torch.empty((4, s.ny, s.nx), dtype=torch.float64, pin_memory=True).numpy()
        ah = torch.empty((s.ny, s.nx), dtype=torch.float64, pin_memory=True).numpy()
        W0, a0, t0, st0 = sol.get_state()
        Wh[...] = W0
        ah[...] = a0
        ke = max(5, min(args.steps, 20))
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        t_cur, step_cur = t0, st0
        for k in range(ke):
            sol.set_state(Wh, ah, t_cur, step_cur)
            sol.step(1)
            _, _, t_cur, step_cur = sol.get_state(out=(Wh, ah))
        torch.cuda.synchronize()
        e_ms = max_over_ranks((time.perf_counter() - e0) * 1e3, ws)
        nbytes = Wh.nbytes + ah.nbytes
        e2e = {"value": replica_throughput(2.0 * cells * ke, ws, e_ms), "unit": UNIT, "steps": ke,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    counters = sol.counters()
    sol.close()
    return {
        "value": value, "ms_per_step": total_ms / args.steps, "wall_s": wall, "launches": launches,
        "roofline": roof, "e2e": e2e, "clocks": clk, "counters": counters, "step_ms": step_ms,
        "per_kernel_ms_per_step": {k: v["ms"] / args.steps for k, v in timing.items()},
    }


BATCH_STEPS = 200       # S2O4 steps of the 64-problem batch


def batch_summary(steps: int = BATCH_STEPS, warmup: int = 3, cpu: bool = True) -> dict:
    """The 64-problem uneven batch (sides 64..512, mixed GKS / L-F, own dt each), advanced `steps`
    S2O4 steps by one launch of a CUDA graph holding all of them, against per-problem launches of
    the single-problem kernels one problem after another on one stream.  Both are timed with CUDA
    events on the stream they run on, after `warmup` untimed steps and a 256 MiB L2 flush, with
    nvidia-smi clocks sampled during both timed regions.  A problem that loses positivity stops at
    its last good step in both paths; only completed cell-stages count."""
    import torch
    from paper_2402_10914_gb300 import _lib, inputs as I
    from paper_2402_10914_gb300.solver import BatchSolver, Solver
    ws = I.batch()
    cells = sum(w.settings.nx * w.settings.ny for w in ws)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    b = BatchSolver([w.settings for w in ws], stream=stream)
    for p, w in enumerate(ws):
        b.set_ic(p, w.W0)
    blocks, _ = b.autotune()
    b.step(warmup, use_graph=True)
    b.prepare(steps)                                    # capture the steps-long graph, untimed
    before = [b.status(p)["step"] for p in range(len(ws))]
    clocks = ClockSampler(torch.cuda.current_device())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    flush.fill_(1.0)
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    rc = b.step(steps, use_graph=True)                  # one graph launch
    e1.record(stream)
    torch.cuda.synchronize()
    clk_b = clocks.stop()
    t_batch = e0.elapsed_time(e1) * 1e-3
    done_batch = [b.status(p)["step"] - before[p] for p in range(len(ws))]
    failed = [p for p in range(len(ws)) if b.status(p)["err"]]
    b.close()
    units = sum(2.0 * w.settings.nx * w.settings.ny * d for w, d in zip(ws, done_batch))
    sols = [Solver(w.settings, stream=stream) for w in ws]
    for sol, w in zip(sols, ws):
        sol.set_ic(w.W0)
        try:
            sol.step(warmup)
        except _lib.DfgksError:
            pass
    before_seq = [sol.get_state()[3] for sol in sols]
    clocks = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    flush.fill_(2.0)
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    for sol in sols:
        try:
            sol.step(steps)
        except _lib.DfgksError:
            pass
    e1.record(stream)
    torch.cuda.synchronize()
    clk_s = clocks.stop()
    t_seq = e0.elapsed_time(e1) * 1e-3
    done_seq = [sol.get_state()[3] - b0 for sol, b0 in zip(sols, before_seq)]
    units_seq = sum(2.0 * w.settings.nx * w.settings.ny * d for w, d in zip(ws, done_seq))
    for sol in sols:
        sol.close()
    out = {"workload": "batch64_uneven_seed1000_%dsteps" % steps, "problems": len(ws), "cells": cells,
           "steps": steps, "warmup": warmup, "value": units / t_batch, "unit": UNIT, "ms": t_batch * 1e3,
           "graph_launches": 1, "kernel_launches_in_graph": 21 * steps, "blocks": blocks, "status": rc,
           "problems_lost_positivity": failed, "cell_stages": units,
           "per_problem_sequential": {"value": units_seq / t_seq, "ms": t_seq * 1e3, "cell_stages": units_seq},
           "speedup_vs_per_problem": (units / t_batch) / (units_seq / t_seq),
           "clocks": clk_b, "clocks_per_problem": clk_s,
           "timing": "CUDA events on the stream both paths run on; 256 MiB L2 flush before each timed region"}
    if cpu:
        try:
            out["cpu_baseline"] = oracle_batch_sample(ws[:16])
        except Exception as e:
            out["cpu_baseline"] = {"value": None, "kind": "oracle", "sample": "failed: %s" % e}
    return out


def bench_batch(args):
    """--workload batch: the batch summary as its own line (steps = --steps, default 200)."""
    steps = args.steps if args.steps != 40 else BATCH_STEPS
    r = batch_summary(steps, max(args.warmup, 3), cpu=not args.no_cpu)
    line = {"metric": "FP64 cell-stage updates/s (64-problem uneven batch, mixed GKS/L-F)", "value": r["value"],
            "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": r["warmup"], "ms_per_step": r["ms"] / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": r["workload"], "problems": r["problems"], "cells": r["cells"],
                       "blocks": r["blocks"], "l2": "one 256 MiB flush before each timed region"},
            "batch": r, "clocks": r["clocks"], "gpu_launches": r["kernel_launches_in_graph"]}
    if "cpu_baseline" in r:
        line["cpu_baseline"] = r["cpu_baseline"]
    print(json.dumps(line))


def oracle_batch_sample(ws):
    """The CPU oracle as it stands on a bounded sample of the batch: one S2O4 step of each given
    problem, one after another, on all host cores."""
    import oracle
    cores = oracle.max_threads()
    units, t = 0.0, 0.0
    for w in ws:
        a0 = oracle.alpha0(w.settings, w.W0)
        t0 = time.perf_counter()
        rc, *_ = oracle.run(w.settings, w.W0, a0, 1)
        t += time.perf_counter() - t0
        if rc == 0:
            units += 2.0 * w.settings.nx * w.settings.ny
    return {"value": units / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one S2O4 step of each of the first %d problems (%.1f s)" % (len(ws), t)}


def bench_blast(args):
    """The extreme robustness run: 1e6 pressure ratio, reflecting walls, GKS, CFL 0.4, run to its end
    time with positivity checked on the device every step.  Reports the whole run's throughput."""
    import torch
    from paper_2402_10914_gb300 import _lib, inputs as I
    from paper_2402_10914_gb300.solver import Solver
    w = I.blast(args.blast_n, t_end=args.blast_t)
    s = w.settings
    sol = Solver(s)
    sol.set_ic(w.W0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    torch.cuda.synchronize()
    clocks.start()
    a.record(sol.stream)
    status = "reached t_end"
    try:
        sol.run(t_end=w.t_end, chunk=256)
    except _lib.DfgksError as e:
        status = "stopped: %s" % e
    b.record(sol.stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b)
    W, alpha, t, steps = sol.get_state()
    cnt = sol.counters()
    p = (s.gamma - 1.0) * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / W[0])
    sol.close()
    units = 2.0 * s.nx * s.ny * steps
    line = {"metric": "FP64 cell-stage updates/s (1e6 pressure-ratio blast, %dx%d, to t=%g)" % (s.nx, s.ny, w.t_end),
            "value": units / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": int(steps), "warmup": 0,
            "ms_per_step": ms / max(steps, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "blast_%dx%d_t%g" % (s.nx, s.ny, w.t_end), "flux": "GKS", "cfl": s.cfl,
                       "bc": "reflecting", "time_limiter": 1},
            "blast": {"status": status, "t": t, "min_rho": float(W[0].min()), "min_p": float(p.min()),
                      "gauss_point_fallbacks": cnt["fallbacks"], "df_normal": cnt["df_normal"],
                      "df_tangential": cnt["df_tangential"], "wall_ms": ms},
            "clocks": clk}
    print(json.dumps(line))


def bench_robustness(args):
    """Sect. 4.3 robustness measure: the largest Mach number at which a run keeps positivity, for
    the hybrid (DF + WENO-AO) and the plain WENO-AO reconstruction (alpha_thres = 0: the DF branch
    never fires), for the hybrid with the DF states taken from the cell averages beside each face
    (df_states = 1, an alternative to the paper's reading) and for the hybrid with alpha^{n+1} from a
    reconstruction of W^{n+1} (alpha_source = 1), GKS (S2O4) and L-F (SSP-RK3), with
    and without the Gauss-point fallback, on the 123 problem, the hurricane-like flow and the
    planar rarefactions (Tables 3-5).  Found by bisection in log Mach between 1 and 256 (12
    halvings; the planar rarefactions from 0.5)."""
    import torch
    from paper_2402_10914_gb300 import _lib, inputs as I
    from paper_2402_10914_gb300.solver import Solver

    def survives(make, ma, flux, thres, fb, dfs=0, asrc=0):
        w = make(ma, flux=flux)
        s = w.settings.with_(alpha_thres=thres, gp_fallback=fb, df_states=dfs, alpha_source=asrc)
        with Solver(s) as sol:
            try:
                sol.set_ic(w.W0)
                if w.t_end:
                    sol.run(t_end=w.t_end, chunk=512)
                else:
                    sol.step(w.steps)
            except _lib.DfgksError:
                return False
            W = sol.get_state()[0]
        return bool(np.isfinite(W).all())

    t0 = time.perf_counter()
    rows = []
    for name, make in (("123 problem (100 cells, t = 0.14)", I.problem_123),
                       ("hurricane-like (400 x 400, 50 steps)", I.hurricane),
                       ("planar rarefactions (400 x 400, t = 0.15)", I.planar_rarefaction)):
        for flux, fname in ((I.GKS, "GKS S2O4"), (I.LF, "L-F SSP-RK3")):
            # the hybrid with the paper's DF states, plain WENO-AO, the hybrid with the DF factor
            # taken from the cell averages beside each face (df_states = 1, not the paper's reading)
            # and the hybrid with alpha^{n+1} from a reconstruction of W^{n+1} (alpha_source = 1)
            for thres, rname, dfs, asrc in ((0.5, "hybrid", 0, 0), (0.0, "WENO-AO", 0, 0),
                                            (0.5, "hybrid, DF from cell averages", 1, 0),
                                            (0.5, "hybrid, DF updated from W^{n+1}", 0, 1)):
                for fb in (0, 1):
                    lo, hi = (0.5 if make is I.planar_rarefaction else 1.0), 256.0
                    if not survives(make, lo, flux, thres, fb, dfs, asrc):
                        res = "< %g" % lo
                    elif survives(make, hi, flux, thres, fb, dfs, asrc):
                        res = ">= 256"
                    else:
                        for _ in range(12):
                            mid = math.sqrt(lo * hi)
                            if survives(make, mid, flux, thres, fb, dfs, asrc):
                                lo = mid
                            else:
                                hi = mid
                        res = round(lo, 2)
                    rows.append({"problem": name, "solver": fname, "reconstruction": rname,
                                 "gauss_point_fallback": fb, "max_mach": res})
                    print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    line = {"metric": "maximum Mach number keeping positivity (Sect. 4.3 robustness measure)", "value": None,
            "unit": "Mach", "n_gpus": 1, "steps": None, "warmup": 0, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic", "config": {"workload": "robustness_123_hurricane_planar_rarefaction"},
            "robustness": rows, "wall_s": time.perf_counter() - t0}
    print(json.dumps(line))


def bench_resolution(args):
    """Sect. 4.2 resolution workloads run to their end times as throughput and regression runs: the
    planar-shock interaction (500 x 500, t = 0.6) and the planar-contact interaction (800 x 800 on
    [0,2]^2, t = 1.6), GKS/S2O4 and L-F/SSP-RK3, hybrid and plain WENO-AO (alpha_thres = 0).  Per run:
    steps, throughput, density extrema, and the density along the horizontal mid line summarised by
    its total variation (more resolved structure, more variation) and its L1 distance to the
    hybrid run's cut."""
    import torch
    from paper_2402_10914_gb300 import inputs as I
    from paper_2402_10914_gb300.solver import Solver
    rows = []
    for make, name in ((I.riemann_cfg3, "planar shocks 500x500 t=0.6"), (I.riemann_cfg6, "planar contacts 800x800 t=1.6")):
        for flux, fname in ((I.GKS, "GKS S2O4"), (I.LF, "L-F SSP-RK3")):
            cut_h = None
            for thres, rname in ((0.5, "hybrid"), (0.0, "WENO-AO")):
                w = make(flux=flux)
                s = w.settings.with_(alpha_thres=thres)
                with Solver(s) as sol:
                    sol.set_ic(w.W0)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    a.record(sol.stream)
                    steps, _ = sol.run(t_end=w.t_end, chunk=512)
                    b.record(sol.stream)
                    torch.cuda.synchronize()
                    ms = a.elapsed_time(b)
                    W, alpha, t, _ = sol.get_state()
                    cnt = sol.counters()
                rho = W[0]
                cut = rho[s.ny // 2]
                if cut_h is None:
                    cut_h = cut
                rows.append({"problem": name, "solver": fname, "reconstruction": rname, "steps": int(steps),
                             "t": t, "cell_stage_per_s": 2.0 * s.nx * s.ny * steps / (ms * 1e-3), "wall_s": ms * 1e-3,
                             "rho_min": float(rho.min()), "rho_max": float(rho.max()),
                             "midline_total_variation": float(np.abs(np.diff(cut)).sum()),
                             "midline_l1_to_hybrid": float(np.abs(cut - cut_h).mean()),
                             "df_cells_normal": cnt["df_normal"], "fallbacks": cnt["fallbacks"]})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    line = {"metric": "Sect. 4.2 resolution runs (throughput and mid-line density statistics)", "value": None,
            "unit": "cell-stage/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "riemann_cfg3_500_cfg6_800"}, "resolution": rows}
    print(json.dumps(line))


def adj_workload(n: int, nsteps: int, ckpt: int = 10) -> str:
    return "vortex_%dx%d_gks_%dsteps_ckpt%d" % (n, n, nsteps, ckpt)


def bench_adjoint(reps: int, warmup: int = 1, n: int = 256, nsteps: int = 100, ckpt: int = 10):
    """Cost of the gradient of J = sum rho^2 after nsteps GKS steps on the isentropic vortex (time
    limiter on), against the plain forward pass: the forward pass that keeps checkpoints plus the
    backward pass (segment recompute + reverse sweeps), divided by the plain forward pass over the
    same steps.  CUDA events on the solver's stream; a 256 MiB L2 flush before each timed region."""
    import torch
    from paper_2402_10914_gb300 import inputs as I
    from paper_2402_10914_gb300.solver import Solver, adjoint_checkpointed, forward_checkpointed
    w = I.vortex(n, steps=nsteps)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
    sol = Solver(w.settings)
    W0 = torch.as_tensor(w.W0, device="cuda")
    stream = sol.stream

    def timed(fn):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), out

    def plain():
        sol.set_ic(W0)
        return timed(lambda: sol.step(nsteps))[0]

    def gradient():
        t_f, dts = timed(lambda: forward_checkpointed(sol, W0, nsteps, ckpt))
        WT = sol.get_state(device=True)[0]
        WTb = torch.zeros_like(WT)
        WTb[0] = 2.0 * WT[0]
        sol.timing(reset=True)
        t_b, g = timed(lambda: adjoint_checkpointed(sol, WTb))
        return t_f, t_b, sol.timing(reset=True)

    sol.set_timing(True)
    for _ in range(warmup):
        plain()
        gradient()
    F, G = [], []
    for _ in range(reps):
        F.append(plain())
        G.append(gradient())
    sol.set_timing(False)
    sol.close()
    fwd = statistics.median(F)
    tf = statistics.median([g[0] for g in G])
    tb = statistics.median([g[1] for g in G])
    rev = G[-1][2]
    return {"workload": adj_workload(n, nsteps, ckpt), "ratio": (tf + tb) / fwd,
            "gradient_cell_stage_per_s": 2.0 * n * n * nsteps / ((tf + tb) * 1e-3), "forward_ms": fwd, "forward_checkpointed_ms": tf,
            "backward_ms": tb, "backward_over_forward": tb / fwd, "reps": reps,
            "backward_kernel_ms": {k: round(v["ms"], 3) for k, v in rev.items()},
            "definition": "(checkpointed forward + backward) / plain forward, same %d steps" % nsteps}


def oracle_adjoint_sample(n=32, steps=1):
    """The CPU oracle as it stands on the gradient of the vortex workload, on a bounded sample: its
    reverse sweep (a recorded forward pass, then the adjoints of every stage from the operation
    tape of its residual) over `steps` steps of the isentropic vortex on an n x n mesh.  That tape
    holds every operation of a stage (about 2 GB per step at 32 x 32), which puts the 256 x 256
    workload itself out of its reach."""
    import numpy as np
    import oracle
    from paper_2402_10914_gb300 import inputs as I
    w = I.vortex(n, steps=steps)
    s = w.settings
    cores = oracle.max_threads()
    dt = oracle.cfl_dt(s, w.W0)
    a0 = oracle.alpha0(s, w.W0)
    t0 = time.perf_counter()
    rc, W, _, _, _, _ = oracle.run(s, w.W0, a0, steps, dt_fixed=dt)
    t_fwd = time.perf_counter() - t0
    assert rc == 0
    WTb = np.zeros_like(W)
    WTb[0] = 2.0 * W[0]
    t0 = time.perf_counter()
    oracle.run_vjp(s, w.W0, [dt] * steps, WTb)
    t_grad = time.perf_counter() - t0
    return {"value": 2.0 * n * n * steps / t_grad, "unit": "cell-stage/s (gradient)", "cores": cores,
            "kind": "oracle", "sample": "gradient of J = sum rho^2 over %d step(s) of the %dx%d vortex" % (steps, n, n),
            "forward_s": t_fwd, "gradient_s": t_grad, "gradient_over_forward": t_grad / t_fwd}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for l in out.splitlines():
            if l.split(":")[0].strip() in ("Model name", "Model"):
                name = l.split(":", 1)[1].strip()
                if name and not name.isdigit():
                    return name
    except Exception:
        pass
    try:
        for l in open("/proc/cpuinfo"):
            if l.lower().startswith(("model name", "cpu model")):
                return l.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def oracle_cpu_baseline(n: int = 400, steps_all: int = CPU_SAMPLE_STEPS) -> dict:
    """The oracle as it stands on bounded samples of the benchmark workload: the first `steps_all`
    S2O4 steps on every host core, and the first step on one core."""
    import oracle
    nproc = oracle.max_threads()
    v, cores, dtw = oracle_sample(steps=steps_all, n=n)
    try:
        v1, _, dt1 = oracle_sample(n_threads=1, steps=1, n=n)
    finally:
        oracle.set_threads(nproc)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": "sample: the first %d S2O4 steps of the %dx%d workload on %d threads (%.1f s)"
                      % (steps_all, n, n, cores, dtw),
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": "sample: the first S2O4 step of the %dx%d workload on one thread (%.1f s)"
                                        % (n, n, dt1)}}


def oracle_sample(n_threads=None, steps=1, n=400):
    """The CPU oracle as it stands on one full S2O4 step of the same workload."""
    import oracle
    from paper_2402_10914_gb300 import inputs as I
    w = I.quadrants(n, seed=SEED)
    if n_threads:
        oracle.set_threads(n_threads)
    cores = oracle.max_threads()
    a0 = oracle.alpha0(w.settings, w.W0)
    t0 = time.perf_counter()
    rc, W, a, t, dts, st = oracle.run(w.settings, w.W0, a0, steps)
    dtw = time.perf_counter() - t0
    assert rc == 0
    return 2.0 * n * n * steps / dtw, cores, dtw


def main():
    args = parse()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        # the reference arm is the CPU oracle, rank 0 only
        if rank != 0:
            return
        import oracle
        oracle.build()
        cores = oracle.max_threads()
        for _ in range(args.warmup):
            oracle_sample(steps=1, n=args.n)
        times = []
        for _ in range(args.steps):
            v, cores, dtw = oracle_sample(steps=1, n=args.n)
            times.append(dtw)
        total = sum(times)
        value = 2.0 * args.n * args.n * args.steps / total
        line = {"metric": metric_name(args.n), "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": workload_name(args.n), "nx": args.n, "ny": args.n, "flux": "GKS", "time_limiter": 1,
                           "cfl": 0.5, "bc": "outflow", "seed": SEED},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": "one full S2O4 step of the %dx%d workload per benchmark step" % (args.n, args.n)},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import __graft_entry__
    __graft_entry__.build()
    if args.workload == "batch":
        if rank == 0:
            bench_batch(args)
        return
    if args.workload == "blast":
        if rank == 0:
            bench_blast(args)
        return
    if args.workload == "robustness":
        if rank == 0:
            bench_robustness(args)
        return
    if args.workload == "resolution":
        if rank == 0:
            bench_resolution(args)
        return
    if args.workload == "adjoint":
        if rank == 0:
            a = bench_adjoint(args.steps, args.warmup, n=args.adj_n, nsteps=args.adj_steps)
            line = {"metric": "adjoint/forward time ratio (gradient of sum rho^2 through %d GKS S2O4 steps)"
                              % args.adj_steps,
                    "value": a["ratio"], "unit": "x", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                    "ms_per_step": (a["forward_checkpointed_ms"] + a["backward_ms"]) / args.adj_steps,
                    "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                    "data": "synthetic", "config": {"workload": a["workload"], "nx": args.adj_n, "ny": args.adj_n,
                                                    "flux": "GKS", "time_limiter": 1, "ckpt_every": 10,
                                                    "l2": "flushed before each timed region"},
                    "adjoint": a}
            if not args.no_cpu:
                line["cpu_baseline"] = oracle_adjoint_sample()
            print(json.dumps(line))
        return
    r = bench_ours(args, ws, rank, local)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu:
        try:
            cpu = oracle_cpu_baseline(args.n)
        except Exception as e:  # the benchmark line must still be printed
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": "failed: %s" % e}
    line = {
        "metric": metric_name(args.n), "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.n), "nx": args.n, "ny": args.n, "flux": "GKS", "time_limiter": 1, "cfl": 0.5,
                   "bc": "outflow", "seed": SEED, "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": "replica per GPU" if ws > 1 else "single GPU"},
        "roofline": r["roofline"], "cpu_baseline": cpu, "e2e": r["e2e"], "gpu_launches": r["launches"],
        "clocks": r["clocks"], "per_kernel_ms_per_step": r["per_kernel_ms_per_step"], "counters": r["counters"],
    }
    if not args.no_batch and ws == 1:
        try:
            line["batch"] = batch_summary(BATCH_STEPS, 3, cpu=not args.no_cpu)
        except Exception as e:  # the benchmark line must still be printed
            line["batch"] = {"workload": "batch64_uneven_seed1000_%dsteps" % BATCH_STEPS, "value": None, "error": str(e)}
    if not args.no_adjoint and ws == 1:
        try:
            line["adjoint"] = bench_adjoint(1, 1)
        except Exception as e:  # the benchmark line must still be printed
            line["adjoint"] = {"workload": adj_workload(256, 100), "ratio": None, "error": str(e)}
        if not args.no_cpu:
            try:
                line["adjoint"]["cpu_baseline"] = oracle_adjoint_sample()
            except Exception as e:
                line["adjoint"]["cpu_baseline"] = {"value": None, "kind": "oracle", "sample": "failed: %s" % e}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
