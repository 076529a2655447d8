"""Benchmark: converged space-time DOF/s of the all-at-once BDF1 Newton solver.

Workload (N = 1): viscous Burgers, 256 x 256 interior nodes on [0,1]^2, nu = 0.01,
zero Dirichlet data, u0 = sin(2 pi x) sin(2 pi y), dt = 1e-3, M = 256 levels,
FP64 throughout, plain initial guess u^n = u^0, Newton to ||R||_inf <= 1e-12.
One step = one converged solve (plain guess -> residual/assembly/level chain per
Newton iteration -> converged U), inputs resident in HBM. The working set
(U, R, five Jacobian planes: ~0.94 GB) is larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun, one rank per GPU) runs independent replicas of the workload
(the single solve does not shard; weak scaling, no data-path collective).
--impl reference times the FP64 CPU oracle (all host cores) on a bounded sample of
the same workload (its first levels: the system is block lower-triangular in time,
so the first L levels form a closed problem).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged space-time DOF/s at ≤1e-10 rel. error; plain vs mixed/batched/learned"
UNIT = "DOF/s"
# GB300's nominal FP64 rate from its unit counts and clock: 152 SMs x 2 FP64 FMA per
# SM-clock x 2 flops x 2.07 GHz. The roofline uses the rate measured in the same run
# (pit_probe_fma_peak); this is only printed beside it.
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Algorithmic FP64 flops (FMA = 2) per unknown: one red-black SOR update
# (4 couplings, rhs, relaxation) and one BiCGStab iteration (2 SpMV + 6 axpy + 5 dots).
FLOPS_PER_SOR_UPDATE = 11
FLOPS_PER_BICGSTAB_ITER = 2 * 9 + 6 * 2 + 5 * 2
# DRAM bytes (read + write) of one wavefront launch on this workload, from an ncu capture
# of the kernel sources whose SHA-256 digests are listed (null once they change).
WAVE_TRAFFIC_BYTES = 579169024 + 293091072
WAVE_TRAFFIC_SOURCES = {
    "paper_2406_00878_gb300/csrc/pit_kernels.cuh": "fd63019189123d130c4fe289b9eb5246bd131938853eac81834b01d5b218b414",
    "paper_2406_00878_gb300/csrc/pit.cu": "f97dba1890ee46fe429a3ce32e51be68be3e33a6cafe4ffb5b5600e038ba9146",
}


def wave_traffic(levels: int):
    import hashlib
    if levels != 256 or not WAVE_TRAFFIC_BYTES or not WAVE_TRAFFIC_SOURCES:
        return None
    root = os.path.dirname(os.path.abspath(__file__))
    for rel, digest in WAVE_TRAFFIC_SOURCES.items():
        with open(os.path.join(root, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    return WAVE_TRAFFIC_BYTES


def host_cores() -> int:
    return len(os.sched_getaffinity(0))


# per node and Newton iteration, Burgers with constant viscosity: residual (convective
# and viscous differences, time term) and the four scaled couplings
FLOPS_PER_RESIDUAL = 18
FLOPS_PER_JACOBIAN = 8


def _dist():
    from paper_2406_00878_gb300 import dist
    return dist.env()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms from before the warm-up
    (the tool takes a while to start); only samples that arrive between region_start()
    and region_end() describe the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []          # (arrival time, line)
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def region_start(self):
        self.t0 = time.monotonic()

    def region_end(self):
        self.t1 = time.monotonic()

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for t, ln in self.lines if self.t0 is not None and self.t0 <= t <= (self.t1 or t) + 0.05]
        for ln in inside:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args, ws, rank, local):
    import torch
    from paper_2406_00878_gb300 import dist as D
    from paper_2406_00878_gb300 import pit
    from paper_2406_00878_gb300 import workloads as W

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = W.burgers256(seed=0, M=args.levels)
    stream = torch.cuda.Stream()
    # the FP64 and FP32 FMA rates of this GPU, measured before the timed region
    fp64_peak = pit.pit_probe_fma_peak(0, stream=stream)
    fp32_peak = pit.pit_probe_fma_peak(1, stream=stream)
    with torch.cuda.stream(stream):
        ctx = pit.context_for(p, stream=stream)
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")

        def step():
            pit.pit_fill_plain_guess(ctx, U)
            return pit.pit_solve(ctx, U)[1]

        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        with ClockSampler(local) as clk:
            for _ in range(max(args.warmup, 0)):
                info = step()
            stream.synchronize()
            D.barrier()
            torch.cuda.synchronize()
            clk.region_start()
            e0.record(stream)
            for _ in range(args.steps):
                infos.append(step())
            e1.record(stream)
            e1.synchronize()
            clk.region_end()
        torch.cuda.synchronize()
        D.barrier()
        ms = D.max_over_ranks(e0.elapsed_time(e1) / args.steps, device="cuda")
        Ug = U.cpu().numpy().reshape(p.M, -1)

        # end to end through the host-buffer entry point: H2D u0 + solve + D2H U
        u0_h = torch.from_numpy(np.ascontiguousarray(p.u0)).pin_memory()
        U_h = torch.empty(p.dof, dtype=torch.float64).pin_memory()
        for _ in range(2):
            pit.pit_solve_host(ctx, u0_h, U_h)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pit.pit_solve_host(ctx, u0_h, U_h)
        e2e_s = D.max_over_ranks((time.perf_counter() - t0) / args.steps, device="cuda")
        ctx.close()

    last = infos[-1]
    k = last["newton_iters"]
    steps = last["steps"]
    wave = last["wave_teams"] > 0
    ms_res = sum(s["ms_residual"] for s in steps)
    ms_asm = sum(s["ms_assemble"] for s in steps)
    ms_sol = sum(s["ms_solve"] for s in steps)
    # algorithmic FP64 flops of the level solves, from the measured sweeps / iterations
    flops = 0.0
    for s in steps:
        it = s["lin_iters_mean"] * p.M
        frac_sor = s["levels_sor"] / p.M
        flops += p.grid.ns * (it * frac_sor * FLOPS_PER_SOR_UPDATE + it * (1 - frac_sor) * FLOPS_PER_BICGSTAB_ITER)
    if wave:
        # one wavefront launch does residual, Jacobian and level solves of every iteration
        launches = 1 + last["wave_launches"] + 1  # plain guess + wavefront + final residual
        flops += k * p.dof * (FLOPS_PER_RESIDUAL + FLOPS_PER_JACOBIAN)
        kernel_ms = last["ms_wave"] / max(last["wave_launches"], 1)
        flops_per_launch = flops / max(last["wave_launches"], 1)
        kernel_name = "wave_kernel (Newton wavefront: residual, Jacobian, nested inverse of eq. 7)"
    else:
        launches = 1 + 3 * k + 1  # plain guess + (residual, assembly, chain) per update + final residual
        kernel_ms = ms_sol / max(k, 1)
        flops_per_launch = flops / max(k, 1)
        kernel_name = "chain_kernel (level chain, eq. 7 nested inverse)"
    achieved_tflops = flops_per_launch / (kernel_ms * 1e-3) / 1e12
    out = None
    if rank == 0:
        value = D.job_throughput([p.dof] * ws, ms * 1e-3)
        acc = oracle_accuracy(p, Ug, 6) if args.check else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"burgers256: 2-D viscous Burgers 256x256 interior, nu=0.01, dt=1e-3, "
                                   f"M={p.M}, u0=sin(2pi x)sin(2pi y), plain guess, Newton to ||R||_inf<=1e-12",
                       "dof_per_solve": p.dof, "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "inputs larger than L2 (U, R, 5 Jacobian planes ~0.94 GB); no flush",
                       "newton_iters": k, "res_inf": last["res_inf"],
                       "lin_iters_mean_per_level": [round(s["lin_iters_mean"], 2) for s in steps],
                       "levels_sor": [s["levels_sor"] for s in steps],
                       "stage_ms": {"residual": ms_res, "assemble": ms_asm, "level_chain": ms_sol},
                       "wavefront": {"teams": last["wave_teams"], "ctas_per_team": last["wave_team_ctas"],
                                     "launches": last["wave_launches"], "ms": last["ms_wave"],
                                     "cta0_us": {"predecessor_wait": round(last["us_pred_wait"], 1),
                                                 "halo_wait": round(last["us_halo_wait"], 1),
                                                 "reduce_wait": round(last["us_reduce_wait"], 1),
                                                 "level_setup": round(last["us_setup"], 1),
                                                 "level_solve": round(last["us_level_solve"], 1),
                                                 "update": round(last["us_update"], 1)}} if wave else None,
                       "accuracy_vs_oracle": acc},
            "gpu_launches": launches * args.steps,
            "e2e": {"value": D.job_throughput([p.dof] * ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(p.grid.ns * 8),
                    "d2h_bytes_per_step": int(p.dof * 8)},
            "roofline": {"kernel": kernel_name, "bound": "alu",
                         "achieved": achieved_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": achieved_tflops / fp64_peak,
                         "traffic": wave_traffic(args.levels) if wave else None,
                         "traffic_unit": "bytes per launch (ncu dram read + write)",
                         "peak_source": "measured in this run: FP64 FMA-chain probe (pit_probe_fma_peak, best of 5)",
                         "nominal_peak": FP64_NOMINAL_TFLOPS, "fp32_peak_measured": fp32_peak},
            "clocks": clk.summary(),
        }
        if args.variants:
            out["variants"] = variants(args, Ug)
        if args.cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return out


# ----------------------------------------------------------------- oracle legs
# The FP64 CPU oracle enters the benchmark in two places only: the CPU baseline
# (cpu_baseline, run_reference) and the accuracy record of every GPU result
# (oracle_accuracy), computed after the timed regions. The timing build of the oracle
# (element-independent loops on all host cores) returns the same bits as the tested
# single-threaded build.

def oracle_accuracy(p, U, levels, bc_q=True):
    """Error of a GPU solution U [M, Ns] against the oracle: the oracle solves the first
    `levels` levels itself (the system is block lower-triangular in time, so they form a
    closed problem) and evaluates its residual of U at every level."""
    import oracle
    from paper_2406_00878_gb300 import workloads as W
    oracle.use_threads(host_cores())
    try:
        L = min(levels, p.M)
        Uo, _, _, _ = oracle.solve(W.truncated(p, L), tol=1e-13)
        err = float(np.abs(U[:L] - Uo).max() / np.abs(Uo).max())
        R = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, U, p.bc, p.q)
        res = float(np.abs(R).max())
    finally:
        oracle.use_threads(1)
    return {"max_rel_err_first_levels_vs_oracle": err, "levels_solved_by_oracle": L,
            "oracle_res_inf_all_levels": res, "ok": bool(err <= 1e-10 and res <= 2e-12)}


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _solve_timed(p, opt, steps, stream):
    """pit_solve of problem p from the plain guess, `steps` times after one warm-up; returns
    (ms per solve, last info, solution [M, Ns] on the host)."""
    import torch
    from paper_2406_00878_gb300 import pit
    with torch.cuda.stream(stream):
        ctx = pit.context_for(p, opt, stream=stream)
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
        pit.pit_fill_plain_guess(ctx, U)
        pit.pit_solve(ctx, U)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            pit.pit_fill_plain_guess(ctx, U)
            _, info = pit.pit_solve(ctx, U)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        Uh = U.cpu().numpy().reshape(p.M, -1)
        ctx.close()
    return ms, info, Uh


def variants(args, U_headline):
    """The other forms of the metric on this GPU, each with its error against the oracle:
    heat32 (the small plain-method workload, with the oracle's CPU seconds), FP32 level
    solves in FP64 Newton on the headline workload, the discontinuous 512 x 512, M = 1024
    workload (FP32 inner, windows of 32) beside its FP64 solve, 64 batched problems in one
    graph-replayed launch beside per-problem loops, the paper's own forms, and the learned
    initial guess with the combined learned + FP32 + batched form."""
    import torch
    from paper_2406_00878_gb300 import pit
    from paper_2406_00878_gb300 import workloads as W
    out = {}
    stream = torch.cuda.Stream()
    out["heat32"] = heat32_variant(args, stream)
    # FP32 level solves on the headline workload
    p = W.burgers256(seed=0, M=args.levels)
    opt = pit.pit_default_options()
    opt.precision = pit.PIT_FP32_INNER
    ms, info, Ug = _solve_timed(p, opt, 3, stream)
    out["mixed_fp32_inner"] = {
        "value": p.dof / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "dof": p.dof, "workload": p.name, "M": p.M,
        "window": 0, "precision": "fp32 level solves / fp64 newton", "newton_iters_total": info["newton_iters_total"],
        "res_inf_final": info["res_inf"][-1], "wave_teams": info["wave_teams"], "ctas_per_team": info["wave_team_ctas"],
        "max_rel_diff_vs_fp64_solution": _rel(Ug, U_headline),
        "accuracy_vs_oracle": oracle_accuracy(p, Ug, 6) if args.check else None}
    del Ug
    # the discontinuous workload: FP32 level solves, and FP64 level solves, windows of 32
    p = W.burgers512(seed=0)
    opt = pit.pit_default_options()
    opt.window = 32
    ms64, info64, U64 = _solve_timed(p, opt, 1, stream)
    opt.precision = pit.PIT_FP32_INNER
    ms, info, Ug = _solve_timed(p, opt, 2, stream)
    out["burgers512_mixed_window32"] = {
        "value": p.dof / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "dof": p.dof, "workload": p.name, "M": p.M,
        "window": 32, "precision": "fp32 level solves / fp64 newton", "newton_iters_total": info["newton_iters_total"],
        "res_inf_final": info["res_inf"][-1], "wave_teams": info["wave_teams"], "ctas_per_team": info["wave_team_ctas"],
        "fp64_same_workload": {"value": p.dof / (ms64 * 1e-3), "ms_per_step": ms64,
                               "newton_iters_total": info64["newton_iters_total"]},
        "max_rel_diff_vs_fp64_solution": _rel(Ug, U64),
        "accuracy_vs_oracle": oracle_accuracy(p, Ug, 2) if args.check else None}
    del Ug, U64
    out["batched64_mixed_window32"] = batched_variant(args, stream)
    out.update(paper_variants(args, U_headline, stream))
    if args.learned:
        out["learned_guess"] = learned_variant(args)
    return out


def heat32_variant(args, stream):
    """The heat32 workload (32 x 32, M = 16, mu = 1 + u^2): GPU DOF/s of the plain FP64 method,
    and the oracle's CPU seconds for sequential BDF1 (O1, one thread) and all-at-once Newton
    (O2, all host cores)."""
    import oracle
    from paper_2406_00878_gb300 import pit
    from paper_2406_00878_gb300 import workloads as W
    p = W.heat32(0)
    ms, info, Ug = _solve_timed(p, pit.pit_default_options(), 50, stream)
    oracle.use_threads(1)
    Uo, it, _, _ = oracle.solve(p, tol=1e-13)
    err = _rel(Ug, Uo)
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.sequential_bdf1(p.grid, p.params, p.M, p.dt, p.u0, p.bc, p.q, tol=1e-14)
    o1 = (time.perf_counter() - t0) / reps
    cores = host_cores()
    oracle.use_threads(cores)
    try:
        t0 = time.perf_counter()
        for _ in range(reps):
            oracle.solve(p, tol=1e-12)
        o2 = (time.perf_counter() - t0) / reps
    finally:
        oracle.use_threads(1)
    return {"value": p.dof / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "dof": p.dof, "workload": p.name,
            "precision": "fp64", "newton_iters": info["newton_iters"], "res_inf_final": info["res_inf"][-1],
            "cpu_seconds": {"o1_sequential_bdf1_1_thread": o1, "o2_all_at_once": o2, "o2_threads": cores},
            "accuracy_vs_oracle": {"max_rel_err_all_levels_vs_oracle": err, "levels_solved_by_oracle": p.M,
                                   "ok": bool(err <= 1e-10)}}


def batched_variant(args, stream):
    """64 independent problems of uneven size in one persistent launch (graph replay), FP32
    level solves, windows of 32, grids of 256^2 and up as wavefront jobs; beside it the same
    problems solved one by one with pit_solve (same windows), FP64 and FP32 level solves.
    Accuracy: the oracle's residual of every batched solution at every level, its solve of
    the first two levels of every problem, and the batched solutions against the FP64 loop's."""
    import torch
    import oracle
    from paper_2406_00878_gb300 import pit
    from paper_2406_00878_gb300 import workloads as W
    probs = W.batched(seed=0)
    dof = sum(p.dof for p in probs)
    opt = pit.pit_default_options()
    opt.precision = pit.PIT_FP32_INNER
    opt.window = 32
    with pit.pit_batch_create(probs, opt) as batch:
        pit.pit_batch_solve(batch)
        st, info = pit.pit_batch_solve(batch)
        res = max(pit.pit_batch_result(batch, i)["res_inf"] for i in range(len(probs)))
        wave_dof = sum(p.dof for i, p in enumerate(probs) if pit.pit_batch_placement(batch, i)["teams"] > 1)
        sols = [t["U"].cpu().numpy().reshape(p.M, -1) for t, p in zip(batch.tensors, probs)]
    loops = {}
    worst_vs_fp64 = 0.0
    for name, prec in (("loop_fp64_pit_solve", pit.PIT_FP64), ("loop_fp32_inner_pit_solve", pit.PIT_FP32_INNER)):
        lopt = pit.pit_default_options()
        lopt.precision = prec
        lopt.window = 32
        total = 0.0
        conv = 0
        with torch.cuda.stream(stream):
            for i, p in enumerate(probs):
                ctx = pit.context_for(p, lopt, stream=stream)
                U = torch.empty(p.dof, dtype=torch.float64, device="cuda")
                pit.pit_fill_plain_guess(ctx, U)
                s, inf = pit.pit_solve(ctx, U, check=False)
                total += inf["ms_total"]
                conv += int(s == pit.PIT_OK)
                if prec == pit.PIT_FP64:
                    worst_vs_fp64 = max(worst_vs_fp64, _rel(sols[i], U.cpu().numpy().reshape(p.M, -1)))
                ctx.close()
        loops[name] = {"value": dof / (total * 1e-3), "ms": total, "converged": conv}
    acc = None
    if args.check:
        oracle.use_threads(host_cores())
        try:
            worst_res, worst_err = 0.0, 0.0
            for p, Ug in zip(probs, sols):
                R = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, Ug, p.bc, p.q)
                worst_res = max(worst_res, float(np.abs(R).max()))
                del R
                Uo, _, _, _ = oracle.solve(W.truncated(p, 2), tol=1e-13)
                worst_err = max(worst_err, _rel(Ug[:2], Uo))
        finally:
            oracle.use_threads(1)
        acc = {"max_rel_err_first_levels_vs_oracle": worst_err, "levels_solved_by_oracle": 2,
               "oracle_res_inf_all_levels": worst_res, "problems_checked": len(probs),
               "ok": bool(worst_err <= 1e-10 and worst_res <= 2e-12)}
    return {
        "value": dof / (info["ms"] * 1e-3), "unit": UNIT, "ms_per_step": info["ms"], "dof": dof,
        "problems": len(probs), "grids": "64..384 squared", "levels": "32..512",
        "precision": "fp32 level solves / fp64 newton", "converged": info["converged"], "max_res_inf_final": res,
        "graph_replay": bool(info["graph"]), "team_ctas": [info["min_team"], info["max_team"]],
        "wave_jobs": info["wave_jobs"], "wave_job_dof": wave_dof, "wave_job_min_nodes": opt.batch_wave_nodes,
        "autotune_ms": info["ms_tuning"], "schedule_estimate_ms": info["est_makespan_ms"],
        "same_problems_one_by_one": loops,
        "speedup_vs_loop_fp64": loops["loop_fp64_pit_solve"]["ms"] / info["ms"],
        "speedup_vs_loop_fp32_inner": loops["loop_fp32_inner_pit_solve"]["ms"] / info["ms"],
        "max_rel_diff_vs_fp64_loop_solutions": worst_vs_fp64,
        "accuracy_vs_oracle": acc}


def _timed(stream, fn, steps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        r = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps, r


def paper_variants(args, U_headline, stream):
    """The paper's own forms: its coarse-grid + spline initial iterate (c_f = 3) on the
    bench workload, and Newton with the literal eq. 8 product form on its Burgers shock
    (63^2 x 12), next to the nested inverse on the same problem."""
    import torch
    from paper_2406_00878_gb300 import pit
    from paper_2406_00878_gb300 import workloads as W
    out = {}
    p = W.burgers256(seed=0, M=args.levels)
    with torch.cuda.stream(stream):
        ctx = pit.context_for(p, stream=stream)
        U = torch.empty(p.dof, dtype=torch.float64, device="cuda")

        def coarse_step():
            _, cinfo = pit.pit_coarse_guess(ctx, 3, U)
            _, info = pit.pit_solve(ctx, U)
            return cinfo, info

        _timed(stream, coarse_step, 1)
        ms, (cinfo, info) = _timed(stream, coarse_step, 2)
        ms_guess, _ = _timed(stream, lambda: pit.pit_coarse_guess(ctx, 3, U), 2)
        _timed(stream, coarse_step, 1)
        Ug = U.cpu().numpy().reshape(p.M, -1)
        ctx.close()
    out["coarse_guess_cf3"] = {
        "value": p.dof / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "ms_guess": ms_guess, "dof": p.dof,
        "workload": p.name, "M": p.M, "precision": "fp64",
        "guess": "coarse 84^2 x 85 solve + natural cubic splines in x, y, t (the paper's initial iterate, c_f = 3)",
        "newton_iters": info["newton_iters"], "coarse_newton_iters": cinfo["newton_iters"],
        "res_inf_first": info["res_inf"][0], "res_inf_final": info["res_inf"][-1],
        "max_rel_diff_vs_plain_guess_solution": _rel(Ug, U_headline),
        "accuracy_vs_oracle": oracle_accuracy(p, Ug, 6) if args.check else None}
    del Ug
    q = W.burgers_shock()
    with torch.cuda.stream(stream):
        ctx = pit.context_for(q, stream=stream)
        U = torch.empty(q.dof, dtype=torch.float64, device="cuda")

        def product_step():
            pit.pit_fill_plain_guess(ctx, U)
            return pit.pit_solve_product(ctx, U)[1]

        def nested_step():
            pit.pit_fill_plain_guess(ctx, U)
            return pit.pit_solve(ctx, U)[1]

        product_step()
        ms_p, ip = _timed(stream, product_step, 2)
        Up = U.cpu().numpy().reshape(q.M, -1)
        nested_step()
        ms_n, inn = _timed(stream, nested_step, 5)
        ctx.close()
    out["product_form_burgers_shock63x12"] = {
        "value": q.dof / (ms_p * 1e-3), "unit": UNIT, "ms_per_step": ms_p, "dof": q.dof, "workload": q.name,
        "precision": "fp64", "solver": "literal eq. 8: P^n by the Sec. 5 recursion, diag(P^n) scaling, banded LU",
        "newton_iters": ip["newton_iters"], "res_inf_final": ip["res_inf"][-1],
        "nested_inverse_same_problem": {"value": q.dof / (ms_n * 1e-3), "ms_per_step": ms_n,
                                        "newton_iters": inn["newton_iters"]},
        "accuracy_vs_oracle": oracle_accuracy(q, Up, q.M) if args.check else None}
    return out


def learned_variant(args):
    """The learned initial iterate on its workload (128^2, M = 128 Burgers, nu log-uniform in
    [1e-3, 1e-1]): `--learned-train` training solutions generated by the batched solver,
    8 epochs, `--learned-held-out` held-out problems solved in four forms (plain FP64
    pit_solve, learned + FP64 pit_solve, batched FP32 from the plain guess, and the
    combined learned + FP32 + batched form), each against the plain FP64 solutions, and the
    combined form's solutions against the oracle."""
    import oracle
    from paper_2406_00878_gb300 import learned
    from paper_2406_00878_gb300 import workloads as W
    cfg = learned.LearnedConfig(train=args.learned_train, held_out=args.learned_held_out, epochs=8)
    rep = learned.run(cfg, keep_solutions=args.check)
    forms = rep["forms"]
    acc = None
    if args.check:
        held, sol = rep["held_out"], rep["solutions"]["combined"]
        oracle.use_threads(host_cores())
        try:
            worst_res, worst_err = 0.0, 0.0
            for i, p in enumerate(held):
                Ug = sol[i].view(p.M, -1).cpu().numpy()
                R = oracle.residual(p.grid, p.params, p.M, p.dt, p.u0, Ug)
                worst_res = max(worst_res, float(np.abs(R).max()))
                if i < 8:
                    Uo, _, _, _ = oracle.solve(W.truncated(p, 4), tol=1e-13)
                    worst_err = max(worst_err, _rel(Ug[:4], Uo))
        finally:
            oracle.use_threads(1)
        acc = {"combined_form": {"oracle_res_inf_all_levels": worst_res, "problems_checked": len(held),
                                 "max_rel_err_first_levels_vs_oracle": worst_err, "levels_solved_by_oracle": 4,
                                 "problems_solved_by_oracle": min(8, len(held)),
                                 "ok": bool(worst_err <= 1e-10 and worst_res <= 2e-12)}}
        del rep["solutions"]
    plain = forms["plain"]["dof_per_s"]
    return {"value": forms["combined"]["dof_per_s"], "unit": UNIT,
            "workload": "burgers 128^2 x 128, nu log-uniform [1e-3, 1e-1], sine-series u0",
            "sample": f"{cfg.train} training solutions, {cfg.epochs} epochs, {cfg.held_out} held-out problems",
            "forms": forms,
            "combined_vs_plain_fp64": forms["combined"]["dof_per_s"] / plain if plain else None,
            "learned_vs_plain_fp64": forms["learned"]["dof_per_s"] / plain if plain else None,
            "learned_fp32_vs_plain_fp64": forms["learned_fp32"]["dof_per_s"] / plain if plain else None,
            "batched_vs_plain_fp64": forms["batched"]["dof_per_s"] / plain if plain else None,
            "newton_iters_plain": rep["newton_iters_plain_mean"],
            "newton_iters_learned": rep["newton_iters_learned_mean"],
            "train_tflops_bf16": rep["train_tflops"], "generation_dof_per_s": rep["generation_dof_per_s"],
            "loss_first_last": [rep["loss_first"], rep["loss_last"]],
            "accuracy_vs_oracle": acc}


def cpu_baseline(args, levels=None):
    """The FP64 oracle on the machine's host cores: all-at-once Newton (O2: the paper's method
    with the nested block inverse, banded LU / BiCGStab level solves) with its
    element-independent loops on every host core, on `levels` levels of the headline
    workload; and sequential BDF1 (O1, the paper's sequential reference, one thread) on
    its first `--o1-levels` levels."""
    import oracle
    from paper_2406_00878_gb300 import workloads as W
    L = levels or args.cpu_levels
    p = W.truncated(W.burgers256(seed=0, M=args.levels), L)
    oracle.build(openmp=True)
    cores = host_cores()
    used = oracle.use_threads(cores)
    try:
        t0 = time.perf_counter()
        oracle.solve(p, tol=1e-12)
        dt = time.perf_counter() - t0
    finally:
        oracle.use_threads(1)
    q = W.truncated(p, min(args.o1_levels, L))
    t0 = time.perf_counter()
    oracle.sequential_bdf1(q.grid, q.params, q.M, q.dt, q.u0, q.bc, q.q, tol=1e-14)
    dt1 = time.perf_counter() - t0
    return {"value": p.dof / dt, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"first {L} of {args.levels} levels of burgers256 ({p.dof} DOF), all-at-once Newton (O2) "
                      f"to 1e-12 on {used} threads, {dt:.1f} s",
            "o1_sequential_bdf1": {"value": q.dof / dt1, "unit": UNIT, "cores": 1, "seconds": dt1,
                                   "sample": f"first {q.M} levels of burgers256, Newton per step to 1e-14"}}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    import oracle
    from paper_2406_00878_gb300 import workloads as W
    p = W.truncated(W.burgers256(seed=0, M=args.levels), args.ref_levels)
    oracle.build(openmp=True)
    used = oracle.use_threads(host_cores())
    vals = []
    try:
        for _ in range(max(args.warmup, 0)):
            oracle.solve(p, tol=1e-12)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            oracle.solve(p, tol=1e-12)
            vals.append(p.dof / (time.perf_counter() - t0))
    finally:
        oracle.use_threads(1)
    value = statistics.median(vals)
    ms = p.dof / value * 1e3
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"burgers256 (first {args.ref_levels} of {args.levels} levels per step)",
                       "dof_per_step": p.dof},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"first {args.ref_levels} levels of burgers256 per step, all-at-once Newton "
                                       f"(O2) on {used} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--levels", type=int, default=256)
    ap.add_argument("--cpu-levels", type=int, default=256)
    ap.add_argument("--o1-levels", type=int, default=32)
    ap.add_argument("--ref-levels", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-check", dest="check", action="store_false")
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--no-learned", dest="learned", action="store_false")
    ap.add_argument("--learned-train", type=int, default=4096)
    ap.add_argument("--learned-held-out", type=int, default=256)
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    else:
        out = run_ours(args, ws, rank, local)
    if out is not None and rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
