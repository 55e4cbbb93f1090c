"""Benchmark of the D4orm denoising hot path on GB300.

One bench step = one full anytime solve (Algorithm 2: `iters` iterations of
`K` denoising steps, each step = sample rollout + fitness of N samples,
softmax weights, weighted-mean update; then apply + rollout + verdict) of the
selected synthetic workload.  Metric: sample-rollouts/s (rollout+fitness),
i.e. N * K * iters sample rollouts per step / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

Default workload: 16 3D holonomic robots on Fibonacci points of a 4 m sphere
with antipodal goals, T = 100, N = 8192, 100 steps x 5 iterations (the
largest single-GPU configuration).
Multi-GPU (torchrun): every rank solves its own replica (independent
instances, weak scaling); value = all ranks' sample rollouts / max time.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the comparison arm; the paper ships no code).
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

import scenarios  # noqa: E402

METRIC = "sample-rollouts/s (rollout+fitness)"
UNIT = "sample-rollouts/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="holo3d_n16",
                    choices=sorted(scenarios.WORKLOADS) + ["mixed512", "warmstart", "mppi_compare", "sensitivity"])
    ap.add_argument("--teams", type=int, default=200, help="held-out teams for --workload warmstart")
    ap.add_argument("--batch-count", type=int, default=512,
                    help="--workload mixed512: problems in the batch (fewer: a smaller case for profiling)")
    ap.add_argument("--batch-steps", type=int, default=100, help="--workload mixed512: denoising steps K")
    ap.add_argument("--batch-iters", type=int, default=5, help="--workload mixed512: iteration budget")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def f32_inst(inst):
    inst.start = inst.start.astype(np.float32).astype(np.float64)
    inst.goal = inst.goal.astype(np.float32).astype(np.float64)
    if inst.obstacles is not None:
        inst.obstacles = np.asarray(inst.obstacles).astype(np.float32).astype(np.float64)
    return inst


# ---------------------------------------------------------------------------
# algorithmic FP32 work of one sample rollout + fitness (FFMA = 2 flops,
# FADD/FMUL/FMNMX/FSETP/MUFU = 1), counted from the method, not the kernel:
#   per robot-timestep: sample u = clip(M + sigma eps): 4 d_u;
#                       Box-Muller per normal: 5;
#                       dynamics step: holonomic 8 d_p, unicycle 31, diff-drive 37;
#                       goal term of Eq. (4) + accumulation: 3 d_p + 4;
#   per unordered robot pair and timestep (Eq. (5)): 3 d_p + 1;
#   per robot, obstacle and timestep (obstacle penalty): 3 d_p + 1.
# ---------------------------------------------------------------------------
DYN_FLOPS = {scenarios.HOLO2D: 16, scenarios.HOLO3D: 24, scenarios.UNICYCLE: 31, scenarios.DIFFDRIVE4: 37}


def flops_per_sample_rollout(inst) -> int:
    d_x, d_u, d_p = inst.dims
    per_robot = 4 * d_u + 5 * d_u + DYN_FLOPS[inst.dyn] + 3 * d_p + 4
    per_pair = 3 * d_p + 1
    n_obs = 0 if inst.obstacles is None else len(inst.obstacles)
    return inst.T * (inst.n * per_robot + inst.n * (inst.n - 1) // 2 * per_pair + inst.n * n_obs * (3 * d_p + 1))


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# dominant kernel, from one ncu --set full capture of the kernel as it is now
# (summaries and commands in profiles/); a kernel changed since its capture
# must be dropped from this table (its traffic is then reported as null).
NCU_TRAFFIC_BYTES = {
    ("k_rollout_fitness_paired", "holo3d_n16_T100_N8192"): 86016,
    ("k_rollout_fitness_pipe", "unicycle_n8_T100_N2048"): 38400,
    ("k_rollout_fitness", "unicycle_n8_T100_N2048"): 45824,
}


def fp32_peak_tflops(sm_count: int, clock_mhz: float) -> float:
    # 128 FP32 lanes per SM, FFMA = 2 flops
    return sm_count * 128 * 2 * clock_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(torch):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(torch, world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(torch, world, value: float) -> float:
    """The largest value over all ranks (the job's time is its slowest rank)."""
    if world == 1:
        return value
    import torch.distributed as dist
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_instance(inst, rank: int):
    """Rank r solves its own replica of the workload: the same problem with
    instance tag r, so every rank draws its own noise (no data-path
    exchange; the job's throughput is the sum over ranks)."""
    inst.tag = rank
    return inst


def job_throughput(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def cpu_oracle_rate(inst, budget_s: float = 15.0, n_sample: int | None = None, threads: int = 1) -> dict:
    """The oracle, as it stands, on a bounded sample: one denoising step over
    the first n_sample samples (fitness of each, weights, weighted-mean
    update), repeated until ~budget_s of wall time, on `threads` host
    threads (the oracle's OpenMP loops over samples and robots)."""
    import oracle
    oracle.set_threads(threads)
    threads = min(threads, oracle.max_threads())
    op = oracle.Problem(n=inst.n, T=inst.T, dyn=inst.dyn, integ=inst.integ, dt=inst.dt, radius=inst.radius,
                        start=inst.start, goal=inst.goal, u_lo=inst.u_lo, u_hi=inst.u_hi,
                        eps_margin=inst.eps_margin, goal_tol=inst.goal_tol, v_max=inst.v_max,
                        obstacles=inst.obstacles)
    d_u = inst.dims[1]
    rng = np.random.default_rng(0)
    u_base = scenarios.random_controls(rng, inst, 0.5)
    du = scenarios.random_deformation(rng, inst, 0.3)
    if n_sample is None:
        # size the sample from a probe of 4 samples
        pp = oracle.Params(N=4, K=inst.K, lam=inst.lam, w_safe=inst.w_safe, beta0=inst.beta0, beta1=inst.beta1,
                           seed=inst.seed, tag=inst.tag)
        t0 = time.perf_counter()
        oracle.denoise_step(op, pp, 0, inst.K, u_base, du)
        per = (time.perf_counter() - t0) / 4
        n_sample = int(max(8, min(inst.N, budget_s / 3 / max(per, 1e-9))))
    pp = oracle.Params(N=n_sample, K=inst.K, lam=inst.lam, w_safe=inst.w_safe, beta0=inst.beta0, beta1=inst.beta1,
                       seed=inst.seed, tag=inst.tag)
    done, t_total, reps = 0, 0.0, 0
    while reps == 0 or (t_total < budget_s and reps < 1000):
        i = inst.K - (reps % inst.K)
        t0 = time.perf_counter()
        oracle.denoise_step(op, pp, 0, i, u_base, du)
        t_total += time.perf_counter() - t0
        done += n_sample
        reps += 1
    return {"value": done / t_total, "unit": UNIT, "cores": threads, "kind": "oracle", "samples": done,
            "sample": f"{reps} denoising step(s) of {n_sample} of the {inst.N} samples of {inst.name} "
                      f"(fitness + weights + update, FP64, {threads} thread(s)), {t_total:.1f} s"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline_line(inst, budget_s: float = 12.0) -> dict:
    """The oracle on every host core (the reported baseline) and on one."""
    cores = host_cores()
    full = cpu_oracle_rate(inst, budget_s=budget_s, threads=cores)
    one = cpu_oracle_rate(inst, budget_s=budget_s / 2, threads=1)
    full["one_thread"] = {"value": one["value"], "sample": one["sample"]}
    return full


def measure_fp32_peak(torch, g, reps: int = 10) -> dict:
    """Measured FP32 peak: the library's FFMA-chain probe over 8 CTAs of 256
    threads per SM (eight independent chains per thread), best of `reps`
    event-timed launches."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads, iters = sms * 8, 256, 4096
    out = torch.empty(blocks * threads, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        g.d4orm_fp32_fma_probe(out, blocks, threads, iters, stream=stream)
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.d4orm_fp32_fma_probe(out, blocks, threads, iters, stream=stream)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    flops = blocks * threads * iters * 16
    return {"tflops": flops / (best / 1e3) / 1e12, "launch_ms": best,
            "how": f"{blocks} x {threads} threads x {iters} iterations x 8 independent FFMA chains, best of {reps}"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    inst = f32_inst(scenarios.WORKLOADS[args.workload]())
    per_step_budget = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    cores = host_cores()
    probe = cpu_oracle_rate(inst, budget_s=0.0, n_sample=4 * cores, threads=cores)
    n_sample = int(max(8, min(inst.N, per_step_budget * probe["value"])))
    rates = []
    for s in range(args.warmup + args.steps):
        # exactly one step of n_sample samples on every host core
        r = cpu_oracle_rate(inst, budget_s=1e-9, n_sample=n_sample, threads=cores)
        if s >= args.warmup:
            rates.append(r["value"])
    value = float(np.mean(rates))
    ms = n_sample / value * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": inst.name, "samples_per_step": n_sample, "of_N": inst.N,
                       "threads": r["cores"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": f"one denoising step over {n_sample} of {inst.N} samples per bench step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


GRAPH_REPS = 50


def rollout_kernel_in_graph_ms(torch, g, prob, params, inst, du) -> float:
    """Average duration of the rollout + fitness kernel inside a CUDA graph:
    GRAPH_REPS calls of d4orm_sample_fitness (steps K, K-1, ...) captured on
    a side stream, replayed 5 times, timed with events on that stream."""
    base = torch.zeros_like(du)
    fit = torch.empty(inst.N, device="cuda")
    side = torch.cuda.Stream()
    g.d4orm_sample_fitness(prob.handle, params, 0, inst.K, base, du, fit, stream=side)   # workspace, attributes
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        for r in range(GRAPH_REPS):
            g.d4orm_sample_fitness(prob.handle, params, 0, inst.K - (r % inst.K), base, du, fit, stream=side)
    times = []
    with torch.cuda.stream(side):
        for rep in range(6):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(side)
            graph.replay()
            b.record(side)
            b.synchronize()
            if rep:
                times.append(a.elapsed_time(b) / GRAPH_REPS)
    return float(np.median(times))


def packing_summary(g, batch, count):
    """Problems rolled out two robots per lane and the autotuner's packing
    pilots (summed device ms per bucket, one robot vs two per lane)."""
    pk = g.d4orm_batch_packing(batch, count)
    names = {g.HOLO2D: "holo2d", g.HOLO3D: "holo3d", g.UNICYCLE: "unicycle", g.DIFFDRIVE4: "diffdrive4"}
    return {"paired_problems": sum(pk["paired"]),
            "pilot_ms_single_paired": {f"{names[d]}_{r}": [round(s * 1e-6, 3), round(q * 1e-6, 3)]
                                       for (d, r), (s, q) in pk["bucket_ns"].items() if s or q}}


def run_batched(args, torch, g, world, rank):
    """512 ragged problems (n ~ U{2..16}, T ~ U{40..120}, 40/30/30 % 2D
    holonomic / 3D holonomic / unicycle, 10 m box), N = 1024, 100 steps x up
    to 5 iterations with stop-on-success, in one persistent graph launch.
    The step's sample-rollout count is summed from each problem's iterations."""
    count, K, iters = args.batch_count, args.batch_steps, args.batch_iters
    insts = [f32_inst(i) for i in scenarios.mixed_batch(count=count, seed=2, N=1024)]
    for i in insts:
        i.K = K
    probs = [g.Problem(i) for i in insts]
    params = g.Params(n_samples=1024, n_steps=K, seed=0, instance_tag=rank * count)
    budget = g.Budget(max_iters=iters, stop_on_success=True)
    workload = "mixed512_batched" if (count, K, iters) == (512, 100, 5) else f"mixed{count}_K{K}_it{iters}_batched"
    outs = [torch.zeros((i.T, i.n, i.dims[1]), device="cuda") for i in insts]
    batch = g.d4orm_batch_create([p.handle for p in probs], params, autotune=True)
    info = g.d4orm_batch_info(batch)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        g.d4orm_batch_solve(batch, budget, outs, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    rollouts, flops, results = 0, 0, None
    barrier(torch, world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for st in range(args.steps):
            flush.zero_()
            ev[st][0].record(stream)
            results = g.d4orm_batch_solve(batch, budget, outs, stream=stream)
            ev[st][1].record(stream)
            for inst, r in zip(insts, results):
                rollouts += inst.N * inst.K * r["iters_run"]
                flops += flops_per_sample_rollout(inst) * inst.N * inst.K * r["iters_run"]
        torch.cuda.synchronize()
    barrier(torch, world)
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ms = max_over_ranks(torch, world, ms)
    per_step = rollouts / args.steps
    value = job_throughput(per_step, world, ms)
    # end to end: descriptors from host arrays, solve, plans read back
    u_host = [torch.empty(o.shape, dtype=torch.float32).pin_memory() for o in outs]
    e2e = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs = [g.Problem(i) for i in insts]
        b2 = g.d4orm_batch_create([h.handle for h in hs], params)
        g.d4orm_batch_solve(b2, budget, outs, stream=stream)
        for o, h in zip(outs, u_host):
            h.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
        g.d4orm_batch_destroy(b2)
        for h in hs:
            h.close()
    e2e_ms = max_over_ranks(torch, world, statistics.median(e2e))
    props = torch.cuda.get_device_properties(0)
    peak = fp32_peak_tflops(props.multi_processor_count, 2070.0)
    achieved = flops / args.steps / (ms / 1e3) / 1e12
    solved = sum(1 for r in results if r["first_success_iter"] >= 0)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on a bounded sample of the batch: one denoising step of
        # 2 s over the first samples of every 64th problem
        picks = insts[::64]
        cores = host_cores()
        parts = [cpu_oracle_rate(i, budget_s=2.0, threads=cores) for i in picks]
        secs = sum(p_["samples"] / p_["value"] for p_ in parts)
        cpu = {"value": sum(p_["samples"] for p_ in parts) / secs, "unit": UNIT, "cores": parts[0]["cores"],
               "kind": "oracle",
               "sample": f"{len(picks)} of the {count} problems (every 64th), one denoising step over their first "
                         f"samples each, FP64, {parts[0]['cores']} thread(s), {secs:.1f} s"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "problems": len(insts), "samples_N": 1024, "denoise_steps": K,
                   "max_iterations": iters, "stop_on_success": True, "sample_rollouts_per_step": per_step,
                   "threads_per_cta": info["threads_per_cta"], "ctas": info["ctas"],
                   "autotune_ms_128_256_512": info["tuned_ms"], "autotune_table": g.d4orm_batch_tuning(batch),
                   "packing": packing_summary(g, batch, len(insts)),
                   "parallelism": f"replicas{world}",
                   "l2": "flushed between timed steps (256 MB write)"},
        "e2e": {"value": per_step * world / (e2e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(sum(2 * i.n * i.dims[0] * 4 for i in insts)),
                "d2h_bytes_per_step": int(sum(i.T * i.n * i.dims[1] * 4 for i in insts)), "ms_per_step": e2e_ms},
        "gpu_launches": args.steps,
        "clocks": clocks.summary(),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_batched_solve",
                     "peak_basis": "FP32 lanes x 2 x 2070 MHz (152 SMs x 128)", "launch_ms": ms},
        "solved": solved,
        # share of the CTAs' time spent inside a problem (device clock of
        # each problem's own solve, summed, over CTAs x the launch): the rest
        # is the tail after the queue ran dry
        "cta_busy_fraction": sum(r["ms_total"] for r in results) / (info["ctas"] * ms),
        "median_ms_to_success": statistics.median([r["ms_to_success"] for r in results if r["ms_to_success"] > 0])
        if solved else None,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.d4orm_batch_destroy(batch)


def run_mppi_compare(args, torch, g, world, rank):
    """Mean time to the first feasible plan (collision-free, every robot within
    0.5 m of its goal) of the method and of MPPI on the same kernels: 16 2D
    holonomic robots on a 4 m antipodal circle (|a| <= 2, |v| <= 1.5),
    N = 2048, 100 steps per iteration, stop on success, 5 s deadline, at most
    50 iterations, --teams evaluation seeds, for each (w, lambda) of a small
    grid (the paper leaves both open); MPPI's sigma is tuned per setting on 8
    other seeds.  One problem at a time on the whole GPU.  The line's value
    is the method's mean time at w = 1, lambda = 0.3."""
    from paper_2503_12204_gb300 import compare as C
    inst = scenarios.holo2d_circle(16, 4.0, a_max=2.0, v_max=1.5)
    inst.goal_tol = 0.5
    grid = []
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for w, lam in C.SETTINGS:
            res = C.compare(torch, inst, 2048, 100, args.teams, C.SIGMAS, w_safe=w, temperature=lam,
                            log=lambda m: None)
            grid.append({"w": w, "lambda": lam, "method": res["method"], "mppi": res["mppi"],
                         "mppi_sigma": res["mppi_sigma"], "speedup_mean_ms": res.get("speedup_mean_ms")})
    primary = next(r for r in grid if r["w"] == 1.0 and r["lambda"] == 0.3)
    line = {
        "metric": "mean ms to first feasible plan (method vs MPPI, same kernels)",
        "value": primary["method"].get("mean_ms"), "unit": "ms", "n_gpus": world, "steps": args.teams, "warmup": 1,
        "ms_per_step": primary["method"].get("mean_ms"), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": inst.name, "robots": 16, "samples_N": 2048, "denoise_steps": 100,
                   "max_iterations": 50, "deadline_ms": 5000, "goal_tol_m": inst.goal_tol,
                   "mppi_sigma_candidates": list(C.SIGMAS), "settings_w_lambda": [list(x) for x in C.SETTINGS]},
        "grid": grid, "clocks": clocks.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sensitivity(args, torch, g, world, rank):
    """Success rate against denoising steps K (50, 100, 200) and iterations
    (1..5) for 10 and 16 robots of each dynamics, --teams runs each (seeds),
    every (dynamics, robots, K) one batched persistent launch; w = 1,
    lambda = 0.3, goals judged at 0.5 m.  The line's value is the 16-robot
    2D holonomic success rate within 5 iterations at K = 100."""
    from paper_2503_12204_gb300 import sweep as SW
    with ClockSampler(torch.cuda.current_device()) as clocks:
        rows = SW.sweep(torch, runs=args.teams, log=lambda m: None)
    primary = next(r for r in rows if r["dynamics"] == "holo2d" and r["robots"] == 16 and r["steps"] == 100)
    line = {
        "metric": "success rate within 5 iterations (16 robots, 2D holonomic, K=100)",
        "value": primary["success_within_iters"][-1], "unit": "fraction", "n_gpus": world, "steps": args.teams,
        "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "sensitivity_K_x_iterations", "runs": args.teams, "samples_N": 2048,
                   "steps_K": [50, 100, 200], "max_iterations": 5, "robots": [10, 16],
                   "dynamics": list(SW.DYNAMICS), "w": 1.0, "lambda": 0.3, "goal_tol_m": 0.5},
        "table": rows, "clocks": clocks.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_warmstart(args, torch, g, world, rank):
    """Median time to a collision-free plan with every robot within 0.5 m of
    its goal, learned warm start vs the plain method, on held-out random 2D
    holonomic teams (n 8..16, T = 80, N = 4096), one problem at a time on
    the whole GPU, with the network trained by paper_2503_12204_gb300.warmstart
    (weights shipped in the package)."""
    from paper_2503_12204_gb300 import warmstart as W
    desc, params_np, meta = W.load_weights(os.path.join(ROOT, "paper_2503_12204_gb300", "weights",
                                                        "setmlp_holo2d_T80.bin"))
    desc.max_batch = 1
    ws = g.d4orm_warmstart_create(desc)
    g.d4orm_warmstart_set_params(ws, params_np)
    teams = scenarios.warmstart_set(args.teams, seed=4)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        res, rows = W.evaluate(torch, ws, teams, g.Params(n_samples=4096, n_steps=100, seed=4), 30, 5,
                               log=lambda m: None)
    g.d4orm_warmstart_destroy(ws)
    a = res["all"]
    line = {
        "metric": "ms to collision-free, goal-reaching plan (median; learned warm start vs plain)",
        "value": a.get("median_ms_warm"), "unit": "ms", "n_gpus": world, "steps": args.teams, "warmup": 1,
        "ms_per_step": a.get("median_ms_warm"), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (set-MLP bf16)", "data": "synthetic",
        "config": {"workload": "warmstart_holo2d_T80", "teams": args.teams, "robots": "8..16", "samples_N": 4096,
                   "start_step": 30, "max_iterations": 5, "goal_tol_m": 0.5},
        "plain_median_ms": a.get("median_ms_plain"), "speedup": a.get("speedup"),
        "median_reward_ratio": a.get("median_reward_ratio"), "judged_worse_rate": a.get("judged_worse_rate"),
        "fallback_rate": a.get("fallback_rate"),
        "solved": {"plain": a["plain_solved"], "warm_after_judge": a["warm_solved"],
                   "warm_raw": a["warm_raw_solved"]},
        "timing": "median over every team; unsolved teams count at their budget time; a warm plan that fails or "
                  "scores > 1 % worse than the plain plan falls back to it with both solves' time charged",
        "n16": res["n16"], "n15_16": res["n15_16"], "by_size": res["by_size"], "batched": res["batched"],
        "clocks": clocks.summary(),
        "training": meta,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    world, rank, local = dist_setup(torch)
    if rank == 0:
        import importlib.util
        spec = importlib.util.spec_from_file_location(
            "d4orm_build", os.path.join(ROOT, "paper_2503_12204_gb300", "_build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()
    barrier(torch, world)
    import paper_2503_12204_gb300 as g

    if args.workload in ("mixed512", "warmstart", "mppi_compare", "sensitivity"):
        {"mixed512": run_batched, "warmstart": run_warmstart, "mppi_compare": run_mppi_compare,
         "sensitivity": run_sensitivity}[args.workload](args, torch, g, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    inst = replica_instance(f32_inst(scenarios.WORKLOADS[args.workload]()), rank)
    d_x, d_u, d_p = inst.dims
    prob = g.Problem(inst)
    params = g.Params(n_samples=inst.N, n_steps=inst.K, temperature=inst.lam, w_safe=inst.w_safe,
                      beta0=inst.beta0, beta1=inst.beta1, seed=inst.seed, instance_tag=inst.tag)
    budget = g.Budget(max_iters=inst.iters)
    stream = torch.cuda.current_stream()
    u_out = torch.zeros((inst.T, inst.n, d_u), device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    rollouts_per_step = inst.N * inst.K * inst.iters
    launches_per_step = inst.iters * (3 * inst.K + 1)

    for _ in range(args.warmup):
        g.d4orm_solve(prob.handle, params, budget, u_out, stream=stream)
    torch.cuda.synchronize()

    # ---------------- timed region: K solves on device-resident inputs
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    results = []
    barrier(torch, world)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for s in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            ev[s][0].record(stream)
            results.append(g.d4orm_solve(prob.handle, params, budget, u_out, stream=stream))
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    barrier(torch, world)
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    ms = max_over_ranks(torch, world, ms)
    value = job_throughput(rollouts_per_step, world, ms)

    # ---------------- end to end through the C ABI with host buffers
    start_h = torch.tensor(inst.start, dtype=torch.float32).pin_memory()
    goal_h = torch.tensor(inst.goal, dtype=torch.float32).pin_memory()
    u_h = torch.empty((inst.T, inst.n, d_u), dtype=torch.float32).pin_memory()
    e2e_ms = []
    for s in range(max(2, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = g.d4orm_problem_create(inst.n, inst.T, inst.dyn, inst.integ, inst.dt, inst.radius, start_h.numpy(),
                                   goal_h.numpy(), eps_margin=inst.eps_margin, goal_tol=inst.goal_tol,
                                   v_max=inst.v_max, u_lo=inst.u_lo, u_hi=inst.u_hi, obstacles=inst.obstacles)
        r = g.d4orm_solve(h, params, budget, u_out, stream=stream)
        u_h.copy_(u_out, non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        g.d4orm_problem_destroy(h)
    e2e = max_over_ranks(torch, world, statistics.median(e2e_ms))
    n_obs = 0 if inst.obstacles is None else len(inst.obstacles)
    h2d = 2 * inst.n * d_x * 4 + n_obs * 16
    d2h = inst.T * inst.n * d_u * 4 + 40  # plan + result struct

    # ---------------- per-kernel breakdown (same kernels, same launch shapes)
    nctrl = (inst.T, inst.n, d_u)
    du_a = torch.zeros(nctrl, device="cuda")
    du_b = torch.zeros(nctrl, device="cuda")
    base = torch.zeros(nctrl, device="cuda")
    kms = []
    for i in range(inst.K, 0, -1):
        kms.append(g.d4orm_denoise_step_timed(prob.handle, params, 0, i, base, du_a, du_b, stream=stream))
        du_a, du_b = du_b, du_a
    kms = np.array(kms)
    # the rollout kernel as the solve runs it: GRAPH_REPS launches of
    # d4orm_sample_fitness (the same kernel, same launch shape) captured in
    # one CUDA graph, replayed with events on the replaying stream
    k2_graph_ms = rollout_kernel_in_graph_ms(torch, g, prob, params, inst, du_a)
    k2_ms = k2_graph_ms
    step_ms = float(kms.sum(axis=1).mean())
    share = (kms.mean(axis=0) / kms.mean(axis=0).sum()).tolist()
    flops = flops_per_sample_rollout(inst) * inst.N
    k2_kind = g.d4orm_problem_rollout_kernel(prob.handle, inst.N)
    k2_name = {g.ROLLOUT_REGISTER: "k_rollout_fitness", g.ROLLOUT_PIPELINE: "k_rollout_fitness_pipe",
               g.ROLLOUT_PAIRED: "k_rollout_fitness_paired"}.get(k2_kind, "?")
    props = torch.cuda.get_device_properties(0)
    csum = clocks.summary()
    peak = fp32_peak_tflops(props.multi_processor_count, 2070.0)
    achieved = flops / (k2_ms / 1e3) / 1e12
    measured = measure_fp32_peak(torch, g)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": inst.name, "dynamics": scenarios.DYN_NAMES[inst.dyn], "robots": inst.n,
                   "horizon_T": inst.T, "samples_N": inst.N, "denoise_steps": inst.K, "iterations": inst.iters,
                   "obstacles": n_obs, "sample_rollouts_per_step": rollouts_per_step, "parallelism": f"replicas{world}",
                   "l2": "flushed between timed steps (256 MB write)"},
        "e2e": {"value": rollouts_per_step * world / (e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": csum,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": NCU_TRAFFIC_BYTES.get((k2_name, inst.name)),
                     "kernel": k2_name, "peak_basis": "FP32 lanes x 2 x 2070 MHz (152 SMs x 128)",
                     "peak_measured": measured["tflops"], "frac_of_measured": achieved / measured["tflops"],
                     "peak_measured_how": measured["how"],
                     "flops_per_launch": flops, "launch_ms": k2_ms,
                     "timing": f"{GRAPH_REPS} launches replayed from one CUDA graph, events on the stream",
                     "eager_event_launch_ms": float(kms[:, 0].mean())},
        "kernel_share": {"rollout_fitness": share[0], "softmax_weights": share[1], "weighted_mean": share[2],
                         "eager_step_ms": step_ms},
        "verdict": results[-1]["verdict"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_line(inst)
    if rank == 0:
        print(json.dumps(line), flush=True)
    prob.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
