"""The method against MPPI on the same kernels: time to the first feasible
plan on antipodal-circle teams (the comparison of Sec. V-B, Fig. 3: MPPI
adapted to sample in the joint control space, success within a 5 s
deadline).

Both update rules run through the same C ABI, the same sampling, rollout,
Eq. (3) fitness and Eq. (6) weights; they differ only in the per-step
constants (the method's schedule, Eq. (12)-(13), or MPPI's constant sigma
around the current deformation).  Each run is one d4orm_solve with stop on
success and a deadline, one problem at a time on the whole GPU; the seed
varies between runs.  MPPI's sigma is chosen on tuning seeds that the
evaluation does not use.

    python -m paper_2503_12204_gb300.compare --runs 30
"""
from __future__ import annotations

import argparse
import statistics
import time

import numpy as np

from . import UPDATE_DENOISE, UPDATE_MPPI, Budget, Params, Problem, d4orm_rollout, d4orm_solve


SIGMAS = (0.02, 0.05, 0.1, 0.2, 0.3, 0.5)
# the reward weight and temperature the paper leaves open, crossed
SETTINGS = ((1.0, 0.1), (1.0, 0.3), (5.0, 0.1), (5.0, 0.3))


def _f32(inst):
    inst.start = inst.start.astype(np.float32).astype(np.float64)
    inst.goal = inst.goal.astype(np.float32).astype(np.float64)
    return inst


def run_method(torch, inst, params: Params, seeds, max_iters: int, deadline_ms: float) -> list[dict]:
    """One solve per seed; the iteration graph of each seed is captured by an
    untimed one-iteration solve first, so the timed solve measures the
    method, not the capture."""
    pr = Problem(_f32(inst))
    d_x, d_u, d_p = inst.dims
    u = torch.zeros((inst.T, inst.n, d_u), device="cuda")
    states = torch.zeros((inst.T + 1, inst.n, d_x), device="cuda")
    goal = np.asarray(inst.goal)[:, :d_p]
    rows = []
    for s in seeds:
        p = Params(**{**params.__dict__, "seed": int(s)})
        d4orm_solve(pr.handle, p, Budget(max_iters=1), u)
        torch.cuda.synchronize()
        r = d4orm_solve(pr.handle, p, Budget(max_iters=max_iters, deadline_ms=deadline_ms, stop_on_success=True), u)
        d4orm_rollout(pr.handle, p, u, states, want_verdict=False)
        final = states[-1, :, :d_p].cpu().numpy()
        rows.append(dict(seed=int(s), ok=r["first_success_iter"] >= 0, first=r["first_success_iter"],
                         ms=r["ms_to_success"] if r["first_success_iter"] >= 0 else None, ms_total=r["ms_total"],
                         reward=r["verdict"]["reward"], iters=r["iters_run"],
                         collision_free=r["verdict"]["collision_free"],
                         max_goal_dist=float(np.linalg.norm(final - goal, axis=1).max())))
    pr.close()
    return rows


def summarize(rows: list[dict]) -> dict:
    ok = [r for r in rows if r["ok"]]
    out = dict(runs=len(rows), success_rate=len(ok) / max(1, len(rows)),
               final_collision_free_rate=sum(r["collision_free"] for r in rows) / max(1, len(rows)),
               median_final_max_goal_dist=statistics.median(r["max_goal_dist"] for r in rows) if rows else None)
    if ok:
        out.update(mean_ms=statistics.mean(r["ms"] for r in ok), median_ms=statistics.median(r["ms"] for r in ok),
                   mean_iterations=statistics.mean(r["first"] + 1 for r in ok),
                   mean_reward=statistics.mean(r["reward"] for r in ok))
    return out


def compare(torch, inst, N: int, K: int, runs: int, sigmas, max_iters: int = 50, deadline_ms: float = 5000.0,
            tune_runs: int = 8, w_safe: float | None = None, temperature: float | None = None, log=print) -> dict:
    """The method and MPPI on `runs` evaluation seeds (1000..), MPPI's sigma
    picked from `sigmas` on `tune_runs` tuning seeds (0..): highest success
    rate, then lowest mean time.  Both use the same reward weight w and
    temperature lambda (the instance's unless given)."""
    base = dict(n_samples=N, n_steps=K, temperature=inst.lam if temperature is None else temperature,
                w_safe=inst.w_safe if w_safe is None else w_safe, beta0=inst.beta0, beta1=inst.beta1,
                instance_tag=0)
    tune = list(range(tune_runs))
    evals = list(range(1000, 1000 + runs))
    tuning = {}
    for sg in sigmas:
        rows = run_method(torch, inst, Params(**base, update_rule=UPDATE_MPPI, mppi_sigma=float(sg)), tune, max_iters,
                          deadline_ms)
        tuning[float(sg)] = summarize(rows)
        log(f"MPPI sigma {sg}: {tuning[float(sg)]}")
    best = max(tuning, key=lambda sg: (tuning[sg]["success_rate"], -tuning[sg].get("mean_ms", 1e30)))
    t0 = time.perf_counter()
    d4 = summarize(run_method(torch, inst, Params(**base, update_rule=UPDATE_DENOISE), evals, max_iters, deadline_ms))
    mp = summarize(run_method(torch, inst, Params(**base, update_rule=UPDATE_MPPI, mppi_sigma=best), evals, max_iters,
                              deadline_ms))
    log(f"method: {d4}\nMPPI (sigma {best}): {mp}  ({time.perf_counter() - t0:.1f} s)")
    res = dict(method=d4, mppi=mp, mppi_sigma=best, tuning=tuning)
    if d4.get("mean_ms") and mp.get("mean_ms"):
        res["speedup_mean_ms"] = mp["mean_ms"] / d4["mean_ms"]
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--runs", type=int, default=30)
    ap.add_argument("--samples", type=int, default=2048)
    ap.add_argument("--robots", type=int, default=16)
    ap.add_argument("--radius", type=float, default=4.0)
    ap.add_argument("--w", type=float, default=1.0)
    ap.add_argument("--lam", type=float, default=0.3)
    args = ap.parse_args(argv)
    import torch

    import scenarios
    inst = scenarios.holo2d_circle(args.robots, args.radius, a_max=2.0, v_max=1.5)
    inst.goal_tol = 0.5
    res = compare(torch, inst, args.samples, 100, args.runs, SIGMAS, w_safe=args.w, temperature=args.lam)
    print(res)


if __name__ == "__main__":
    main()
