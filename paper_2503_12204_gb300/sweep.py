"""Success rate against denoising steps and iterations (the sensitivity study
of Sec. V-A, Fig. 2: 10 and 16 robots, three dynamics, 30 runs with
different seeds; the figure's values are not recoverable, so this rebuilds
the experiment, not its numbers).

For every (dynamics, robots, K) the 30 runs are 30 problems of one batched
persistent launch (problem b draws its noise with instance tag b, i.e. its
own seed), solved with stop on success for up to `max_iters` iterations;
the success rate within i iterations is the share of runs whose first
success came at iteration < i.

    python -m paper_2503_12204_gb300.sweep
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import Budget, Params, Problem, d4orm_batch_create, d4orm_batch_destroy, d4orm_batch_solve

DYNAMICS = ("holo2d", "holo3d", "diffdrive4")


def instance(dyn: str, n: int, N: int):
    """Antipodal circle (2D) or Fibonacci sphere (3D) of radius 4 m (Sec. V-A);
    |a| <= 2, |v| <= 1.5 for the double integrators; the differential drive
    with omega, a in [-1, 1] and |v| <= 1.5; goals judged at 0.5 m."""
    import scenarios
    if dyn == "holo2d":
        inst = scenarios.holo2d_circle(n, 4.0, N=N, a_max=2.0, v_max=1.5)
    elif dyn == "holo3d":
        p = scenarios.fibonacci_sphere(n, 4.0)
        s, g = scenarios._full_state(scenarios.HOLO3D, p, -p)
        inst = scenarios.Instance(f"holo3d_sphere_n{n}", scenarios.HOLO3D, scenarios.RK4, n, 100, 0.1, 0.2,
                                  (-2.0, -2.0, -2.0), (2.0, 2.0, 2.0), 1.5, s, g, N=N)
    elif dyn == "diffdrive4":
        p = scenarios.circle_antipodal(n, 4.0)
        s, g = scenarios._full_state(scenarios.DIFFDRIVE4, p, -p)
        inst = scenarios.Instance(f"diffdrive4_circle_n{n}", scenarios.DIFFDRIVE4, scenarios.RK4, n, 100, 0.1, 0.2,
                                  (-1.0, -1.0), (1.0, 1.0), 1.5, s, g, N=N)
    else:
        raise ValueError(dyn)
    inst.goal_tol = 0.5
    inst.start = inst.start.astype(np.float32).astype(np.float64)
    inst.goal = inst.goal.astype(np.float32).astype(np.float64)
    return inst


def sweep(torch, dynamics=DYNAMICS, robots=(10, 16), steps=(50, 100, 200), runs: int = 30, max_iters: int = 5,
          N: int = 2048, w_safe: float = 1.0, temperature: float = 0.3, log=print) -> list[dict]:
    rows = []
    for dyn in dynamics:
        for n in robots:
            inst = instance(dyn, n, N)
            probs = [Problem(inst) for _ in range(runs)]
            outs = [torch.zeros((inst.T, n, inst.dims[1]), device="cuda") for _ in range(runs)]
            for K in steps:
                params = Params(n_samples=N, n_steps=K, temperature=temperature, w_safe=w_safe, seed=0,
                                instance_tag=0)
                batch = d4orm_batch_create([p.handle for p in probs], params, autotune=False)
                t0 = time.perf_counter()
                res = d4orm_batch_solve(batch, Budget(max_iters=max_iters, stop_on_success=True), outs)
                wall = time.perf_counter() - t0
                d4orm_batch_destroy(batch)
                first = [r["first_success_iter"] for r in res]
                rate = [sum(1 for f in first if 0 <= f < i) / runs for i in range(1, max_iters + 1)]
                rows.append(dict(dynamics=dyn, robots=n, steps=K, success_within_iters=rate,
                                 collision_free_final=sum(r["verdict"]["collision_free"] for r in res) / runs,
                                 wall_s=wall, runs=[dict(first_success_iter=r["first_success_iter"],
                                                         iters_run=r["iters_run"], verdict=r["verdict"])
                                                    for r in res]))
                log(f"{dyn} n={n} K={K}: success within 1..{max_iters} iterations {rate}")
            for p in probs:
                p.close()
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--runs", type=int, default=30)
    args = ap.parse_args(argv)
    import torch
    sweep(torch, runs=args.runs)


if __name__ == "__main__":
    main()
