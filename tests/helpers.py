"""Test helpers: build the oracle's and the CUDA library's views of one
seeded scenario from identical (binary32-rounded) inputs."""
from __future__ import annotations

import copy
import importlib.util
import os

import numpy as np

import scenarios


def f32(x):
    return float(np.float32(x))


def round_instance(inst: scenarios.Instance) -> scenarios.Instance:
    """Round every real input to binary32 so that both implementations see
    exactly the same problem (the CUDA path takes float inputs)."""
    r = copy.deepcopy(inst)
    r.start = inst.start.astype(np.float32).astype(np.float64)
    r.goal = inst.goal.astype(np.float32).astype(np.float64)
    for name in ("dt", "radius", "v_max", "lam", "w_safe", "eps_margin", "goal_tol", "beta0", "beta1"):
        setattr(r, name, f32(getattr(inst, name)))
    r.u_lo = tuple(f32(v) for v in inst.u_lo)
    r.u_hi = tuple(f32(v) for v in inst.u_hi)
    if inst.obstacles is not None:
        r.obstacles = np.asarray(inst.obstacles).astype(np.float32).astype(np.float64)
    return r


def oracle_problem(o, inst: scenarios.Instance):
    return o.Problem(n=inst.n, T=inst.T, dyn=inst.dyn, integ=inst.integ, dt=inst.dt, radius=inst.radius,
                     start=inst.start, goal=inst.goal, u_lo=inst.u_lo, u_hi=inst.u_hi,
                     eps_margin=inst.eps_margin, goal_tol=inst.goal_tol, v_max=inst.v_max,
                     obstacles=inst.obstacles)


def oracle_params(o, inst: scenarios.Instance, N: int | None = None, update=(0, 0.0)):
    """update = (rule, mppi_sigma): rule 0 is the method, 1 is MPPI."""
    return o.Params(N=N or inst.N, K=inst.K, lam=inst.lam, w_safe=inst.w_safe, beta0=inst.beta0,
                    beta1=inst.beta1, seed=inst.seed, tag=inst.tag, update_rule=update[0], mppi_sigma=update[1])


def gpu_params(g, inst: scenarios.Instance, N: int | None = None, update=(0, 0.0)):
    return g.Params(n_samples=N or inst.N, n_steps=inst.K, temperature=inst.lam, w_safe=inst.w_safe,
                    beta0=inst.beta0, beta1=inst.beta1, seed=inst.seed, instance_tag=inst.tag,
                    update_rule=update[0], mppi_sigma=update[1])


def small_instance(dyn: int, n: int, T: int, N: int, integ: int = scenarios.RK4, seed: int = 0,
                   K: int = 20, layout_seed: int = 7, tag: int = 0) -> scenarios.Instance:
    """A random box instance of the requested size (for parity cases)."""
    rng = np.random.default_rng(layout_seed)
    inst = scenarios.box_instance(rng, dyn, n, T, N, side=4.0 + n * 0.5, min_sep=0.6, K=K, seed=seed, tag=tag)
    inst.integ = integ
    return round_instance(inst)


def build_library() -> None:
    """Compile libd4orm.so if it is missing or stale (the build script is
    loaded by path: importing the package loads the library)."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("d4orm_build", os.path.join(root, "paper_2503_12204_gb300",
                                                                               "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()


def add_obstacles(inst: scenarios.Instance, count: int, seed: int, r_lo: float = 0.2, r_hi: float = 0.6,
                  reach: float = 0.8):
    """Place `count` obstacles at points along random robots' straight
    start-goal segments, a fraction U(reach / 4, reach) of the way (so that
    many samples touch them: short horizons want a small reach), radius
    U(r_lo, r_hi); returns a binary32-rounded copy of the instance."""
    rng = np.random.default_rng(seed)
    d_p = inst.dims[2]
    obs = np.zeros((count, 4))
    for o in range(count):
        k = int(rng.integers(inst.n))
        a = rng.uniform(reach / 4, reach)
        obs[o, :d_p] = (1 - a) * inst.start[k, :d_p] + a * inst.goal[k, :d_p] + rng.normal(0, 0.2, d_p)
        obs[o, 3] = rng.uniform(r_lo, r_hi)
    r = copy.deepcopy(inst)
    r.obstacles = obs
    return round_instance(r)


def obstacle_safety_gap(inst: scenarios.Instance, states: np.ndarray) -> float:
    """min over t in 0..T, robots and obstacles of | |p - c| - (r_o + R_a) |:
    how far a plan is from flipping the obstacle part of the safety verdict."""
    if inst.obstacles is None or len(inst.obstacles) == 0:
        return np.inf
    d_p = inst.dims[2]
    p = states[:, :, None, :d_p]                               # [T+1][n][1][d_p]
    c = np.asarray(inst.obstacles)[None, None, :, :d_p]        # [1][1][m][d_p]
    d = np.sqrt(((p - c) ** 2).sum(-1))
    return float(np.abs(d - (np.asarray(inst.obstacles)[:, 3] + inst.radius)).min())

