"""Seeded synthetic inputs for the D4orm hot path.

This module is shared by the tests, the benchmark and both implementations'
callers.  It holds NONE of the method's arithmetic (no noise, dynamics,
reward, schedule or update): it only lays out problem instances and random
inputs with numpy's own generator (PCG64), never with the Philox stream the
method draws its samples from.

Instance shapes follow the paper's evaluation (Sec. V-A: robots on a circle /
sphere with antipodal goals; Appendix: random starts and goals in a D x D
square), with the sizes of the workloads this library is measured on.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

HOLO2D, HOLO3D, UNICYCLE, DIFFDRIVE4 = 0, 1, 2, 3
EULER, RK4 = 0, 1
DIMS = {HOLO2D: (4, 2, 2), HOLO3D: (6, 3, 3), UNICYCLE: (3, 2, 2), DIFFDRIVE4: (4, 2, 2)}
DYN_NAMES = {HOLO2D: "holo2d", HOLO3D: "holo3d", UNICYCLE: "unicycle", DIFFDRIVE4: "diffdrive4"}


@dataclass
class Instance:
    """One planning problem with its denoising parameters (all plain data)."""
    name: str
    dyn: int
    integ: int
    n: int
    T: int
    dt: float
    radius: float
    u_lo: tuple
    u_hi: tuple
    v_max: float
    start: np.ndarray            # [n][d_x] float64
    goal: np.ndarray             # [n][d_x] float64
    N: int
    K: int = 100
    iters: int = 1
    seed: int = 0
    tag: int = 0
    lam: float = 0.1
    w_safe: float = 5.0
    eps_margin: float = 0.05
    goal_tol: float = 0.1
    beta0: float = 1e-4
    beta1: float = 1e-2
    obstacles: np.ndarray | None = None   # [m][4]: centre x, y, z, radius (Appendix)
    extra: dict = field(default_factory=dict)

    @property
    def dims(self):
        return DIMS[self.dyn]


def _full_state(dyn: int, pos: np.ndarray, goal_pos: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Start/goal states from positions: holonomic robots start at rest;
    heading robots start facing their own goal."""
    n, d_p = pos.shape
    d_x = DIMS[dyn][0]
    s = np.zeros((n, d_x))
    g = np.zeros((n, d_x))
    s[:, :d_p] = pos
    g[:, :d_p] = goal_pos
    if dyn in (UNICYCLE, DIFFDRIVE4):
        heading = np.arctan2(goal_pos[:, 1] - pos[:, 1], goal_pos[:, 0] - pos[:, 0])
        s[:, 2] = heading
        g[:, 2] = heading
    return s, g


def circle_antipodal(n: int, r: float) -> np.ndarray:
    """Start positions evenly spaced on a circle of radius r (angle 2 pi k / n)."""
    ang = 2.0 * np.pi * np.arange(n) / n
    return np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)


def fibonacci_sphere(n: int, r: float) -> np.ndarray:
    """Start positions on Fibonacci points of a sphere of radius r:
    z_k = 1 - 2 (k + 1/2) / n, phi_k = k pi (3 - sqrt 5)."""
    k = np.arange(n)
    z = 1.0 - 2.0 * (k + 0.5) / n
    phi = k * np.pi * (3.0 - math.sqrt(5.0))
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return r * np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def box_points(rng: np.random.Generator, n: int, d_p: int, half: float, min_sep: float) -> np.ndarray:
    """n points uniform in [-half, half]^d_p, pairwise >= min_sep apart
    (rejection sampling, one point at a time)."""
    pts = np.zeros((n, d_p))
    placed = 0
    tries = 0
    while placed < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("box_points: could not place points")
        q = rng.uniform(-half, half, size=d_p)
        if placed == 0 or np.min(np.linalg.norm(pts[:placed] - q, axis=1)) >= min_sep:
            pts[placed] = q
            placed += 1
    return pts


# ---------------------------------------------------------------------------
# The measured workloads (sizes as stated in the benchmark configuration).
# ---------------------------------------------------------------------------

def holo2d_circle_n4() -> Instance:
    """2D holonomic, 4 robots, Euler dt 0.1, T=50, circle r=3 m antipodal,
    R_a 0.2 m, |a|<=1, |v|<=1, N=256, 100 steps, 1 iteration, seed 0."""
    p = circle_antipodal(4, 3.0)
    s, g = _full_state(HOLO2D, p, -p)
    return Instance("holo2d_n4_T50_N256", HOLO2D, EULER, 4, 50, 0.1, 0.2, (-1.0, -1.0), (1.0, 1.0), 1.0,
                    s, g, N=256, K=100, iters=1, seed=0)


def unicycle_circle_n8(jitter_seed: int = 1) -> Instance:
    """Unicycle (x, y, theta; v in [0,1], omega in [-1,1]), 8 robots, RK4 dt
    0.1, T=100, circle r=4 m antipodal + U(+-0.3 m) jitter on every start and
    goal coordinate, R_a 0.2 m, N=2048, 100 steps, 5 iterations."""
    rng = np.random.default_rng(jitter_seed)
    p = circle_antipodal(8, 4.0)
    gp = -p
    p = p + rng.uniform(-0.3, 0.3, size=p.shape)
    gp = gp + rng.uniform(-0.3, 0.3, size=gp.shape)
    s, g = _full_state(UNICYCLE, p, gp)
    return Instance("unicycle_n8_T100_N2048", UNICYCLE, RK4, 8, 100, 0.1, 0.2, (0.0, -1.0), (1.0, 1.0), 0.0,
                    s, g, N=2048, K=100, iters=5, seed=0)


def holo3d_sphere_n16() -> Instance:
    """3D holonomic, 16 robots, RK4 dt 0.1, T=100, Fibonacci sphere r=4 m
    antipodal, R_a 0.25 m, |a|<=2, |v|<=1.5, N=8192, 100 steps, 5 iterations."""
    p = fibonacci_sphere(16, 4.0)
    s, g = _full_state(HOLO3D, p, -p)
    return Instance("holo3d_n16_T100_N8192", HOLO3D, RK4, 16, 100, 0.1, 0.25, (-2.0, -2.0, -2.0),
                    (2.0, 2.0, 2.0), 1.5, s, g, N=8192, K=100, iters=5, seed=0)


_DYN_DEFAULTS = {
    HOLO2D: dict(u_lo=(-1.0, -1.0), u_hi=(1.0, 1.0), v_max=1.0, radius=0.2),
    HOLO3D: dict(u_lo=(-2.0, -2.0, -2.0), u_hi=(2.0, 2.0, 2.0), v_max=1.5, radius=0.25),
    UNICYCLE: dict(u_lo=(0.0, -1.0), u_hi=(1.0, 1.0), v_max=0.0, radius=0.2),
    DIFFDRIVE4: dict(u_lo=(-1.0, -1.0), u_hi=(1.0, 1.0), v_max=1.0, radius=0.2),
}


def holo2d_circle(n: int = 16, r: float = 4.0, N: int = 2048, a_max: float = 1.0, v_max: float = 1.0) -> Instance:
    """n 2D holonomic robots evenly spaced on a circle of radius r with
    antipodal goals (Sec. V-A), RK4 dt 0.1, T = 100 (H = 100, dt = 0.1 as in
    Sec. V), R_a 0.2 m, |a| <= a_max, |v| <= v_max, N samples, 100 steps."""
    p = circle_antipodal(n, r)
    s, g = _full_state(HOLO2D, p, -p)
    return Instance(f"holo2d_circle_n{n}_r{r:g}_a{a_max:g}_v{v_max:g}_T100_N{N}", HOLO2D, RK4, n, 100, 0.1, 0.2,
                    (-a_max, -a_max), (a_max, a_max), v_max, s, g, N=N, K=100, iters=50, seed=0)


def circle_obstacles_n16(n_obstacles: int = 4, N: int = 4096) -> Instance:
    """16 2D holonomic robots on a circle of radius 4 m with antipodal goals
    (Sec. V-A layout) and 1..4 static disc obstacles of radius 0.4 m across
    the crossing region (Appendix, obstacle study: 16 robots, 1-4
    obstacles, at most 50 iterations): one at the centre, the others on a
    1.6 m circle at angles 2 pi o / (m - 1) + pi / 4.  RK4 dt 0.1, T = 100,
    R_a 0.2 m, |a| <= 1, |v| <= 1, N samples, 100 steps, 50 iterations."""
    if not 1 <= n_obstacles <= 16:
        raise ValueError("n_obstacles must be in 1..16")
    p = circle_antipodal(16, 4.0)
    s, g = _full_state(HOLO2D, p, -p)
    obs = [[0.0, 0.0, 0.0, 0.4]]
    m = n_obstacles - 1
    for o in range(m):
        a = 2.0 * np.pi * o / m + np.pi / 4
        obs.append([1.6 * np.cos(a), 1.6 * np.sin(a), 0.0, 0.4])
    inst = Instance(f"obstacles{n_obstacles}_holo2d_n16_T100_N{N}", HOLO2D, RK4, 16, 100, 0.1, 0.2, (-1.0, -1.0),
                    (1.0, 1.0), 1.0, s, g, N=N, K=100, iters=50, seed=0)
    inst.obstacles = np.array(obs)
    return inst


def box_instance(rng: np.random.Generator, dyn: int, n: int, T: int, N: int, *, side: float = 10.0,
                 min_sep: float = 0.6, K: int = 100, iters: int = 5, tag: int = 0, seed: int = 0) -> Instance:
    """Random starts, then goals, uniform in a side x side box (cube in 3D),
    each set >= min_sep apart (Appendix, generic target assignment)."""
    d_p = DIMS[dyn][2]
    p = box_points(rng, n, d_p, side / 2, min_sep)
    gp = box_points(rng, n, d_p, side / 2, min_sep)
    s, g = _full_state(dyn, p, gp)
    dd = _DYN_DEFAULTS[dyn]
    return Instance(f"box_{DYN_NAMES[dyn]}_n{n}_T{T}", dyn, RK4, n, T, 0.1, dd["radius"], dd["u_lo"], dd["u_hi"],
                    dd["v_max"], s, g, N=N, K=K, iters=iters, seed=seed, tag=tag)


def mixed_batch(count: int = 512, seed: int = 2, N: int = 1024) -> list[Instance]:
    """Ragged batch: n ~ U{2..16}, T ~ U{40..120}, dynamics 40 % 2D
    holonomic / 30 % 3D holonomic / 30 % differential drive (unicycle),
    10 m box, >= 0.6 m separation, N samples each, instance tags 0..count-1."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(rng.integers(2, 17))
        T = int(rng.integers(40, 121))
        u = rng.uniform()
        dyn = HOLO2D if u < 0.4 else (HOLO3D if u < 0.7 else UNICYCLE)
        out.append(box_instance(rng, dyn, n, T, N, tag=b, seed=0))
    return out


def reachable_box_instance(rng: np.random.Generator, n: int, T: int, N: int, *, side: float = 10.0,
                           min_sep: float = 0.6, max_axis: float = 6.0, K: int = 100, iters: int = 5,
                           tag: int = 0, seed: int = 0) -> Instance:
    """2D holonomic team: starts uniform in a side x side box (>= min_sep
    apart); each robot's goal uniform in the part of the box within max_axis
    metres of its start along each axis (goals also >= min_sep apart), so
    that every goal is reachable within T steps at |v|, |a| <= 1 with room
    for detours (a 10 m box allows displacements the horizon cannot cover)."""
    half = side / 2
    p = box_points(rng, n, 2, half, min_sep)
    gp = np.zeros_like(p)
    for k in range(n):
        lo = np.maximum(-half, p[k] - max_axis)
        hi = np.minimum(half, p[k] + max_axis)
        for _ in range(100000):
            q = rng.uniform(lo, hi)
            if k == 0 or np.min(np.linalg.norm(gp[:k] - q, axis=1)) >= min_sep:
                gp[k] = q
                break
        else:
            raise RuntimeError("reachable_box_instance: could not place a goal")
    s, g = _full_state(HOLO2D, p, gp)
    dd = _DYN_DEFAULTS[HOLO2D]
    return Instance(f"reach_holo2d_n{n}_T{T}", HOLO2D, RK4, n, T, 0.1, dd["radius"], dd["u_lo"], dd["u_hi"],
                    dd["v_max"], s, g, N=N, K=K, iters=iters, seed=seed, tag=tag)


def warmstart_set(count: int, seed: int, N: int = 4096, T: int = 80, n_lo: int = 8, n_hi: int = 16,
                  max_axis: float = 4.0, goal_tol: float = 0.5, large_share: float = 0.0,
                  large_lo: int = 13) -> list[Instance]:
    """Teams of n ~ U{n_lo..n_hi} 2D holonomic robots for the learned warm
    start (training and held-out sets use disjoint seeds); goals within
    max_axis metres per axis of their starts; a plan reaches its goals when
    every robot ends within goal_tol.  With large_share > 0 that share of the
    teams draws n from U{large_lo..n_hi} instead (training sets that hold
    enough of the largest teams)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        lo = large_lo if large_share > 0.0 and rng.uniform() < large_share else n_lo
        inst = reachable_box_instance(rng, int(rng.integers(lo, n_hi + 1)), T, N, max_axis=max_axis)
        inst.goal_tol = goal_tol
        out.append(inst)
    return out


def random_controls(rng: np.random.Generator, inst: Instance, scale: float = 1.0) -> np.ndarray:
    """Uniform controls inside the box (scaled about its centre), [T][n][d_u]."""
    d_u = inst.dims[1]
    lo = np.array(inst.u_lo)
    hi = np.array(inst.u_hi)
    mid = 0.5 * (lo + hi)
    half = 0.5 * (hi - lo) * scale
    return mid + half * rng.uniform(-1.0, 1.0, size=(inst.T, inst.n, d_u))


def random_deformation(rng: np.random.Generator, inst: Instance, scale: float = 0.3) -> np.ndarray:
    """A normal deformation dU of standard deviation `scale`, [T][n][d_u]."""
    return scale * rng.standard_normal(size=(inst.T, inst.n, inst.dims[1]))


WORKLOADS = {
    "holo2d_n4": holo2d_circle_n4,
    "unicycle_n8": unicycle_circle_n8,
    "holo3d_n16": holo3d_sphere_n16,
    "obstacles4_n16": circle_obstacles_n16,
}
