"""FP64 CPU oracle of the D4orm denoising hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The CUDA library
(``paper_2503_12204_gb300``) never imports it, and the two share no code: the
oracle is plain C (``d4orm_oracle.c``) compiled with gcc into
``liboracle.so`` and wrapped here with ctypes over numpy float64 arrays.

Paper: Zhang et al., "D4orm: Multi-Robot Trajectories with Dynamics-aware
Diffusion Denoised Deformations" (IROS 2025).  Function-by-function citations
are in ``d4orm_oracle.c``:

* ``philox4x32_10`` / ``box_muller`` / ``noise`` -- sample noise of Eq. (12)
  (Philox from Salmon et al., SC'11; Box-Muller 1958).
* ``schedule``         -- alpha_i, alpha_bar_i (Sec. IV-B, under Eq. (10)).
* ``rollout``          -- Eq. (1) feasibility with the Sec. V dynamics.
* ``reward``           -- Eq. (3)-(5).
* ``verdict``          -- Eq. (1) safety/terminal conditions, Eq. (2) objective.
* ``weights``          -- Sec. IV-C batch normalisation + Eq. (6) softmax.
* ``denoise_step``     -- Algorithm 1 body on deformations (Eq. (12)-(13)).
* ``solve``            -- Algorithm 2 with an iteration budget.

Parity status: every function is pinned by tests under ``tests/test_oracle_*``
(closed forms, brute force, invariants, an independent Philox).  The absolute
reward values depend on silent constants of the paper (epsilon, w, lambda,
beta schedule), which are inputs; only invariants pin them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "d4orm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

HOLO2D, HOLO3D, UNICYCLE, DIFFDRIVE4 = 0, 1, 2, 3
EULER, RK4 = 0, 1
DIMS = {HOLO2D: (4, 2, 2), HOLO3D: (6, 3, 3), UNICYCLE: (3, 2, 2), DIFFDRIVE4: (4, 2, 2)}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C11, no FMA contraction so x86 and
    Arm hosts round identically)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "d4orm_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP splits independent samples (fitness) and robots (weighted
        # mean) over threads; every sum keeps its order, so the results do
        # not depend on the thread count.  Without OpenMP the loops run serially.
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("T", ctypes.c_int), ("dyn", ctypes.c_int), ("integ", ctypes.c_int),
        ("dt", ctypes.c_double), ("radius", ctypes.c_double), ("eps_margin", ctypes.c_double),
        ("goal_tol", ctypes.c_double), ("v_max", ctypes.c_double),
        ("u_lo", ctypes.c_double * 3), ("u_hi", ctypes.c_double * 3),
        ("start", ctypes.POINTER(ctypes.c_double)), ("goal", ctypes.POINTER(ctypes.c_double)),
        ("n_obs", ctypes.c_int), ("obstacles", ctypes.POINTER(ctypes.c_double)),
    ]


class _Params(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int), ("K", ctypes.c_int), ("lam", ctypes.c_double),
        ("w_safe", ctypes.c_double), ("beta0", ctypes.c_double), ("beta1", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("tag", ctypes.c_uint32),
        ("update_rule", ctypes.c_int), ("mppi_sigma", ctypes.c_double),
    ]


DENOISE, MPPI = 0, 1


class _Verdict(ctypes.Structure):
    _fields_ = [
        ("collision_free", ctypes.c_int), ("goal_reached", ctypes.c_int),
        ("reward", ctypes.c_double), ("objective", ctypes.c_double),
        ("min_pair_dist", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i32, u32 = P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_uint32)
        lib.orc_philox4x32_10.argtypes = [u32, u32, u32]
        lib.orc_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, d, d]
        lib.orc_noise.argtypes = [P(_Params), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.orc_noise.restype = ctypes.c_double
        lib.orc_schedule.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, d, d]
        lib.orc_dynamics.argtypes = [ctypes.c_int, d, d, d]
        lib.orc_integrate.argtypes = [P(_Problem), d, d, d]
        lib.orc_rollout.argtypes = [P(_Problem), d, d]
        lib.orc_reward.argtypes = [P(_Problem), ctypes.c_double, d, d]
        lib.orc_reward.restype = ctypes.c_double
        lib.orc_verdict_of.argtypes = [P(_Problem), ctypes.c_double, d, P(_Verdict)]
        lib.orc_weights.argtypes = [ctypes.c_int, d, ctypes.c_double, d]
        lib.orc_sample_fitness.argtypes = [P(_Problem), P(_Params), ctypes.c_int, ctypes.c_int, d, d,
                                           ctypes.c_int, i32, d, d, ctypes.c_double, i32]
        lib.orc_fragile.argtypes = [P(_Problem), d, ctypes.c_double]
        lib.orc_fragile.restype = ctypes.c_int
        lib.orc_denoise_step.argtypes = [P(_Problem), P(_Params), ctypes.c_int, ctypes.c_int, d, d, d, d, d, d]
        lib.orc_weighted_update.argtypes = [P(_Problem), P(_Params), ctypes.c_int, ctypes.c_int, d, d, d]
        lib.orc_apply.argtypes = [P(_Problem), d, d, d]
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_max_threads.restype = ctypes.c_int
        lib.orc_solve.argtypes = [P(_Problem), P(_Params), ctypes.c_int, ctypes.c_int, ctypes.c_int, d, d,
                                  P(_Verdict), i32]
        lib.orc_solve.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Problem:
    """Problem of Sec. III: n robots, horizon T, dynamics, start S and goal T."""
    n: int
    T: int
    dyn: int
    integ: int
    dt: float
    radius: float
    start: np.ndarray          # [n][d_x]
    goal: np.ndarray           # [n][d_x]
    u_lo: tuple
    u_hi: tuple
    eps_margin: float = 0.05
    goal_tol: float = 0.1
    v_max: float = 0.0
    obstacles: np.ndarray | None = None   # [m][4]: centre x, y, z, radius (Appendix)
    _c: _Problem = field(default=None, init=False, repr=False)

    @property
    def dims(self):
        return DIMS[self.dyn]

    def c(self) -> _Problem:
        d_x, d_u, _ = self.dims
        self._start = np.ascontiguousarray(self.start, dtype=np.float64).reshape(self.n, d_x)
        self._goal = np.ascontiguousarray(self.goal, dtype=np.float64).reshape(self.n, d_x)
        lo = (ctypes.c_double * 3)(*(list(self.u_lo) + [0.0] * (3 - d_u)))
        hi = (ctypes.c_double * 3)(*(list(self.u_hi) + [0.0] * (3 - d_u)))
        if self.obstacles is not None and len(self.obstacles):
            self._obs = np.ascontiguousarray(self.obstacles, dtype=np.float64).reshape(-1, 4)
            n_obs, obs = self._obs.shape[0], _dp(self._obs)
        else:
            n_obs, obs = 0, None
        self._c = _Problem(self.n, self.T, self.dyn, self.integ, self.dt, self.radius, self.eps_margin,
                           self.goal_tol, self.v_max, lo, hi, _dp(self._start), _dp(self._goal), n_obs, obs)
        return self._c

    @property
    def n_ctrl(self) -> int:
        return self.T * self.n * self.dims[1]


@dataclass
class Params:
    """Denoising parameters: samples N (the paper's M), steps K (the paper's
    N), temperature lambda, safety weight w, schedule (beta0, beta1), seed."""
    N: int
    K: int = 100
    lam: float = 0.1
    w_safe: float = 5.0
    beta0: float = 1e-4
    beta1: float = 1e-2
    seed: int = 0
    tag: int = 0
    update_rule: int = 0       # DENOISE (Eq. (12)-(13)) or MPPI
    mppi_sigma: float = 0.0    # MPPI exploration standard deviation

    def c(self) -> _Params:
        return _Params(self.N, self.K, self.lam, self.w_safe, self.beta0, self.beta1, self.seed, self.tag,
                       self.update_rule, self.mppi_sigma)


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def box_muller(a: int, b: int) -> tuple[float, float]:
    lib = _load()
    z0, z1 = ctypes.c_double(), ctypes.c_double()
    lib.orc_box_muller(a, b, ctypes.byref(z0), ctypes.byref(z1))
    return z0.value, z1.value


def noise(params: Params, it: int, i: int, j: int, k: int, e: int) -> float:
    lib = _load()
    pc = params.c()
    return lib.orc_noise(ctypes.byref(pc), it, i, j, k, e)


def noise_block(prob: Problem, params: Params, it: int, i: int, j: int) -> np.ndarray:
    """eps[t][k][d] of sample j (loops over orc_noise)."""
    d_u = prob.dims[1]
    out = np.empty((prob.T, prob.n, d_u))
    lib = _load()
    pc = params.c()
    for t in range(prob.T):
        for k in range(prob.n):
            for d in range(d_u):
                out[t, k, d] = lib.orc_noise(ctypes.byref(pc), it, i, j, k, t * d_u + d)
    return out


def schedule(K: int, beta0: float, beta1: float):
    lib = _load()
    a = np.zeros(K + 1)
    ab = np.zeros(K + 1)
    lib.orc_schedule(K, beta0, beta1, _dp(a), _dp(ab))
    return a, ab


def dynamics(dyn: int, x, u) -> np.ndarray:
    lib = _load()
    d_x = DIMS[dyn][0]
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(d_x)
    lib.orc_dynamics(dyn, _dp(x), _dp(u), _dp(out))
    return out


def integrate(prob: Problem, x, u) -> np.ndarray:
    lib = _load()
    pc = prob.c()
    x = np.ascontiguousarray(x, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(prob.dims[0])
    lib.orc_integrate(ctypes.byref(pc), _dp(x), _dp(u), _dp(out))
    return out


def rollout(prob: Problem, u: np.ndarray) -> np.ndarray:
    """states[T+1][n][d_x] from controls u[T][n][d_u]."""
    lib = _load()
    pc = prob.c()
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(prob.T, prob.n, prob.dims[1])
    st = np.zeros((prob.T + 1, prob.n, prob.dims[0]))
    lib.orc_rollout(ctypes.byref(pc), _dp(u), _dp(st))
    return st


def reward(prob: Problem, w_safe: float, states: np.ndarray):
    """(r, threshold_gap) of Eq. (3)."""
    lib = _load()
    pc = prob.c()
    states = np.ascontiguousarray(states, dtype=np.float64)
    gap = ctypes.c_double()
    r = lib.orc_reward(ctypes.byref(pc), w_safe, _dp(states), ctypes.byref(gap))
    return r, gap.value


def verdict(prob: Problem, w_safe: float, states: np.ndarray) -> dict:
    lib = _load()
    pc = prob.c()
    states = np.ascontiguousarray(states, dtype=np.float64)
    v = _Verdict()
    lib.orc_verdict_of(ctypes.byref(pc), w_safe, _dp(states), ctypes.byref(v))
    return dict(collision_free=bool(v.collision_free), goal_reached=bool(v.goal_reached),
                reward=v.reward, objective=v.objective, min_pair_dist=v.min_pair_dist)


def weights(r: np.ndarray, lam: float) -> np.ndarray:
    lib = _load()
    r = np.ascontiguousarray(r, dtype=np.float64)
    w = np.zeros_like(r)
    lib.orc_weights(len(r), _dp(r), lam, _dp(w))
    return w


def sample_fitness(prob: Problem, params: Params, it: int, i: int, u_base, du_in, js, delta: float = 0.0,
                   with_fragile: bool = False):
    """(fitness[len(js)], threshold_gap[len(js)]) for the listed samples, plus
    the per-sample fragile robot-timestep counts when with_fragile."""
    lib = _load()
    pc, pp = prob.c(), params.c()
    u_base = np.ascontiguousarray(u_base, dtype=np.float64)
    du_in = np.ascontiguousarray(du_in, dtype=np.float64)
    js = np.ascontiguousarray(js, dtype=np.int32)
    f = np.zeros(len(js))
    g = np.zeros(len(js))
    fr = np.zeros(len(js), dtype=np.int32)
    lib.orc_sample_fitness(ctypes.byref(pc), ctypes.byref(pp), it, i, _dp(u_base), _dp(du_in), len(js),
                           js.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(f), _dp(g), delta,
                           fr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if with_fragile else None)
    return (f, g, fr) if with_fragile else (f, g)


def fragile(prob: Problem, states: np.ndarray, delta: float) -> int:
    lib = _load()
    pc = prob.c()
    states = np.ascontiguousarray(states, dtype=np.float64)
    return lib.orc_fragile(ctypes.byref(pc), _dp(states), delta)


def denoise_step(prob: Problem, params: Params, it: int, i: int, u_base, du_in, fitness_in=None):
    """(du_out[T][n][d_u], fitness[N]) for one step; fitness_in overrides
    the oracle's own rewards when given."""
    lib = _load()
    pc, pp = prob.c(), params.c()
    u_base = np.ascontiguousarray(u_base, dtype=np.float64)
    du_in = np.ascontiguousarray(du_in, dtype=np.float64)
    out = np.zeros_like(du_in)
    fit = np.zeros(params.N)
    fin = None if fitness_in is None else np.ascontiguousarray(fitness_in, dtype=np.float64)
    lib.orc_denoise_step(ctypes.byref(pc), ctypes.byref(pp), it, i, _dp(u_base), _dp(du_in), _dp(out),
                         _dp(fit), _dp(fin), None)
    return out, fit


def weighted_update(prob: Problem, params: Params, it: int, i: int, du_in, w) -> np.ndarray:
    lib = _load()
    pc, pp = prob.c(), params.c()
    du_in = np.ascontiguousarray(du_in, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros_like(du_in)
    lib.orc_weighted_update(ctypes.byref(pc), ctypes.byref(pp), it, i, _dp(du_in), _dp(w), _dp(out))
    return out


def apply(prob: Problem, u_base, du0) -> np.ndarray:
    lib = _load()
    pc = prob.c()
    u_base = np.ascontiguousarray(u_base, dtype=np.float64)
    du0 = np.ascontiguousarray(du0, dtype=np.float64)
    out = np.zeros_like(u_base)
    lib.orc_apply(ctypes.byref(pc), _dp(u_base), _dp(du0), _dp(out))
    return out


def solve(prob: Problem, params: Params, max_iters: int, stop_on_success: bool = False,
          start_step: int = 0, du_init=None):
    """Algorithm 2.  Returns (u_out, verdicts per iteration, first_success_iter)."""
    lib = _load()
    pc, pp = prob.c(), params.c()
    u_out = np.zeros((prob.T, prob.n, prob.dims[1]))
    vs = (_Verdict * max_iters)()
    iters = ctypes.c_int()
    dui = None if du_init is None else np.ascontiguousarray(du_init, dtype=np.float64)
    first = lib.orc_solve(ctypes.byref(pc), ctypes.byref(pp), max_iters, int(stop_on_success),
                          start_step, _dp(dui), _dp(u_out), vs, ctypes.byref(iters))
    verdicts = [dict(collision_free=bool(v.collision_free), goal_reached=bool(v.goal_reached),
                     reward=v.reward, objective=v.objective, min_pair_dist=v.min_pair_dist)
                for v in list(vs)[: iters.value]]
    return u_out, verdicts, first


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel sample loops (1 = serial)."""
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())
