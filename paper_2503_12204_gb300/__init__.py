"""Python binding of libd4orm.so, the GB300 (sm_103a) D4orm hot path.

A thin ctypes layer over the C ABI in ``include/d4orm.h``: functions keep the
C names and only marshal arguments (device pointers may be given as ints or
as objects with ``data_ptr()``, e.g. torch tensors; streams as ints, None, or
objects with ``cuda_stream``).  Every step of the denoising path runs in the
library's CUDA kernels; there is no CPU fallback, and importing this package
raises if the compiled library is missing.

Paper: Zhang et al., "D4orm: Multi-Robot Trajectories with Dynamics-aware
Diffusion Denoised Deformations" (IROS 2025) -- Eq. (1)-(13), Algorithms 1-2.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libd4orm.so")

HOLO2D, HOLO3D, UNICYCLE, DIFFDRIVE4 = 0, 1, 2, 3
EULER, RK4 = 0, 1
ROLLOUT_AUTO, ROLLOUT_REGISTER, ROLLOUT_PIPELINE, ROLLOUT_PAIRED = 0, 1, 2, 3
STOP_BUDGET, STOP_DEADLINE, STOP_CANCELLED = 0, 1, 2
PACK_SINGLE, PACK_PAIRED = 0, 1
ERR_TIMEOUT, ERR_CANCELLED = 5, 6
UPDATE_DENOISE, UPDATE_MPPI = 0, 1
DIMS = {HOLO2D: (4, 2, 2), HOLO3D: (6, 3, 3), UNICYCLE: (3, 2, 2), DIFFDRIVE4: (4, 2, 2)}
MAX_ROBOTS = 32
MAX_ITERS = 4096
MAX_TAG = (1 << 20) - 1
MAX_CTRL = 49152
NOALLOC_SCRATCH_FLOATS = 1 << 19
NOALLOC_MAX_SAMPLES = 65536

STATUS = {0: "D4ORM_OK", 1: "D4ORM_ERR_INVALID_ARG", 2: "D4ORM_ERR_UNSUPPORTED", 3: "D4ORM_ERR_OOM",
          4: "D4ORM_ERR_CUDA", 5: "D4ORM_ERR_TIMEOUT", 6: "D4ORM_ERR_CANCELLED"}

# Every entry point declared in include/d4orm.h.
EXPORTS = (
    "d4orm_problem_create", "d4orm_problem_destroy", "d4orm_problem_set_rollout_kernel",
    "d4orm_problem_rollout_kernel", "d4orm_problem_graph_captures", "d4orm_rollout", "d4orm_sample_fitness",
    "d4orm_denoise_step",
    "d4orm_denoise_step_timed", "d4orm_denoise_step_noalloc", "d4orm_solve", "d4orm_problem_cancel",
    "d4orm_sample_noise", "d4orm_philox4x32_10", "d4orm_fp32_fma_probe", "d4orm_status_string", "d4orm_last_error",
    "d4orm_batch_create", "d4orm_batch_solve", "d4orm_batch_info", "d4orm_batch_tuning", "d4orm_batch_cancel",
    "d4orm_batch_set_packing", "d4orm_batch_packing", "d4orm_batch_destroy",
    "d4orm_solve_batched",
    "d4orm_warmstart_create", "d4orm_warmstart_destroy", "d4orm_warmstart_param_count",
    "d4orm_warmstart_get_params", "d4orm_warmstart_set_params", "d4orm_warmstart_forward",
    "d4orm_warmstart_loss_grad", "d4orm_warmstart_train_step", "d4orm_warmstart_features",
    "d4orm_warmstart_predict",
)
WS_FEATURES = 16
BATCH_MAX_SAMPLES = 8192


class D4ormError(RuntimeError):
    """A non-OK status.  For D4ORM_ERR_CANCELLED and D4ORM_ERR_TIMEOUT of a
    solve, `results` holds what the call wrote (the anytime plans' results)."""

    def __init__(self, status: int, message: str, results=None):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.results = results


class _Desc(ctypes.Structure):
    _fields_ = [
        ("n_robots", ctypes.c_int), ("T", ctypes.c_int), ("dyn", ctypes.c_int), ("integ", ctypes.c_int),
        ("dt", ctypes.c_float), ("radius", ctypes.c_float), ("eps_margin", ctypes.c_float),
        ("goal_tol", ctypes.c_float), ("v_max", ctypes.c_float),
        ("start", ctypes.POINTER(ctypes.c_float)), ("goal", ctypes.POINTER(ctypes.c_float)),
        ("u_lo", ctypes.POINTER(ctypes.c_float)), ("u_hi", ctypes.POINTER(ctypes.c_float)),
        ("n_obstacles", ctypes.c_int), ("obstacles", ctypes.POINTER(ctypes.c_float)),
    ]


class _Params(ctypes.Structure):
    _fields_ = [
        ("n_samples", ctypes.c_int), ("n_steps", ctypes.c_int), ("temperature", ctypes.c_float),
        ("w_safe", ctypes.c_float), ("beta0", ctypes.c_float), ("beta1", ctypes.c_float),
        ("seed", ctypes.c_uint64), ("instance_tag", ctypes.c_uint32),
        ("update_rule", ctypes.c_int), ("mppi_sigma", ctypes.c_float),
    ]


class _Budget(ctypes.Structure):
    _fields_ = [
        ("max_iters", ctypes.c_int), ("deadline_ms", ctypes.c_double), ("stop_on_success", ctypes.c_int),
        ("start_step", ctypes.c_int),
    ]


class _WsDesc(ctypes.Structure):
    _fields_ = [
        ("n_max", ctypes.c_int), ("T", ctypes.c_int), ("d_u", ctypes.c_int), ("width", ctypes.c_int),
        ("max_batch", ctypes.c_int), ("seed", ctypes.c_uint64), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("weight_decay", ctypes.c_float),
        ("pos_scale", ctypes.c_float),
    ]


class _Verdict(ctypes.Structure):
    _fields_ = [
        ("collision_free", ctypes.c_int), ("goal_reached", ctypes.c_int), ("reward", ctypes.c_float),
        ("objective", ctypes.c_float), ("min_pair_dist", ctypes.c_float),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("verdict", _Verdict), ("iters_run", ctypes.c_int), ("first_success_iter", ctypes.c_int),
        ("ms_to_success", ctypes.c_double), ("ms_total", ctypes.c_double), ("stop_reason", ctypes.c_int),
    ]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32
    lib.d4orm_problem_create.argtypes = [ctypes.POINTER(_Desc), ctypes.POINTER(vp)]
    lib.d4orm_problem_create.restype = i
    lib.d4orm_problem_destroy.argtypes = [vp]
    lib.d4orm_problem_destroy.restype = None
    lib.d4orm_problem_set_rollout_kernel.argtypes = [vp, i]
    lib.d4orm_problem_set_rollout_kernel.restype = i
    lib.d4orm_problem_rollout_kernel.argtypes = [vp, i]
    lib.d4orm_problem_rollout_kernel.restype = i
    lib.d4orm_rollout.argtypes = [vp, ctypes.POINTER(_Params), vp, vp, ctypes.POINTER(_Verdict), vp]
    lib.d4orm_rollout.restype = i
    lib.d4orm_sample_fitness.argtypes = [vp, ctypes.POINTER(_Params), i, i, vp, vp, vp, vp]
    lib.d4orm_sample_fitness.restype = i
    lib.d4orm_denoise_step.argtypes = [vp, ctypes.POINTER(_Params), i, i, vp, vp, vp, vp, vp]
    lib.d4orm_denoise_step.restype = i
    lib.d4orm_denoise_step_timed.argtypes = [vp, ctypes.POINTER(_Params), i, i, vp, vp, vp, vp,
                                             ctypes.POINTER(ctypes.c_float), vp]
    lib.d4orm_denoise_step_timed.restype = i
    lib.d4orm_denoise_step_noalloc.argtypes = [vp, ctypes.POINTER(_Params), i, i, vp, vp, vp, vp, vp]
    lib.d4orm_denoise_step_noalloc.restype = i
    lib.d4orm_solve.argtypes = [vp, ctypes.POINTER(_Params), ctypes.POINTER(_Budget), vp, vp,
                                ctypes.POINTER(_Result), vp]
    lib.d4orm_solve.restype = i
    lib.d4orm_sample_noise.argtypes = [vp, ctypes.POINTER(_Params), i, i, i, i, vp, vp]
    lib.d4orm_sample_noise.restype = i
    lib.d4orm_problem_graph_captures.argtypes = [vp]
    lib.d4orm_problem_graph_captures.restype = ctypes.c_longlong
    lib.d4orm_philox4x32_10.argtypes = [vp, u32, u32, i, vp, vp]
    lib.d4orm_philox4x32_10.restype = i
    lib.d4orm_fp32_fma_probe.argtypes = [vp, i, i, i, vp]
    lib.d4orm_fp32_fma_probe.restype = i
    PP = ctypes.POINTER(vp)
    lib.d4orm_batch_create.argtypes = [PP, i, ctypes.POINTER(_Params), i, ctypes.POINTER(vp)]
    lib.d4orm_batch_create.restype = i
    lib.d4orm_batch_solve.argtypes = [vp, ctypes.POINTER(_Budget), PP, PP, ctypes.POINTER(_Result), vp]
    lib.d4orm_batch_solve.restype = i
    lib.d4orm_batch_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_float)]
    lib.d4orm_batch_info.restype = i
    lib.d4orm_batch_cancel.argtypes = [vp]
    lib.d4orm_batch_cancel.restype = i
    lib.d4orm_problem_cancel.argtypes = [vp]
    lib.d4orm_problem_cancel.restype = i
    lib.d4orm_batch_tuning.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                       ctypes.POINTER(ctypes.c_float)]
    lib.d4orm_batch_tuning.restype = i
    lib.d4orm_batch_set_packing.argtypes = [vp, i]
    lib.d4orm_batch_set_packing.restype = i
    lib.d4orm_batch_packing.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)]
    lib.d4orm_batch_packing.restype = i
    lib.d4orm_batch_destroy.argtypes = [vp]
    lib.d4orm_batch_destroy.restype = None
    lib.d4orm_solve_batched.argtypes = [PP, i, ctypes.POINTER(_Params), ctypes.POINTER(_Budget), PP,
                                        ctypes.POINTER(_Result), vp]
    lib.d4orm_solve_batched.restype = i
    fp = ctypes.POINTER(ctypes.c_float)
    lib.d4orm_warmstart_create.argtypes = [ctypes.POINTER(_WsDesc), ctypes.POINTER(vp)]
    lib.d4orm_warmstart_create.restype = i
    lib.d4orm_warmstart_destroy.argtypes = [vp]
    lib.d4orm_warmstart_destroy.restype = None
    lib.d4orm_warmstart_param_count.argtypes = [vp]
    lib.d4orm_warmstart_param_count.restype = i
    lib.d4orm_warmstart_get_params.argtypes = [vp, fp, i]
    lib.d4orm_warmstart_get_params.restype = i
    lib.d4orm_warmstart_set_params.argtypes = [vp, fp, i]
    lib.d4orm_warmstart_set_params.restype = i
    lib.d4orm_warmstart_forward.argtypes = [vp, vp, vp, i, vp, vp]
    lib.d4orm_warmstart_forward.restype = i
    lib.d4orm_warmstart_loss_grad.argtypes = [vp, vp, vp, vp, i, fp, vp, vp]
    lib.d4orm_warmstart_loss_grad.restype = i
    lib.d4orm_warmstart_train_step.argtypes = [vp, vp, vp, vp, vp, i, fp, vp]
    lib.d4orm_warmstart_train_step.restype = i
    lib.d4orm_warmstart_features.argtypes = [vp, i, ctypes.c_float, fp, fp]
    lib.d4orm_warmstart_features.restype = i
    lib.d4orm_warmstart_predict.argtypes = [vp, vp, ctypes.POINTER(_Params), i, vp, vp]
    lib.d4orm_warmstart_predict.restype = i
    lib.d4orm_status_string.argtypes = [i]
    lib.d4orm_status_string.restype = ctypes.c_char_p
    lib.d4orm_last_error.argtypes = []
    lib.d4orm_last_error.restype = ctypes.c_char_p
    return lib


lib = _load()


def _check(status: int) -> None:
    if status != 0:
        raise D4ormError(status, lib.d4orm_last_error().decode())


def _ptr(x) -> ctypes.c_void_p | None:
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError(f"cannot take a device pointer from {type(x)!r}")


def _stream(s) -> ctypes.c_void_p | None:
    if s is None:
        return None
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    raise TypeError(f"cannot take a stream handle from {type(s)!r}")


def _fbuf(values, count: int):
    vals = [float(v) for v in values]
    if len(vals) != count:
        raise ValueError(f"expected {count} values, got {len(vals)}")
    return (ctypes.c_float * count)(*vals)


@dataclass
class Params:
    """Denoising parameters (d4orm_params)."""
    n_samples: int
    n_steps: int = 100
    temperature: float = 0.1
    w_safe: float = 5.0
    beta0: float = 1e-4
    beta1: float = 1e-2
    seed: int = 0
    instance_tag: int = 0
    update_rule: int = 0       # UPDATE_DENOISE or UPDATE_MPPI
    mppi_sigma: float = 0.0

    def c(self) -> _Params:
        return _Params(self.n_samples, self.n_steps, self.temperature, self.w_safe, self.beta0, self.beta1,
                       self.seed, self.instance_tag, self.update_rule, self.mppi_sigma)


@dataclass
class Budget:
    """Anytime budget (d4orm_budget)."""
    max_iters: int = 1
    deadline_ms: float = 0.0
    stop_on_success: bool = False
    start_step: int = 0

    def c(self) -> _Budget:
        return _Budget(self.max_iters, self.deadline_ms, int(self.stop_on_success), self.start_step)


def _verdict(v: _Verdict) -> dict:
    return dict(collision_free=bool(v.collision_free), goal_reached=bool(v.goal_reached), reward=v.reward,
                objective=v.objective, min_pair_dist=v.min_pair_dist)


def d4orm_problem_create(n_robots: int, T: int, dyn: int, integ: int, dt: float, radius: float, start, goal,
                         eps_margin: float = 0.05, goal_tol: float = 0.1, v_max: float = 0.0,
                         u_lo=None, u_hi=None, obstacles=None) -> ctypes.c_void_p:
    """Create a problem handle; start/goal are host sequences of n*d_x floats;
    obstacles (optional) rows of (x, y, z, radius)."""
    d_x, d_u, _ = DIMS.get(dyn, (4, 2, 2))
    flat_s = [float(v) for v in _flatten(start)]
    flat_g = [float(v) for v in _flatten(goal)]
    s = (ctypes.c_float * max(1, len(flat_s)))(*flat_s)
    g = (ctypes.c_float * max(1, len(flat_g)))(*flat_g)
    if n_robots >= 1 and (len(flat_s) != n_robots * d_x or len(flat_g) != n_robots * d_x):
        raise ValueError("start/goal must hold n_robots * d_x values")
    lo = _fbuf(u_lo, d_u) if u_lo is not None else None
    hi = _fbuf(u_hi, d_u) if u_hi is not None else None
    obs_flat = [float(v) for v in _flatten(obstacles)] if obstacles is not None else []
    n_obs = len(obs_flat) // 4
    obs = (ctypes.c_float * max(1, len(obs_flat)))(*obs_flat)
    desc = _Desc(n_robots, T, dyn, integ, dt, radius, eps_margin, goal_tol, v_max, s, g,
                 ctypes.cast(lo, ctypes.POINTER(ctypes.c_float)) if lo is not None else None,
                 ctypes.cast(hi, ctypes.POINTER(ctypes.c_float)) if hi is not None else None,
                 n_obs, ctypes.cast(obs, ctypes.POINTER(ctypes.c_float)) if n_obs else None)
    h = ctypes.c_void_p()
    _check(lib.d4orm_problem_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def d4orm_problem_destroy(handle) -> None:
    lib.d4orm_problem_destroy(handle)


def d4orm_problem_set_rollout_kernel(handle, kernel: int) -> None:
    _check(lib.d4orm_problem_set_rollout_kernel(handle, kernel))


def d4orm_problem_rollout_kernel(handle, n_samples: int) -> int:
    return lib.d4orm_problem_rollout_kernel(handle, n_samples)


def d4orm_rollout(handle, params: Params | None, u_dev, states_dev=None, want_verdict: bool = True, stream=None):
    v = _Verdict()
    pc = params.c() if params is not None else None
    _check(lib.d4orm_rollout(handle, ctypes.byref(pc) if pc is not None else None, _ptr(u_dev), _ptr(states_dev),
                             ctypes.byref(v) if want_verdict else None, _stream(stream)))
    return _verdict(v) if want_verdict else None


def d4orm_sample_fitness(handle, params: Params, iter: int, step_i: int, u_base_dev, du_in_dev, fitness_dev,
                         stream=None) -> None:
    """Eq. (3) fitness of the N samples of step i (no update)."""
    pc = params.c()
    _check(lib.d4orm_sample_fitness(handle, ctypes.byref(pc), iter, step_i, _ptr(u_base_dev), _ptr(du_in_dev),
                                    _ptr(fitness_dev), _stream(stream)))


def d4orm_denoise_step(handle, params: Params, iter: int, step_i: int, u_base_dev, du_in_dev, du_out_dev,
                       fitness_dev=None, stream=None) -> None:
    pc = params.c()
    _check(lib.d4orm_denoise_step(handle, ctypes.byref(pc), iter, step_i, _ptr(u_base_dev), _ptr(du_in_dev),
                                  _ptr(du_out_dev), _ptr(fitness_dev), _stream(stream)))


def d4orm_denoise_step_timed(handle, params: Params, iter: int, step_i: int, u_base_dev, du_in_dev, du_out_dev,
                             fitness_dev=None, stream=None) -> list[float]:
    """Same as d4orm_denoise_step; returns the per-kernel device times [ms]
    (rollout+fitness, softmax weights, weighted noise sum with the update)."""
    pc = params.c()
    ms = (ctypes.c_float * 3)()
    _check(lib.d4orm_denoise_step_timed(handle, ctypes.byref(pc), iter, step_i, _ptr(u_base_dev), _ptr(du_in_dev),
                                        _ptr(du_out_dev), _ptr(fitness_dev), ms, _stream(stream)))
    return list(ms)


def d4orm_denoise_step_noalloc(handle, params: Params, iter: int, step_i: int, u_base_dev, du_in_dev, du_out_dev,
                               fitness_dev=None, stream=None) -> None:
    """d4orm_denoise_step for callers that cannot allocate device memory: the
    scratch lives in a fixed array of the library's device image (shared by
    all calls on a device; overlapping calls race)."""
    pc = params.c()
    _check(lib.d4orm_denoise_step_noalloc(handle, ctypes.byref(pc), iter, step_i, _ptr(u_base_dev),
                                          _ptr(du_in_dev), _ptr(du_out_dev), _ptr(fitness_dev), _stream(stream)))


def _anytime_check(status: int, results) -> None:
    """Raise for a non-OK status; a cancelled or timed-out solve carries the
    results it wrote."""
    if status in (ERR_TIMEOUT, ERR_CANCELLED):
        raise D4ormError(status, lib.d4orm_last_error().decode(errors="replace"), results)
    _check(status)


def _result(r) -> dict:
    return dict(verdict=_verdict(r.verdict), iters_run=r.iters_run, first_success_iter=r.first_success_iter,
                ms_to_success=r.ms_to_success, ms_total=r.ms_total, stop_reason=r.stop_reason)


def d4orm_solve(handle, params: Params, budget: Budget, u_out_dev, du_init_dev=None, stream=None) -> dict:
    pc, bc = params.c(), budget.c()
    r = _Result()
    status = lib.d4orm_solve(handle, ctypes.byref(pc), ctypes.byref(bc), _ptr(du_init_dev), _ptr(u_out_dev),
                             ctypes.byref(r), _stream(stream))
    _anytime_check(status, _result(r))
    return _result(r)


def d4orm_problem_cancel(handle) -> None:
    """Stop the running (or next) solve of this problem before its next iteration."""
    _check(lib.d4orm_problem_cancel(handle))


def d4orm_batch_cancel(batch) -> None:
    """Stop the running (or next) batched solve at every CTA's next step."""
    _check(lib.d4orm_batch_cancel(batch))


def d4orm_sample_noise(handle, params: Params, iter: int, step_i: int, j0: int, count: int, eps_dev,
                       stream=None) -> None:
    pc = params.c()
    _check(lib.d4orm_sample_noise(handle, ctypes.byref(pc), iter, step_i, j0, count, _ptr(eps_dev),
                                  _stream(stream)))


def d4orm_problem_graph_captures(handle) -> int:
    """Iteration graphs captured on this handle so far."""
    return int(lib.d4orm_problem_graph_captures(handle))


def d4orm_philox4x32_10(ctr_dev, key0: int, key1: int, count: int, out_dev, stream=None) -> None:
    _check(lib.d4orm_philox4x32_10(_ptr(ctr_dev), key0 & 0xFFFFFFFF, key1 & 0xFFFFFFFF, count, _ptr(out_dev),
                                   _stream(stream)))


def d4orm_fp32_fma_probe(out_dev, blocks: int, threads: int, iters: int, stream=None) -> None:
    """blocks * threads * iters * 16 FP32 FLOPs of independent FFMA chains."""
    _check(lib.d4orm_fp32_fma_probe(_ptr(out_dev), blocks, threads, iters, _stream(stream)))


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for b, x in enumerate(items):
        p = _ptr(x)
        arr[b] = p.value if p is not None else None
    return arr


def _results(res, count):
    return [_result(r) for r in list(res)[:count]]


def d4orm_batch_create(handles, params: Params, autotune: bool = False) -> ctypes.c_void_p:
    """Batch over problem handles (they must outlive the batch)."""
    hs = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    pc = params.c()
    out = ctypes.c_void_p()
    _check(lib.d4orm_batch_create(hs, len(handles), ctypes.byref(pc), int(autotune), ctypes.byref(out)))
    return out


def d4orm_batch_solve(batch, budget: Budget, u_out_devs, du_init_devs=None, stream=None) -> list[dict]:
    bc = budget.c()
    outs = _ptr_array(u_out_devs)
    inits = _ptr_array(du_init_devs) if du_init_devs is not None else None
    res = (_Result * len(u_out_devs))()
    status = lib.d4orm_batch_solve(batch, ctypes.byref(bc), inits, outs, res, _stream(stream))
    _anytime_check(status, _results(res, len(u_out_devs)))
    return _results(res, len(u_out_devs))


def d4orm_batch_tuning(batch) -> list[dict]:
    """Every autotuner pilot: threads per CTA, CTAs per SM, ms."""
    n = ctypes.c_int()
    _check(lib.d4orm_batch_tuning(batch, 0, ctypes.byref(n), None, None, None))
    w, o = (ctypes.c_int * max(1, n.value))(), (ctypes.c_int * max(1, n.value))()
    ms = (ctypes.c_float * max(1, n.value))()
    _check(lib.d4orm_batch_tuning(batch, n.value, ctypes.byref(n), w, o, ms))
    return [dict(threads_per_cta=w[k], ctas_per_sm=o[k], ms=ms[k]) for k in range(n.value)]


def d4orm_batch_set_packing(batch, mode: int) -> None:
    """PACK_SINGLE or PACK_PAIRED for every problem (paired only where the
    kernel has the two-robots-per-lane rollout: teams of 5..16 robots)."""
    _check(lib.d4orm_batch_set_packing(batch, int(mode)))


def d4orm_batch_packing(batch, count: int) -> dict:
    """Per-problem packing (1 = two robots per lane) and the packing
    pilots' summed device ns per bucket: {(dyn, "5-8"|"9-16"): (single, paired)}."""
    paired = (ctypes.c_int * max(1, count))()
    ns = (ctypes.c_longlong * 16)()
    _check(lib.d4orm_batch_packing(batch, count, paired, ns))
    names = [(d, r) for d in (HOLO2D, HOLO3D, UNICYCLE, DIFFDRIVE4) for r in ("5-8", "9-16")]
    return dict(paired=[paired[b] for b in range(count)],
                bucket_ns={names[k]: (ns[2 * k], ns[2 * k + 1]) for k in range(8)})


def d4orm_batch_info(batch) -> dict:
    t, c = ctypes.c_int(), ctypes.c_int()
    ms = (ctypes.c_float * 3)()
    _check(lib.d4orm_batch_info(batch, ctypes.byref(t), ctypes.byref(c), ms))
    return dict(threads_per_cta=t.value, ctas=c.value, tuned_ms=list(ms))


def d4orm_batch_destroy(batch) -> None:
    lib.d4orm_batch_destroy(batch)


def d4orm_solve_batched(handles, params: Params, budget: Budget, u_out_devs, stream=None) -> list[dict]:
    hs = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    pc, bc = params.c(), budget.c()
    res = (_Result * len(handles))()
    _check(lib.d4orm_solve_batched(hs, len(handles), ctypes.byref(pc), ctypes.byref(bc), _ptr_array(u_out_devs),
                                   res, _stream(stream)))
    return _results(res, len(handles))


@dataclass
class WarmStartDesc:
    """Shape and optimiser settings of the set-MLP (d4orm_warmstart_desc)."""
    n_max: int = 16
    T: int = 80
    d_u: int = 2
    width: int = 256
    max_batch: int = 256
    seed: int = 0
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    weight_decay: float = 1e-4
    pos_scale: float = 5.0

    def c(self) -> _WsDesc:
        return _WsDesc(self.n_max, self.T, self.d_u, self.width, self.max_batch, self.seed, self.lr, self.beta1,
                       self.beta2, self.eps, self.weight_decay, self.pos_scale)


def d4orm_warmstart_create(desc: WarmStartDesc) -> ctypes.c_void_p:
    dc = desc.c()
    out = ctypes.c_void_p()
    _check(lib.d4orm_warmstart_create(ctypes.byref(dc), ctypes.byref(out)))
    return out


def d4orm_warmstart_destroy(ws) -> None:
    lib.d4orm_warmstart_destroy(ws)


def d4orm_warmstart_param_count(ws) -> int:
    return lib.d4orm_warmstart_param_count(ws)


def d4orm_warmstart_get_params(ws):
    import numpy as np
    n = lib.d4orm_warmstart_param_count(ws)
    out = np.zeros(n, dtype=np.float32)
    _check(lib.d4orm_warmstart_get_params(ws, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n))
    return out


def d4orm_warmstart_set_params(ws, params) -> None:
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib.d4orm_warmstart_set_params(ws, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(p)))


def d4orm_warmstart_forward(ws, x_dev, mask_dev, B: int, y_dev, stream=None) -> None:
    _check(lib.d4orm_warmstart_forward(ws, _ptr(x_dev), _ptr(mask_dev), B, _ptr(y_dev), _stream(stream)))


def d4orm_warmstart_loss_grad(ws, x_dev, mask_dev, y_dev, B: int, grad_dev=None, stream=None) -> float:
    loss = ctypes.c_float()
    _check(lib.d4orm_warmstart_loss_grad(ws, _ptr(x_dev), _ptr(mask_dev), _ptr(y_dev), B, ctypes.byref(loss),
                                         _ptr(grad_dev), _stream(stream)))
    return loss.value


def d4orm_warmstart_train_step(ws, x_all, mask_all, y_all, B: int, idx_dev=None, want_loss: bool = True,
                               stream=None):
    loss = ctypes.c_float()
    _check(lib.d4orm_warmstart_train_step(ws, _ptr(x_all), _ptr(mask_all), _ptr(y_all), _ptr(idx_dev), B,
                                          ctypes.byref(loss) if want_loss else None, _stream(stream)))
    return loss.value if want_loss else None


def d4orm_warmstart_features(handle, n_max: int, pos_scale: float = 5.0):
    import numpy as np
    x = np.zeros((n_max, WS_FEATURES), dtype=np.float32)
    m = np.zeros(n_max, dtype=np.float32)
    _check(lib.d4orm_warmstart_features(handle, n_max, pos_scale, x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        m.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return x, m


def d4orm_warmstart_predict(ws, handle, params: Params, start_step: int, du_seed_dev, stream=None) -> None:
    pc = params.c()
    _check(lib.d4orm_warmstart_predict(ws, handle, ctypes.byref(pc), start_step, _ptr(du_seed_dev),
                                       _stream(stream)))


def d4orm_status_string(status: int) -> str:
    return lib.d4orm_status_string(status).decode()


def d4orm_last_error() -> str:
    return lib.d4orm_last_error().decode()


def _flatten(x):
    if hasattr(x, "ravel"):
        return list(x.ravel())
    out = []
    for v in x:
        if isinstance(v, (list, tuple)) or hasattr(v, "__len__"):
            out.extend(_flatten(v))
        else:
            out.append(v)
    return out


class Problem:
    """Owning wrapper of a d4orm_problem handle built from a scenario-like
    object (fields n, T, dyn, integ, dt, radius, start, goal, u_lo, u_hi,
    v_max, eps_margin, goal_tol)."""

    def __init__(self, inst):
        self.inst = inst
        self.n, self.T, self.dyn = inst.n, inst.T, inst.dyn
        self.d_x, self.d_u, self.d_p = DIMS[inst.dyn]
        self.handle = d4orm_problem_create(inst.n, inst.T, inst.dyn, inst.integ, inst.dt, inst.radius,
                                           inst.start, inst.goal, eps_margin=inst.eps_margin,
                                           goal_tol=inst.goal_tol, v_max=inst.v_max, u_lo=inst.u_lo,
                                           u_hi=inst.u_hi, obstacles=getattr(inst, "obstacles", None))

    def close(self):
        if self.handle:
            d4orm_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
