"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs and the same Philox noise.

Tolerances (FP32 path vs FP64 oracle):
* Philox words: bit-exact.
* eps: |d| <= 1.2e-6 r + min(2.4e-7 / r, 7e-4) + 1e-7 with r the Box-Muller
  radius of the element's pair -- the error bound of the special-function
  unit's log2, sqrt and sin/cos that the kernels use (margins of 20 %).
* rollout states: <= 1e-4 absolute (metres, m/s, rad).
* per-sample fitness: |d| <= 1e-3 |r| + 1e-5, plus w/(nT) per fragile
  robot-timestep -- one whose Eq. (5) indicator sits within 2e-4 m of its
  threshold, where FP32 and FP64 positions may fall on different sides (each
  flip moves Eq. (3) by exactly w/(nT)).  Fragile samples are counted.
* weighted-mean update: max-norm difference <= 1e-3 ||dU||_inf + 1e-6 ||dU||_inf,
  with the oracle's Eq. (6)/(12)/(13) run on the GPU's own fitness vector
  (stage isolation), and again on the oracle's own fitness when no sample is
  fragile.
"""
import copy
import math

import numpy as np
import pytest

import scenarios
from helpers import (add_obstacles, gpu_params, obstacle_safety_gap, oracle_params, oracle_problem, round_instance,
                     small_instance)

pytestmark = pytest.mark.gpu

DELTA = 2e-4


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    return torch


@pytest.fixture(scope="module")
def g(torch):
    from helpers import build_library
    build_library()
    import paper_2503_12204_gb300 as g
    return g


def dev(torch, a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float32, device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


# ----------------------------------------------------------------------------- noise

def test_philox_bit_exact(torch, g, oracle_lib):
    rng = np.random.default_rng(123)
    ctr = rng.integers(0, 2**32, size=(2048, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [0xFFFFFFFF, 0, 0xFFFFFFFF, 0]]
    key = (0x9E3779B9, 0xDEADBEEF)
    c_dev = torch.as_tensor(ctr.view(np.int32), device="cuda")
    out = torch.zeros_like(c_dev)
    g.d4orm_philox4x32_10(c_dev, key[0], key[1], len(ctr), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    for i in range(len(ctr)):
        assert np.array_equal(got[i], oracle_lib.philox4x32_10(ctr[i], key)), i


@pytest.mark.parametrize("dyn,n,T", [(0, 3, 13), (1, 5, 7), (2, 8, 10), (3, 1, 9)])
def test_sample_noise_matches_oracle(torch, g, oracle_lib, dyn, n, T):
    inst = small_instance(dyn, n, T, N=16, seed=0xABCDEF0123, tag=77)
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    op = oracle_params(oracle_lib, inst)
    j0, count, it, i = 5, 6, 3, 11
    eps = torch.zeros((count, T, n, inst.dims[1]), device="cuda")
    g.d4orm_sample_noise(prob.handle, p, it, i, j0, count, eps)
    torch.cuda.synchronize()
    got = host(eps)
    d_u = inst.dims[1]
    for s in range(count):
        want = oracle_lib.noise_block(oracle_problem(oracle_lib, inst), op, it, i, j0 + s)
        # Box-Muller radius of each element's pair (stream elements 4q+0/1 and 4q+2/3)
        r = np.zeros_like(want)
        for t in range(T):
            for k in range(n):
                for d in range(d_u):
                    e = t * d_u + d
                    other = oracle_lib.noise(op, it, i, j0 + s, k, e ^ 1)
                    r[t, k, d] = np.hypot(want[t, k, d], other)
        err = np.abs(got[s] - want)
        tol = 1.2e-6 * r + np.minimum(2.4e-7 / np.maximum(r, 1e-30), 7e-4) + 1e-7
        assert (err <= tol).all(), (err / tol).max()


# ----------------------------------------------------------------------------- rollout

ROLLOUT_CASES = [(0, 0, 4, 50), (0, 1, 5, 37), (1, 1, 16, 100), (1, 0, 3, 11), (2, 1, 8, 100), (2, 0, 6, 23),
                 (3, 1, 7, 41), (3, 0, 2, 5), (0, 1, 32, 20), (2, 1, 1, 1)]


@pytest.mark.parametrize("dyn,integ,n,T", ROLLOUT_CASES)
def test_rollout_states_and_verdict(torch, g, oracle_lib, dyn, integ, n, T):
    inst = small_instance(dyn, n, T, N=8, integ=integ)
    rng = np.random.default_rng(n * 100 + T)
    u = scenarios.random_controls(rng, inst, scale=1.4).astype(np.float32)  # some outside the box
    prob = g.Problem(inst)
    states = torch.zeros((T + 1, n, inst.dims[0]), device="cuda")
    v = g.d4orm_rollout(prob.handle, gpu_params(g, inst), dev(torch, u), states)
    op = oracle_problem(oracle_lib, inst)
    want = oracle_lib.rollout(op, u.astype(np.float64))
    got = host(states)
    assert np.abs(got - want).max() <= 1e-4, np.abs(got - want).max()
    vo = oracle_lib.verdict(op, inst.w_safe, want)
    if abs(vo["min_pair_dist"] - 2 * inst.radius) > DELTA:
        assert v["collision_free"] == vo["collision_free"]
    final = np.linalg.norm(want[-1, :, :inst.dims[2]] - inst.goal[:, :inst.dims[2]], axis=1)
    if np.all(np.abs(final - inst.goal_tol) > DELTA):
        assert v["goal_reached"] == vo["goal_reached"]
    frag = oracle_lib.fragile(op, want, DELTA)
    assert abs(v["reward"] - vo["reward"]) <= 1e-3 * abs(vo["reward"]) + 1e-5 + frag * inst.w_safe / (n * T)
    if n > 1:
        assert abs(v["min_pair_dist"] - vo["min_pair_dist"]) <= 2e-4


# ----------------------------------------------------------------------------- one step

def _check_step(torch, g, o, inst, it, i, max_oracle_samples=None, seed=0, kernel=0, update=(0, 0.0)):
    rng = np.random.default_rng(seed)
    d_u = inst.dims[1]
    u_base = scenarios.random_controls(rng, inst, scale=0.5).astype(np.float32)
    du_in = scenarios.random_deformation(rng, inst, scale=0.3).astype(np.float32)
    prob = g.Problem(inst)
    g.d4orm_problem_set_rollout_kernel(prob.handle, kernel)
    if kernel:
        assert g.d4orm_problem_rollout_kernel(prob.handle, inst.N) == kernel
    p = gpu_params(g, inst, update=update)
    fit = torch.zeros(inst.N, device="cuda")
    du_out = torch.zeros_like(dev(torch, du_in))
    g.d4orm_denoise_step(prob.handle, p, it, i, dev(torch, u_base), dev(torch, du_in), du_out, fit)
    torch.cuda.synchronize()
    fit_g = host(fit)
    out_g = host(du_out)
    op = oracle_problem(o, inst)
    pp = oracle_params(o, inst, update=update)
    ub64, du64 = u_base.astype(np.float64), du_in.astype(np.float64)
    # per-sample fitness
    if max_oracle_samples and inst.N > max_oracle_samples:
        js = np.sort(rng.choice(inst.N, size=max_oracle_samples, replace=False))
    else:
        js = np.arange(inst.N)
    f_o, _, frag = o.sample_fitness(op, pp, it, i, ub64, du64, js, delta=DELTA, with_fragile=True)
    tol = 1e-3 * np.abs(f_o) + 1e-5 + frag * inst.w_safe / (inst.n * inst.T)
    err = np.abs(fit_g[js] - f_o)
    assert (err <= tol).all(), (err.max(), int((err > tol).sum()))
    n_fragile = int((frag > 0).sum())
    # update from the GPU's fitness vector (stage isolation)
    out_o, _ = o.denoise_step(op, pp, it, i, ub64, du64, fitness_in=fit_g)
    scale = max(np.abs(out_o).max(), 1e-30)
    assert np.abs(out_g - out_o).max() <= (1e-3 + 1e-6) * scale, np.abs(out_g - out_o).max() / scale
    return dict(n_fragile=n_fragile, checked=len(js), fit_g=fit_g, out_g=out_g, u_base=ub64, du_in=du64)


STEP_CASES = [
    # dyn, integ, n, T, N, it, i
    (0, 0, 3, 13, 200, 0, 20),     # ragged: 3 robots in 4-lane segments, T % 4 = 1, partial CTA
    (1, 1, 5, 7, 77, 2, 1),        # 3D, d_u = 3, T * d_u % 4 = 1, last step (sigma small)
    (2, 1, 1, 9, 33, 1, 7),        # one robot: segment of one lane
    (3, 1, 7, 21, 130, 0, 13),     # 4-state differential drive
    (0, 1, 32, 10, 64, 1, 5),      # 32 robots: a whole warp per sample
    (1, 1, 16, 1, 1, 0, 3),        # N = 1, T = 1
    (2, 0, 6, 30, 300, 4095, 20),  # largest iteration index
    (0, 1, 2, 8, 9000, 0, 10),     # N > 8192: softmax re-reads fitness instead of holding it in registers
]


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["register", "pipeline", "paired"])
@pytest.mark.parametrize("dyn,integ,n,T,N,it,i", STEP_CASES)
def test_denoise_step_parity(torch, g, oracle_lib, dyn, integ, n, T, N, it, i, kernel):
    inst = small_instance(dyn, n, T, N, integ=integ, seed=7, K=20)
    r = _check_step(torch, g, oracle_lib, inst, it, i, kernel=kernel)
    assert r["n_fragile"] <= max(2, 0.02 * N)


OBSTACLE_CASES = [
    # dyn, integ, n, T, N, obstacles, reach (fraction of the start-goal segment)
    (0, 1, 5, 40, 300, 3, 0.8),
    (1, 1, 9, 23, 200, 16, 0.4),   # 3D, the maximum obstacle count
    (2, 1, 8, 50, 257, 4, 0.8),
    (3, 0, 3, 17, 64, 2, 0.1),     # diff-drive from rest barely leaves its start in 17 steps
    (0, 1, 32, 12, 70, 12, 0.05),
]


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["register", "pipeline", "paired"])
@pytest.mark.parametrize("dyn,integ,n,T,N,m,reach", OBSTACLE_CASES)
def test_denoise_step_parity_obstacles(torch, g, oracle_lib, dyn, integ, n, T, N, m, reach, kernel):
    """Appendix obstacle term inside the fused rollout + fitness: the same
    per-sample tolerance as without obstacles (fragile indicators now also
    count obstacle distances near r_o + R_a + eps), and the obstacles must
    change the fitness of a good share of the samples (not vacuous).
    Robots cross obstacle boundaries far more often than they pass another
    robot at exactly 2R + eps, so up to a quarter of the samples may carry a
    fragile indicator; the rest are held to the strict tolerance."""
    inst = add_obstacles(small_instance(dyn, n, T, N, integ=integ, seed=7, K=20), m, seed=n + T, reach=reach)
    r = _check_step(torch, g, oracle_lib, inst, 1, 11, kernel=kernel)
    assert r["n_fragile"] <= max(2, 0.25 * N)
    free = copy.deepcopy(inst)
    free.obstacles = None
    f_free, _ = oracle_lib.sample_fitness(oracle_problem(oracle_lib, free), oracle_params(oracle_lib, free), 1, 11,
                                          r["u_base"], r["du_in"], np.arange(N))
    changed = np.abs(r["fit_g"] - f_free) > 0.5 * inst.w_safe / (n * T)
    assert changed.mean() >= 0.2, changed.mean()


@pytest.mark.parametrize("dyn,integ,n,T,m", [(0, 1, 6, 60, 5), (1, 1, 4, 40, 3), (2, 1, 8, 80, 8)])
def test_rollout_verdict_obstacles(torch, g, oracle_lib, dyn, integ, n, T, m):
    """Eq. (1) safety with obstacles on the rollout entry point: the GPU's
    collision_free flag equals the oracle's away from both thresholds, and
    the reward carries the obstacle penalty within the fragile allowance."""
    inst = add_obstacles(small_instance(dyn, n, T, N=8, integ=integ), m, seed=3 * n)
    op = oracle_problem(oracle_lib, inst)
    prob = g.Problem(inst)
    robust = 0
    for trial in range(6):
        rng = np.random.default_rng(100 * trial + n)
        u = scenarios.random_controls(rng, inst, scale=1.2).astype(np.float32)
        v = g.d4orm_rollout(prob.handle, gpu_params(g, inst), dev(torch, u))
        want = oracle_lib.rollout(op, u.astype(np.float64))
        vo = oracle_lib.verdict(op, inst.w_safe, want)
        if (n < 2 or abs(vo["min_pair_dist"] - 2 * inst.radius) > DELTA) and obstacle_safety_gap(inst, want) > DELTA:
            assert v["collision_free"] == vo["collision_free"]
            robust += 1
        frag = oracle_lib.fragile(op, want, DELTA)
        assert abs(v["reward"] - vo["reward"]) <= 1e-3 * abs(vo["reward"]) + 1e-5 + frag * inst.w_safe / (n * T)
    assert robust >= 3


def test_verdict_unsafe_only_because_of_an_obstacle(torch, g):
    """One robot holding still: clear of a distant obstacle it is safe;
    with the obstacle's safety radius reaching its start it is not."""
    start = np.array([[0.0, 0.0, 0.0, 0.0]])
    inst = scenarios.Instance("still", 0, 1, 1, 10, 0.1, 0.2, (-1.0, -1.0), (1.0, 1.0), 1.0, start, start, N=8)
    u = torch.zeros((10, 1, 2), device="cuda")
    for centre, safe in (([3.0, 0.0, 0.0, 0.5], True), ([0.6, 0.0, 0.0, 0.5], False)):
        inst.obstacles = np.array([centre])
        prob = g.Problem(round_instance(inst))
        v = g.d4orm_rollout(prob.handle, gpu_params(g, inst), u)
        assert v["collision_free"] is safe
        assert v["goal_reached"]


MPPI_CASES = [
    # dyn, integ, n, T, N, it, i, sigma
    (0, 1, 4, 30, 256, 0, 50, 0.5),
    (1, 1, 7, 13, 100, 2, 1, 1.0),
    (2, 1, 8, 40, 300, 1, 99, 0.3),
    (3, 0, 5, 21, 9000, 0, 10, 0.8),   # N > 8192
]


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["register", "pipeline", "paired"])
@pytest.mark.parametrize("dyn,integ,n,T,N,it,i,sigma", MPPI_CASES)
def test_mppi_step_parity(torch, g, oracle_lib, dyn, integ, n, T, N, it, i, sigma, kernel):
    """The MPPI update rule on the same kernels: constant sigma around the
    current deformation, new deformation = weighted mean; same fitness and
    update tolerances as the method's step."""
    inst = small_instance(dyn, n, T, N, integ=integ, seed=5, K=100)
    sig = float(np.float32(sigma))
    r = _check_step(torch, g, oracle_lib, inst, it, i, kernel=kernel, update=(1, sig),
                    max_oracle_samples=600 if N > 2000 else None)
    assert r["n_fragile"] <= max(2, 0.05 * min(N, 600))


def test_mppi_differs_from_the_schedule(torch, g):
    """Same samples, same fitness: MPPI's step is not the method's step (the
    schedule's c, sigma, g differ), and beta0/beta1 do not change MPPI."""
    inst = small_instance(0, 4, 20, 128, seed=2, K=50)
    rng = np.random.default_rng(3)
    ub = dev(torch, scenarios.random_controls(rng, inst, 0.5))
    du = dev(torch, scenarios.random_deformation(rng, inst))
    prob = g.Problem(inst)
    outs = []
    for update, betas in (((0, 0.0), (1e-4, 1e-2)), ((1, 0.5), (1e-4, 1e-2)), ((1, 0.5), (0.1, 0.3))):
        p = gpu_params(g, inst, update=update)
        p.beta0, p.beta1 = betas
        o = torch.zeros_like(du)
        g.d4orm_denoise_step(prob.handle, p, 0, 20, ub, du, o, torch.zeros(128, device="cuda"))
        outs.append(host(o))
    assert np.abs(outs[0] - outs[1]).max() > 1e-2
    assert np.array_equal(outs[1], outs[2])


@pytest.mark.parametrize("N", [200, 3000, 9000])
def test_equal_rewards_give_uniform_weights(torch, g, N):
    """Sec. IV-C normalisation when every sample scores the same: a spread
    of 1e-30 around a mean of whole controls moves no position in binary32,
    so all N rewards are bit-equal, the population std is 0 and the weights
    fall back to uniform (no division by zero, no NaN): the MPPI update then
    returns the deformation it was given to within 1e-30 * max|eps|.  N
    spans one and several rewards per softmax thread and the re-reading
    path above 8192."""
    inst = small_instance(0, 4, 20, N, seed=2, K=50)
    rng = np.random.default_rng(9)
    ub = dev(torch, np.round(scenarios.random_controls(rng, inst, 0.5), 1))
    du = torch.zeros_like(ub)
    prob = g.Problem(inst)
    p = gpu_params(g, inst, update=(1, 1e-30))
    o, f = torch.full_like(du, float("nan")), torch.zeros(N, device="cuda")
    g.d4orm_denoise_step(prob.handle, p, 0, 20, ub, du, o, f)
    torch.cuda.synchronize()
    fit = host(f)
    assert np.all(fit == fit[0])
    out = host(o)
    assert np.all(np.isfinite(out)) and np.abs(out).max() <= 1e-28


def test_mppi_solve_verdict_parity(torch, g, oracle_lib):
    """A 2-robot swap solved with the MPPI rule by both implementations: the
    oracle re-judges the GPU's plan with the GPU's verdict, and both reach
    the same verdict flags."""
    start = np.array([[-1.5, 0, 0, 0], [1.5, 0, 0, 0]])
    inst = scenarios.Instance("swap", 0, 1, 2, 60, 0.1, 0.2, (-1.0, -1.0), (1.0, 1.0), 1.0, start, -start,
                              N=256, K=20, iters=4, seed=0)
    inst = round_instance(inst)
    upd = (1, float(np.float32(0.4)))
    prob = g.Problem(inst)
    u_out = torch.zeros((inst.T, 2, 2), device="cuda")
    res = g.d4orm_solve(prob.handle, gpu_params(g, inst, update=upd), g.Budget(max_iters=4), u_out)
    op = oracle_problem(oracle_lib, inst)
    _, verdicts, _ = oracle_lib.solve(op, oracle_params(oracle_lib, inst, update=upd), 4)
    v_g = oracle_lib.verdict(op, inst.w_safe, oracle_lib.rollout(op, host(u_out)))
    if abs(v_g["min_pair_dist"] - 0.4) > DELTA:
        assert res["verdict"]["collision_free"] == v_g["collision_free"]
    assert res["verdict"]["goal_reached"] == v_g["goal_reached"]
    assert abs(res["verdict"]["reward"] - verdicts[-1]["reward"]) < 0.05


@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["register", "pipeline", "paired"])
@pytest.mark.parametrize("dyn,n,T,N", [(0, 5, 23, 300), (2, 8, 40, 257), (1, 3, 17, 64)])
def test_sample_fitness_entry_point(torch, g, oracle_lib, dyn, n, T, N, kernel):
    """d4orm_sample_fitness writes exactly the fitness the full step writes,
    and those values match the oracle within the step's tolerance."""
    inst = small_instance(dyn, n, T, N, seed=9, K=30)
    rng = np.random.default_rng(4)
    ub = scenarios.random_controls(rng, inst, 0.5).astype(np.float32)
    du = scenarios.random_deformation(rng, inst).astype(np.float32)
    prob = g.Problem(inst)
    g.d4orm_problem_set_rollout_kernel(prob.handle, kernel)
    p = gpu_params(g, inst)
    f1 = torch.zeros(N, device="cuda")
    f2 = torch.zeros(N, device="cuda")
    g.d4orm_sample_fitness(prob.handle, p, 3, 17, dev(torch, ub), dev(torch, du), f1)
    g.d4orm_denoise_step(prob.handle, p, 3, 17, dev(torch, ub), dev(torch, du), torch.zeros_like(dev(torch, du)), f2)
    torch.cuda.synchronize()
    assert torch.equal(f1, f2)
    f_o, _, frag = oracle_lib.sample_fitness(oracle_problem(oracle_lib, inst), oracle_params(oracle_lib, inst), 3, 17,
                                             ub.astype(np.float64), du.astype(np.float64), np.arange(N), delta=DELTA,
                                             with_fragile=True)
    tol = 1e-3 * np.abs(f_o) + 1e-5 + frag * inst.w_safe / (n * T)
    assert (np.abs(host(f1) - f_o) <= tol).all()
    with pytest.raises(g.D4ormError):
        g.d4orm_sample_fitness(prob.handle, p, 0, 0, dev(torch, ub), dev(torch, du), f1)


def test_timed_and_noalloc_steps_equal_the_step(torch, g):
    """d4orm_denoise_step_timed and d4orm_denoise_step_noalloc run the same
    kernels with the same launch shapes as d4orm_denoise_step: identical
    fitness and update bits; the timed call reports three positive kernel
    times (rollout + fitness, softmax weights, weighted mean)."""
    inst = small_instance(1, 12, 41, 1500, seed=6, K=20)
    rng = np.random.default_rng(8)
    ub = dev(torch, scenarios.random_controls(rng, inst, 0.5))
    du = dev(torch, scenarios.random_deformation(rng, inst))
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    outs, fits = [], []
    for call in ("step", "timed", "noalloc"):
        o, f = torch.zeros_like(du), torch.zeros(inst.N, device="cuda")
        if call == "step":
            g.d4orm_denoise_step(prob.handle, p, 1, 13, ub, du, o, f)
        elif call == "timed":
            ms = g.d4orm_denoise_step_timed(prob.handle, p, 1, 13, ub, du, o, f)
            assert len(ms) == 3 and all(t > 0 for t in ms)
        else:
            g.d4orm_denoise_step_noalloc(prob.handle, p, 1, 13, ub, du, o, f)
        torch.cuda.synchronize()
        outs.append(o)
        fits.append(f)
    for o, f in zip(outs[1:], fits[1:]):
        assert torch.equal(f, fits[0]) and torch.equal(o, outs[0])


@pytest.mark.parametrize("dyn,n,T,N,m", [(0, 4, 50, 256, 0), (2, 8, 100, 700, 0), (1, 16, 37, 300, 0),
                                         (3, 32, 9, 40, 0), (0, 16, 51, 256, 7), (1, 11, 30, 200, 16)])
def test_rollout_kernels_agree(torch, g, dyn, n, T, N, m):
    """The register, pipeline and paired kernels evaluate the same samples
    with the same arithmetic; only the order of the fitness summation
    differs (m > 0: with obstacles on the start-goal segments)."""
    inst = small_instance(dyn, n, T, N, seed=13, K=20)
    if m:
        inst = add_obstacles(inst, m, seed=n + T)
    rng = np.random.default_rng(2)
    ub = dev(torch, scenarios.random_controls(rng, inst, 0.5))
    du = dev(torch, scenarios.random_deformation(rng, inst))
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    fits = []
    for kernel in (1, 2, 3):
        g.d4orm_problem_set_rollout_kernel(prob.handle, kernel)
        f = torch.zeros(N, device="cuda")
        o = torch.zeros_like(du)
        g.d4orm_denoise_step(prob.handle, p, 2, 9, ub, du, o, f)
        fits.append(host(f))
    torch.cuda.synchronize()
    for f in fits[1:]:
        assert np.abs(fits[0] - f).max() <= 2e-6 * max(1.0, np.abs(fits[0]).max())


def test_denoise_step_own_fitness_when_robust(torch, g, oracle_lib):
    """Full oracle step (its own fitness) vs the GPU when no sample is fragile."""
    inst = small_instance(0, 4, 30, 256, seed=3, K=20)
    r = _check_step(torch, g, oracle_lib, inst, 0, 20)
    if r["n_fragile"] == 0:
        out_o, _ = oracle_lib.denoise_step(oracle_problem(oracle_lib, inst), oracle_params(oracle_lib, inst), 0, 20,
                                           r["u_base"], r["du_in"])
        scale = np.abs(out_o).max()
        assert np.abs(r["out_g"] - out_o).max() <= 2e-3 * scale


@pytest.mark.parametrize("name,it,i,cap", [("holo2d_n4", 0, 100, None), ("unicycle_n8", 3, 100, None),
                                           ("unicycle_n8", 4, 1, 512), ("holo3d_n16", 1, 60, 384)])
def test_denoise_step_parity_full_size(torch, g, oracle_lib, name, it, i, cap):
    """The measured workloads at full size (same launch configuration as the
    benchmark); the oracle checks all samples or a random subset."""
    inst = round_instance(scenarios.WORKLOADS[name]())
    _check_step(torch, g, oracle_lib, inst, it, i, max_oracle_samples=cap, seed=1)


def test_denoise_step_at_the_control_size_limit(torch, g, oracle_lib):
    """T * n * d_u = D4ORM_MAX_CTRL (32 robots, 768 steps, 2 controls): the
    register kernel stages 192 KB of mean controls (200 KB opt-in), AUTO
    picks it because the pipelined kernel's shared memory would not fit,
    and the step matches the oracle on a sample of the batch."""
    inst = small_instance(0, 32, 768, 64, seed=5, K=10)
    assert inst.T * inst.n * 2 == g.MAX_CTRL
    prob = g.Problem(inst)
    assert g.d4orm_problem_rollout_kernel(prob.handle, inst.N) == g.ROLLOUT_REGISTER
    r = _check_step(torch, g, oracle_lib, inst, 0, 7, max_oracle_samples=12, seed=2)
    assert r["checked"] == 12


def test_auto_rollout_kernel_choice(torch, g):
    """AUTO on the 152-SM GB300: two robots per lane for holonomic teams of
    5+ robots from 6 paired warps per SM (12 with obstacles), never for
    unicycle teams; the pipelined kernel for the small 4-robot workload."""
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("thresholds are stated for 152 SMs")
    expect = [("holo3d_n16", None, g.ROLLOUT_PAIRED), ("holo3d_n16", 4096, g.ROLLOUT_PAIRED),
              ("holo3d_n16", 3072, g.ROLLOUT_REGISTER), ("obstacles4_n16", None, g.ROLLOUT_REGISTER),
              ("obstacles4_n16", 8192, g.ROLLOUT_PAIRED), ("unicycle_n8", None, g.ROLLOUT_REGISTER),
              ("unicycle_n8", 65536, g.ROLLOUT_REGISTER), ("holo2d_n4", None, g.ROLLOUT_PIPELINE),
              ("holo2d_n4", 65536, g.ROLLOUT_REGISTER)]
    for name, N, kind in expect:
        inst = round_instance(scenarios.WORKLOADS[name]())
        prob = g.Problem(inst)
        assert g.d4orm_problem_rollout_kernel(prob.handle, N or inst.N) == kind, (name, N)


@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_denoise_step_is_deterministic(torch, g, kernel):
    inst = small_instance(1, 9, 40, 1000, seed=5)
    prob = g.Problem(inst)
    g.d4orm_problem_set_rollout_kernel(prob.handle, kernel)
    p = gpu_params(g, inst)
    rng = np.random.default_rng(0)
    ub = dev(torch, scenarios.random_controls(rng, inst, 0.5))
    du = dev(torch, scenarios.random_deformation(rng, inst))
    outs = []
    for _ in range(2):
        o = torch.zeros_like(du)
        f = torch.zeros(inst.N, device="cuda")
        g.d4orm_denoise_step(prob.handle, p, 1, 10, ub, du, o, f)
        outs.append((o.clone(), f.clone()))
    torch.cuda.synchronize()
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_denoise_step_argument_errors(torch, g):
    inst = small_instance(0, 2, 5, 8)
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    a = torch.zeros((5, 2, 2), device="cuda")
    b = torch.zeros_like(a)
    for it, i in ((0, 0), (0, inst.K + 1), (-1, 1), (4096, 1)):
        with pytest.raises(g.D4ormError) as ei:
            g.d4orm_denoise_step(prob.handle, p, it, i, a, a, b)
        assert ei.value.status == 1
    with pytest.raises(g.D4ormError):
        g.d4orm_denoise_step(prob.handle, p, 0, 1, a, a, a)   # du_out aliases du_in
    bad = gpu_params(g, inst)
    bad.temperature = 0.0
    with pytest.raises(g.D4ormError):
        g.d4orm_denoise_step(prob.handle, bad, 0, 1, a, a, b)
    for rule, sigma in ((2, 0.5), (1, 0.0), (1, float("nan")), (-1, 0.5)):
        with pytest.raises(g.D4ormError) as ei:
            g.d4orm_denoise_step(prob.handle, gpu_params(g, inst, update=(rule, sigma)), 0, 1, a, a, b)
        assert ei.value.status == 1


# ----------------------------------------------------------------------------- solve

def test_solve_matches_eager_steps(torch, g):
    """One solve iteration (graph replay) equals K eager denoise steps followed
    by tau.u = clip(0 + dU_0), bit for bit."""
    inst = small_instance(0, 4, 24, 128, seed=9, K=12)
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    nctrl = (inst.T, inst.n, 2)
    u_out = torch.zeros(nctrl, device="cuda")
    # a new handle runs its first iteration eagerly and captures the graph
    # the second time: both forms give the same bits
    g.d4orm_solve(prob.handle, p, g.Budget(max_iters=1), u_out)
    first = u_out.clone()
    res = g.d4orm_solve(prob.handle, p, g.Budget(max_iters=1), u_out)
    assert torch.equal(first, u_out)
    zero = torch.zeros(nctrl, device="cuda")
    du = torch.zeros(nctrl, device="cuda")
    for i in range(inst.K, 0, -1):
        nxt = torch.zeros_like(du)
        g.d4orm_denoise_step(prob.handle, p, 0, i, zero, du, nxt)
        du = nxt
    lo = torch.tensor(inst.u_lo, device="cuda")
    hi = torch.tensor(inst.u_hi, device="cuda")
    want = torch.minimum(torch.maximum(du, lo), hi)
    torch.cuda.synchronize()
    assert torch.equal(u_out, want)
    assert res["iters_run"] == 1
    v = g.d4orm_rollout(prob.handle, p, u_out)
    assert v == res["verdict"]


@pytest.mark.parametrize("stop", [False, True])
def test_solve_eager_then_graph_iterations(torch, g, stop):
    """Three iterations on a new handle (the first eager, the second captured
    and replayed, the third replayed) equal three iterations on a handle
    whose graph is already captured, bit for bit, verdicts included."""
    inst = small_instance(2, 5, 30, 200, seed=3, K=15)
    p = gpu_params(g, inst)
    budget = g.Budget(max_iters=3, stop_on_success=stop, deadline_ms=0.0)
    outs, results = [], []
    for _ in range(2):
        prob = g.Problem(inst)
        u = torch.zeros((inst.T, inst.n, 2), device="cuda")
        if results:  # second handle: capture first
            g.d4orm_solve(prob.handle, p, g.Budget(max_iters=2, stop_on_success=stop), u)
        results.append(g.d4orm_solve(prob.handle, p, budget, u))
        outs.append(u)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])
    assert results[0]["verdict"] == results[1]["verdict"]
    assert results[0]["iters_run"] == results[1]["iters_run"]


def test_solve_verdict_parity_holo2d_n4(torch, g, oracle_lib):
    """The 4-robot Euler workload solved end to end by both implementations:
    identical collision-free / goal-reached verdicts, and the oracle's
    verdict of the GPU's own plan agrees with the GPU's."""
    inst = round_instance(scenarios.holo2d_circle_n4())
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    u_out = torch.zeros((inst.T, inst.n, 2), device="cuda")
    res = g.d4orm_solve(prob.handle, p, g.Budget(max_iters=1), u_out)
    op, pp = oracle_problem(oracle_lib, inst), oracle_params(oracle_lib, inst)
    u_o, verdicts, _ = oracle_lib.solve(op, pp, 1)
    st_g = oracle_lib.rollout(op, host(u_out))
    v_g = oracle_lib.verdict(op, inst.w_safe, st_g)
    assert res["verdict"]["collision_free"] == v_g["collision_free"]
    assert res["verdict"]["goal_reached"] == v_g["goal_reached"]
    assert res["verdict"]["collision_free"] == verdicts[-1]["collision_free"]
    assert res["verdict"]["goal_reached"] == verdicts[-1]["goal_reached"] is False  # 6 m in 5 s is infeasible


def test_solve_swap_succeeds_like_oracle(torch, g, oracle_lib):
    start = np.array([[-1.5, 0, 0, 0], [1.5, 0, 0, 0]])
    inst = scenarios.Instance("swap", 0, 1, 2, 60, 0.1, 0.2, (-1.0, -1.0), (1.0, 1.0), 1.0, start, -start,
                              N=256, K=100, iters=6, seed=0)
    inst = round_instance(inst)
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    u_out = torch.zeros((inst.T, 2, 2), device="cuda")
    res = g.d4orm_solve(prob.handle, p, g.Budget(max_iters=6, stop_on_success=True), u_out)
    _, verdicts, first = oracle_lib.solve(oracle_problem(oracle_lib, inst), oracle_params(oracle_lib, inst), 6,
                                          stop_on_success=True)
    assert first >= 0 and res["first_success_iter"] >= 0
    assert res["verdict"]["collision_free"] and res["verdict"]["goal_reached"]
    assert res["iters_run"] == res["first_success_iter"] + 1


def test_solve_budget_paths(torch, g):
    inst = small_instance(2, 3, 20, 64, seed=4, K=10)
    prob = g.Problem(inst)
    p = gpu_params(g, inst)
    u_out = torch.zeros((inst.T, 3, 2), device="cuda")
    r = g.d4orm_solve(prob.handle, p, g.Budget(max_iters=3), u_out)
    assert r["iters_run"] == 3 and r["ms_total"] > 0
    r2 = g.d4orm_solve(prob.handle, p, g.Budget(max_iters=3, deadline_ms=1e-6), u_out)
    assert r2["iters_run"] == 1
    # warm start: first iteration runs steps start_step..1 from du_init
    du0 = torch.full((inst.T, 3, 2), 0.05, device="cuda")
    r3 = g.d4orm_solve(prob.handle, p, g.Budget(max_iters=2, start_step=4), u_out, du_init_dev=du0)
    assert r3["iters_run"] == 2
    with pytest.raises(g.D4ormError):
        g.d4orm_solve(prob.handle, p, g.Budget(max_iters=2, start_step=0), u_out, du_init_dev=du0)
    with pytest.raises(g.D4ormError):
        g.d4orm_solve(prob.handle, p, g.Budget(max_iters=0), u_out)
