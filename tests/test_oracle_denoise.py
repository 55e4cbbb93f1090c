"""Pins for the oracle's schedule and one-step denoise (Eq. (10)-(13),
Algorithm 1 on deformations per Algorithm 2), and for the solve loop.
"""
import math

import numpy as np
import pytest

import scenarios


def _small(o, dyn=0, n=3, T=12, N=64, seed=5):
    d_x, d_u, d_p = o.DIMS[dyn]
    rng = np.random.default_rng(11)
    start = np.zeros((n, d_x))
    start[:, :d_p] = rng.uniform(-2, 2, size=(n, d_p))
    goal = np.zeros((n, d_x))
    goal[:, :d_p] = rng.uniform(-2, 2, size=(n, d_p))
    lo = tuple([-1.0] * d_u)
    hi = tuple([1.0] * d_u)
    pr = o.Problem(n=n, T=T, dyn=dyn, integ=o.RK4, dt=0.1, radius=0.2, start=start, goal=goal, u_lo=lo,
                   u_hi=hi, v_max=1.0)
    pp = o.Params(N=N, K=10, seed=seed)
    return pr, pp


def test_schedule_constant_beta_closed_form(oracle_lib):
    """beta0 = beta1 = b: alpha_bar_i = (1 - b)^i, alpha_bar_0 = 1."""
    a, ab = oracle_lib.schedule(50, 0.02, 0.02)
    for i in range(51):
        assert abs(ab[i] - 0.98**i) < 1e-14
    a, ab = oracle_lib.schedule(100, 1e-4, 1e-2)
    assert ab[0] == 1.0 and np.all(np.diff(ab) < 0)
    assert abs(a[1] - (1 - 1e-4)) < 1e-16 and abs(a[100] - (1 - 1e-2)) < 1e-16


B_CONST = 0.05   # constant beta: alpha_i = 1 - b, abar_i = (1 - b)^i in closed form


def _far_goal_problem(o, G=1.0e4):
    """One 2D holonomic robot at rest at the origin, one control step, goal
    G metres along x, no control box and no speed bound.  The exact update
    gives p_1 = u dt^2 / 2, so Eq. (4)'s reward is r = 1 - |p_1 - g| / G and
    the applied x-control is recovered from the reward alone:
    u_x = 2 (G - sqrt(G^2 (1 - r)^2 - (dt^2 u_y / 2)^2)) / dt^2, where the
    u_y term moves u_x by under 1e-8 for |u_y| < 10."""
    start = np.zeros((1, 4))
    goal = np.array([[G, 0.0, 0.0, 0.0]])
    pr = o.Problem(n=1, T=1, dyn=o.HOLO2D, integ=o.RK4, dt=0.1, radius=0.2, start=start, goal=goal,
                   u_lo=(-1e6, -1e6), u_hi=(1e6, 1e6), v_max=0.0)
    return pr, G


def _recover_ux(r, G, dt):
    return 2.0 * G * r / dt**2   # first order in u_y^2 / G, see _far_goal_problem


def test_samples_have_eq12_moments_through_the_rollout(oracle_lib):
    """Eq. (12): the deformation samples of step i are distributed as
    N(dU_i / sqrt(abar_i), (1/abar_i - 1) I).  The samples are observed only
    through the rollout and reward of each (the fitness path), and the
    expected moments come from the closed-form constant-beta schedule, not
    from the oracle: 4000 samples, mean within 4.5 standard errors and
    variance within 15 % (about 6.7 standard errors of a variance of 4000
    draws).  A spread of sqrt(1 - abar_i), or a mean scale of 1 or
    sqrt(abar_i), fails by far more (abar_20 = 0.358)."""
    o = oracle_lib
    pr, G = _far_goal_problem(o)
    K, i, N = 30, 20, 4000
    pp = o.Params(N=N, K=K, beta0=B_CONST, beta1=B_CONST, seed=9, w_safe=0.0)
    abar_i = (1 - B_CONST) ** i
    du = np.array([[[0.7, -0.4]]])
    ub = np.array([[[0.25, 0.1]]])
    f, _ = o.sample_fitness(pr, pp, 0, i, ub, du, np.arange(N))
    samples = _recover_ux(np.asarray(f), G, pr.dt) - ub[0, 0, 0]
    mean_want = du[0, 0, 0] / math.sqrt(abar_i)
    var_want = 1.0 / abar_i - 1.0
    se = math.sqrt(var_want / N)
    assert abs(samples.mean() - mean_want) < 4.5 * se, (samples.mean(), mean_want, se)
    assert abs(samples.var() / var_want - 1.0) < 0.15, (samples.var(), var_want)


def test_one_hot_update_returns_the_rolled_out_sample(oracle_lib):
    """Eq. (13) with all weight on sample j: dU_{i-1} = sqrt(abar_{i-1}) times
    the very sample j whose rollout gave fitness j.  The sample is read back
    from its reward (fitness path), the factor is the closed-form
    (1 - b)^((i-1)/2); nothing is taken from the oracle's own noise."""
    o = oracle_lib
    pr, G = _far_goal_problem(o)
    K, i, N = 30, 12, 24
    pp = o.Params(N=N, K=K, beta0=B_CONST, beta1=B_CONST, seed=4)
    du = np.array([[[-0.3, 0.5]]])
    ub = np.zeros((1, 1, 2))
    f, _ = o.sample_fitness(pr, pp, 2, i, ub, du, np.arange(N))
    ux = _recover_ux(np.asarray(f), G, pr.dt)
    g = (1 - B_CONST) ** ((i - 1) / 2)
    for j in (0, 7, 23):
        w = np.zeros(N)
        w[j] = 1.0
        out = o.weighted_update(pr, pp, 2, i, du, w)
        assert abs(out[0, 0, 0] / g - ux[j]) < 1e-6, (j, out[0, 0, 0] / g, ux[j])


def test_uniform_weights_follow_eq10_with_eq11_score(oracle_lib):
    """Eq. (10) with the Monte Carlo score of Eq. (11): as the weights become
    uniform over many samples the weighted mean tends to the sample mean
    dU_i / sqrt(abar_i), so dU_{i-1} -> dU_i / sqrt(alpha_i) (alpha_i = 1 - b
    for a constant beta).  The residual is sqrt(abar_{i-1}) sqrt(1/abar_i - 1)
    times the mean of N standard normals per entry: its 320 entries must
    have a variance within 35 % of abar_{i-1} (1/abar_i - 1) / N (about 4.4
    standard errors) and none beyond 5 standard deviations."""
    o = oracle_lib
    T, n, N, K, i = 40, 4, 20000, 30, 20
    start = np.zeros((n, 4))
    goal = np.ones((n, 4))
    pr = o.Problem(n=n, T=T, dyn=o.HOLO2D, integ=o.RK4, dt=0.1, radius=0.2, start=start, goal=goal,
                   u_lo=(-1, -1), u_hi=(1, 1), v_max=1.0)
    pp = o.Params(N=N, K=K, beta0=B_CONST, beta1=B_CONST, seed=13)
    rng = np.random.default_rng(8)
    du = rng.uniform(-1.0, 1.0, size=(T, n, 2))
    out = o.weighted_update(pr, pp, 1, i, du, np.full(N, 1.0 / N))
    resid = out - du / math.sqrt(1 - B_CONST)
    abar_i, abar_im1 = (1 - B_CONST) ** i, (1 - B_CONST) ** (i - 1)
    var_want = abar_im1 * (1.0 / abar_i - 1.0) / N
    assert abs((resid**2).mean() / var_want - 1.0) < 0.35, ((resid**2).mean(), var_want)
    assert np.abs(resid).max() < 5.0 * math.sqrt(var_want)
    # the mean path itself: the least-squares slope of dU_{i-1} on dU_i is
    # 1 / sqrt(alpha_i) = 1.026 within 5 standard errors (5.6e-4), and a
    # factor of 1 would sit about 46 standard errors away
    slope = float((out * du).sum() / (du * du).sum())
    se_slope = math.sqrt(var_want / (du * du).sum())
    assert abs(slope - 1.0 / math.sqrt(1 - B_CONST)) < 5.0 * se_slope, (slope, se_slope)
    assert abs(slope - 1.0) > 20.0 * se_slope


def test_uniform_weights_mean_noise_shrinks(oracle_lib):
    """Uniform weights and dU_i = 0: dU_{i-1} = g sigma mean_j eps_j, whose
    entries are N(0, (g sigma)^2 / N): all within 5 standard errors."""
    o = oracle_lib
    pr, pp = _small(o, n=2, T=10, N=2000)
    i = 10
    w = np.full(pp.N, 1.0 / pp.N)
    out = o.weighted_update(pr, pp, 0, i, np.zeros((pr.T, pr.n, 2)), w)
    a, ab = o.schedule(pp.K, pp.beta0, pp.beta1)
    se = math.sqrt(ab[i - 1]) * math.sqrt(1 / ab[i] - 1) / math.sqrt(pp.N)
    assert np.abs(out).max() < 5 * se
    assert np.abs(out).max() > 0.05 * se


def test_denoise_invariant_to_affine_reward(oracle_lib):
    """Batch normalisation (Sec. IV-C) makes the step invariant to r -> a r + b, a > 0."""
    o = oracle_lib
    pr, pp = _small(o, dyn=2, n=3, T=10, N=48)
    rng = np.random.default_rng(3)
    du = 0.2 * rng.standard_normal((pr.T, pr.n, 2))
    ub = np.zeros_like(du)
    out, fit = o.denoise_step(pr, pp, 1, 6, ub, du)
    out2, _ = o.denoise_step(pr, pp, 1, 6, ub, du, fitness_in=2.5 * fit - 7.0)
    np.testing.assert_allclose(out2, out, rtol=1e-9, atol=1e-13)


def test_sample_fitness_matches_manual_rollout(oracle_lib):
    """Sample j's fitness is Eq. (3) of rollout(S, u_base + dU_j), with dU_j
    assembled from the pinned noise and schedule."""
    o = oracle_lib
    pr, pp = _small(o, dyn=0, n=3, T=10, N=8)
    rng = np.random.default_rng(4)
    du = 0.2 * rng.standard_normal((pr.T, pr.n, 2))
    ub = 0.3 * rng.standard_normal((pr.T, pr.n, 2))
    i, j = 3, 5
    f, _ = o.sample_fitness(pr, pp, 0, i, ub, du, [j])
    a, ab = o.schedule(pp.K, pp.beta0, pp.beta1)
    samp = du / math.sqrt(ab[i]) + math.sqrt(1 / ab[i] - 1) * o.noise_block(pr, pp, 0, i, j)
    st = o.rollout(pr, ub + samp)
    assert abs(f[0] - o.reward(pr, pp.w_safe, st)[0]) < 1e-13


def test_two_robot_swap_becomes_feasible(oracle_lib):
    """The method's own claim (Sec. V-B): a small swap is deconflicted.  Two
    2D-holonomic robots exchange places along a line; after a few iterations
    the plan is collision-free and reaches both goals."""
    o = oracle_lib
    start = np.array([[-1.5, 0, 0, 0], [1.5, 0, 0, 0]], float)
    goal = np.array([[1.5, 0, 0, 0], [-1.5, 0, 0, 0]], float)
    pr = o.Problem(n=2, T=60, dyn=o.HOLO2D, integ=o.RK4, dt=0.1, radius=0.2, start=start, goal=goal,
                   u_lo=(-1, -1), u_hi=(1, 1), v_max=1.0, goal_tol=0.1)
    pp = o.Params(N=256, K=100, seed=0)
    u, verdicts, first = o.solve(pr, pp, max_iters=6, stop_on_success=True)
    assert first >= 0, verdicts
    st = o.rollout(pr, u)
    v = o.verdict(pr, pp.w_safe, st)
    assert v["collision_free"] and v["goal_reached"]


def test_scenarios_shapes():
    inst = scenarios.holo3d_sphere_n16()
    r = np.linalg.norm(inst.start[:, :3], axis=1)
    np.testing.assert_allclose(r, 4.0, rtol=1e-12)
    np.testing.assert_allclose(inst.goal[:, :3], -inst.start[:, :3])
    inst = scenarios.holo2d_circle_n4()
    np.testing.assert_allclose(inst.start[:, :2], [[3, 0], [0, 3], [-3, 0], [0, -3]], atol=1e-12)
    batch = scenarios.mixed_batch(count=24, seed=2)
    for b in batch:
        d_p = b.dims[2]
        for pts in (b.start[:, :d_p], b.goal[:, :d_p]):
            dd = np.linalg.norm(pts[:, None] - pts[None], axis=-1) + np.eye(b.n) * 1e9
            assert dd.min() >= 0.6 and np.abs(pts).max() <= 5.0
        assert 2 <= b.n <= 16 and 40 <= b.T <= 120
