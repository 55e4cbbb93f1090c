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


def test_denoise_equals_eq10_eq11_form(oracle_lib):
    """Eq. (13) (tau_{i-1} = sqrt(abar_{i-1}) tau_bar) must agree with the
    longer route of Eq. (10) with the Monte Carlo score of Eq. (11)."""
    o = oracle_lib
    pr, pp = _small(o)
    rng = np.random.default_rng(1)
    du = 0.2 * rng.standard_normal((pr.T, pr.n, 2))
    ub = 0.1 * rng.standard_normal((pr.T, pr.n, 2))
    i = 7
    out, _ = o.denoise_step(pr, pp, 0, i, ub, du)
    a, ab = o.schedule(pp.K, pp.beta0, pp.beta1)
    tau_bar = out / math.sqrt(ab[i - 1])
    score = -du / (1 - ab[i]) + math.sqrt(ab[i]) / (1 - ab[i]) * tau_bar
    eq10 = (du + (1 - ab[i]) * score) / math.sqrt(a[i])
    np.testing.assert_allclose(eq10, out, rtol=1e-10, atol=1e-12)


def test_one_hot_weights_pick_one_sample(oracle_lib):
    """With all weight on sample j, dU_{i-1} = sqrt(abar_{i-1}) times that
    sample, dU_i / sqrt(abar_i) + sqrt(1/abar_i - 1) eps_j (Eq. (12))."""
    o = oracle_lib
    pr, pp = _small(o, dyn=1, n=2, T=9, N=16)
    rng = np.random.default_rng(2)
    du = 0.3 * rng.standard_normal((pr.T, pr.n, 3))
    i, j = 4, 11
    w = np.zeros(pp.N)
    w[j] = 1.0
    out = o.weighted_update(pr, pp, 0, i, du, w)
    a, ab = o.schedule(pp.K, pp.beta0, pp.beta1)
    eps = o.noise_block(pr, pp, 0, i, j)
    want = math.sqrt(ab[i - 1]) * (du / math.sqrt(ab[i]) + math.sqrt(1 / ab[i] - 1) * eps)
    np.testing.assert_allclose(out, want, rtol=1e-13, atol=1e-15)


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
