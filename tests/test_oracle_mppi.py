"""Pins for the oracle's MPPI update rule: the softmax update the paper
contrasts its noise schedule with (Sec. IV-B; Williams et al., "Information
Theoretic MPC for Model-Based Reinforcement Learning", ICRA 2017/2018):
samples dU + sigma eps around the current deformation, new deformation =
their softmax-weighted mean, no schedule.

Expected values are built from the noise function (pinned separately by
the Philox known-answer and Box-Muller tests) and the textbook update
dU' = dU + sigma * sum_j w_j eps_j, never from the update code itself.
"""
import numpy as np
import pytest


def _prob(o, n=2, T=6):
    start = np.array([[0.0, 0.0, 0.0, 0.0], [1.0, 0.0, 0.0, 0.0]])[:n]
    goal = np.array([[1.0, 1.0, 0.0, 0.0], [0.0, 1.0, 0.0, 0.0]])[:n]
    return o.Problem(n=n, T=T, dyn=o.HOLO2D, integ=o.RK4, dt=0.1, radius=0.2, start=start, goal=goal,
                     u_lo=(-1, -1), u_hi=(1, 1))


def _params(o, N, sigma=0.7, **kw):
    return o.Params(N=N, K=10, lam=0.1, w_safe=5.0, seed=11, tag=3, update_rule=o.MPPI, mppi_sigma=sigma, **kw)


def test_single_sample_moves_by_sigma_eps(oracle_lib):
    """N = 1: the only weight is 1, so dU' = dU + sigma eps_0."""
    o = oracle_lib
    pr = _prob(o)
    pp = _params(o, 1)
    rng = np.random.default_rng(0)
    du = rng.normal(size=(pr.T, pr.n, 2))
    out = o.weighted_update(pr, pp, 2, 7, du, np.array([1.0]))
    eps = o.noise_block(pr, pp, 2, 7, 0)
    assert np.abs(out - (du + 0.7 * eps)).max() < 1e-14


def test_uniform_weights_average_the_noise(oracle_lib):
    """Equal fitness (degenerate batch, uniform weights): dU' = dU + sigma mean_j eps_j."""
    o = oracle_lib
    pr = _prob(o)
    N = 16
    pp = _params(o, N, sigma=0.3)
    du = np.full((pr.T, pr.n, 2), 0.25)
    out, _ = o.denoise_step(pr, pp, 0, 4, np.zeros_like(du), du, fitness_in=np.full(N, 0.5))
    mean_eps = np.mean([o.noise_block(pr, pp, 0, 4, j) for j in range(N)], axis=0)
    assert np.abs(out - (du + 0.3 * mean_eps)).max() < 1e-13


def test_dominant_sample_takes_all_weight(oracle_lib):
    """One sample of nine scored 1, the rest 0: z-scores 2.83 vs -0.35, so
    at lambda = 0.1 its logit leads by 31.8 and the other eight weights
    total 1e-13: dU' = dU + sigma eps_best to 1e-12."""
    o = oracle_lib
    pr = _prob(o)
    N = 9
    pp = _params(o, N, sigma=0.5)
    fit = np.zeros(N)
    fit[5] = 1.0
    du = np.zeros((pr.T, pr.n, 2))
    out, _ = o.denoise_step(pr, pp, 1, 2, du, du, fitness_in=fit)
    assert np.abs(out - 0.5 * o.noise_block(pr, pp, 1, 2, 5)).max() < 1e-12


def test_no_schedule(oracle_lib):
    """The update does not depend on beta0/beta1 or on the step's place in
    the schedule (only the Philox counter carries the step index)."""
    o = oracle_lib
    pr = _prob(o)
    N = 8
    rng = np.random.default_rng(1)
    du = rng.normal(size=(pr.T, pr.n, 2))
    w = rng.dirichlet(np.ones(N))
    a = o.weighted_update(pr, _params(o, N, beta0=1e-4, beta1=1e-2), 0, 3, du, w)
    b = o.weighted_update(pr, _params(o, N, beta0=0.2, beta1=0.5), 0, 3, du, w)
    assert np.array_equal(a, b)
    want = du + 0.7 * sum(w[j] * o.noise_block(pr, _params(o, N), 0, 3, j) for j in range(N))
    assert np.abs(a - want).max() < 1e-13


def test_denoise_rule_differs(oracle_lib):
    """Same samples' noise under the D4orm rule: dU' = g (c dU + s sum w eps)
    with the schedule's c = 1/sqrt(abar_i), s = sqrt(1/abar_i - 1),
    g = sqrt(abar_{i-1}) -- the closed forms, from the schedule of Sec. IV-B."""
    o = oracle_lib
    pr = _prob(o)
    N = 4
    rng = np.random.default_rng(2)
    du = rng.normal(size=(pr.T, pr.n, 2))
    w = rng.dirichlet(np.ones(N))
    pp = o.Params(N=N, K=10, lam=0.1, w_safe=5.0, seed=11, tag=3)
    i = 6
    beta = 1e-4 + (1e-2 - 1e-4) * np.arange(10) / 9
    abar = np.concatenate([[1.0], np.cumprod(1 - beta)])
    c, s, g = 1 / np.sqrt(abar[i]), np.sqrt(1 / abar[i] - 1), np.sqrt(abar[i - 1])
    want = g * (c * du + s * sum(w[j] * o.noise_block(pr, pp, 0, i, j) for j in range(N)))
    got = o.weighted_update(pr, pp, 0, i, du, w)
    assert np.abs(got - want).max() < 1e-12


@pytest.mark.parametrize("sigma", [0.3, 1.0])
def test_mppi_solve_improves_the_reward(oracle_lib, sigma):
    """Property: two robots swapping places; MPPI iterations from zero
    controls raise the Eq. (3) reward above that of the zero plan."""
    o = oracle_lib
    start = np.array([[-1.0, 0.0, 0.0, 0.0], [1.0, 0.0, 0.0, 0.0]])
    pr = o.Problem(n=2, T=30, dyn=o.HOLO2D, integ=o.RK4, dt=0.1, radius=0.2, start=start, goal=-start,
                   u_lo=(-1, -1), u_hi=(1, 1), v_max=1.0)
    pp = o.Params(N=64, K=5, lam=0.1, w_safe=5.0, seed=1, update_rule=o.MPPI, mppi_sigma=sigma)
    zero = o.verdict(pr, 5.0, o.rollout(pr, np.zeros((30, 2, 2))))["reward"]
    _, verdicts, _ = o.solve(pr, pp, 3)
    assert verdicts[-1]["reward"] > zero + 0.1
