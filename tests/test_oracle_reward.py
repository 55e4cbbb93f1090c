"""Pins for the oracle's reward (Eq. (3)-(5)), verdict (Eq. (1)-(2)) and
sample weights (Sec. IV-C normalisation, Eq. (6) softmax).

Trajectories are built by hand (states written directly), so collision
timesteps and goal distances have closed forms independent of the oracle.
"""
import math

import numpy as np
import pytest


def _prob2d(o, n, T, start, goal, radius=0.2, eps=0.05, tol=0.1):
    return o.Problem(n=n, T=T, dyn=o.HOLO2D, integ=o.RK4, dt=0.1, radius=radius, start=np.array(start, float),
                     goal=np.array(goal, float), u_lo=(-1, -1), u_hi=(1, 1), eps_margin=eps, goal_tol=tol)


def _states(paths, d_x=4):
    """paths: list over robots of arrays [T+1][2] positions."""
    T1 = len(paths[0])
    st = np.zeros((T1, len(paths), d_x))
    for k, p in enumerate(paths):
        st[:, k, :2] = p
    return st


def test_head_on_pair_closed_form(oracle_lib):
    """Two robots approach head-on along x at 0.1 m per step from x = -+2
    and pass through each other: separation s_t = |4 - 0.2 t|.  r_safe = -1
    exactly when s_t <= 2R+eps = 0.45, i.e. for t = 18..22 (5 steps)."""
    o = oracle_lib
    T, w = 25, 5.0
    t = np.arange(T + 1)
    x1 = -2.0 + 0.1 * t
    p1 = np.stack([x1, np.zeros_like(x1)], 1)
    p2 = np.stack([-x1, np.zeros_like(x1)], 1)
    start = [[-2, 0, 0, 0], [2, 0, 0, 0]]
    goal = [[2, 0, 0, 0], [-2, 0, 0, 0]]
    pr = _prob2d(o, 2, T, start, goal)
    st = _states([p1, p2])
    r, gap = o.reward(pr, w, st)
    n_coll = 5
    # r_goal for robot 1 at t: 1 - |x1 - 2| / 4 = 1 - (4 - 0.1 t) / 4 = 0.025 t; same for robot 2.
    goal_sum = 2 * sum(0.025 * tt for tt in range(1, T + 1))
    want = (goal_sum - w * 2 * n_coll) / (2 * T)
    assert abs(r - want) < 1e-12
    # gap: closest approach of a separation to 0.45 over t = 1..T
    assert abs(gap - min(abs(abs(4 - 0.2 * tt) - 0.45) for tt in range(1, T + 1))) < 1e-12
    v = o.verdict(pr, w, st)
    assert abs(v["min_pair_dist"]) < 1e-12          # they meet at t = 20
    assert v["collision_free"] is False


def test_r_safe_is_an_indicator_not_a_count(oracle_lib):
    """Robot 0 sits between robots 1 and 2, both within 2R+eps: it still
    receives -1 per timestep, not -2."""
    o = oracle_lib
    T, w = 4, 1.0
    st = _states([np.tile([0.0, 0.0], (T + 1, 1)), np.tile([0.3, 0.0], (T + 1, 1)),
                  np.tile([-0.3, 0.0], (T + 1, 1))])
    start = [[0, 0, 0, 0], [0.3, 0, 0, 0], [-0.3, 0, 0, 0]]
    goal = [[0, 5, 0, 0], [0.3, 5, 0, 0], [-0.3, 5, 0, 0]]
    pr = _prob2d(o, 3, T, start, goal)
    r, _ = o.reward(pr, w, st)
    # every robot stays at its start: r_goal = 0; robots 1, 2 are 0.6 apart (> 0.45).
    assert abs(r - (-(T * 3) * w) / (3 * T)) < 1e-15


def test_parked_at_goal_and_at_start(oracle_lib):
    o = oracle_lib
    T = 10
    start = [[0, 0, 0, 0], [3, 0, 0, 0]]
    goal = [[0, 2, 0, 0], [3, 2, 0, 0]]
    pr = _prob2d(o, 2, T, start, goal)
    at_goal = _states([np.tile([0.0, 2.0], (T + 1, 1)), np.tile([3.0, 2.0], (T + 1, 1))])
    at_start = _states([np.tile([0.0, 0.0], (T + 1, 1)), np.tile([3.0, 0.0], (T + 1, 1))])
    assert abs(o.reward(pr, 5.0, at_goal)[0] - 1.0) < 1e-15
    assert abs(o.reward(pr, 5.0, at_start)[0]) < 1e-15
    v = o.verdict(pr, 5.0, at_goal)
    assert v["goal_reached"] and v["collision_free"] and v["objective"] == 1.0
    v = o.verdict(pr, 5.0, at_start)
    assert not v["goal_reached"] and v["objective"] == 0.0


def test_goal_on_start_uses_radius_denominator(oracle_lib):
    """A goal placed on its start: d0 = 0 is replaced by R_a, so a robot
    displaced by R_a gets r_goal = 0."""
    o = oracle_lib
    T = 3
    pr = _prob2d(o, 1, T, [[1, 1, 0, 0]], [[1, 1, 0, 0]], radius=0.2)
    st = _states([np.tile([1.2, 1.0], (T + 1, 1))])
    assert abs(o.reward(pr, 5.0, st)[0]) < 1e-12


def test_safety_uses_2R_not_margin(oracle_lib):
    """Eq. (1) safety is |p_k - p_l| > 2 R_a (no epsilon); Eq. (5) uses 2 R_a + eps."""
    o = oracle_lib
    T = 2
    st = _states([np.tile([0.0, 0.0], (T + 1, 1)), np.tile([0.42, 0.0], (T + 1, 1))])
    pr = _prob2d(o, 2, T, [[0, 0, 0, 0], [0.42, 0, 0, 0]], [[0, 9, 0, 0], [0.42, 9, 0, 0]])
    v = o.verdict(pr, 5.0, st)
    assert v["collision_free"]          # 0.42 > 0.4
    assert v["reward"] < 0              # 0.42 <= 0.45: penalised
    assert abs(v["min_pair_dist"] - 0.42) < 1e-15


def test_objective_counts_time_at_goal(oracle_lib):
    """Eq. (2): robot reaches its goal at t = 6 of T = 10 and stays: 5 of 10
    states at goal (t = 6..10)."""
    o = oracle_lib
    T = 10
    xs = np.minimum(np.arange(T + 1) * 0.5, 3.0)
    pr = _prob2d(o, 1, T, [[0, 0, 0, 0]], [[3, 0, 0, 0]])
    st = _states([np.stack([xs, np.zeros_like(xs)], 1)])
    v = o.verdict(pr, 5.0, st)
    assert abs(v["objective"] - 5 / 10) < 1e-15 and v["goal_reached"]


# ------------------------------------------------------------------ weights

def test_weights_two_samples_closed_form(oracle_lib):
    """N = 2, r = (0, 1): population z-score gives z = (-1, +1), so
    w_1 = 1 / (1 + exp(-2 / lambda))."""
    o = oracle_lib
    for lam in (0.1, 0.5, 2.0):
        w = o.weights(np.array([0.0, 1.0]), lam)
        assert abs(w[1] - 1.0 / (1.0 + math.exp(-2.0 / lam))) < 1e-15
        assert abs(w.sum() - 1.0) < 1e-15


def test_weights_sum_to_one_and_invariance(oracle_lib):
    o = oracle_lib
    rng = np.random.default_rng(0)
    r = rng.normal(size=777)
    w = o.weights(r, 0.1)
    assert abs(w.sum() - 1.0) < 1e-12 and (w >= 0).all()
    for a, b in ((3.0, 0.0), (0.01, -5.0), (1.0, 1e3)):
        np.testing.assert_allclose(o.weights(a * r + b, 0.1), w, rtol=1e-9, atol=1e-300)


def test_weights_equal_rewards_uniform(oracle_lib):
    o = oracle_lib
    w = o.weights(np.full(100, 0.37), 0.1)
    np.testing.assert_allclose(w, 0.01, rtol=1e-14)


def test_weights_zero_temperature_limit(oracle_lib):
    """As lambda -> 0 the weights collapse onto the argmax, or become uniform
    over exact ties."""
    o = oracle_lib
    r = np.array([0.1, 0.9, 0.5, 0.2])
    w = o.weights(r, 1e-4)
    np.testing.assert_allclose(w, [0, 1, 0, 0], atol=1e-12)
    r = np.array([0.1, 0.9, 0.5, 0.9])
    w = o.weights(r, 1e-4)
    np.testing.assert_allclose(w, [0, 0.5, 0, 0.5], atol=1e-12)
