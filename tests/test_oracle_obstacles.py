"""Pins for the oracle's obstacle term (Appendix, "presence of obstacles": a
binary penalty per state that collides with an obstacle, added to the
Eq. (3) reward; Eq. (1) safety extended to obstacle clearance).

Readings pinned here: a state collides for the penalty when its distance
to an obstacle's centre is at most r_o + R_a + eps (the Eq. (5) margin),
the penalty weight is the w of Eq. (3), the term is an indicator over
obstacles (two overlapping obstacles cost one w), it adds to the robot-pair
indicator, it counts for t >= 1 like Eq. (3), and safety needs a distance
above r_o + R_a at every t in 0..T.  Trajectories are written by hand, so
every count has a closed form independent of the oracle.
"""
import math

import numpy as np


def _prob(o, n, T, start, goal, obstacles, dyn=None, radius=0.2, eps=0.05, tol=0.1):
    dyn = o.HOLO2D if dyn is None else dyn
    d_u = 3 if dyn == o.HOLO3D else 2
    return o.Problem(n=n, T=T, dyn=dyn, integ=o.RK4, dt=0.1, radius=radius, start=np.array(start, float),
                     goal=np.array(goal, float), u_lo=(-1,) * d_u, u_hi=(1,) * d_u, eps_margin=eps,
                     goal_tol=tol, obstacles=None if obstacles is None else np.array(obstacles, float))


def _states(paths, d_x=4, d_p=2):
    st = np.zeros((len(paths[0]), len(paths), d_x))
    for k, p in enumerate(paths):
        st[:, k, :d_p] = p
    return st


def _line(T, x0=0.0, step=1.0, y=0.0):
    t = np.arange(T + 1)
    return np.stack([x0 + step * t, np.full(T + 1, y)], 1)


def test_single_robot_passes_one_obstacle(oracle_lib):
    """One robot at (t, 0), t = 0..4; obstacle at (2, 0.5), r_o = 0.3.
    Penalty radius 0.3 + 0.2 + 0.05 = 0.55: only t = 2 (distance 0.5) is
    inside; the reward drops by exactly w / (nT) = w / 4."""
    o = oracle_lib
    T, w = 4, 5.0
    start, goal = [[0, 0, 0, 0]], [[4, 0, 0, 0]]
    st = _states([_line(T)])
    r0, _ = o.reward(_prob(o, 1, T, start, goal, None), w, st)
    r1, gap = o.reward(_prob(o, 1, T, start, goal, [[2.0, 0.5, 0.0, 0.3]]), w, st)
    # r_goal at t: 1 - (4 - t) / 4 = t / 4
    assert abs(r0 - sum(t / 4 for t in range(1, 5)) / 4) < 1e-12
    assert abs((r0 - r1) - w / 4) < 1e-12
    dists = [math.hypot(t - 2.0, 0.5) for t in range(1, 5)]
    assert abs(gap - min(abs(d - 0.55) for d in dists)) < 1e-12


def test_overlapping_obstacles_cost_one_w(oracle_lib):
    """Two obstacles that both cover the state at t = 2 cost one w there (an
    indicator over obstacles); a third far away costs nothing."""
    o = oracle_lib
    T, w = 4, 3.0
    start, goal = [[0, 0, 0, 0]], [[4, 0, 0, 0]]
    st = _states([_line(T)])
    r0, _ = o.reward(_prob(o, 1, T, start, goal, None), w, st)
    obs = [[2.0, 0.1, 0.0, 0.3], [2.1, -0.1, 0.0, 0.3], [50.0, 50.0, 0.0, 1.0]]
    r1, _ = o.reward(_prob(o, 1, T, start, goal, obs), w, st)
    assert abs((r0 - r1) - w / 4) < 1e-12


def test_obstacle_and_pair_penalties_add(oracle_lib):
    """Robots 0 and 1 stay 0.3 m apart (inside 2R + eps = 0.45) next to an
    obstacle that covers both at every t >= 1: each robot-step costs 2w."""
    o = oracle_lib
    T, w = 3, 2.0
    p0 = np.tile([0.0, 0.0], (T + 1, 1))
    p1 = np.tile([0.3, 0.0], (T + 1, 1))
    start, goal = [[0, 0, 0, 0], [0.3, 0, 0, 0]], [[0, 0, 0, 0], [0.3, 0, 0, 0]]
    st = _states([p0, p1])
    obs = [[0.15, 0.4, 0.0, 0.2]]   # distance 0.427 from both, below 0.2 + 0.2 + 0.05
    r, _ = o.reward(_prob(o, 2, T, start, goal, obs), w, st)
    # goals are the starts: r_goal = 1 everywhere; penalty 2w per robot-step
    assert abs(r - (1.0 - 2.0 * w)) < 1e-12


def test_penalty_boundary_is_inclusive(oracle_lib):
    """A state exactly at r_o + R_a + eps is penalised (<=), one just
    outside is not.  Distances are exact binary fractions."""
    o = oracle_lib
    T, w = 1, 1.0
    obs = [[0.0, 0.0, 0.0, 0.25]]   # threshold 0.25 + 0.25 + 0.0 = 0.5 with eps = 0
    for y, pen in ((0.5, 1), (0.5 + 2.0 ** -20, 0)):
        st = _states([np.array([[0.0, 5.0], [0.0, y]])])
        pr = _prob(o, 1, T, [[0, 5, 0, 0]], [[0, y, 0, 0]], obs, radius=0.25, eps=0.0)
        r, _ = o.reward(pr, w, st)
        assert abs(r - (1.0 - pen * w)) < 1e-12


def test_verdict_safety_uses_radius_without_margin(oracle_lib):
    """Safety (Eq. (1) with obstacles) needs |p - c_o| > r_o + R_a = 0.5;
    the margin eps only enters the penalty.  At distance 0.52 the plan is
    penalised but safe; at 0.48 it collides; a start inside an obstacle
    (t = 0, not part of Eq. (3)) also makes it unsafe."""
    o = oracle_lib
    T, w = 2, 1.0
    obs = [[0.0, 0.0, 0.0, 0.3]]
    for d, safe in ((0.52, True), (0.48, False)):
        st = _states([np.array([[3.0, 0.0], [d, 0.0], [3.0, 0.0]])])
        v = o.verdict(_prob(o, 1, T, [[3, 0, 0, 0]], [[3, 0, 0, 0]], obs), w, st)
        assert v["collision_free"] is safe
    st = _states([np.array([[0.1, 0.0], [3.0, 0.0], [3.0, 0.0]])])
    v = o.verdict(_prob(o, 1, T, [[0.1, 0, 0, 0]], [[3, 0, 0, 0]], obs), w, st)
    assert v["collision_free"] is False
    r, _ = o.reward(_prob(o, 1, T, [[0.1, 0, 0, 0]], [[3, 0, 0, 0]], obs), w, st)
    # t = 1, 2 at the goal: r_goal = 1, no penalty (t = 0 is not rewarded)
    assert abs(r - 1.0) < 1e-12


def test_3d_uses_z_and_2d_ignores_it(oracle_lib):
    """In 3D the obstacle's z counts: a robot at the obstacle's (x, y) but
    1 m below is clear.  In 2D the same obstacle row (z = 1) covers the
    robot, because only (x, y) are positions."""
    o = oracle_lib
    T, w = 1, 1.0
    obs = [[0.0, 0.0, 1.0, 0.3]]
    st3 = np.zeros((2, 1, 6))
    st3[:, 0, :3] = [[0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]
    pr3 = _prob(o, 1, T, [[0, 0, 0, 0, 0, 0]], [[0, 0, 0, 0, 0, 0]], obs, dyn=o.HOLO3D)
    r3, _ = o.reward(pr3, w, st3)
    assert abs(r3 - 1.0) < 1e-12
    st2 = _states([np.array([[0.0, 0.0], [0.0, 0.0]])])
    r2, _ = o.reward(_prob(o, 1, T, [[0, 0, 0, 0]], [[0, 0, 0, 0]], obs), w, st2)
    assert abs(r2 - (1.0 - w)) < 1e-12


def test_fragile_counts_obstacle_indicators(oracle_lib):
    """A state 1e-5 m from the obstacle's penalty threshold is one fragile
    indicator; moving it 1 mm away makes it robust."""
    o = oracle_lib
    T = 1
    obs = [[0.0, 0.0, 0.0, 0.3]]
    for d, want in ((0.55 + 1e-5, 1), (0.551, 0)):
        st = _states([np.array([[3.0, 0.0], [d, 0.0]])])
        pr = _prob(o, 1, T, [[3, 0, 0, 0]], [[d, 0, 0, 0]], obs)
        assert o.fragile(pr, st, 1e-4) == want


def test_sample_fitness_sees_obstacles(oracle_lib):
    """Through the whole sample path (noise, rollout, Eq. (3)): an obstacle
    that covers the entire reachable region costs every sample exactly w."""
    o = oracle_lib
    T, N = 10, 8
    pr0 = _prob(o, 2, T, [[0, 0, 0, 0], [1, 0, 0, 0]], [[1, 1, 0, 0], [0, 1, 0, 0]], None)
    pr1 = _prob(o, 2, T, [[0, 0, 0, 0], [1, 0, 0, 0]], [[1, 1, 0, 0], [0, 1, 0, 0]], [[0.5, 0.5, 0.0, 100.0]])
    pp = o.Params(N=N, K=10, lam=0.1, w_safe=4.0, beta0=1e-4, beta1=1e-2, seed=3, tag=0)
    u = np.zeros((T, 2, 2))
    du = np.zeros((T, 2, 2))
    js = np.arange(N)
    f0, _ = o.sample_fitness(pr0, pp, 0, 9, u, du, js)
    f1, _ = o.sample_fitness(pr1, pp, 0, 9, u, du, js)
    assert np.allclose(f0 - f1, 4.0, atol=1e-12)
