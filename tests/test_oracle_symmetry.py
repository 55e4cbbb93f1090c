"""Symmetry pins of the oracle's rollout and Eq. (3)-(5) reward.

Each property holds exactly in real arithmetic and catches a class of
index mistakes that closed-form cases can miss: a robot index crossed
between the pair loop and the goal term breaks permutation invariance; a
coordinate mixed up in the dynamics or in a distance breaks translation or
rotation invariance.
- Translation: moving every start, goal and obstacle by one vector moves
  every trajectory by it (the dynamics do not depend on absolute position),
  so every distance, the reward and the verdict are unchanged.
- Permutation: relabelling the robots (starts, goals, controls together)
  leaves the team reward and the verdict unchanged.
- Rotation (unicycle): the control box acts on (v, omega), so rotating
  starts, goals, obstacles and initial headings about the origin rotates the
  trajectories; distances, reward and verdict are unchanged.
"""
import math

import numpy as np
import pytest

DYN = {"holo2d": (0, 4, 2, 2), "holo3d": (1, 6, 3, 3), "unicycle": (2, 3, 2, 2), "diffdrive4": (3, 4, 2, 2)}


def _problem(o, dyn, start, goal, obstacles, T):
    d, d_x, d_u, d_p = DYN[dyn]
    lo, hi = ((0.0, -1.0), (1.0, 1.0)) if dyn == "unicycle" else ((-1.0,) * d_u, (1.0,) * d_u)
    return o.Problem(n=start.shape[0], T=T, dyn=d, integ=o.RK4, dt=0.1, radius=0.2, start=start, goal=goal,
                     u_lo=lo, u_hi=hi, v_max=1.5 if dyn in ("holo2d", "holo3d", "diffdrive4") else 0.0,
                     obstacles=obstacles)


def _instance(rng, dyn, n, m):
    d, d_x, d_u, d_p = DYN[dyn]
    start = np.zeros((n, d_x))
    goal = np.zeros((n, d_x))
    start[:, :d_p] = rng.uniform(-2, 2, (n, d_p))
    goal[:, :d_p] = rng.uniform(-2, 2, (n, d_p))
    if dyn in ("unicycle", "diffdrive4"):
        start[:, 2] = rng.uniform(-math.pi, math.pi, n)
    obs = np.zeros((m, 4))
    obs[:, :d_p] = rng.uniform(-1.5, 1.5, (m, d_p))
    obs[:, 3] = rng.uniform(0.1, 0.4, m)
    return start, goal, obs


def _score(o, pr, u):
    st = o.rollout(pr, u)
    r, _ = o.reward(pr, 3.0, st)
    return r, o.verdict(pr, 3.0, st), st


@pytest.mark.parametrize("dyn", ["holo2d", "holo3d", "unicycle", "diffdrive4"])
def test_translation_invariance(oracle_lib, dyn):
    o = oracle_lib
    rng = np.random.default_rng(1)
    d, d_x, d_u, d_p = DYN[dyn]
    T, n = 25, 5
    for trial in range(4):
        start, goal, obs = _instance(rng, dyn, n, 3)
        u = rng.uniform(-1.2, 1.2, (T, n, d_u))
        shift = rng.uniform(-3, 3, d_p)
        s2, g2, o2 = start.copy(), goal.copy(), obs.copy()
        s2[:, :d_p] += shift
        g2[:, :d_p] += shift
        o2[:, :d_p] += shift
        r1, v1, st1 = _score(o, _problem(o, dyn, start, goal, obs, T), u)
        r2, v2, st2 = _score(o, _problem(o, dyn, s2, g2, o2, T), u)
        assert np.allclose(st2[:, :, :d_p] - shift, st1[:, :, :d_p], atol=1e-9)
        assert abs(r1 - r2) < 1e-9
        assert v1["collision_free"] == v2["collision_free"] and v1["goal_reached"] == v2["goal_reached"]
        assert abs(v1["min_pair_dist"] - v2["min_pair_dist"]) < 1e-9


@pytest.mark.parametrize("dyn", ["holo2d", "holo3d", "unicycle", "diffdrive4"])
def test_robot_permutation_invariance(oracle_lib, dyn):
    o = oracle_lib
    rng = np.random.default_rng(2)
    d, d_x, d_u, d_p = DYN[dyn]
    T, n = 20, 6
    for trial in range(4):
        start, goal, obs = _instance(rng, dyn, n, 2)
        # a crowded start so that some pairs collide and the pair loop matters
        start[:, :d_p] *= 0.3
        u = rng.uniform(-1.2, 1.2, (T, n, d_u))
        perm = rng.permutation(n)
        r1, v1, _ = _score(o, _problem(o, dyn, start, goal, obs, T), u)
        r2, v2, _ = _score(o, _problem(o, dyn, start[perm], goal[perm], obs, T), u[:, perm])
        assert abs(r1 - r2) < 1e-12
        assert v1 == pytest.approx(v2, abs=1e-12)


def test_unicycle_rotation_invariance(oracle_lib):
    o = oracle_lib
    rng = np.random.default_rng(3)
    T, n = 30, 4
    for trial in range(4):
        start, goal, obs = _instance(rng, "unicycle", n, 3)
        start[:, :2] *= 0.5
        u = np.stack([rng.uniform(0, 1, (T, n)), rng.uniform(-1, 1, (T, n))], axis=2)
        a = rng.uniform(-math.pi, math.pi)
        R = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
        s2, g2, o2 = start.copy(), goal.copy(), obs.copy()
        s2[:, :2] = start[:, :2] @ R.T
        s2[:, 2] = start[:, 2] + a
        g2[:, :2] = goal[:, :2] @ R.T
        o2[:, :2] = obs[:, :2] @ R.T
        r1, v1, st1 = _score(o, _problem(o, "unicycle", start, goal, obs, T), u)
        r2, v2, st2 = _score(o, _problem(o, "unicycle", s2, g2, o2, T), u)
        assert np.allclose(st2[:, :, :2], st1[:, :, :2] @ R.T, atol=1e-9)
        assert abs(r1 - r2) < 1e-9
        assert abs(v1["min_pair_dist"] - v2["min_pair_dist"]) < 1e-9
