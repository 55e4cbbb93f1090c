"""Pins for the oracle's dynamics and rollout (Sec. III Eq. (1), Sec. V).

Closed forms of the integrators on constant controls:
* double integrator, forward Euler: p_t = p0 + v0 t dt + a dt^2 t (t-1) / 2;
* double integrator, RK4 (exact for a constant acceleration):
  p_t = p0 + v0 t dt + a (t dt)^2 / 2;
* the per-axis speed bound applied after each step (accelerate, then each
  later step adds v_max dt + a dt^2 / 2);
* unicycle with omega = 0: a straight line; with constant omega: the exact
  circular arc (RK4 to O(dt^4)), and forward Euler's geometric sum;
* differential drive (4-state) with omega = 0: a straight line with the
  speed ramp.
"""
import math

import numpy as np
import pytest


def _prob(o, dyn, integ, n=1, T=40, dt=0.1, v_max=0.0, start=None, lo=None, hi=None):
    d_x, d_u, d_p = o.DIMS[dyn]
    if start is None:
        start = np.zeros((n, d_x))
    lo = lo if lo is not None else tuple([-10.0] * d_u)
    hi = hi if hi is not None else tuple([10.0] * d_u)
    return o.Problem(n=n, T=T, dyn=dyn, integ=integ, dt=dt, radius=0.2, start=np.array(start, float),
                     goal=np.zeros((n, d_x)), u_lo=lo, u_hi=hi, v_max=v_max)


@pytest.mark.parametrize("dyn", [0, 1])
def test_double_integrator_euler_closed_form(oracle_lib, dyn):
    o = oracle_lib
    d_x, d_u, d_p = o.DIMS[dyn]
    start = np.zeros((1, d_x))
    p0 = np.array([0.3, -1.2, 0.7][:d_p])
    v0 = np.array([0.05, -0.02, 0.01][:d_p])
    a = np.array([0.011, -0.007, 0.003][:d_p])
    start[0, :d_p] = p0
    start[0, d_p:] = v0
    T, dt = 40, 0.1
    pr = _prob(o, dyn, o.EULER, T=T, dt=dt, start=start)
    st = o.rollout(pr, np.tile(a, (T, 1, 1)))
    for t in range(T + 1):
        want_p = p0 + v0 * t * dt + a * dt * dt * t * (t - 1) / 2.0
        want_v = v0 + a * t * dt
        np.testing.assert_allclose(st[t, 0, :d_p], want_p, atol=1e-13)
        np.testing.assert_allclose(st[t, 0, d_p:], want_v, atol=1e-13)


@pytest.mark.parametrize("dyn", [0, 1])
def test_double_integrator_rk4_closed_form(oracle_lib, dyn):
    o = oracle_lib
    d_x, d_u, d_p = o.DIMS[dyn]
    start = np.zeros((1, d_x))
    p0 = np.array([-2.0, 1.0, 0.5][:d_p])
    v0 = np.array([0.1, 0.0, -0.3][:d_p])
    a = np.array([0.02, -0.01, 0.015][:d_p])
    start[0, :d_p] = p0
    start[0, d_p:] = v0
    T, dt = 60, 0.1
    pr = _prob(o, dyn, o.RK4, T=T, dt=dt, start=start)
    st = o.rollout(pr, np.tile(a, (T, 1, 1)))
    for t in range(T + 1):
        want_p = p0 + v0 * t * dt + 0.5 * a * (t * dt) ** 2
        np.testing.assert_allclose(st[t, 0, :d_p], want_p, atol=1e-12)
        np.testing.assert_allclose(st[t, 0, d_p:], v0 + a * t * dt, atol=1e-12)


def test_speed_bound_after_step(oracle_lib):
    """a = 1, dt = 0.1, v_max = 1 from rest (RK4): the speed reaches 1 at
    t = 10 (p = 0.5); afterwards each step adds v_max dt + a dt^2 / 2 = 0.105."""
    o = oracle_lib
    T = 30
    pr = _prob(o, 0, o.RK4, T=T, v_max=1.0)
    st = o.rollout(pr, np.tile([1.0, 0.0], (T, 1, 1)))
    for t in range(T + 1):
        want = 0.005 * t * t if t <= 10 else 0.5 + 0.105 * (t - 10)
        assert abs(st[t, 0, 0] - want) < 1e-12
        assert abs(st[t, 0, 2] - min(0.1 * t, 1.0)) < 1e-12
        assert st[t, 0, 1] == 0.0


def test_control_box_clips(oracle_lib):
    o = oracle_lib
    T = 20
    pr = _prob(o, 0, o.RK4, T=T, lo=(-1.0, -0.5), hi=(1.0, 0.5))
    big = o.rollout(pr, np.tile([7.0, -9.0], (T, 1, 1)))
    edge = o.rollout(pr, np.tile([1.0, -0.5], (T, 1, 1)))
    np.testing.assert_array_equal(big, edge)


@pytest.mark.parametrize("integ", [0, 1])
def test_unicycle_straight_line(oracle_lib, integ):
    o = oracle_lib
    th = 0.7
    T, dt, v = 50, 0.1, 0.8
    pr = _prob(o, o.UNICYCLE, integ, T=T, dt=dt, start=[[1.0, -2.0, th]])
    st = o.rollout(pr, np.tile([v, 0.0], (T, 1, 1)))
    for t in range(T + 1):
        assert abs(st[t, 0, 0] - (1.0 + v * t * dt * math.cos(th))) < 1e-12
        assert abs(st[t, 0, 1] - (-2.0 + v * t * dt * math.sin(th))) < 1e-12
        assert abs(st[t, 0, 2] - th) < 1e-15


def test_unicycle_arc_rk4(oracle_lib):
    o = oracle_lib
    th0, v, w = 0.3, 0.9, 0.6
    T, dt = 100, 0.1
    pr = _prob(o, o.UNICYCLE, o.RK4, T=T, dt=dt, start=[[0.5, 0.25, th0]])
    st = o.rollout(pr, np.tile([v, w], (T, 1, 1)))
    for t in range(T + 1):
        tt = t * dt
        x = 0.5 + v / w * (math.sin(th0 + w * tt) - math.sin(th0))
        y = 0.25 + v / w * (math.cos(th0) - math.cos(th0 + w * tt))
        assert abs(st[t, 0, 0] - x) < 1e-6 and abs(st[t, 0, 1] - y) < 1e-6
        assert abs(st[t, 0, 2] - (th0 + w * tt)) < 1e-12


def test_unicycle_euler_geometric_sum(oracle_lib):
    o = oracle_lib
    th0, v, w = -0.4, 0.7, 0.9
    T, dt = 60, 0.1
    pr = _prob(o, o.UNICYCLE, o.EULER, T=T, dt=dt, start=[[0.0, 0.0, th0]])
    st = o.rollout(pr, np.tile([v, w], (T, 1, 1)))
    q = complex(math.cos(w * dt), math.sin(w * dt))
    for t in range(T + 1):
        s = complex(math.cos(th0), math.sin(th0)) * (1 - q ** t) / (1 - q) * v * dt
        assert abs(st[t, 0, 0] - s.real) < 1e-12 and abs(st[t, 0, 1] - s.imag) < 1e-12


def test_diffdrive4_straight_ramp(oracle_lib):
    o = oracle_lib
    th, v0, a = 1.1, 0.2, 0.05
    T, dt = 40, 0.1
    pr = _prob(o, o.DIFFDRIVE4, o.RK4, T=T, dt=dt, start=[[0.0, 1.0, th, v0]])
    st = o.rollout(pr, np.tile([0.0, a], (T, 1, 1)))
    for t in range(T + 1):
        s = v0 * t * dt + 0.5 * a * (t * dt) ** 2
        assert abs(st[t, 0, 0] - s * math.cos(th)) < 1e-12
        assert abs(st[t, 0, 1] - (1.0 + s * math.sin(th))) < 1e-12
        assert abs(st[t, 0, 3] - (v0 + a * t * dt)) < 1e-12


def test_dynamics_fields(oracle_lib):
    """The vector fields of Sec. V at one point each."""
    o = oracle_lib
    np.testing.assert_array_equal(o.dynamics(o.HOLO2D, [1, 2, 3, 4], [5, 6]), [3, 4, 5, 6])
    np.testing.assert_array_equal(o.dynamics(o.HOLO3D, [1, 2, 3, 4, 5, 6], [7, 8, 9]), [4, 5, 6, 7, 8, 9])
    f = o.dynamics(o.UNICYCLE, [1, 2, math.pi / 2], [2.0, 0.5])
    np.testing.assert_allclose(f, [0.0, 2.0, 0.5], atol=1e-15)
    f = o.dynamics(o.DIFFDRIVE4, [1, 2, math.pi, 3.0], [0.25, -1.0])
    np.testing.assert_allclose(f, [-3.0, 0.0, 0.25, -1.0], atol=1e-14)


def test_variable_count_matches_paper(oracle_lib):
    """Sec. V-A: 16 2D-holonomic robots over H = 100 have 3200 control
    variables, d_u x H x n; the control layout has exactly that many."""
    o = oracle_lib
    pr = _prob(o, o.HOLO2D, o.RK4, n=16, T=100)
    assert pr.n_ctrl == 3200
