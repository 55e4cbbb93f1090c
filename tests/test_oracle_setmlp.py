"""Pins for the FP64 set-MLP oracle (oracle/setmlp.py): its hand-written
gradient against central finite differences, the masked pooling's
invariances, and the first AdamW step's closed form."""
import numpy as np
import pytest

from oracle import setmlp


def _tiny(seed=0, B=3, n_max=4, width=16, D=6):
    rng = np.random.default_rng(seed)
    _, count = setmlp.layout(width, D)
    p = rng.normal(scale=0.4, size=count)
    x = rng.normal(size=(B, n_max, setmlp.N_FEAT))
    mask = np.ones((B, n_max))
    mask[1, 3] = 0.0
    mask[2, 2:] = 0.0
    x *= mask[:, :, None]
    t = rng.normal(size=(B, n_max, D))
    return p, x, mask, t, width, D


def test_gradient_matches_finite_differences():
    p, x, mask, t, W, D = _tiny()
    loss, g = setmlp.loss_and_grad(p, x, mask, t, W, D)
    rng = np.random.default_rng(1)
    idx = rng.choice(len(p), size=60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (setmlp.loss_and_grad(pp, x, mask, t, W, D)[0] - setmlp.loss_and_grad(pm, x, mask, t, W, D)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, fd, g[i])


def test_masked_robots_do_not_matter():
    """Changing a padded robot's features changes neither the real robots'
    outputs nor the loss."""
    p, x, mask, t, W, D = _tiny(seed=2)
    y0, _ = setmlp.forward(p, x, mask, W, D)
    x2 = x.copy()
    x2[2, 3] = 7.0          # padded robot of team 2
    t2 = t.copy()
    t2[2, 3] = -3.0
    y1, _ = setmlp.forward(p, x2, mask, W, D)
    np.testing.assert_allclose(y1[2, :2], y0[2, :2], rtol=0, atol=1e-14)
    l0, _ = setmlp.loss_and_grad(p, x, mask, t, W, D)
    l1, _ = setmlp.loss_and_grad(p, x2, mask, t2, W, D)
    assert abs(l0 - l1) < 1e-14


def test_team_order_equivariance():
    """Permuting a team's robots permutes its outputs (set model)."""
    p, x, mask, t, W, D = _tiny(seed=3)
    perm = np.array([2, 0, 3, 1])
    y0, _ = setmlp.forward(p, x, mask, W, D)
    y1, _ = setmlp.forward(p, x[:, perm], mask[:, perm], W, D)
    np.testing.assert_allclose(y1[0], y0[0][perm], atol=1e-12)


def test_adamw_first_step_closed_form():
    """t = 1: m_hat = g, v_hat = g^2, so p <- p - lr (g / (|g| + eps) + wd p)."""
    rng = np.random.default_rng(4)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m, v = setmlp.adamw_step(p, g, np.zeros(50), np.zeros(50), 1, 1e-3, 0.9, 0.999, 1e-8, 0.01)
    np.testing.assert_allclose(p1, p - 1e-3 * (g / (np.abs(g) + 1e-8) + 0.01 * p), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_features_layout():
    start = np.array([[1.0, -2.0, 0.0, 0.0], [0.5, 0.5, 0.0, 0.0]])
    goal = np.array([[4.0, 2.0, 0.0, 0.0], [0.5, 0.5, 0.0, 0.0]])
    x, m = setmlp.features(start, goal, 2, 3, 5.0)
    np.testing.assert_allclose(x[0, :11], [0.2, -0.4, 0, 0.8, 0.4, 0, 0.6, 0.8, 0, 1.0, 1.0])
    assert x[1, 9] == 0.0 and x[1, 10] == 1.0
    np.testing.assert_array_equal(m, [1, 1, 0])
    assert not x[2].any()
