"""GPU parity of the learned warm start's kernels (BF16 tensor-core GEMMs,
pooling, loss, AdamW) against the FP64 oracle (oracle/setmlp.py).

The GPU rounds weights and activations to BF16 (8 significant bits, unit
roundoff 2^-9) and accumulates in FP32.  Forward outputs are compared in
relative Frobenius norm at 3e-2 (six layers of BF16 operands); gradients
per tensor at 8e-2 -- the first layer's weight gradient sits behind eleven
BF16 GEMMs, each adding ~2^-9 relative per operand -- together with a
direction check (cosine >= 0.995) that a wrong index or transposition would
fail.  The oracle is fed the GPU's own BF16-rounded weights and inputs.  AdamW is compared elementwise (FP32 vs FP64 arithmetic) on the
GPU's own gradient.
"""
import math

import numpy as np
import pytest

import scenarios
from helpers import round_instance
from oracle import setmlp

pytestmark = pytest.mark.gpu


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


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _net(g, width=64, T=10, d_u=2, n_max=6, B=5, seed=0):
    desc = g.WarmStartDesc(n_max=n_max, T=T, d_u=d_u, width=width, max_batch=8, seed=seed, lr=3e-3,
                           weight_decay=1e-2)
    ws = g.d4orm_warmstart_create(desc)
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(B, n_max, 16)).astype(np.float32)
    mask = np.ones((B, n_max), dtype=np.float32)
    mask[0, 4:] = 0
    mask[3, 2:] = 0
    x *= mask[:, :, None]
    y = rng.uniform(-1, 1, size=(B, n_max, T * d_u)).astype(np.float32)
    return ws, desc, x, mask, y


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_forward_matches_oracle(torch, g):
    ws, desc, x, mask, _ = _net(g)
    D = desc.T * desc.d_u
    p = g.d4orm_warmstart_get_params(ws)
    y_dev = torch.zeros((x.shape[0], desc.n_max, D), device="cuda")
    g.d4orm_warmstart_forward(ws, torch.as_tensor(x, device="cuda"), torch.as_tensor(mask, device="cuda"),
                              x.shape[0], y_dev)
    torch.cuda.synchronize()
    y_o, _ = setmlp.forward(bf16(p), bf16(x), mask.astype(np.float64), desc.width, D)
    real = mask > 0
    assert _rel(y_dev.cpu().numpy()[real], y_o[real]) <= 3e-2
    g.d4orm_warmstart_destroy(ws)


def test_gradients_match_oracle(torch, g):
    ws, desc, x, mask, y = _net(g, seed=1)
    D = desc.T * desc.d_u
    p = g.d4orm_warmstart_get_params(ws)
    grad = torch.zeros(len(p), device="cuda")
    loss = g.d4orm_warmstart_loss_grad(ws, torch.as_tensor(x, device="cuda"), torch.as_tensor(mask, device="cuda"),
                                       torch.as_tensor(y, device="cuda"), x.shape[0], grad_dev=grad)
    loss_o, grad_o = setmlp.loss_and_grad(bf16(p), bf16(x), mask.astype(np.float64), y.astype(np.float64),
                                          desc.width, D)
    assert abs(loss - loss_o) <= 2e-2 * loss_o
    gg = grad.cpu().numpy()
    lay, _ = setmlp.layout(desc.width, D)
    def cos(a, b):
        return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))

    for (o, i, w, b) in lay:
        for lo, hi, what in ((w, w + o * i, "weight"), (b, b + o, "bias")):
            assert _rel(gg[lo:hi], grad_o[lo:hi]) <= 8e-2, (o, i, what)
            assert cos(gg[lo:hi].astype(np.float64), grad_o[lo:hi]) >= 0.995, (o, i, what)
    g.d4orm_warmstart_destroy(ws)


def test_adamw_step_matches_oracle(torch, g):
    ws, desc, x, mask, y = _net(g, seed=2)
    p0 = g.d4orm_warmstart_get_params(ws).astype(np.float64)
    xd, md, yd = (torch.as_tensor(a, device="cuda") for a in (x, mask, y))
    grad = torch.zeros(len(p0), device="cuda")
    g.d4orm_warmstart_loss_grad(ws, xd, md, yd, x.shape[0], grad_dev=grad)
    g.d4orm_warmstart_train_step(ws, xd, md, yd, x.shape[0])
    p1 = g.d4orm_warmstart_get_params(ws).astype(np.float64)
    gg = grad.cpu().numpy().astype(np.float64)
    want, _, _ = setmlp.adamw_step(p0, gg, np.zeros_like(p0), np.zeros_like(p0), 1, desc.lr, desc.beta1,
                                   desc.beta2, desc.eps, desc.weight_decay)
    assert np.abs(p1 - want).max() <= 1e-6 + 1e-5 * desc.lr
    g.d4orm_warmstart_destroy(ws)


def test_training_reduces_loss(torch, g):
    """A learnable target (a fixed random linear map of the features, kept
    in [-1, 1]) is fitted: the loss falls by 5x within 300 AdamW steps."""
    ws, desc, x, mask, _ = _net(g, width=64, seed=3, B=8)
    rng = np.random.default_rng(7)
    A = rng.normal(scale=0.3, size=(16, desc.T * desc.d_u))
    X = rng.uniform(-1, 1, size=(64, desc.n_max, 16)).astype(np.float32)
    M = np.ones((64, desc.n_max), dtype=np.float32)
    Y = np.tanh(X @ A).astype(np.float32)
    Xd, Md, Yd = (torch.as_tensor(a, device="cuda") for a in (X, M, Y))
    idx = torch.zeros(8, dtype=torch.int32, device="cuda")
    losses = []
    for s in range(300):
        idx.copy_(torch.as_tensor(rng.integers(0, 64, size=8), dtype=torch.int32))
        losses.append(g.d4orm_warmstart_train_step(ws, Xd, Md, Yd, 8, idx_dev=idx))
    assert np.mean(losses[-20:]) < 0.2 * np.mean(losses[:20])
    g.d4orm_warmstart_destroy(ws)


def test_predict_seeds_scaled_plan(torch, g):
    inst = round_instance(scenarios.box_instance(np.random.default_rng(3), scenarios.HOLO2D, 6, 10, 64))
    prob = g.Problem(inst)
    ws, desc, _, _, _ = _net(g, width=64, T=10, d_u=2, n_max=8, seed=4)
    params = g.Params(n_samples=64, n_steps=100)
    seed = torch.zeros((10, 6, 2), device="cuda")
    g.d4orm_warmstart_predict(ws, prob.handle, params, 30, seed)
    x, m = g.d4orm_warmstart_features(prob.handle, 8, desc.pos_scale)
    y = torch.zeros((1, 8, 20), device="cuda")
    g.d4orm_warmstart_forward(ws, torch.as_tensor(x[None], device="cuda"), torch.as_tensor(m[None], device="cuda"),
                              1, y)
    torch.cuda.synchronize()
    _, ab = __import__("oracle").schedule(100, 1e-4, 1e-2)
    want = math.sqrt(ab[30]) * y.cpu().numpy()[0, :6].reshape(6, 10, 2).transpose(1, 0, 2)
    np.testing.assert_allclose(seed.cpu().numpy(), want, rtol=2e-6, atol=1e-7)
    g.d4orm_warmstart_destroy(ws)


def test_trained_network_beats_untrained_and_zero_seed(torch, g):
    """Ablation: the shipped network (trained on the method's own plans)
    against the same architecture untrained and against no seed at all.
    Each held-out team runs one iteration from step 30 of 100 (the warm
    start's budget); the trained seed ends with a clearly higher Eq. (3)
    reward and the robots closer to their goals."""
    import os
    import scenarios
    from paper_2503_12204_gb300 import warmstart as W
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    desc, trained, _ = W.load_weights(os.path.join(root, "paper_2503_12204_gb300", "weights", "setmlp_holo2d_T80.bin"))
    desc.max_batch = 1
    nets = {}
    for name in ("trained", "untrained"):
        ws = g.d4orm_warmstart_create(desc)
        if name == "trained":
            g.d4orm_warmstart_set_params(ws, trained)
        nets[name] = ws
    teams = scenarios.warmstart_set(24, seed=4)
    params = g.Params(n_samples=1024, n_steps=100, seed=4)
    reward = {k: [] for k in ("trained", "untrained", "zero")}
    for b, inst in enumerate(teams):
        inst = round_instance(inst)
        prob = g.Problem(inst)
        p = g.Params(**{**params.__dict__, "instance_tag": b})
        u = torch.zeros((inst.T, inst.n, 2), device="cuda")
        for name in reward:
            seed = torch.zeros_like(u)
            if name != "zero":
                g.d4orm_warmstart_predict(nets[name], prob.handle, p, 30, seed)
            r = g.d4orm_solve(prob.handle, p, g.Budget(max_iters=1, start_step=30), u, du_init_dev=seed)
            reward[name].append(r["verdict"]["reward"])
    for ws in nets.values():
        g.d4orm_warmstart_destroy(ws)
    mean = {k: float(np.mean(v)) for k, v in reward.items()}
    assert mean["trained"] > mean["untrained"] + 0.05, mean
    assert mean["trained"] > mean["zero"] + 0.05, mean
    wins = sum(t > z for t, z in zip(reward["trained"], reward["zero"]))
    assert wins >= 20, (wins, mean)
