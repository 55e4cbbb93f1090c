"""FP64 oracle of the learned warm start (numpy) -- TEST INFRASTRUCTURE ONLY.

The set-MLP the CUDA library trains (see include/d4orm.h, learned warm
start), written out in plain FP64 numpy: features of a team, forward pass,
masked mean squared error, its gradient by hand-written backpropagation, and
one AdamW step (Loshchilov & Hutter, "Decoupled Weight Decay
Regularization", 2019).  Pinned by central finite differences
(tests/test_oracle_setmlp.py).  The method of the paper has no learning
component; this is the oracle of the library's own addition.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 16


def layout(width: int, D: int, n_feat: int = N_FEAT):
    """[(out, in, w_offset, b_offset)] of the six layers and the total count.
    Flat order: W1, b1, W2, b2, ..., W6, b6; W row-major [out][in]."""
    shapes = [(width, n_feat), (width, width), (width, width), (width, 2 * width), (width, width), (D, width)]
    out, off = [], 0
    for o, i in shapes:
        w = off
        off += o * i
        b = off
        off += o
        out.append((o, i, w, b))
    return out, off


def unpack(params: np.ndarray, width: int, D: int):
    lay, _ = layout(width, D)
    return [(params[w:w + o * i].reshape(o, i), params[b:b + o]) for (o, i, w, b) in lay]


def features(start: np.ndarray, goal: np.ndarray, d_p: int, n_max: int, pos_scale: float):
    """x [n_max][16]: start/s, goal/s, (goal - start)/s (3 slots each, unused
    slots 0), |goal - start|/s, 1; mask [n_max]: 1 for real robots."""
    n = start.shape[0]
    x = np.zeros((n_max, N_FEAT))
    m = np.zeros(n_max)
    for k in range(n):
        s = start[k, :d_p] / pos_scale
        g = goal[k, :d_p] / pos_scale
        x[k, 0:d_p] = s
        x[k, 3:3 + d_p] = g
        x[k, 6:6 + d_p] = g - s
        x[k, 9] = np.sqrt(np.sum((g - s) ** 2))
        x[k, 10] = 1.0
        m[k] = 1.0
    return x, m


def forward(params, x, mask, width: int, D: int):
    """Y [B][n_max][D] and the cached activations."""
    (W1, b1), (W2, b2), (W3, b3), (W4, b4), (W5, b5), (W6, b6) = unpack(params, width, D)
    relu = lambda z: np.maximum(z, 0.0)  # noqa: E731
    H1 = relu(x @ W1.T + b1)
    H2 = relu(H1 @ W2.T + b2)
    H3 = relu(H2 @ W3.T + b3)
    cnt = np.maximum(mask.sum(axis=1), 1.0)                       # [B]
    P = (mask[:, :, None] * H3).sum(axis=1) / cnt[:, None]       # [B][W]
    C = np.concatenate([H3, np.broadcast_to(P[:, None, :], H3.shape)], axis=2)
    H4 = relu(C @ W4.T + b4)
    H5 = relu(H4 @ W5.T + b5)
    Y = H5 @ W6.T + b6
    return Y, dict(x=x, H1=H1, H2=H2, H3=H3, C=C, H4=H4, H5=H5, cnt=cnt)


def loss_and_grad(params, x, mask, target, width: int, D: int):
    """Masked MSE  L = sum_k mask (Y - T)^2 / (sum mask * D)  and dL/dparams."""
    Y, c = forward(params, x, mask, width, D)
    Ws = unpack(params, width, D)
    denom = max(mask.sum(), 1.0) * D
    E = (Y - target) * mask[:, :, None]
    loss = float((E ** 2).sum() / denom)
    dY = 2.0 * E / denom
    grads = [None] * 6

    def lin_back(dZ, A, l):
        W, _ = Ws[l]
        dW = np.einsum("bko,bki->oi", dZ, A)
        db = dZ.sum(axis=(0, 1))
        grads[l] = (dW, db)
        return dZ @ W

    dH5 = lin_back(dY, c["H5"], 5) * (c["H5"] > 0)
    dH4 = lin_back(dH5, c["H4"], 4) * (c["H4"] > 0)
    dC = lin_back(dH4, c["C"], 3)
    Wd = c["H3"].shape[2]
    dP = dC[:, :, Wd:].sum(axis=1)                                  # [B][W]
    dH3 = (dC[:, :, :Wd] + mask[:, :, None] * (dP / c["cnt"][:, None])[:, None, :]) * (c["H3"] > 0)
    dH2 = lin_back(dH3, c["H2"], 2) * (c["H2"] > 0)
    dH1 = lin_back(dH2, c["H1"], 1) * (c["H1"] > 0)
    lin_back(dH1, c["x"], 0)
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return loss, flat


def adamw_step(p, g, m, v, t: int, lr: float, b1: float, b2: float, eps: float, wd: float):
    """One AdamW step (decoupled decay, bias-corrected moments); returns p, m, v."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    p = p - lr * (mh / (np.sqrt(vh) + eps) + wd * p)
    return p, m, v
