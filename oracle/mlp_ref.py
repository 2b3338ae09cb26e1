"""Double-precision reference of the proposal network (the learned subQUBO
selection added to IC-D2S; readings S21, S22) and of its training step.

TEST INFRASTRUCTURE ONLY: used by the tests; the product library never
imports it.  Plain numpy; a matrix product is the only library step.

Network: 6 features -> 64 (ReLU) -> 64 (ReLU) -> 1 score, parameters flat in
the order W1[64][6], b1[64], W2[64][64], b2[64], w3[64], b3 (4673 values).
The weights the network computes with are the BF16 roundings of float32
master weights; this reference evaluates those BF16 values in double.

Loss: binary cross-entropy on the score as a logit, the positive term
weighted by ``pos_weight``, averaged over the rows:
    l(s, y) = pos_weight * y * softplus(-s) + (1 - y) * softplus(s).
Optimiser: Adam (Kingma & Ba, ICLR'15) on the float32 master weights.
"""
from __future__ import annotations

import numpy as np

NPAR = 4673
H = 64
OFF_W1, OFF_B1, OFF_W2, OFF_B2, OFF_W3, OFF_B3 = 0, 384, 448, 4544, 4608, 4672


def unpack(W):
    W = np.asarray(W, dtype=np.float64)
    assert W.shape == (NPAR,)
    return (W[OFF_W1:OFF_B1].reshape(H, 6), W[OFF_B1:OFF_W2], W[OFF_W2:OFF_B2].reshape(H, H),
            W[OFF_B2:OFF_W3], W[OFF_W3:OFF_B3], W[OFF_B3])


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def bf16_round(a):
    """Round float32 values to the nearest BF16 value (ties to even), returned
    as float32: keep the top 16 bits after adding 0x7FFF plus the lowest kept bit."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).reshape(a.shape)


def forward(W, F):
    """Scores (double) of the rows F [rows][6] and the activations."""
    W1, b1, W2, b2, w3, b3 = unpack(W)
    F = np.asarray(F, dtype=np.float64).reshape(-1, 6)
    a1 = F @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    s = h2 @ w3 + b3
    return s, (F, a1, h1, a2, h2)


def softplus(v):
    return np.maximum(v, 0.0) + np.log1p(np.exp(-np.abs(v)))


def sigmoid(v):
    return 0.5 * (1.0 + np.tanh(0.5 * v))


def loss(W, F, y, pos_weight=1.0):
    s, _ = forward(W, F)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    return float(np.mean(pos_weight * y * softplus(-s) + (1.0 - y) * softplus(s)))


def loss_and_grad(W, F, y, pos_weight=1.0):
    """Mean loss and its gradient (double, flat NPAR) by backpropagation."""
    W1, b1, W2, b2, w3, b3 = unpack(W)
    s, (F, a1, h1, a2, h2) = forward(W, F)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    B = s.shape[0]
    L = float(np.mean(pos_weight * y * softplus(-s) + (1.0 - y) * softplus(s)))
    sg = sigmoid(s)
    ds = (pos_weight * y * (sg - 1.0) + (1.0 - y) * sg) / B       # dL/ds
    gw3 = h2.T @ ds
    gb3 = ds.sum()
    d2 = np.outer(ds, w3) * (a2 > 0)                                # dL/da2
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (a1 > 0)                                       # dL/da1
    gW1 = d1.T @ F
    gb1 = d1.sum(axis=0)
    return L, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def adam(master, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1), in double; returns new (master, m, v)."""
    g = np.asarray(grad, dtype=np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return np.asarray(master, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v
