"""FP64 reference of the warm-start MLP — TEST INFRASTRUCTURE.

Plain NumPy forward and backward of h_{l+1} = relu(h_l W_l + b_l) (no ReLU
after the last layer), masked softmax over the first nact entries, weighted
cross entropy averaged over the batch. With bf16_operands=True every product
rounds both operands to BF16 (round to nearest even) first, as the GPU
kernels do, so GPU gradients can be compared tightly; with False it is the
exact FP64 model that finite differences pin.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _mm(a, b, bf16):
    if bf16:
        return bf16_round(a) @ bf16_round(b)
    return a @ b


def forward(W, b, X, bf16=False):
    acts = [X]
    h = X
    for l in range(len(W)):
        z = _mm(h, W[l], bf16) + b[l]
        h = np.maximum(z, 0.0) if l < len(W) - 1 else z
        acts.append(h)
    return acts


def loss_and_grads(W, b, X, nact, target, weight=None, bf16=False):
    B = X.shape[0]
    acts = forward(W, b, X, bf16)
    z = acts[-1]
    mask = np.arange(z.shape[1])[None, :] < nact[:, None]
    zm = np.where(mask, z, -np.inf)
    mx = zm.max(axis=1, keepdims=True)
    lse = mx + np.log(np.exp(zm - mx).sum(axis=1, keepdims=True))
    p = np.where(mask, np.exp(zm - lse), 0.0)
    w = np.ones(B) if weight is None else weight
    logp = np.where(mask, z - lse, 0.0)
    loss = float((-(target * logp).sum(axis=1) * w).sum() / B)
    d = (p - target) * mask * w[:, None] / B
    gW, gb = [None] * len(W), [None] * len(W)
    for l in range(len(W) - 1, -1, -1):
        gW[l] = _mm(acts[l].T, d, bf16)
        gb[l] = d.sum(axis=0)
        if l > 0:
            d = _mm(d, W[l].T, bf16) * (acts[l] > 0)
    return loss, gW, gb
