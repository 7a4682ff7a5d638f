"""CPU oracle of the edge-scoring MLP used by the learned schedule.

TEST INFRASTRUCTURE ONLY (tests and the smoke check call it; the product
library never does).  The thesis has no learned component; this network only
orders the worklist of the colour-index rules (Section 4.2) and can never
change the kernel, because the greatest fixpoint of monotone deletion rules
is unique.

Network: 16 -> 64 -> 64 -> 1, ReLU after the two hidden layers, a logistic
output, binary cross-entropy against "the edge fails the edge rule in this
pass".  Everything here is plain numpy in float64: a reader can check each
line against the textbook definitions.  ``forward_bf16`` and
``loss_and_grad_bf16`` are the same network with the kernels' bf16 product
operands (see the comment above them).

Weights are stored as a dict of arrays:
    W1 [64, 16], b1 [64], W2 [64, 64], b2 [64], w3 [64], b3 [] (scalar)
"""
from __future__ import annotations

import numpy as np

SHAPES = {"W1": (64, 16), "b1": (64,), "W2": (64, 64), "b2": (64,), "w3": (64,), "b3": ()}
ORDER = ["W1", "b1", "W2", "b2", "w3", "b3"]


def init(seed: int) -> dict:
    """He-style initialisation (deterministic)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0.0, np.sqrt(2.0 / 16), (64, 16)),
        "b1": np.zeros(64),
        "W2": rng.normal(0.0, np.sqrt(2.0 / 64), (64, 64)),
        "b2": np.zeros(64),
        "w3": rng.normal(0.0, np.sqrt(1.0 / 64), 64),
        "b3": np.zeros(()),
    }


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], np.float64).reshape(-1) for k in ORDER])


def unflatten(v: np.ndarray) -> dict:
    out, o = {}, 0
    for k in ORDER:
        size = int(np.prod(SHAPES[k])) if SHAPES[k] else 1
        out[k] = np.asarray(v[o:o + size], np.float64).reshape(SHAPES[k])
        o += size
    return out


def forward(p: dict, X: np.ndarray):
    """X [B, 16] -> (logits [B], cache)."""
    X = np.asarray(X, np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    logit = h2 @ p["w3"] + p["b3"]
    return logit, (X, z1, h1, z2, h2)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def bce_loss(logit: np.ndarray, y: np.ndarray) -> float:
    """Mean binary cross-entropy of sigmoid(logit) against labels y in {0,1},
    written in the overflow-free form max(l,0) - l*y + log(1 + exp(-|l|))."""
    logit = np.asarray(logit, np.float64)
    y = np.asarray(y, np.float64)
    return float(np.mean(np.maximum(logit, 0.0) - logit * y + np.log1p(np.exp(-np.abs(logit)))))


def loss_and_grad(p: dict, X: np.ndarray, y: np.ndarray):
    """Loss and the gradient of the mean BCE with respect to every weight."""
    logit, (X, z1, h1, z2, h2) = forward(p, X)
    B = len(y)
    loss = bce_loss(logit, y)
    dlogit = (sigmoid(logit) - np.asarray(y, np.float64)) / B      # d loss / d logit
    g = {}
    g["w3"] = h2.T @ dlogit
    g["b3"] = np.asarray(dlogit.sum())
    dh2 = np.outer(dlogit, p["w3"])
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return loss, g


# ---------------------------------------------------------------------------
# the network with bf16 operands and wide accumulation
# ---------------------------------------------------------------------------
#
# The learned schedule's network keeps bf16 weights and accumulates in fp32
# (the tensor-core products of the kernels take bf16 operands).  The functions
# below are the same network with every product operand rounded to bf16 at
# the points where the kernels round it, and everything else exact (float64
# here): the only difference left against the kernels is the order and width
# of the accumulation.  Rounding points:
#
#   forward   parameters p -> bf16(p) (all of them);  x -> bf16(x);
#             z1 = bf16(x) W1^T + b1;  h1 = bf16(relu(z1));
#             z2 = h1 W2^T + b2;  h2 = relu(z2) (not rounded);
#             logit = h2 . w3 + b3
#   backward  dl = (sigmoid(logit) - y) / B;  g_w3 = h2^T dl;  g_b3 = sum dl;
#             dz2 = bf16(dl w3^T * [z2 > 0]);  g_W2 = dz2^T h1;  g_b2 = sum dz2;
#             dz1 = bf16((dz2 W2) * [z1 > 0]);  g_W1 = dz1^T bf16(x);  g_b1 = sum dz1
#
# The gradient is taken with respect to the rounded parameters (the fp32
# master copy receives it unchanged in the Adam step).

def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 value, ties to even (the IEEE rule on
    the top 16 bits of a float32), returned as float64.  Values are first
    rounded to float32, as a kernel holds them."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def quantized(p: dict) -> dict:
    return {k: bf16(v) for k, v in p.items()}


def forward_bf16(p: dict, X: np.ndarray):
    """Forward pass with bf16 operands (rounding points above)."""
    q = quantized(p)
    Xr = bf16(X)
    z1 = Xr @ q["W1"].T + q["b1"]
    h1 = bf16(np.maximum(z1, 0.0))
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, 0.0)
    logit = h2 @ q["w3"] + q["b3"]
    return logit, (Xr, z1, h1, z2, h2, q)


def loss_and_grad_bf16(p: dict, X: np.ndarray, y: np.ndarray):
    """Loss and gradient of the bf16-operand network (rounding points above)."""
    logit, (Xr, z1, h1, z2, h2, q) = forward_bf16(p, X)
    B = len(y)
    loss = bce_loss(logit, y)
    dlogit = (sigmoid(logit) - np.asarray(y, np.float64)) / B
    g = {}
    g["w3"] = h2.T @ dlogit
    g["b3"] = np.asarray(dlogit.sum())
    dz2 = bf16(np.outer(dlogit, q["w3"]) * (z2 > 0))
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = bf16((dz2 @ q["W2"]) * (z1 > 0))
    g["W1"] = dz1.T @ Xr
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adam_step(p: dict, g: dict, state: dict, lr: float, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
    """One Adam update in place (Kingma and Ba, Algorithm 1)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in ORDER:
        m = state.setdefault("m_" + k, np.zeros_like(np.asarray(p[k], np.float64)))
        v = state.setdefault("v_" + k, np.zeros_like(np.asarray(p[k], np.float64)))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] * g[k]
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mhat / (np.sqrt(vhat) + eps)
