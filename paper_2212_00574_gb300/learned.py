"""Training and use of the edge-scoring MLP of the learned schedule.

Everything runs through the library's C ABI (include/kz_learned.h): the
training data comes from kz_collect_trace (plain Jacobi sweeps on the GPU),
gradients from kz_mlp_grad and updates from kz_mlp_adam -- the project's own
forward and backward kernels.  PyTorch only holds the device buffers.
"""
from __future__ import annotations

import numpy as np

from . import (KZ_MLP_PARAMS, KernelGraph, kz_collect_trace, kz_mlp_adam, kz_mlp_grad, kz_model_create,
               kz_model_get, synth)


def init_weights(seed: int = 0) -> np.ndarray:
    """He-style initial weights in the flat KZ_MLP_PARAMS layout."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2 / 16), 64 * 16), np.zeros(64), rng.normal(0, np.sqrt(2 / 64), 64 * 64),
             np.zeros(64), rng.normal(0, np.sqrt(1 / 64), 64), np.zeros(1)]
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == KZ_MLP_PARAMS
    return w


def cascade_specs(count: int, seed: int, n_lo: int = 256, n_hi: int = 32768):
    """Batch-style graphs (random k-partite, a planted clique on every other
    one) in the regime where the plain method cascades over many sweeps, at
    every scale from n_lo to n_hi: n log-uniform, k uniform in 8..32, and p
    set so that an edge expects mu = U[3, 9] common neighbours per class
    (p = sqrt(mu k / n)), the range in which a sweep's deletions make further
    edges fail.  (n, k, p, planted, graph seed) per graph."""
    rng = np.random.default_rng(seed)
    specs = []
    for j in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        k = int(rng.integers(8, 33))
        mu = float(rng.uniform(3.0, 9.0))
        p = float(min(0.6, max(0.02, np.sqrt(mu * k / n))))
        specs.append((n, k, p, j % 2 == 0, int(seed * 1000003 + j)))
    return specs


def collect(specs, per_sweep_cap: int = 4096, seed: int = 1) -> tuple:
    """Features and labels of plain-method sweeps over the given graphs."""
    Xs, ys = [], []
    for i, (n, k, p, planted, gseed) in enumerate(specs):
        g = synth.kpartite(n, k, p, gseed, planted=planted)
        with KernelGraph.from_synth(g) as kg:
            X, y = kz_collect_trace(kg.h, per_sweep_cap, seed + i, cap=per_sweep_cap * 128)
        Xs.append(X)
        ys.append(y)
    return np.concatenate(Xs), np.concatenate(ys)


def train(X: np.ndarray, y: np.ndarray, steps: int = 400, batch: int = 4096, lr: float = 3e-3, seed: int = 0,
          weights: np.ndarray | None = None, pos_weight_balance: bool = True):
    """Adam on the mean BCE, on the GPU.  Returns (model handle, losses).
    Positive samples are repeated so that the classes are about balanced
    (failures are rare in most sweeps)."""
    import torch
    dev = torch.device("cuda")
    rng = np.random.default_rng(seed)
    if pos_weight_balance and 0 < y.sum() < len(y):
        pos = np.nonzero(y)[0]
        reps = max(1, int(round((len(y) - len(pos)) / len(pos))))
        idx = np.concatenate([np.arange(len(y)), np.repeat(pos, reps - 1)])
        X, y = X[idx], y[idx]
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    yd = torch.from_numpy(np.ascontiguousarray(y, np.float32)).to(dev)
    m = kz_model_create(init_weights(seed) if weights is None else weights)
    grad = torch.zeros(KZ_MLP_PARAMS, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    losses = []
    n = len(y)
    for step in range(steps):
        sel = torch.from_numpy(rng.integers(0, n, size=min(batch, n))).to(dev)
        xb = Xd.index_select(0, sel).contiguous()
        yb = yd.index_select(0, sel).contiguous()
        kz_mlp_grad(m, xb.data_ptr(), yb.data_ptr(), len(sel), grad.data_ptr(), loss.data_ptr())
        kz_mlp_adam(m, grad.data_ptr(), lr)
        if step % 20 == 0 or step == steps - 1:
            losses.append(float(loss.item()))
    return m, losses


def weights_of(m: int) -> np.ndarray:
    return kz_model_get(m)
