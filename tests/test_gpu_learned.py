"""Learned schedule (GPU): the project's MLP kernels against the CPU oracle of
the network, training on plain-method traces, and the schedule's result
against the plain method's (bit-identical survivors)."""
import numpy as np
import pytest

import oracle
import paper_2212_00574_gb300 as kz
from oracle import mlp
from paper_2212_00574_gb300 import learned, synth

pytestmark = pytest.mark.gpu


def _bf16_round(w):
    """Round-to-nearest-even to bf16, kept in float64 (the inference weights)."""
    u = np.asarray(w, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_forward_matches_oracle_with_bf16_weights():
    import torch
    rng = np.random.default_rng(0)
    w = learned.init_weights(3) + rng.normal(0, 0.05, kz.KZ_MLP_PARAMS).astype(np.float32)
    X = rng.normal(size=(3000, 16)).astype(np.float32)
    m = kz.kz_model_create(w)
    try:
        Xd = torch.from_numpy(X).cuda()
        out = torch.zeros(len(X), dtype=torch.float32, device="cuda")
        kz.kz_mlp_forward(m, Xd.data_ptr(), len(X), out.data_ptr())
        got = out.cpu().numpy().astype(np.float64)
    finally:
        kz.kz_model_free(m)
    want, _ = mlp.forward(mlp.unflatten(_bf16_round(w)), X.astype(np.float64))
    # bf16 weights on both sides; fp32 accumulation of ~5k products vs fp64
    assert np.max(np.abs(got - want)) < 1e-4 * (1 + np.max(np.abs(want)))


def test_gradient_matches_oracle():
    import torch
    rng = np.random.default_rng(1)
    w = learned.init_weights(5)
    X = rng.normal(size=(1000, 16)).astype(np.float32)
    y = (rng.random(1000) < 0.3).astype(np.float32)
    m = kz.kz_model_create(w)
    try:
        grad = torch.zeros(kz.KZ_MLP_PARAMS, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
        kz.kz_mlp_grad(m, Xd.data_ptr(), yd.data_ptr(), len(y), grad.data_ptr(), loss.data_ptr())
        g_gpu = grad.cpu().numpy().astype(np.float64)
        l_gpu = float(loss.item())
    finally:
        kz.kz_model_free(m)
    l_ref, g_ref = mlp.loss_and_grad(mlp.unflatten(w.astype(np.float64)), X.astype(np.float64), y)
    g_ref = mlp.flatten(g_ref)
    assert abs(l_gpu - l_ref) < 1e-5 * (1 + abs(l_ref))
    # fp32 sums of 1000 samples against fp64
    assert np.max(np.abs(g_gpu - g_ref)) < 1e-5 + 1e-3 * np.max(np.abs(g_ref))


def test_adam_matches_oracle():
    import torch
    rng = np.random.default_rng(2)
    w = learned.init_weights(7)
    g = rng.normal(0, 1e-2, kz.KZ_MLP_PARAMS).astype(np.float32)
    m = kz.kz_model_create(w)
    try:
        gd = torch.from_numpy(g).cuda()
        for _ in range(3):
            kz.kz_mlp_adam(m, gd.data_ptr(), 1e-3)
        got = kz.kz_model_get(m).astype(np.float64)
    finally:
        kz.kz_model_free(m)
    p = mlp.unflatten(w.astype(np.float64))
    st = {}
    for _ in range(3):
        mlp.adam_step(p, mlp.unflatten(g.astype(np.float64)), st, lr=1e-3)
    assert np.max(np.abs(got - mlp.flatten(p))) < 1e-6


def test_trace_labels_match_plain_sweeps():
    """The first sweep's labels are exactly the oracle's first-sweep edge
    failures (all edges sampled)."""
    g = synth.tiny_random(41, 300, 6, 0.12, planted=True)
    with kz.KernelGraph.from_synth(g) as kg:
        X, y = kz.kz_collect_trace(kg.h, 10 ** 9, 0, cap=200000)
    orc = oracle.fixpoint(g.colour, g.edges, g.k)
    first = int(np.sum(orc["e_rule_sweep"] == 1))
    # records of sweep 0 come first; the round index feature is column 9
    n0 = int(np.sum(X[:, 9] == 0))
    assert n0 == len(g.edges) and int(y[:n0].sum()) == first
    assert X.shape[1] == 16 and np.all(np.isfinite(X))


@pytest.fixture(scope="module")
def trained():
    X, y = learned.collect(learned.cascade_specs(24, 901), per_sweep_cap=3000)
    m, losses = learned.train(X, y, steps=300, batch=4096, lr=3e-3)
    yield m, losses, (X, y)
    kz.kz_model_free(m)


def test_training_reduces_loss(trained):
    m, losses, (X, y) = trained
    assert 0 < y.mean() < 1
    assert losses[-1] < 0.8 * losses[0], losses


@pytest.mark.parametrize("threshold", [0.0, 0.5, 0.95])
def test_learned_schedule_is_bit_identical(trained, threshold):
    m = trained[0]
    for i, (n, k, p, planted, seed) in enumerate(learned.cascade_specs(6, 77)):
        g = synth.kpartite(n, k, p, seed, planted=planted)
        orc = oracle.fixpoint(g.colour, g.get_edges(), g.k)
        with kz.KernelGraph.from_synth(g) as kg:
            kz.kz_attach_model(kg.h, m, threshold)
            kg.kernelize(schedule="learned")
            alive, edges, st = kg.fetch()
        assert np.array_equal(alive, orc["vlive"])
        assert np.array_equal(edges, g.get_edges()[orc["elive"].astype(bool)])


def test_learned_gain_over_plain(trained):
    """On held-out cascading graphs the trained schedule tests fewer edges than
    the plain Jacobi sweeps; the numbers are printed for the record."""
    m = trained[0]
    tot = {"plain": 0, "frontier": 0, "learned": 0}
    for (n, k, p, planted, seed) in learned.cascade_specs(12, 4040):
        g = synth.kpartite(n, k, p, seed, planted=planted)
        for name, kw, thr in (("plain", {}, None), ("frontier", {"schedule": "learned"}, 0.0),
                              ("learned", {"schedule": "learned"}, 0.5)):
            with kz.KernelGraph.from_synth(g) as kg:
                if thr is not None:
                    kz.kz_attach_model(kg.h, m, thr)
                kg.kernelize(path="bitset", **kw)
                tot[name] += kg.stats()["edge_tests"]
    print("edge tests over held-out graphs:", tot)
    assert tot["learned"] < tot["plain"]
