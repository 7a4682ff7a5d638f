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


def test_forward_matches_oracle_with_bf16_operands():
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
    want, _ = mlp.forward_bf16(mlp.unflatten(w.astype(np.float64)), X.astype(np.float64))
    assert_logits_close(got, want)


def assert_logits_close(got, want):
    """The same bf16 operands on both sides, so what is left is fp32
    accumulation of at most 64 products per sum (relative 64 * 2^-24), and,
    rarely, a hidden value whose fp32 and fp64 sums lie on either side of a
    bf16 rounding boundary: that row moves by about one bf16 ulp of one hidden
    unit's contribution.  So: nearly every row agrees to fp32 accumulation
    error, and every row to within bf16 precision."""
    err = np.abs(got - want)
    tight = err < 1e-5 * (1 + np.abs(want))
    assert tight.mean() > 0.998, tight.mean()
    assert np.all(err < 2.0 ** -7 * (1 + np.abs(want))), np.max(err)


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
    l_ref, g_ref = mlp.loss_and_grad_bf16(mlp.unflatten(w.astype(np.float64)), X.astype(np.float64), y)
    g_ref = mlp.flatten(g_ref)
    assert abs(l_gpu - l_ref) < 1e-5 * (1 + abs(l_ref))
    # the same bf16 product operands on both sides (tensor-core MMAs on the
    # GPU); fp32 sums of 1000 samples against fp64
    assert np.max(np.abs(g_gpu - g_ref)) < 1e-5 + 1e-3 * np.max(np.abs(g_ref))
    # and the bf16 network's gradient stays within bf16 rounding of the exact
    # network's (pinned by finite differences on the CPU)
    _, g_exact = mlp.loss_and_grad(mlp.unflatten(w.astype(np.float64)), X.astype(np.float64), y)
    g_exact = mlp.flatten(g_exact)
    assert np.linalg.norm(g_gpu - g_exact) < 2.0 ** -5 * np.linalg.norm(g_exact)


def test_gradient_matches_oracle_on_ragged_batches():
    # batch sizes that leave the last 64-sample chunk partly empty, and more
    # chunks than the grid has CTAs
    import torch
    rng = np.random.default_rng(3)
    w = learned.init_weights(9) + rng.normal(0, 0.05, kz.KZ_MLP_PARAMS).astype(np.float32)
    for B in (1, 17, 64, 65, 200, 40000):
        X = rng.normal(size=(B, 16)).astype(np.float32)
        y = (rng.random(B) < 0.4).astype(np.float32)
        m = kz.kz_model_create(w)
        try:
            grad = torch.zeros(kz.KZ_MLP_PARAMS, dtype=torch.float32, device="cuda")
            loss = torch.zeros(1, dtype=torch.float32, device="cuda")
            Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
            kz.kz_mlp_grad(m, Xd.data_ptr(), yd.data_ptr(), B, grad.data_ptr(), loss.data_ptr())
            g_gpu = grad.cpu().numpy().astype(np.float64)
            l_gpu = float(loss.item())
        finally:
            kz.kz_model_free(m)
        l_ref, g_ref = mlp.loss_and_grad_bf16(mlp.unflatten(w.astype(np.float64)), X.astype(np.float64), y)
        g_ref = mlp.flatten(g_ref)
        assert abs(l_gpu - l_ref) < 1e-5 * (1 + abs(l_ref)), B
        assert np.max(np.abs(g_gpu - g_ref)) < 1e-5 + 1e-3 * np.max(np.abs(g_ref)), B


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
    X, y = learned.collect(learned.cascade_specs(24, 901, n_hi=8192), per_sweep_cap=3000)
    m, losses = learned.train(X, y, steps=300, batch=4096, lr=3e-3)
    yield m, losses, (X, y)
    kz.kz_model_free(m)


def test_training_reduces_loss(trained):
    m, losses, (X, y) = trained
    assert 0 < y.mean() < 1
    assert losses[-1] < 0.8 * losses[0], losses


@pytest.mark.parametrize("path", ["auto", "tensor"])
@pytest.mark.parametrize("threshold", [0.0, 0.5, 0.95])
def test_learned_schedule_is_bit_identical(trained, threshold, path):
    # full passes on the bitset sweep (AUTO on these sizes) or the tensor form
    m = trained[0]
    for i, (n, k, p, planted, seed) in enumerate(learned.cascade_specs(6, 77, n_hi=2048)):
        g = synth.kpartite(n, k, p, seed, planted=planted)
        orc = oracle.fixpoint(g.colour, g.get_edges(), g.k)
        with kz.KernelGraph.from_synth(g) as kg:
            kz.kz_attach_model(kg.h, m, threshold)
            kg.kernelize(schedule="learned", path=path)
            alive, edges, st = kg.fetch()
            assert st["path"] == (4 if path == "tensor" else 1)
        assert np.array_equal(alive, orc["vlive"])
        assert np.array_equal(edges, g.get_edges()[orc["elive"].astype(bool)])


def test_learned_gain_over_plain(trained):
    """On held-out cascading graphs the trained schedule tests fewer edges than
    the plain Jacobi sweeps; the numbers are printed for the record."""
    m = trained[0]
    tot = {"plain": 0, "frontier": 0, "learned": 0}
    for (n, k, p, planted, seed) in learned.cascade_specs(12, 4040, n_hi=8192):
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


def test_forward_ragged_sizes():
    import torch
    rng = np.random.default_rng(4)
    w = learned.init_weights(13) + rng.normal(0, 0.05, kz.KZ_MLP_PARAMS).astype(np.float32)
    m = kz.kz_model_create(w)
    try:
        for B in (1, 31, 33, 100003):
            X = rng.normal(size=(B, 16)).astype(np.float32)
            out = torch.full((B,), float("nan"), dtype=torch.float32, device="cuda")
            kz.kz_mlp_forward(m, torch.from_numpy(X).cuda().data_ptr(), B, out.data_ptr())
            got = out.cpu().numpy().astype(np.float64)
            want, _ = mlp.forward_bf16(mlp.unflatten(w.astype(np.float64)), X.astype(np.float64))
            assert_logits_close(got, want)
    finally:
        kz.kz_model_free(m)
