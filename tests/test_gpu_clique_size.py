"""Clique size q below the colour count k (thresholds q-1 and q-2, thesis
Section 4.2 Remarks) through the C ABI, against the oracle (GPU only).
Bit-exact: survivors, sweeps, passes, per-sweep counts, tests."""
import numpy as np
import pytest

import oracle
import paper_2212_00574_gb300 as kz
from paper_2212_00574_gb300 import synth
from tests.test_gpu_parity import assert_parity, gpu_run

pytestmark = pytest.mark.gpu

CASES = [(5100 + i, n, k, p) for i, (n, k, p) in enumerate(
    [(40, 5, 0.5), (90, 7, 0.35), (150, 9, 0.45), (200, 12, 0.3), (70, 33, 0.8), (300, 6, 0.12)])]


def _qs(k):
    return sorted({k - 1, k - 2, max(1, k // 2), 2, 1} - {0, k})


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"s{c[0]}-n{c[1]}-k{c[2]}")
@pytest.mark.parametrize("path", ["bitset", "small", "sparse", "tensor"])
def test_clique_size_parity(case, path):
    seed, n, k, p = case
    g = synth.tiny_random(seed, n, k, p, planted=n >= k)
    if path == "small" and n > 200:
        pytest.skip("larger than the in-CTA path's shared memory")
    for q in _qs(k):
        orc = oracle.fixpoint(g.colour, g.get_edges(), k, clique_k=q)
        res = gpu_run(g, path=path, clique_k=q)
        assert res["stats"]["clique_k"] == q
        assert_parity(g, res, orc=orc)


@pytest.mark.parametrize("plane0", [1, 2, 3])
def test_clique_size_plane0_forms(plane0):
    # dense and sparse graphs with several planes per class, each first test
    for seed, n, k, p in [(5201, 700, 8, 0.85), (5202, 900, 6, 0.2)]:
        g = synth.kpartite(n, k, p, seed, planted=True)
        for q in (k - 1, k - 3):
            orc = oracle.fixpoint(g.colour, g.get_edges(), k, clique_k=q)
            assert_parity(g, gpu_run(g, path="bitset", dense=True, plane0=plane0, clique_k=q), orc=orc)


def test_clique_size_changes_on_one_handle():
    # the cached launch graphs of the bitset path must follow q between runs
    g = synth.tiny_random(5301, 400, 7, 0.3, planted=True)
    with kz.KernelGraph.from_synth(g) as kg:
        for q in (7, 5, 7, 3, 5):
            for use_graph in (1, 2):
                kg.reset().kernelize(path="bitset", clique_k=q, use_graph=use_graph)
                alive, edges, st = kg.fetch()
                orc = oracle.fixpoint(g.colour, g.get_edges(), g.k, clique_k=q)
                assert np.array_equal(alive, orc["vlive"])
                assert np.array_equal(edges, g.get_edges()[orc["elive"].astype(bool)])
                assert st["sweeps"] == orc["sweeps"] and st["clique_k"] == q


@pytest.mark.parametrize("mode", ["concurrent", "sequential"])
def test_clique_size_batch(mode):
    graphs = [synth.tiny_random(5400 + i, 60 + 40 * i, 6 + i % 3, 0.25 + 0.05 * i, planted=True) for i in range(6)]
    handles = [kz.KernelGraph.from_synth(g) for g in graphs]
    try:
        kz.kz_kernelize_batch([h.h for h in handles], kz.kz_default_options(batch=mode, clique_k=4))
        for g, h in zip(graphs, handles):
            alive, edges, st = h.fetch()
            orc = oracle.fixpoint(g.colour, g.get_edges(), g.k, clique_k=4)
            assert np.array_equal(alive, orc["vlive"]) and st["sweeps"] == orc["sweeps"]
            assert np.array_equal(edges, g.get_edges()[orc["elive"].astype(bool)])
    finally:
        for h in handles:
            h.close()


def test_clique_size_errors():
    g = synth.tiny_random(5501, 50, 5, 0.5, planted=True)
    with kz.KernelGraph.from_synth(g) as kg:
        for bad in (6, -1):
            with pytest.raises(kz.KzError) as e:
                kg.kernelize(clique_k=bad)
            assert e.value.status == kz.KZ_ERR_ARG
        with pytest.raises(kz.KzError) as e:
            kg.kernelize(schedule="support", clique_k=4)
        assert e.value.status == kz.KZ_ERR_UNSUPPORTED
        # q = k through clique_k is the default rule
        kg.kernelize(clique_k=5)
        alive, _, st = kg.fetch()
        assert st["clique_k"] == 5
        assert np.array_equal(alive, oracle.fixpoint(g.colour, g.get_edges(), 5)["vlive"])
    with kz.KernelGraph.from_synth(g) as kg:
        with pytest.raises(kz.KzError) as e:
            kz.kz_kernelize_batch([kg.h], kz.kz_default_options(batch="fused", clique_k=4))
        assert e.value.status == kz.KZ_ERR_UNSUPPORTED
