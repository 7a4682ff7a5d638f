"""Vertex dominance rounds (thesis Section 4.3, Definition 4.3.1) after the
colour-index fixpoint, through the C ABI, against the oracle (GPU only).
Bit-exact: surviving vertices and edges, dominance rounds, vertices deleted."""
import numpy as np
import pytest

import oracle
import paper_2212_00574_gb300 as kz
from paper_2212_00574_gb300 import synth
from tests import refs

pytestmark = pytest.mark.gpu


def _run(g, **opts):
    with kz.KernelGraph.from_synth(g) as kg:
        kg.kernelize(dominance=1, **opts)
        alive, edges, st = kg.fetch()
    return alive, edges, st


def _check(g, alive, edges, st, q=None):
    orc = oracle.fixpoint_dominance(g.colour, g.get_edges(), g.k, clique_k=q)
    assert np.array_equal(alive, orc["vlive"]), "surviving vertices differ"
    assert np.array_equal(edges, g.get_edges()[orc["elive"].astype(bool)]), "surviving edges differ"
    assert st["dominance_rounds"] == orc["rounds"] and st["dominated"] == orc["dominated"]
    return orc


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("path", ["bitset", "small", "tensor"])
def test_dominance_parity(seed, path):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(10, 160))
    k = int(rng.integers(3, 12))
    p = float(rng.uniform(0.3, 0.9))
    g = synth.tiny_random(7000 + seed, n, k, p, planted=bool(seed % 2))
    alive, edges, st = _run(g, path=path)
    _check(g, alive, edges, st)


@pytest.mark.parametrize("path", ["bitset", "tensor"])
def test_dominance_larger_graphs_and_clique_size(path):
    for seed, n, k, p in [(7101, 600, 8, 0.5), (7102, 900, 12, 0.8), (7103, 400, 5, 0.3)]:
        g = synth.kpartite(n, k, p, seed, planted=True)
        for q in (k, k - 1):
            alive, edges, st = _run(g, path=path, clique_k=q)
            _check(g, alive, edges, st, q=q)


def test_dominance_keeps_a_planted_clique():
    g = synth.workload("c1")
    alive, edges, st = _run(g)
    orc = _check(g, alive, edges, st)
    assert st["dominated"] > 0 or orc["rounds"] == 0
    assert refs.has_q_clique(g.n, g.k, g.colour, edges)  # the clique number k is kept


def test_dominance_refused_where_unsupported():
    g = synth.tiny_random(7201, 60, 5, 0.5, planted=True)
    with kz.KernelGraph.from_synth(g) as kg:
        for opts in (dict(path="sparse"), dict(schedule="support"), dict(dominance=2)):
            with pytest.raises(kz.KzError) as e:
                kg.kernelize(**{"dominance": 1, **opts})
            assert e.value.status in (kz.KZ_ERR_UNSUPPORTED, kz.KZ_ERR_ARG)
        with pytest.raises(kz.KzError) as e:
            kz.kz_kernelize_batch([kg.h], kz.kz_default_options(dominance=1))
        assert e.value.status == kz.KZ_ERR_UNSUPPORTED
