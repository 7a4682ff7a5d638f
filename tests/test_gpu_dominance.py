"""Vertex dominance rounds (thesis Section 4.3, Definition 4.3.1) and edge
dominance rounds (Definitions 4.3.2 and 4.3.3) after the colour-index
fixpoint, through the C ABI, against the oracle (GPU only).  Bit-exact:
surviving vertices and edges, dominance rounds, elements deleted."""
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
        for opts in (dict(path="sparse"), dict(schedule="support"), dict(dominance=3),
                     dict(dominance=2, clique_k=2)):
            with pytest.raises(kz.KzError) as e:
                kg.kernelize(**{"dominance": 1, **opts})
            assert e.value.status in (kz.KZ_ERR_UNSUPPORTED, kz.KZ_ERR_ARG)
        with pytest.raises(kz.KzError) as e:
            kz.kz_kernelize_batch([kg.h], kz.kz_default_options(dominance=1))
        assert e.value.status == kz.KZ_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# edge dominance
# ---------------------------------------------------------------------------

def _run_edge(g, **opts):
    with kz.KernelGraph.from_synth(g) as kg:
        kg.kernelize(dominance=2, **opts)
        alive, edges, st = kg.fetch()
    return alive, edges, st


def _check_edge(g, alive, edges, st, q=None):
    orc = oracle.fixpoint_edge_dominance(g.colour, g.get_edges(), g.k, clique_k=q)
    assert np.array_equal(alive, orc["vlive"]), "surviving vertices differ"
    assert np.array_equal(edges, g.get_edges()[orc["elive"].astype(bool)]), "surviving edges differ"
    assert st["dominance_rounds"] == orc["rounds"] and st["dominated"] == orc["deleted"]
    return orc


@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("path", ["bitset", "small", "tensor"])
def test_edge_dominance_parity(seed, path):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(8, 60))
    k = int(rng.integers(3, 9))
    p = float(rng.uniform(0.35, 0.95))
    g = synth.tiny_random(7300 + seed, n, k, p, planted=bool(seed % 2))
    alive, edges, st = _run_edge(g, path=path)
    orc = _check_edge(g, alive, edges, st)
    # the clique number is kept: a k-clique survives exactly when there was one
    assert refs.has_q_clique(g.n, g.k, g.colour, g.get_edges()) == (
        len(edges) > 0 and refs.has_q_clique(g.n, g.k, g.colour, edges))


@pytest.mark.parametrize("path", ["bitset", "tensor"])
def test_edge_dominance_larger_graphs_and_clique_size(path):
    # several classes of more than 32 vertices (rows of several planes) and
    # the clique size below the colour count
    for seed, n, k, p in [(7401, 160, 4, 0.3), (7402, 130, 3, 0.2), (7403, 90, 5, 0.6)]:
        g = synth.kpartite(n, k, p, seed, planted=True)
        for q in (k, k - 1):
            if q < 3:
                continue
            alive, edges, st = _run_edge(g, path=path, clique_k=q)
            _check_edge(g, alive, edges, st, q=q)


def test_edge_dominance_examples_of_the_definitions():
    # Definition 4.3.2 (shared vertex) and 4.3.3 (disjoint edges): the hand
    # examples the oracle is pinned on
    for colour, edges, k in (([0, 1, 0, 2], [[0, 1], [1, 2], [0, 3], [1, 3], [2, 3]], 3),
                             ([0, 1, 2, 3, 0, 1], [[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3], [4, 5], [2, 4],
                                                   [3, 4], [2, 5], [3, 5]], 4),
                             ([0, 1, 2, 0, 1, 2], [[0, 1], [0, 2], [1, 2], [3, 4], [2, 3], [2, 4], [3, 5], [4, 5]], 3)):
        g = synth.Graph(n=len(colour), k=k, colour=np.asarray(colour, np.int32),
                        edges=synth.canonical_edges(np.asarray(edges)))
        for path in ("bitset", "small"):
            alive, kept, st = _run_edge(g, path=path)
            _check_edge(g, alive, kept, st)
