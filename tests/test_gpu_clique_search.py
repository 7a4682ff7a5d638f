"""The kernel's consumer: q-clique search on the kernel and the maximum-clique
driver (kernelize for q = k, k-1, ...), against exhaustive enumeration on the
CPU (GPU only: every search runs on a kernel the CUDA path produced)."""
import numpy as np
import pytest

import paper_2212_00574_gb300 as kz
from paper_2212_00574_gb300 import synth
from tests import refs

pytestmark = pytest.mark.gpu


def _is_clique(edges, vs):
    es = {tuple(e) for e in np.asarray(edges).tolist()}
    return all((min(a, b), max(a, b)) in es for i, a in enumerate(vs) for b in vs[i + 1:])


def _omega(g):
    for q in range(g.k, 0, -1):
        if refs.q_cliques(g.n, q, g.colour, g.get_edges()):
            return q
    return 0


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("path", ["bitset", "sparse", "tensor"])
def test_max_clique_matches_enumeration(seed, path):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(12, 40))
    k = int(rng.integers(3, 8))
    p = float(rng.uniform(0.25, 0.8))
    g = synth.tiny_random(6000 + seed, n, k, p, planted=bool(seed % 3 == 0))
    with kz.KernelGraph.from_synth(g) as kg:
        q, clique = kz.kz_max_clique(kg.h, g.k, kz.kz_default_options(path=path))
        assert q == _omega(g)
        assert len(clique) == q and len(set(clique.tolist())) == q
        assert _is_clique(g.get_edges(), clique.tolist())
        assert len(set(g.colour[clique].tolist())) == q
        assert kg.stats()["clique_k"] == q


def test_find_clique_on_the_dense_kernel():
    # the dense workload scaled down: the planted k-clique survives and is found
    g = synth.workload("c2", 0.125)
    with kz.KernelGraph.from_synth(g, dense=True) as kg:
        kg.kernelize()
        found, clique = kz.kz_find_clique(kg.h, g.k)
        assert found and len(clique) == g.k
        bits = g.get_bits()
        for i, a in enumerate(clique.tolist()):
            for b in clique.tolist()[i + 1:]:
                assert (int(bits[a, b // 64]) >> (b % 64)) & 1


def test_clique_search_limits_and_absence():
    # a complete 4-partite graph on classes of 3 has 4-cliques but no 5 colours
    colour, edges = refs.complete_kpartite([3, 3, 3, 3])
    with kz.KernelGraph(12, 4, colour, edges=edges) as kg:
        kg.kernelize()
        found, clique = kz.kz_find_clique(kg.h, 4)
        assert found and _is_clique(edges, clique.tolist())
        with pytest.raises(kz.KzError) as e:
            kz.kz_find_clique(kg.h, 5)
        assert e.value.status == kz.KZ_ERR_ARG
    # remove one class's edges to another: no 4-clique; the kernel for q = 4
    # is empty, and a 3-clique is the maximum
    keep = [e for e in np.asarray(edges).tolist() if not ({colour[e[0]], colour[e[1]]} == {0, 1})]
    with kz.KernelGraph(12, 4, colour, edges=np.array(keep, np.int32)) as kg:
        q, clique = kz.kz_max_clique(kg.h, 4)
        assert q == 3 and _is_clique(keep, clique.tolist())
    # a node budget of one cannot finish a search that has to branch
    g = synth.tiny_random(6101, 60, 6, 0.6, planted=False)
    with kz.KernelGraph.from_synth(g) as kg:
        kg.kernelize(clique_k=4)
        if kg.stats()["n_live"] > 0:
            with pytest.raises(kz.KzError) as e:
                kz.kz_find_clique(kg.h, 4, node_limit=1)
            assert e.value.status == kz.KZ_ERR_LIMIT


@pytest.mark.parametrize("name", ["c1", "c3"])
def test_workload_kernels_keep_a_clique(name):
    # the sparse large workload: every planted 12-clique survives its 34
    # sweeps, and the search finds a k-clique in what is left
    g = synth.workload(name)
    with kz.KernelGraph.from_synth(g) as kg:
        kg.kernelize()
        found, clique = kz.kz_find_clique(kg.h, g.k)
        assert found and _is_clique(g.get_edges(), clique.tolist())
