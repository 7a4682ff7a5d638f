"""Tensor-core edge rule (tcgen05.mma kind::f8f6f4) against the oracle, through
the C ABI (GPU only).  Bit-exact: survivors, sweeps, per-sweep counts."""
import numpy as np
import pytest

import paper_2212_00574_gb300 as kz
from paper_2212_00574_gb300 import synth
from tests import refs
from tests.test_gpu_parity import _graph, _tiny_cases, assert_parity, gpu_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", _tiny_cases()[::2], ids=lambda c: f"s{c[0]}-n{c[1]}-k{c[2]}")
def test_tensor_tiny(case):
    seed, n, k, p, planted = case
    g = synth.tiny_random(5000 + seed, n, k, p, planted=planted and n >= k)
    assert_parity(g, gpu_run(g, path="tensor"))


@pytest.mark.parametrize("sizes", [[31, 32, 33], [64, 65, 1, 96], [5, 0, 7], [2] * 33])
def test_tensor_shapes(sizes):
    colour, edges = refs.complete_kpartite(sizes)
    g = _graph(colour, edges, len(sizes))
    assert_parity(g, gpu_run(g, path="tensor"))


def test_tensor_cascades_and_large_classes():
    for seed in range(4):
        g = synth.tiny_random(700 + seed, 400, 6, 0.06 + 0.01 * seed, planted=bool(seed % 2))
        assert_parity(g, gpu_run(g, path="tensor"))
    g = synth.tiny_random(61, 600, 4, 0.03, planted=True)
    assert_parity(g, gpu_run(g, path="tensor"))


@pytest.mark.parametrize("scale", [0.0625, 0.125])
def test_tensor_dense_workload_reduced(scale):
    g = synth.workload("c2", scale)
    assert_parity(g, gpu_run(g, path="tensor", dense=True))


def test_tensor_matches_bitset_on_batch_members():
    for (n, k, p, planted, seed) in synth.batch_specs(6, 515, n_hi=900):
        g = synth.kpartite(n, k, p, seed, planted=planted)
        a = gpu_run(g, path="tensor", dense=True)
        b = gpu_run(g, path="bitset", dense=True)
        assert np.array_equal(a["alive"], b["alive"]) and np.array_equal(a["edges"], b["edges"])
        assert a["stats"]["sweeps"] == b["stats"]["sweeps"]


@pytest.mark.parametrize("seed,n,k,p", [(84, 2300, 8, 0.1), (86, 2300, 4, 0.04), (81, 2300, 8, 0.3)])
def test_tensor_more_tiles_than_ctas(seed, n, k, p):
    # 18 x 18 tiles (171 upper-triangle tiles: more than one per SM), classes
    # of up to 18 K-steps (several pipeline stages per class), cascades over
    # several sweeps, and a graph where nothing is deleted
    g = synth.tiny_random(seed, n, k, p, planted=True)
    assert_parity(g, gpu_run(g, path="tensor"))


def test_auto_picks_tensor_for_a_larger_sparser_graph():
    # n = 4500, k = 12, density about 0.12 falls in a bin where the tensor
    # form measured faster; a dense graph of the same size stays on the bitset
    # sweep.  The result is the same whichever path runs.
    g = synth.kpartite(4500, 12, 0.12, 77, planted=True)
    a = gpu_run(g, path="auto", dense=True)
    b = gpu_run(g, path="bitset", dense=True)
    assert a["stats"]["path"] == 4
    assert np.array_equal(a["alive"], b["alive"]) and np.array_equal(a["edges"], b["edges"])
    assert a["stats"]["sweeps"] == b["stats"]["sweeps"]
    g2 = synth.kpartite(4500, 12, 0.6, 78, planted=True)
    assert gpu_run(g2, path="auto", dense=True)["stats"]["path"] == 1


@pytest.mark.parametrize("case", _tiny_cases()[1::4], ids=lambda c: f"s{c[0]}-n{c[1]}-k{c[2]}")
def test_tensor_bf16_tiny(case):
    # BF16 0/1 operands through kind::f16: the same exact counts
    seed, n, k, p, planted = case
    g = synth.tiny_random(5000 + seed, n, k, p, planted=planted and n >= k)
    assert_parity(g, gpu_run(g, path="tensor", tensor_precision=1))


@pytest.mark.parametrize("seed,n,k,p", [(84, 2300, 8, 0.1), (86, 2300, 4, 0.04)])
def test_tensor_bf16_more_tiles_than_ctas(seed, n, k, p):
    g = synth.tiny_random(seed, n, k, p, planted=True)
    a = gpu_run(g, path="tensor", tensor_precision=1)
    assert_parity(g, a)
    # switching precision on one handle keeps both buffer sets apart
    with kz.KernelGraph.from_synth(g) as kg:
        for prec in (0, 1, 0):
            kg.reset().kernelize(path="tensor", tensor_precision=prec)
            alive, edges, st = kg.fetch()
            assert np.array_equal(alive, a["alive"]) and np.array_equal(edges, a["edges"])
