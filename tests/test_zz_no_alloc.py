"""The allocation-free entry point, kz_kernelize_dense_noalloc (GPU only).

Some callers cannot allocate device memory. For example, a process may have
handed all of the GPU's memory to another allocator's pool. A caller may also
run inside such an allocator's own callbacks. Or it may be a latency-critical
loop in which cudaMalloc, which can synchronise the device, is not acceptable.
The entry point serves those callers from one fixed static scratch array. These
tests check its output against the ordinary entry points (kz_load_graph_dense +
kz_kernelize + kz_fetch_kernel_dense) and against the CPU oracle, so that a
mistake the two CUDA paths might share is still caught. The comparison is
exact, since this is integer work. They run it on calls in a row, so that nothing left in the shared
scratch by one call leaks into the next.

This file is collected last on purpose: when it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import paper_2212_00574_gb300 as kz
from paper_2212_00574_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(g, max_sweeps=0):
    import torch
    dev = torch.device("cuda", 0)
    bits = g.get_bits()
    n, rw = g.n, max(bits.shape[1], 1)
    colour_d = torch.from_numpy(np.ascontiguousarray(g.colour, np.int32)).to(dev)
    bits_d = torch.from_numpy(np.ascontiguousarray(bits).view(np.int64)).to(dev)
    alive_d = torch.full((max(n, 1),), 7, dtype=torch.uint8, device=dev)          # garbage to overwrite
    out_d = torch.full((max(n, 1), rw), -1, dtype=torch.int64, device=dev)
    counts_d = torch.full((4,), -5, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info(dev)[0]
    st = kz.kz_kernelize_dense_noalloc(n, g.k, colour_d.data_ptr(), bits_d.data_ptr(), rw, max_sweeps,
                                       alive_d.data_ptr(), out_d.data_ptr(), counts_d.data_ptr())
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info(dev)[0]
    return dict(status=st, alive=alive_d.cpu().numpy()[:n], bits=out_d.cpu().numpy().view(np.uint64)[:n],
                counts=counts_d.cpu().numpy(), free_delta=free_before - free_after)


def _reference(g, max_sweeps=0):
    with kz.KernelGraph.from_synth(g, dense=True) as kg:
        kg.kernelize(path="bitset", max_sweeps=max_sweeps)
        alive, bits, stats = kg.fetch_dense(allow=(kz.KZ_OK, kz.KZ_ERR_LIMIT))
    return alive, bits, stats


def _check_same(g, max_sweeps=0):
    r = _noalloc(g, max_sweeps)
    alive, bits, stats = _reference(g, max_sweeps)
    assert r["status"] == stats["status"] == int(r["counts"][3])
    assert np.array_equal(r["alive"], alive), "vertex survivors differ from the ordinary entry points"
    assert np.array_equal(r["bits"], bits), "edge survivors differ from the ordinary entry points"
    assert list(r["counts"][:3]) == [stats["sweeps"], stats["passes"], stats["edge_tests"]]
    # the oracle: survivors and productive sweeps (and, without a limit, the
    # passes and live-edge tests too)
    edges = g.get_edges()
    orc = oracle.fixpoint(g.colour, edges, g.k, max_sweeps=max_sweeps, raise_on_limit=False)
    assert np.array_equal(r["alive"], orc["vlive"]), "vertex survivors differ from the oracle"
    kept = synth.bits_to_edges(np.ascontiguousarray(r["bits"]), g.n)
    assert np.array_equal(kept, edges[orc["elive"].astype(bool)]), "edge survivors differ from the oracle"
    assert int(r["counts"][0]) == orc["sweeps"]
    if orc["status"] == 0:
        assert [int(r["counts"][1]), int(r["counts"][2])] == [orc["passes"], orc["tests"]]
    return r


def test_noalloc_matches_ordinary_entry_points_on_calls_in_a_row():
    first = synth.tiny_random(7001, 900, 7, 0.06, planted=True)    # cascades over several sweeps
    second = synth.kpartite(300, 10, 0.7, seed=7002)              # dense, already a fixpoint
    r1 = _check_same(first)
    assert r1["counts"][0] >= 2
    r2 = _check_same(second)
    assert r2["counts"][0] == 0 and r2["counts"][1] == 1
    r3 = _check_same(first)   # the scratch keeps the previous call's contents: must not matter
    assert list(r3["counts"]) == list(r1["counts"])
    # after the first call on this device the entry point allocates nothing
    assert r2["free_delta"] == 0 and r3["free_delta"] == 0


def test_noalloc_sweep_limit_and_global_mode():
    # 4000 vertices in 4 classes: too large for one CTA's shared memory, so the
    # fixpoint runs on the scratch array's ping-pong buffers
    g = synth.tiny_random(7003, 4000, 4, 0.004, planted=True)
    _check_same(g)
    _check_same(g, max_sweeps=1)


def test_noalloc_rejects_sizes_beyond_its_limits():
    g = synth.tiny_random(7004, 40, 3, 0.5)
    r = _noalloc(g)
    assert r["status"] == kz.KZ_OK
    # n above KZ_NOALLOC_MAX_N: refused on the host
    big = synth.Graph(n=4097, k=2, colour=np.arange(4097, dtype=np.int32) % 2,
                      edges=np.zeros((0, 2), np.int32))
    assert _noalloc(big)["status"] == kz.KZ_ERR_UNSUPPORTED
    # one class of 4065 vertices with k = 32: rows of 4096 words exceed the scratch
    colour = np.zeros(4096, np.int32)
    colour[:31] = np.arange(1, 32)
    lop = synth.Graph(n=4096, k=32, colour=colour, edges=np.zeros((0, 2), np.int32))
    r = _noalloc(lop)
    assert r["status"] == kz.KZ_ERR_UNSUPPORTED
    # refused on the device: the outputs are defined (empty kernel, zero counts)
    assert not r["alive"].any() and not r["bits"].any() and list(r["counts"]) == [0, 0, 0, r["status"]]
    # a colour outside [0, k) and an edge inside one class: found on the device
    bad = synth.tiny_random(7006, 60, 4, 0.5)
    bad.colour = bad.colour.copy()
    bad.colour[5] = 4
    r = _noalloc(bad)
    assert r["status"] == kz.KZ_ERR_COLOUR_RANGE
    assert not r["alive"].any() and not r["bits"].any() and list(r["counts"]) == [0, 0, 0, r["status"]]
    mono = synth.Graph(n=3, k=2, colour=np.array([0, 0, 1], np.int32), edges=np.array([[0, 1]], np.int32))
    r = _noalloc(mono)
    assert r["status"] == kz.KZ_ERR_ILLEGAL_COLOURING
    assert not r["alive"].any() and not r["bits"].any()
    # and a correct call right after the refusals
    _check_same(synth.kpartite(200, 8, 0.6, seed=7005))
