"""Allocator-failure injection through the caller-supplied allocator (GPU
only): every load path reports KZ_ERR_OOM, releases what it got, and the
library works again once a working allocator is back."""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_2212_00574_gb300 as kz
from paper_2212_00574_gb300 import synth

pytestmark = pytest.mark.gpu


def _install(fail_after):
    """An allocator that serves `fail_after` requests through torch's caching
    allocator and fails every later one; returns (allocator, counters)."""
    import torch
    state = {"alloc": 0, "freed": 0, "live": set()}

    def _alloc(nbytes, stream, ctx):
        state["alloc"] += 1
        if state["alloc"] > fail_after:
            return None
        p = int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0)))
        state["live"].add(p)
        return p

    def _free(ptr, nbytes, stream, ctx):
        state["freed"] += 1
        if ptr in state["live"]:
            state["live"].discard(ptr)
            torch.cuda.caching_allocator_delete(int(ptr))

    a = kz.kz_allocator(kz._ALLOC_FN(_alloc), kz._FREE_FN(_free), None)
    assert kz._lib().kz_set_allocator(C.byref(a)) == kz.KZ_OK
    return a, state


def _load(g, dense):
    if dense:
        return kz.kz_load_graph_dense(g.n, g.k, g.colour, g.get_bits())
    return kz.kz_load_graph(g.n, g.k, g.colour, g.get_edges())


@pytest.mark.parametrize("dense", [False, True])
def test_allocation_failure_reports_oom(dense):
    g = synth.tiny_random(4101, 90, 6, 0.4, planted=True)
    # how many requests a successful load makes
    a, state = _install(1 << 30)
    try:
        kz.kz_free_graph(_load(g, dense))
        total = state["alloc"]
        assert total >= 1 and not state["live"]
    finally:
        kz.use_default_allocator()
    for fail_after in sorted({0, total // 2, total - 1}):
        a, state = _install(fail_after)
        try:
            with pytest.raises(kz.KzError) as e:
                _load(g, dense)
            assert e.value.status == kz.KZ_ERR_OOM
            assert state["alloc"] == fail_after + 1  # the load stopped at the failed request
            assert not state["live"]                 # and gave back everything it got
        finally:
            kz.use_default_allocator()
    with kz.KernelGraph.from_synth(g, dense=dense) as kg:
        kg.kernelize()
        alive, edges, st = kg.fetch()
    orc = oracle.fixpoint(g.colour, g.get_edges(), g.k)
    assert np.array_equal(alive, orc["vlive"])
    assert np.array_equal(edges, g.get_edges()[orc["elive"].astype(bool)])
