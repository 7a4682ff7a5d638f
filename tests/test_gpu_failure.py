"""Failure detection without a GPU fault (GPU only): a bounded wait that runs
out must leave an error status the host can read and a usable context."""
import numpy as np
import pytest

import oracle
import paper_2212_00574_gb300 as kz
from paper_2212_00574_gb300 import synth

pytestmark = pytest.mark.gpu


def test_grid_barrier_timeout_reports_and_recovers():
    g = synth.tiny_random(5, 400, 6, 0.1, planted=True)
    with kz.KernelGraph.from_synth(g) as kg:
        # a barrier that waits for an arrival nobody makes: every wait gives up
        kz.kz_probe_barrier_timeout(kg.h, spin_limit=1 << 12)
        st = kg.stats(allow=(kz.KZ_ERR_TIMEOUT,))
        assert st["status"] == kz.KZ_ERR_TIMEOUT
        assert st["sweeps"] == 0          # no pass was applied
        # the context and the graph are still usable
        kg.reset().kernelize(path="bitset")
        alive, edges, st2 = kg.fetch()
    orc = oracle.fixpoint(g.colour, g.edges, g.k)
    assert np.array_equal(alive, orc["vlive"])
    assert np.array_equal(edges, g.edges[orc["elive"].astype(bool)])


def test_sweep_limit_on_every_path():
    g = synth.tiny_random(31, 60, 6, 0.35)
    for path in ("bitset", "small", "sparse", "tensor"):
        with kz.KernelGraph.from_synth(g) as kg:
            kg.kernelize(path=path, max_sweeps=1)
            st = kg.stats(allow=(kz.KZ_ERR_LIMIT,))
            assert st["status"] == kz.KZ_ERR_LIMIT and st["sweeps"] == 1, path
