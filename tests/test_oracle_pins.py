"""The oracle against its pins (CPU only)."""
import pytest

import oracle
from tests import pins


@pytest.fixture(scope="module")
def orc():
    return oracle.Oracle()


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    msg = pin(orc)
    assert msg is None, msg


def test_fig8_fixpoint_runs(orc):
    """The rebuilt Figure 8 graph has no 4-clique, so its kernel is empty."""
    from tests import refs
    fx = refs.load_fig8()
    r = orc.fixpoint(fx["colour"], fx["edges"], fx["k"])
    assert not r["vlive"].any() and not r["elive"].any()
    assert r["sweeps"] >= 1


def test_sweep_limit(orc):
    """A cascading graph stopped after one sweep reports the limit."""
    from paper_2212_00574_gb300 import synth
    g = synth.tiny_random(31, 60, 6, 0.35)
    full = orc.fixpoint(g.colour, g.edges, 6)
    assert full["sweeps"] >= 2
    r = orc.fixpoint(g.colour, g.edges, 6, max_sweeps=1, raise_on_limit=False)
    assert r["status"] == -7 and r["sweeps"] == 1


def test_dense_indices_fig8(orc):
    """The dense-matrix form of the colour indices gives the values the thesis
    prints for the Section 4.2 worked example."""
    import numpy as np
    from paper_2212_00574_gb300 import synth
    from tests import refs
    fx = refs.load_fig8()
    bits = synth.edges_to_bits(len(fx["colour"]), fx["edges"])
    verts = [v for v, _ in fx["expect_vertex"]]
    pairs = [(u, v) for u, v, _ in fx["expect_edge"]]
    iv, ie = orc.dense_indices(fx["colour"], bits, fx["k"], verts=verts, pairs=pairs)
    assert list(iv) == [x for _, x in fx["expect_vertex"]]
    assert list(ie) == [x for _, _, x in fx["expect_edge"]]


def test_dense_indices_match_list_form_on_live_states(orc):
    """Both oracle forms agree on random live states (vertices and edges
    deleted at random, in the matrix by clearing bits)."""
    import numpy as np
    from paper_2212_00574_gb300 import synth
    rng = np.random.default_rng(5)
    for s in range(10):
        g = synth.tiny_random(300 + s, 70, int(rng.integers(3, 9)), float(rng.uniform(0.2, 0.8)))
        e = g.edges
        vlive = (rng.random(g.n) < 0.85).astype(np.uint8)
        elive = (rng.random(len(e)) < 0.85).astype(np.uint8)
        elive &= vlive[e[:, 0]] & vlive[e[:, 1]]
        bits = synth.edges_to_bits(g.n, e[elive.astype(bool)])
        verts = np.nonzero(vlive)[0]
        eids = np.nonzero(elive)[0]
        iv1, ie1 = orc.indices(g.colour, e, g.k, verts=verts, edge_ids=eids, vlive=vlive, elive=elive)
        iv2, ie2 = orc.dense_indices(g.colour, bits, g.k, verts=verts, pairs=e[eids], vlive=vlive)
        assert np.array_equal(iv1, iv2) and np.array_equal(ie1, ie2)


def test_session_matches_indices():
    import numpy as np
    import oracle
    from paper_2212_00574_gb300 import synth
    g = synth.tiny_random(21, 120, 6, 0.5, planted=True)
    ids = np.arange(len(g.edges))
    s = oracle.Session(g.colour, g.edges, g.k)
    _, ref = oracle.indices(g.colour, g.edges, g.k, edge_ids=ids)
    assert np.array_equal(s.edge_index(ids), ref)
    s.close()
