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
