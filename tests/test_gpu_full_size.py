"""Full-size workloads against the oracle, bit for bit (GPU only).

The oracle takes minutes to hours on these graphs, so its results were
computed once, on the CPU, by ``tests/golden/make_full_size_digests.py`` (which
calls nothing but ``oracle/`` and the seeded generators) and stored as
digests under ``tests/golden/full_size/``.  Each test regenerates the same
seeded input, checks that it is the input the digest was made from, runs the
CUDA path in the configuration the benchmark uses (and on every other path
that can hold the graph), and compares, exactly:

* the surviving vertices and edges (sha256 of the flags and of the sorted
  surviving edge list),
* the productive sweeps, the passes and the live-edge tests,
* the vertices and edges that failed in each productive sweep,
* the sweep in which each vertex was deleted (sha256).

The dense workload at n = 32,768 and p = 0.85 (437M edges) is beyond the
oracle's reach as a whole fixpoint; there the GPU kernel is checked for
closure on sampled elements, one oracle call each, for the plain and the
learned schedule alike.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import paper_2212_00574_gb300 as kz
from paper_2212_00574_gb300 import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
DIGESTS = os.path.join(HERE, "golden", "full_size")


def _sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _digest(name: str) -> dict:
    path = os.path.join(DIGESTS, f"{name}.json")
    with open(path) as f:
        return json.load(f)


def _check_input(g, want: dict, cut=None):
    got = _sha(np.asarray(g.colour, np.int32), np.asarray(g.get_edges(), np.int32))
    if cut:
        got = got[:cut]
    assert got == want["input_sha256"], (
        "the seeded generator drew a different graph on this machine than the one the digest was made from")


def _result_digest(alive, kept, v_sweep, cut=None) -> dict:
    f = (lambda s: s[:cut]) if cut else (lambda s: s)
    return dict(vlive_sha256=f(_sha(np.asarray(alive, np.uint8))),
                kept_sha256=f(_sha(np.asarray(kept, np.int32).reshape(-1, 2))),
                v_sweep_sha256=f(_sha(np.asarray(v_sweep, np.int32))))


def _compare(want: dict, alive, kept, stats, dv, de, v_sweep, cut=None, tests=True):
    got = _result_digest(alive, kept, v_sweep, cut)
    assert stats["n_live"] == want["n_live"] and stats["m_live"] == want["m_live"], (
        (stats["n_live"], stats["m_live"]), (want["n_live"], want["m_live"]))
    assert stats["sweeps"] == want["sweeps"], (stats["sweeps"], want["sweeps"])
    assert stats["passes"] == want["passes"], (stats["passes"], want["passes"])
    if tests:
        assert stats["edge_tests"] == want["tests"], (stats["edge_tests"], want["tests"])
    assert [int(x) for x in dv[:stats["sweeps"]]] == want["dv"], "per-sweep vertex deletions differ"
    assert [int(x) for x in de[:stats["sweeps"]]] == want["de"], "per-sweep edge deletions differ"
    assert got["vlive_sha256"] == want["vlive_sha256"], "surviving vertices differ"
    assert got["kept_sha256"] == want["kept_sha256"], "surviving edges differ"
    assert got["v_sweep_sha256"] == want["v_sweep_sha256"], "vertex deletion sweeps differ"


def _run_and_compare(g, want, dense, tests=True, **opts):
    with kz.KernelGraph.from_synth(g, dense=dense) as kg:
        kg.kernelize(**opts)
        alive, kept, stats = kg.fetch()
        dv, de, vs = kg.trace()
    _compare(want, alive, kept, stats, dv, de, vs, tests=tests)
    return stats


# ---------------------------------------------------------------------------
# n = 4096, k = 20, p = 0.92 (7.33M edges)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c2():
    g = synth.workload("c2")
    want = _digest("c2")
    _check_input(g, want)
    return g, want


@pytest.mark.parametrize("path", ["auto", "bitset", "tensor"])
def test_c2_full_size_matches_oracle(c2, path):
    g, want = c2
    st = _run_and_compare(g, want, dense=True, path=path)
    assert st["path"] == {"auto": 1, "bitset": 1, "tensor": 4}[path]


# ---------------------------------------------------------------------------
# Chung-Lu n = 200,000, k = 12 (about 6M edges, dozens of sweeps)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c3():
    g = synth.workload("c3")
    want = _digest("c3")
    _check_input(g, want)
    return g, want


def test_c3_full_size_matches_oracle(c3):
    g, want = c3
    st = _run_and_compare(g, want, dense=False)
    assert st["path"] == 3


def test_c3_full_size_support_schedule_matches_oracle(c3):
    # the support schedule makes fewer tests by design; everything else is equal
    g, want = c3
    st = _run_and_compare(g, want, dense=False, tests=False, schedule="support")
    assert st["edge_tests"] <= want["tests"]


# ---------------------------------------------------------------------------
# n = 32,768, k = 24, p = 0.12 (61.7M edges; the tensor form's regime)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c5c():
    g = synth.workload("c5c")
    want = _digest("c5c")
    _check_input(g, want)
    return g, want


@pytest.mark.parametrize("path", ["auto", "bitset"])
def test_c5c_full_size_matches_oracle(c5c, path):
    g, want = c5c
    st = _run_and_compare(g, want, dense=True, path=path)
    assert st["path"] == {"auto": 4, "bitset": 1}[path]


# ---------------------------------------------------------------------------
# the 1024-graph batch
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c4():
    want = _digest("c4")
    specs = synth.batch_specs(want["count"], want["seed"])
    graphs = [synth.kpartite(n, k, p, seed, planted=pl) for (n, k, p, pl, seed) in specs]
    cut = want["digest_hex_chars"]
    for g, w in zip(graphs, want["graphs"]):
        assert (g.n, g.k) == (w["n"], w["k"])
        _check_input(g, w, cut=cut)
    return graphs, want


@pytest.mark.parametrize("mode", ["concurrent", "fused", "sequential"])
def test_c4_full_batch_matches_oracle(c4, mode):
    graphs, want = c4
    cut = want["digest_hex_chars"]
    hs = [kz.KernelGraph.from_synth(g, dense=True) for g in graphs]
    try:
        kz.kz_kernelize_batch([h.h for h in hs], kz.kz_default_options(batch=mode))
        for i, (h, w) in enumerate(zip(hs, want["graphs"])):
            alive, kept, stats = h.fetch()
            dv, de, vs = h.trace()
            try:
                _compare(w, alive, kept, stats, dv, de, vs, cut=cut)
            except AssertionError as e:
                raise AssertionError(f"graph {i} (n={w['n']}, k={w['k']}, p={w['p']:.3f}): {e}") from None
    finally:
        for h in hs:
            h.close()


# ---------------------------------------------------------------------------
# n = 32,768, k = 24, p = 0.85 (437M edges): sampled closure, plain and learned
# ---------------------------------------------------------------------------

def _closure_sample(g, alive, bits, rng, n_pairs=3000):
    verts = rng.choice(g.n, size=400, replace=False).astype(np.int32)
    # sampled surviving edges, straight from the output bit matrix
    us = rng.integers(0, g.n, size=4 * n_pairs)
    vs = rng.integers(0, g.n, size=4 * n_pairs)
    a, b = np.minimum(us, vs), np.maximum(us, vs)
    on = ((bits[a, b >> 6] >> (b & 63).astype(np.uint64)) & np.uint64(1)).astype(bool) & (a != b)
    pairs = np.stack([a[on], b[on]], axis=1)[:n_pairs].astype(np.int32)
    iv, ie = oracle.dense_indices(g.colour, bits, g.k, verts=verts, pairs=pairs, vlive=alive)
    return verts, pairs, iv, ie


def test_c5_full_size_plain_and_learned_sampled_closure():
    from paper_2212_00574_gb300 import learned

    g = synth.workload("c5")
    bits_in = g.get_bits()
    X, y = learned.collect(learned.cascade_specs(6, synth.SEED_BASE + 950), per_sweep_cap=2000)
    model, _ = learned.train(X, y, steps=60, batch=2048, lr=3e-3)
    try:
        outs = {}
        with kz.KernelGraph(g.n, g.k, g.colour, bits=bits_in) as kg:
            kz.kz_attach_model(kg.h, model, 0.5)
            for schedule in ("plain", "learned"):
                kg.reset().kernelize(schedule=schedule)
                alive, bits, st = kg.fetch_dense()
                outs[schedule] = (alive, bits, st)
    finally:
        kz.kz_model_free(model)
    pa, pb, ps = outs["plain"]
    la, lb, ls = outs["learned"]
    assert np.array_equal(pa, la) and np.array_equal(pb, lb), "learned and plain kernels differ"
    # no element fails on the input (every sampled one passes, below), so the
    # fixpoint is the input itself after one certifying pass
    assert ps["sweeps"] == 0 and ps["passes"] == 1 and ps["edge_tests"] == ps["m"]
    assert pa.all() and np.array_equal(pb, bits_in)
    rng = np.random.default_rng(5)
    verts, pairs, iv, ie = _closure_sample(g, pa, pb, rng)
    assert len(pairs) >= 2000
    assert (iv >= g.k - 1).all(), "a surviving vertex fails the vertex rule"
    assert (ie >= g.k - 2).all(), "a surviving edge fails the edge rule"
