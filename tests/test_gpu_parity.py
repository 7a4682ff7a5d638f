"""CUDA path against the CPU oracle, through the C ABI (GPU only).

Integer graph work: everything is compared exactly -- surviving vertices and
edges, productive sweep count, passes, per-sweep deletion counts, the sweep
in which each vertex died, and the number of live-edge tests.
"""
import numpy as np
import pytest

import oracle
import paper_2212_00574_gb300 as kz
from paper_2212_00574_gb300 import synth
from tests import refs

pytestmark = pytest.mark.gpu


def gpu_run(g, dense=False, **opts):
    with kz.KernelGraph.from_synth(g, dense=dense) as kg:
        kg.kernelize(**opts)
        alive, edges, stats = kg.fetch(allow=(kz.KZ_OK, kz.KZ_ERR_LIMIT))
        dv, de, vs = kg.trace()
    return dict(alive=alive, edges=edges, stats=stats, dv=dv[:stats["sweeps"]], de=de[:stats["sweeps"]], v_sweep=vs)


def assert_parity(g, res, orc=None, max_sweeps=0):
    edges = g.get_edges()
    if orc is None:
        orc = oracle.fixpoint(g.colour, edges, g.k, max_sweeps=max_sweeps, raise_on_limit=False)
    want_edges = edges[orc["elive"].astype(bool)]
    st = res["stats"]
    assert np.array_equal(res["alive"], orc["vlive"]), "surviving vertices differ"
    assert np.array_equal(res["edges"], want_edges), "surviving edges differ"
    assert st["sweeps"] == orc["sweeps"], (st["sweeps"], orc["sweeps"])
    assert st["passes"] == orc["passes"], (st["passes"], orc["passes"])
    assert st["edge_tests"] == orc["tests"], (st["edge_tests"], orc["tests"])
    assert np.array_equal(res["dv"], orc["dv"]), "per-sweep vertex deletions differ"
    assert np.array_equal(res["de"], orc["de"]), "per-sweep edge deletions differ"
    assert np.array_equal(res["v_sweep"], orc["v_sweep"]), "vertex deletion sweeps differ"
    assert st["n_live"] == int(orc["vlive"].sum()) and st["m_live"] == len(want_edges)
    return orc


# ---------------------------------------------------------------------------
# many small random graphs (several blocks, ragged class tails)
# ---------------------------------------------------------------------------

def _tiny_cases():
    rng = np.random.default_rng(2024)
    cases = []
    for i in range(48):
        n = int(rng.integers(1, 160))
        k = int(rng.integers(1, 14))
        p = float(rng.uniform(0.05, 0.95))
        cases.append((i, n, k, p, bool(i % 2)))
    for i, (n, k) in enumerate([(40, 33), (90, 40), (200, 64), (70, 32), (300, 48), (128, 20)]):
        cases.append((100 + i, n, k, 0.8, True))
    return cases


@pytest.mark.parametrize("path", ["bitset", "small", "sparse"])
@pytest.mark.parametrize("case", _tiny_cases(), ids=lambda c: f"s{c[0]}-n{c[1]}-k{c[2]}-p{c[3]:.2f}")
def test_tiny_random(case, path):
    seed, n, k, p, planted = case
    g = synth.tiny_random(5000 + seed, n, k, p, planted=planted and n >= k)
    assert_parity(g, gpu_run(g, path=path))


# ---------------------------------------------------------------------------
# shapes chosen to hit edge cases
# ---------------------------------------------------------------------------

def _graph(colour, edges, k):
    colour = np.asarray(colour, np.int32)
    return synth.Graph(n=len(colour), k=k, colour=colour, edges=synth.canonical_edges(np.asarray(edges).reshape(-1, 2)))


def test_empty_graph():
    g = _graph([], np.zeros((0, 2)), 3)
    assert_parity(g, gpu_run(g))


def test_isolated_vertices_only():
    for k in (1, 2, 5):
        g = _graph(np.arange(7) % k, np.zeros((0, 2)), k)
        assert_parity(g, gpu_run(g))


@pytest.mark.parametrize("sizes", [[1, 1, 1], [31, 32, 33], [64, 65, 1, 96], [33] * 5, [1] * 32, [2] * 33,
                                   [100, 3, 57]])
def test_complete_kpartite(sizes):
    colour, edges = refs.complete_kpartite(sizes)
    g = _graph(colour, edges, len(sizes))
    r = gpu_run(g)
    assert r["stats"]["sweeps"] == 0 and r["alive"].all()
    assert_parity(g, r)


@pytest.mark.parametrize("sizes", [[5, 0, 7], [0, 40, 40, 40], [33, 33, 0]])
def test_empty_class(sizes):
    colour, edges = refs.complete_kpartite(sizes)
    g = _graph(colour, edges, len(sizes))
    r = gpu_run(g)
    assert r["stats"]["sweeps"] == 1 and not r["alive"].any()
    assert_parity(g, r)


def test_k_greater_than_n():
    g = synth.tiny_random(3, 10, 16, 0.9)
    assert_parity(g, gpu_run(g))


def test_large_class_slow_path():
    """Classes of 150 vertices (5 planes) with sparse edges: plane-0 words are
    often empty, so the exact recount over all planes decides."""
    for seed in range(4):
        g = synth.tiny_random(60 + seed, 600, 4, 0.02 + 0.01 * seed, planted=True)
        assert_parity(g, gpu_run(g))


@pytest.mark.parametrize("path", ["bitset", "small", "sparse"])
def test_cascades(path):
    """Sparse graphs that take many sweeps."""
    seen = 0
    for seed in range(12):
        g = synth.tiny_random(700 + seed, 400, 6, 0.06 + 0.01 * (seed % 5), planted=bool(seed % 2))
        orc = assert_parity(g, gpu_run(g, path=path))
        seen = max(seen, orc["sweeps"])
    assert seen >= 3


# ---------------------------------------------------------------------------
# options, reset, limits, input forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("loop", [0, 1, 2])
def test_pass_loops_agree(loop):
    """Host-driven loop, one persistent launch, CUDA-graph while loop."""
    for seed in (42, 43):
        g = synth.tiny_random(seed, 300, 7, 0.12, planted=True)
        assert_parity(g, gpu_run(g, path="bitset", use_graph=loop))
    g = synth.workload("c2", 0.125)
    assert_parity(g, gpu_run(g, path="bitset", use_graph=loop, dense=True))


def test_dense_input_equals_edge_input():
    g = synth.kpartite(500, 9, 0.35, seed=17)
    a = gpu_run(g, dense=True)
    b = gpu_run(g, dense=False)
    assert np.array_equal(a["alive"], b["alive"]) and np.array_equal(a["edges"], b["edges"])
    assert_parity(g, a)


def _pack_bool_rows(mat: np.ndarray, row_words: int) -> np.ndarray:
    """uint64[n, row_words] with bit j % 64 of word j // 64 = mat[i, j]."""
    n = mat.shape[0]
    by = np.packbits(mat, axis=1, bitorder="little")
    out = np.zeros((n, row_words * 8), np.uint8)
    out[:, :by.shape[1]] = by
    return out.view(np.uint64)


@pytest.mark.parametrize("n,k,classes", [(12000, 6, "geometric"), (11777, 37, "uniform"), (515, 3, "geometric"),
                                         (6000, 64, "one large")])
def test_dense_load_fetch_round_trip(n, k, classes):
    """A graph dense enough that the rules delete nothing comes back exactly:
    the upper triangle of the input, mirrored, whatever the lower triangle
    and the diagonal hold, through a padded row stride.  The larger sizes
    move in row chunks overlapped with the packing and unpacking; k = 6 and
    k = 3 put several rounds of a class in one group of the symmetrizer,
    skewed classes leave blocks missing, and one class of 3000 vertices makes
    rows too long for the unpacker's tile form (its row form runs).  Every
    class has enough members that no edge of the 0.9-dense graph fails."""
    rng = np.random.default_rng(n + k)
    if classes == "geometric":
        w = 0.6 ** np.arange(k)
        colour = rng.choice(k, size=n, p=w / w.sum()).astype(np.int32)
    elif classes == "one large":
        colour = np.concatenate([np.zeros(3000, np.int32), rng.integers(1, k, size=n - 3000).astype(np.int32)])
        colour = colour[rng.permutation(n)]
    else:
        colour = rng.integers(0, k, size=n).astype(np.int32)
    upper = np.triu(rng.integers(0, 10, size=(n, n), dtype=np.uint8) < 9, 1)
    upper &= colour[:, None] != colour[None, :]
    garbage = np.tril(rng.integers(0, 2, size=(n, n), dtype=np.uint8) == 1, 0)
    row_words = (n + 63) // 64 + 1
    bits_in = _pack_bool_rows(upper | garbage, row_words)
    del garbage
    full = upper | upper.T
    h = kz.kz_load_graph_dense(n, k, colour, bits_in)
    try:
        kz.kz_kernelize(h)
        alive, bits, st = kz.kz_fetch_kernel_dense(h, n, out_bits=np.zeros((n, row_words), np.uint64))
    finally:
        kz.kz_free_graph(h)
    assert st["sweeps"] == 0 and alive.all()
    assert st["m"] == int(upper.sum()) and st["m_live"] == st["m"]
    assert np.array_equal(bits, _pack_bool_rows(full, row_words))


def test_dense_load_beyond_the_tile_packer():
    """A dense input of more than 49,152 vertices takes the packer's row form
    (its column words no longer fit in shared memory); sparse enough that the
    oracle runs in seconds."""
    rng = np.random.default_rng(50)
    n, k = 50200, 8
    colour = rng.integers(0, k, size=n).astype(np.int32)
    a, b = rng.integers(0, n, size=300000), rng.integers(0, n, size=300000)
    ok = (a != b) & (colour[a] != colour[b])
    edges = np.unique(np.sort(np.stack([a[ok], b[ok]], 1), axis=1), axis=0).astype(np.int32)
    bits = synth.edges_to_bits(n, edges)
    orc = oracle.fixpoint(colour, edges, k)
    h = kz.kz_load_graph_dense(n, k, colour, bits)
    try:
        kz.kz_kernelize(h)
        alive, kept, st = kz.kz_fetch_kernel(h, n)
        assert st["m"] == len(edges)
    finally:
        kz.kz_free_graph(h)
    assert np.array_equal(alive, orc["vlive"]) and np.array_equal(kept, edges[orc["elive"].astype(bool)])
    assert st["sweeps"] == orc["sweeps"]


def test_reset_and_rerun():
    g = synth.tiny_random(8, 250, 6, 0.1, planted=True)
    with kz.KernelGraph.from_synth(g) as kg:
        kg.kernelize()
        a1, e1, s1 = kg.fetch()
        kg.kernelize()               # already a fixpoint: one certifying pass
        a2, e2, s2 = kg.fetch()
        assert s2["sweeps"] == 0 and s2["passes"] == 1
        assert np.array_equal(a1, a2) and np.array_equal(e1, e2)
        kg.reset().kernelize()
        a3, e3, s3 = kg.fetch()
        assert np.array_equal(a1, a3) and np.array_equal(e1, e3) and s3["sweeps"] == s1["sweeps"]
    assert s1["sweeps"] >= 1


def test_sweep_limit():
    g = synth.tiny_random(31, 60, 6, 0.35)
    orc_full = oracle.fixpoint(g.colour, g.edges, 6)
    assert orc_full["sweeps"] >= 2
    r = gpu_run(g, max_sweeps=1)
    assert r["stats"]["status"] == kz.KZ_ERR_LIMIT and r["stats"]["sweeps"] == 1
    orc = oracle.fixpoint(g.colour, g.edges, 6, max_sweeps=1, raise_on_limit=False)
    assert np.array_equal(r["alive"], orc["vlive"])
    assert np.array_equal(r["edges"], g.edges[orc["elive"].astype(bool)])


def test_duplicates():
    g = synth.tiny_random(12, 50, 4, 0.3)
    dup = np.concatenate([g.edges, g.edges[:5, ::-1], g.edges[5:9]])
    with pytest.raises(kz.KzError) as ei:
        kz.kz_load_graph(g.n, g.k, g.colour, dup)
    assert ei.value.status == kz.KZ_ERR_DUPLICATE_EDGE
    with kz.KernelGraph(g.n, g.k, g.colour, edges=dup, flags=kz.KZ_DEDUP) as kg:
        kg.kernelize()
        alive, edges, st = kg.fetch()
        assert st["m"] == len(g.edges)
    orc = oracle.fixpoint(g.colour, g.edges, g.k)
    assert np.array_equal(alive, orc["vlive"]) and np.array_equal(edges, g.edges[orc["elive"].astype(bool)])


@pytest.mark.parametrize("path", ["sparse", "auto"])
def test_device_csr_shapes(path):
    """The CSR is sorted and deduplicated on the device: edge lists given in
    both orientations and shuffled, with repeats (KZ_DEDUP), many isolated
    vertices (more vertices than edges: the rank sort is longer than the edge
    sort) and a hub of high degree, against the oracle on the sparse path."""
    rng = np.random.default_rng(77)
    n, k = 5000, 7
    colour = rng.integers(0, k, size=n).astype(np.int32)
    hub = 0
    others = np.nonzero(colour != colour[hub])[0][:1500]
    e = [np.stack([np.full(len(others), hub), others], 1)]
    a, b = rng.integers(0, 600, size=4000), rng.integers(0, 600, size=4000)
    ok = (a != b) & (colour[a] != colour[b])
    e.append(np.stack([a[ok], b[ok]], 1))
    edges = np.concatenate(e).astype(np.int32)
    canon = np.unique(np.sort(edges, axis=1), axis=0)
    shuffled = edges[rng.permutation(len(edges))]
    flip = rng.random(len(shuffled)) < 0.5
    shuffled[flip] = shuffled[flip][:, ::-1]
    with_repeats = np.concatenate([shuffled, shuffled[:300]])
    with kz.KernelGraph(n, k, colour, edges=with_repeats, flags=kz.KZ_DEDUP) as kg:
        kg.kernelize(path=path)
        alive, kept, st = kg.fetch()
    assert st["m"] == len(canon)
    orc = oracle.fixpoint(colour, canon, k)
    assert np.array_equal(alive, orc["vlive"]) and np.array_equal(kept, canon[orc["elive"].astype(bool)])
    with pytest.raises(kz.KzError) as ei:
        kz.kz_load_graph(n, k, colour, with_repeats)
    assert ei.value.status == kz.KZ_ERR_DUPLICATE_EDGE


def test_dense_illegal_colouring_found_on_device():
    colour = np.array([0, 1, 1], np.int32)
    bits = synth.edges_to_bits(3, np.array([[0, 1], [1, 2]]))
    with pytest.raises(kz.KzError) as ei:
        kz.kz_load_graph_dense(3, 2, colour, bits)
    assert ei.value.status == kz.KZ_ERR_ILLEGAL_COLOURING


def test_fetch_before_kernelize_and_small_buffer():
    g = synth.tiny_random(4, 30, 3, 0.5)
    with kz.KernelGraph.from_synth(g) as kg:
        with pytest.raises(kz.KzError) as ei:
            kg.fetch()
        assert ei.value.status == kz.KZ_ERR_NOT_READY
        kg.kernelize()
        with pytest.raises(kz.KzError) as ei:
            kz.kz_fetch_kernel(kg.h, g.n, cap=0)
        assert ei.value.status == kz.KZ_ERR_BUFFER


# ---------------------------------------------------------------------------
# the workloads, reduced and full
# ---------------------------------------------------------------------------

def test_c1_full():
    g = synth.workload("c1")
    assert_parity(g, gpu_run(g, dense=True))


@pytest.mark.parametrize("scale", [0.0625, 0.125])
def test_c2_reduced(scale):
    g = synth.workload("c2", scale)
    assert_parity(g, gpu_run(g, dense=True))


def test_c5_reduced():
    g = synth.workload("c5", 1 / 32)
    assert_parity(g, gpu_run(g, dense=True))


@pytest.mark.parametrize("path", ["auto", "sparse"])
def test_c3_reduced_cascade(path):
    g = synth.workload("c3", 0.02)
    orc = assert_parity(g, gpu_run(g, path=path))
    assert orc["sweeps"] >= 2


def test_sparse_edge_cases():
    for g in (_graph([], np.zeros((0, 2)), 3), _graph(np.arange(7) % 3, np.zeros((0, 2)), 3)):
        assert_parity(g, gpu_run(g, path="sparse"))
    for sizes in ([1, 1, 1], [31, 32, 33], [5, 0, 7], [2] * 33):
        colour, edges = refs.complete_kpartite(sizes)
        g = _graph(colour, edges, len(sizes))
        assert_parity(g, gpu_run(g, path="sparse"))


def test_sparse_limit():
    g = synth.tiny_random(31, 60, 6, 0.35)
    r = gpu_run(g, path="sparse", max_sweeps=1)
    assert r["stats"]["status"] == kz.KZ_ERR_LIMIT and r["stats"]["sweeps"] == 1
    orc = oracle.fixpoint(g.colour, g.edges, 6, max_sweeps=1, raise_on_limit=False)
    assert np.array_equal(r["alive"], orc["vlive"])
    assert np.array_equal(r["edges"], g.edges[orc["elive"].astype(bool)])


def test_switching_paths_on_one_handle():
    """Each path continues from the state another path left: a sweep limit
    stops one path part-way, the next path finishes the fixpoint."""
    g = synth.tiny_random(77, 500, 6, 0.05, planted=True)
    orc = oracle.fixpoint(g.colour, g.edges, g.k)
    want = g.edges[orc["elive"].astype(bool)]
    for first, second in (("sparse", "bitset"), ("bitset", "sparse"), ("small", "sparse"), ("sparse", "small")):
        with kz.KernelGraph.from_synth(g) as kg:
            kg.kernelize(path=first, max_sweeps=1)
            kg.kernelize(path=second)
            alive, edges, st = kg.fetch()
            assert np.array_equal(alive, orc["vlive"]) and np.array_equal(edges, want), (first, second)
            kg.reset().kernelize(path=second)
            alive, edges, st = kg.fetch()
            assert np.array_equal(edges, want) and st["sweeps"] == orc["sweeps"]


def test_c4_style_batch_members():
    for (n, k, p, planted, seed) in synth.batch_specs(10, 99, n_hi=700):
        g = synth.kpartite(n, k, p, seed, planted=planted)
        assert_parity(g, gpu_run(g, dense=True))


def _sampled_closure(g, alive, bits_out, n_pairs=1500, seed=0):
    """On the GPU's kernel, sampled surviving vertices and edges must pass the
    rules (oracle, one element at a time), and sampled deleted edges of the
    input must not be re-derivable... only survivors are checked here."""
    rng = np.random.default_rng(seed)
    verts = rng.choice(g.n, size=min(g.n, 300), replace=False).astype(np.int32)
    verts = verts[alive[verts] == 1]
    edges = synth.bits_to_edges(bits_out, g.n) if g.n <= 8192 else None
    if edges is None or len(edges) == 0:
        pairs = np.zeros((0, 2), np.int32)
    else:
        pairs = edges[rng.choice(len(edges), size=min(n_pairs, len(edges)), replace=False)]
    iv, ie = oracle.dense_indices(g.colour, bits_out, g.k, verts=verts, pairs=pairs, vlive=alive)
    assert (iv >= g.k - 1).all(), "a surviving vertex fails the vertex rule"
    assert (ie >= g.k - 2).all(), "a surviving edge fails the edge rule"


def test_c2_full_size_sampled():
    """Full 4096-vertex dense workload in the benchmark's configuration: the
    kernel is closed on sampled elements (oracle, one element at a time), and
    no element is deleted, as the fixpoint of a graph with no failing element
    must be."""
    g = synth.workload("c2")
    with kz.KernelGraph.from_synth(g, dense=True) as kg:
        kg.kernelize()
        alive, bits, st = kg.fetch_dense()
    assert st["sweeps"] == 0 and st["passes"] == 1 and st["edge_tests"] == g.m
    assert np.array_equal(bits, g.get_bits()) and alive.all()
    _sampled_closure(g, alive, bits)
    # the same full-size input, sampled elements on the *input* graph
    rng = np.random.default_rng(1)
    e = synth.bits_to_edges(g.get_bits(), g.n)
    pairs = e[rng.choice(len(e), size=2000, replace=False)]
    _, ie = oracle.dense_indices(g.colour, g.get_bits(), g.k, pairs=pairs)
    assert (ie >= g.k - 2).all()


# ---------------------------------------------------------------------------
# whole fixpoint in one CTA, and the batched persistent launch
# ---------------------------------------------------------------------------

def test_small_path_global_mode():
    """A graph too large for shared memory runs the in-CTA kernel on its
    global ping-pong buffers."""
    g = synth.tiny_random(77, 2000, 6, 0.02, planted=True)
    r = gpu_run(g, path="small")
    assert_parity(g, r)


def test_small_path_limit_and_rerun():
    g = synth.tiny_random(31, 60, 6, 0.35)
    r = gpu_run(g, path="small", max_sweeps=1)
    assert r["stats"]["status"] == kz.KZ_ERR_LIMIT and r["stats"]["sweeps"] == 1
    orc = oracle.fixpoint(g.colour, g.edges, 6, max_sweeps=1, raise_on_limit=False)
    assert np.array_equal(r["alive"], orc["vlive"])
    with kz.KernelGraph.from_synth(g) as kg:
        kg.kernelize(path="small")
        a1, e1, s1 = kg.fetch()
        kg.kernelize(path="bitset")      # continues from the in-CTA result
        a2, e2, s2 = kg.fetch()
        assert s2["sweeps"] == 0 and np.array_equal(a1, a2) and np.array_equal(e1, e2)


def _batch_graphs():
    gs = [synth.kpartite(n, k, p, seed, planted=pl) for (n, k, p, pl, seed) in synth.batch_specs(40, 4242, n_hi=1500)]
    gs += [synth.tiny_random(900 + i, 300 + 40 * i, 5 + i, 0.08, planted=bool(i % 2)) for i in range(8)]
    gs += [synth.tiny_random(950, 2000, 6, 0.02, planted=True)]     # global mode inside the batch
    gs += [synth.tiny_random(951, 120, 40, 0.9, planted=True)]      # k > 32: its own KMAX group
    return gs


@pytest.mark.parametrize("path,batch", [("auto", "concurrent"), ("auto", "sequential"), ("auto", "fused"),
                                        ("bitset", "concurrent"), ("small", "concurrent"), ("small", "fused"),
                                        ("sparse", "concurrent")])
def test_batch_matches_oracle(path, batch):
    gs = _batch_graphs()
    if path == "sparse":
        gs = gs[:20]
    handles = [kz.KernelGraph.from_synth(g, dense=False) for g in gs]
    try:
        kz.kz_kernelize_batch([h.h for h in handles], kz.kz_default_options(path=path, batch=batch))
        for g, h in zip(gs, handles):
            alive, edges, stats = h.fetch()
            dv, de, vs = h.trace()
            res = dict(alive=alive, edges=edges, stats=stats, dv=dv[:stats["sweeps"]], de=de[:stats["sweeps"]],
                       v_sweep=vs)
            assert_parity(g, res)
    finally:
        for h in handles:
            h.close()


@pytest.mark.parametrize("path,batch", [("auto", "concurrent"), ("auto", "fused"), ("small", "fused")])
def test_batch_c4_reduced(path, batch):
    """The batched workload's recipe at reduced size (64 graphs, n <= 1024)."""
    specs = synth.batch_specs(64, synth.SEED_BASE + 4, n_hi=1024)
    gs = [synth.kpartite(n, k, p, seed, planted=pl) for (n, k, p, pl, seed) in specs]
    handles = [kz.KernelGraph.from_synth(g) for g in gs]
    try:
        kz.kz_kernelize_batch([h.h for h in handles], kz.kz_default_options(path=path, batch=batch))
        for g, h in zip(gs, handles):
            alive, edges, stats = h.fetch()
            orc = oracle.fixpoint(g.colour, g.get_edges(), g.k)
            assert np.array_equal(alive, orc["vlive"])
            assert np.array_equal(edges, g.get_edges()[orc["elive"].astype(bool)])
            assert stats["sweeps"] == orc["sweeps"] and stats["edge_tests"] == orc["tests"]
    finally:
        for h in handles:
            h.close()


def test_batch_limit_and_repeat():
    """A batch run twice without reset certifies in one pass per graph; a
    sweep limit applies per graph."""
    gs = [synth.tiny_random(1300 + i, 200, 6, 0.1, planted=True) for i in range(6)]
    handles = [kz.KernelGraph.from_synth(g) for g in gs]
    try:
        hs = [h.h for h in handles]
        kz.kz_kernelize_batch(hs, kz.kz_default_options(max_sweeps=1))
        for g, h in zip(gs, handles):
            alive, edges, st = h.fetch(allow=(kz.KZ_OK, kz.KZ_ERR_LIMIT))
            orc = oracle.fixpoint(g.colour, g.edges, g.k, max_sweeps=1, raise_on_limit=False)
            assert np.array_equal(alive, orc["vlive"]) and st["sweeps"] == orc["sweeps"]
        for h in handles:
            h.reset()
        kz.kz_kernelize_batch(hs)
        kz.kz_kernelize_batch(hs)
        for h in handles:
            st = h.stats()
            assert st["sweeps"] == 0 and st["passes"] == 1
        with pytest.raises(kz.KzError):  # a fused batch has no multi-CTA per-graph form
            kz.kz_kernelize_batch(hs, kz.kz_default_options(path="bitset", batch="fused"))
    finally:
        for h in handles:
            h.close()


def test_fused_batch_replays_plans_and_limits():
    """The fused batch replays its captured launch on repeated calls, builds a
    new plan when the set of graphs changes, gives large graphs multi-CTA
    groups and applies a sweep limit per graph; every graph matches the
    oracle each time."""
    gs = [synth.kpartite(3000, 12, 0.5, 61, planted=True),                      # a multi-CTA group
          synth.kpartite(2500, 20, 0.35, 62, planted=False)]
    gs += [synth.tiny_random(1400 + i, 150 + 60 * i, 5 + (i % 4), 0.1, planted=bool(i % 2)) for i in range(10)]
    orcs = [oracle.fixpoint(g.colour, g.get_edges(), g.k) for g in gs]
    handles = [kz.KernelGraph.from_synth(g, dense=True) for g in gs]
    fused = kz.kz_default_options(batch="fused")

    def check(sub, limit=0):
        for i in sub:
            alive, edges, st = handles[i].fetch(allow=(kz.KZ_OK, kz.KZ_ERR_LIMIT))
            orc = orcs[i] if not limit else oracle.fixpoint(gs[i].colour, gs[i].get_edges(), gs[i].k,
                                                            max_sweeps=limit, raise_on_limit=False)
            assert np.array_equal(alive, orc["vlive"]), i
            assert np.array_equal(edges, gs[i].get_edges()[orc["elive"].astype(bool)]), i
            assert st["sweeps"] == orc["sweeps"], i
            if not limit:
                assert st["passes"] == orc["passes"] and st["edge_tests"] == orc["tests"], i

    try:
        every = list(range(len(gs)))
        for _ in range(3):
            for h in handles:
                h.reset()
            kz.kz_kernelize_batch([h.h for h in handles], fused)
            check(every)
        sub = every[::2]
        for i in sub:
            handles[i].reset()
        kz.kz_kernelize_batch([handles[i].h for i in sub], fused)
        check(sub)
        for h in handles:
            h.reset()
        kz.kz_kernelize_batch([h.h for h in handles], kz.kz_default_options(batch="fused", max_sweeps=1))
        check(every, limit=1)
    finally:
        for h in handles:
            h.close()


def test_fused_batch_groups_larger_than_their_work():
    """Groups of many CTAs on graphs with only a few work items per pass: most
    members of a group then have no item at all and may join late.  The
    group's continue decision is taken at its barrier, so every member leaves
    on the same pass; every graph matches the oracle."""
    gs = [synth.tiny_random(1500 + i, 40 + 17 * i, 4 + (i % 5), 0.15 + 0.05 * (i % 4), planted=bool(i % 2))
          for i in range(16)]
    handles = [kz.KernelGraph.from_synth(g, dense=True) for g in gs]
    try:
        for spread, ipw, group in ((1e6, 1, 64), (1e6, 16, 456), (0, 0, 0)):
            kz.kz_set_batch_tuning(spread, ipw, group)
            for h in handles:
                h.reset()
            kz.kz_kernelize_batch([h.h for h in handles], kz.kz_default_options(batch="fused"))
            for g, h in zip(gs, handles):
                alive, edges, st = h.fetch()
                orc = oracle.fixpoint(g.colour, g.get_edges(), g.k)
                assert np.array_equal(alive, orc["vlive"]) and st["sweeps"] == orc["sweeps"], (spread, g.name)
                assert np.array_equal(edges, g.get_edges()[orc["elive"].astype(bool)]), (spread, g.name)
    finally:
        kz.kz_set_batch_tuning(0, 0, 0)
        for h in handles:
            h.close()


# ---------------------------------------------------------------------------
# multi-CTA sweep: equal-cost warp ranges and change-tagged writes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("loop", [0, 1, 2])
def test_warp_ranges_multi_sweep(loop):
    """Graphs with thousands of units (several per warp, ranges crossing block
    boundaries) that take several sweeps: only words that changed in this or
    the previous sweep are rewritten, so every sweep checks the protocol."""
    for (n, k, p, seed) in ((3000, 10, 0.1, 5), (2500, 8, 0.07, 5)):
        g = synth.tiny_random(seed, n, k, p, planted=True)
        orc = assert_parity(g, gpu_run(g, path="bitset", use_graph=loop))
        assert orc["sweeps"] >= 3


def test_sweep_by_sweep_continuation():
    """One sweep per call, continued on the same handle until the fixpoint:
    the state after each call equals the oracle's after that many sweeps."""
    g = synth.tiny_random(5, 2500, 8, 0.07, planted=True)
    edges = g.get_edges()
    orc = oracle.fixpoint(g.colour, edges, g.k)
    with kz.KernelGraph.from_synth(g) as kg:
        for s in range(1, orc["sweeps"] + 2):
            kg.kernelize(path="bitset", max_sweeps=1)
            alive, got, st = kg.fetch(allow=(kz.KZ_OK, kz.KZ_ERR_LIMIT))
            want = oracle.fixpoint(g.colour, edges, g.k, max_sweeps=s, raise_on_limit=False)
            assert np.array_equal(alive, want["vlive"]), s
            assert np.array_equal(got, edges[want["elive"].astype(bool)]), s
        assert st["status"] == kz.KZ_OK and st["sweeps"] == 0


@pytest.mark.parametrize("first", ["small", "tensor", "sparse"])
def test_bitset_after_other_path(first):
    """Another path writes the rows part-way (one sweep); the multi-CTA sweep
    then writes every word once and finishes the fixpoint."""
    g = synth.tiny_random(5, 2500, 8, 0.07, planted=True)
    edges = g.get_edges()
    orc = oracle.fixpoint(g.colour, edges, g.k)
    with kz.KernelGraph.from_synth(g) as kg:
        kg.kernelize(path="bitset")          # rows in step after a converged run
        kg.reset()
        kg.kernelize(path=first, max_sweeps=1)
        kg.kernelize(path="bitset")
        alive, got, st = kg.fetch()
    assert np.array_equal(alive, orc["vlive"])
    assert np.array_equal(got, edges[orc["elive"].astype(bool)])


def _two_density_graph(seed, n, k, n_dense, p_dense, p_sparse):
    """k-partite graph whose first n_dense classes are joined densely and the
    rest sparsely: dense overall (the half-word plane-0 test is taken) while
    many pairs need the recount and the sparse classes cascade."""
    rng = np.random.default_rng(seed)
    colour = np.sort(rng.integers(0, k, size=n)).astype(np.int32)
    iu, iv = np.triu_indices(n, 1)
    cu, cv = colour[iu], colour[iv]
    p = np.where((cu < n_dense) & (cv < n_dense), p_dense, p_sparse)
    keep = (cu != cv) & (rng.random(len(iu)) < p)
    edges = np.stack([iu[keep], iv[keep]], axis=1).astype(np.int32)
    return synth.Graph(n=n, k=k, colour=colour, edges=synth.canonical_edges(edges), name="two-density")


@pytest.mark.parametrize("loop,plane0", [(0, 0), (1, 0), (1, 1), (2, 2), (1, 3), (2, 3)])
def test_half_word_plane0_with_recounts(loop, plane0):
    """Densities 0.65 to 0.95: the half-word test with and without the
    whole-block fold, blocks that fall back to per-pair results."""
    for seed, (n, k, nd, pd, ps) in enumerate(((1200, 12, 10, 0.95, 0.05), (900, 8, 6, 0.97, 0.3),
                                               (700, 20, 18, 0.9, 0.1), (800, 24, 23, 0.95, 0.05),
                                               (1500, 16, 14, 0.99, 0.4))):
        g = _two_density_graph(seed, n, k, nd, pd, ps)
        cross = (n * n - np.sum(np.bincount(g.colour, minlength=k) ** 2)) / 2
        assert len(g.edges) >= 0.6 * cross  # dense
        assert_parity(g, gpu_run(g, path="bitset", use_graph=loop, plane0=plane0))


@pytest.mark.parametrize("plane0", [1, 2, 3])
def test_forced_plane0_forms(plane0):
    """Every first test on graphs of any density, sparse ones included (the
    half-word form then sends most pairs to the recount; the two-plane form
    falls back to full words where a class has one block or k > 32)."""
    for (n, k, p, seed) in ((3000, 10, 0.1, 5), (600, 7, 0.5, 6), (400, 33, 0.9, 7), (1000, 64, 0.97, 8),
                            (1100, 29, 0.35, 9), (1500, 6, 0.3, 10)):
        g = synth.tiny_random(seed, n, k, p, planted=True)
        assert_parity(g, gpu_run(g, path="bitset", plane0=plane0))


# ---------------------------------------------------------------------------
# CSR path with incremental support counts (schedule SUPPORT)
# ---------------------------------------------------------------------------

def assert_support_parity(g, res, max_sweeps=0):
    """Same Jacobi sweeps as the oracle, fewer or equal tests."""
    edges = g.get_edges()
    orc = oracle.fixpoint(g.colour, edges, g.k, max_sweeps=max_sweeps, raise_on_limit=False)
    st = res["stats"]
    assert np.array_equal(res["alive"], orc["vlive"]), "surviving vertices differ"
    assert np.array_equal(res["edges"], edges[orc["elive"].astype(bool)]), "surviving edges differ"
    assert st["sweeps"] == orc["sweeps"]
    assert np.array_equal(res["dv"], orc["dv"]) and np.array_equal(res["de"], orc["de"])
    assert np.array_equal(res["v_sweep"], orc["v_sweep"])
    if orc["status"] == 0:  # under a sweep limit the refused pass is counted differently
        assert st["passes"] == orc["passes"]
        assert 0 < st["edge_tests"] <= orc["tests"] or orc["tests"] == 0
    return orc


def test_support_schedule_cascades():
    seen = 0
    for seed in range(12):
        g = synth.tiny_random(700 + seed, 400, 6, 0.06 + 0.01 * (seed % 5), planted=bool(seed % 2))
        orc = assert_support_parity(g, gpu_run(g, schedule="support"))
        seen = max(seen, orc["sweeps"])
    assert seen >= 3
    for case in _tiny_cases()[:30]:
        (i, n, k, p, planted) = case
        g = synth.tiny_random(i, n, k, p, planted=planted)
        assert_support_parity(g, gpu_run(g, schedule="support"))


def test_support_schedule_c3_reduced_and_dense():
    g = synth.workload("c3", 0.02)
    orc = assert_support_parity(g, gpu_run(g, schedule="support"))
    assert orc["sweeps"] >= 2
    for seed, (n, k, nd, pd, ps) in enumerate(((1200, 12, 10, 0.95, 0.05), (700, 20, 18, 0.9, 0.1))):
        g = _two_density_graph(seed, n, k, nd, pd, ps)
        assert_support_parity(g, gpu_run(g, schedule="support"))


def test_support_schedule_limit_rerun_and_switch():
    g = synth.tiny_random(5, 2500, 8, 0.07, planted=True)
    edges = g.get_edges()
    orc = oracle.fixpoint(g.colour, edges, g.k)
    r = gpu_run(g, schedule="support", max_sweeps=1)
    assert r["stats"]["status"] == kz.KZ_ERR_LIMIT
    assert_support_parity(g, r, max_sweeps=1)
    with kz.KernelGraph.from_synth(g, dense=False) as kg:
        for s in range(1, orc["sweeps"] + 2):   # one sweep per call, continued on the handle
            kg.kernelize(schedule="support", max_sweeps=1)
            alive, got, st = kg.fetch(allow=(kz.KZ_OK, kz.KZ_ERR_LIMIT))
            want = oracle.fixpoint(g.colour, edges, g.k, max_sweeps=s, raise_on_limit=False)
            assert np.array_equal(alive, want["vlive"]) and np.array_equal(got, edges[want["elive"].astype(bool)])
        kg.reset()
        kg.kernelize(path="bitset", max_sweeps=1)      # another path part-way, then the support schedule
        kg.kernelize(schedule="support")
        alive, got, st = kg.fetch()
        assert np.array_equal(alive, orc["vlive"]) and np.array_equal(got, edges[orc["elive"].astype(bool)])
    with kz.KernelGraph.from_synth(g, dense=True) as kg:   # no CSR state: the bitset rows' re-check sweeps
        kg.kernelize(schedule="support")
        alive, got, st = kg.fetch()
        assert np.array_equal(alive, orc["vlive"]) and np.array_equal(got, edges[orc["elive"].astype(bool)])
        assert st["sweeps"] == orc["sweeps"] and st["passes"] == orc["passes"]
    with kz.KernelGraph.from_synth(g) as kg:
        with pytest.raises(kz.KzError):
            kg.kernelize(schedule="support", path="small")


# ---------------------------------------------------------------------------
# schedule SUPPORT on the bitset rows (re-check sweeps)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("path", ["bitset", "tensor", "dense-auto"])
def test_dense_support_matches_jacobi(path):
    """The re-check sweeps are the oracle's Jacobi sweeps: same survivors,
    sweeps, per-sweep deletions and vertex deletion sweeps, no more tests."""
    seen = 0
    cases = [synth.tiny_random(900 + s, 400, 6, 0.06 + 0.01 * (s % 5), planted=bool(s % 2)) for s in range(6)]
    cases += [synth.kpartite(1500, 12, 0.3, seed=3), synth.kpartite(2100, 20, 0.45, seed=4),
              _two_density_graph(7, 1200, 12, 10, 0.95, 0.05)]
    for g in cases:
        if path == "dense-auto":
            res = gpu_run(g, dense=True, schedule="support")
        else:
            res = gpu_run(g, schedule="support", path=path)
        orc = assert_support_parity(g, res)
        seen = max(seen, orc["sweeps"])
    assert seen >= 3


def test_dense_support_refusals():
    """The re-check sweeps follow the thesis's thresholds only and run on their
    own: a clique size below the colour count, dominance rounds and the in-CTA
    path are refused, and the handle stays usable."""
    g = synth.kpartite(600, 8, 0.4, seed=21)
    edges = g.get_edges()
    orc = oracle.fixpoint(g.colour, edges, g.k)
    with kz.KernelGraph.from_synth(g, dense=True) as kg:
        for opts in ({"clique_k": g.k - 1}, {"dominance": 1}, {"path": "small"}, {"path": "sparse"}):
            with pytest.raises(kz.KzError) as ei:
                kg.kernelize(schedule="support", **opts)
            assert ei.value.status in (kz.KZ_ERR_UNSUPPORTED, kz.KZ_ERR_ARG), (opts, ei.value.status)
        kg.kernelize(schedule="support")
        alive, kept, st = kg.fetch()
    assert np.array_equal(alive, orc["vlive"]) and np.array_equal(kept, edges[orc["elive"].astype(bool)])


def test_dense_support_tiny_cases():
    """Every tiny case (n from 1, k from 1 to 64, all densities) on the bitset
    rows' re-check sweeps, against the oracle's Jacobi sweeps."""
    for (i, n, k, p, planted) in _tiny_cases():
        g = synth.tiny_random(i, n, k, p, planted=planted)
        assert_support_parity(g, gpu_run(g, dense=True, schedule="support"))


def test_dense_support_limits_and_continuation():
    g = synth.kpartite(1800, 12, 0.2, seed=11)
    edges = g.get_edges()
    orc = oracle.fixpoint(g.colour, edges, g.k)
    assert orc["sweeps"] >= 3
    with kz.KernelGraph.from_synth(g, dense=True) as kg:
        for s in range(1, orc["sweeps"] + 2):   # one sweep per call, continued on the handle
            kg.kernelize(schedule="support", max_sweeps=1)
            alive, got, st = kg.fetch(allow=(kz.KZ_OK, kz.KZ_ERR_LIMIT))
            want = oracle.fixpoint(g.colour, edges, g.k, max_sweeps=s, raise_on_limit=False)
            assert np.array_equal(alive, want["vlive"]) and np.array_equal(got, edges[want["elive"].astype(bool)])
        kg.reset()
        kg.kernelize(schedule="support", max_sweeps=2)
        alive, got, st = kg.fetch(allow=(kz.KZ_ERR_LIMIT,))
        want = oracle.fixpoint(g.colour, edges, g.k, max_sweeps=2, raise_on_limit=False)
        assert st["sweeps"] == 2 and np.array_equal(got, edges[want["elive"].astype(bool)])
        kg.kernelize()                            # plain sweeps finish from there
        alive, got, st = kg.fetch()
        assert np.array_equal(alive, orc["vlive"]) and np.array_equal(got, edges[orc["elive"].astype(bool)])
