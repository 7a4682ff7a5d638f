"""The pins that fix the oracle's result, written as functions of an oracle
instance so that the same pins can be run against deliberately broken
builds of the oracle (``test_oracle_mutants.py``).

Each pin returns None when it holds, else a short message.
"""
from __future__ import annotations

import numpy as np

from paper_2212_00574_gb300 import synth
from tests import refs


def _graph(seed, n, k, p, planted=False):
    g = synth.tiny_random(seed, n, k, p, planted=planted)
    return g.colour, g.edges


def pin_fig8(orc):
    """Section 4.2 worked example: the thesis prints the colour index of
    vertices a and d and of edges {a,d} and {h,i}."""
    fx = refs.load_fig8()
    edges = [tuple(e) for e in fx["edges"].tolist()]
    verts = [v for v, _ in fx["expect_vertex"]]
    eids = []
    for u, v, _ in fx["expect_edge"]:
        eids.append(edges.index((u, v)) if (u, v) in edges else edges.index((v, u)))
    got_v, got_e = orc.indices(fx["colour"], fx["edges"], fx["k"], verts=verts, edge_ids=eids)
    want_v = [x for _, x in fx["expect_vertex"]]
    want_e = [x for _, _, x in fx["expect_edge"]]
    if list(got_v) != want_v or list(got_e) != want_e:
        return f"fig8: vertex {list(got_v)} vs {want_v}, edge {list(got_e)} vs {want_e}"
    return None


def pin_brute_force(orc, cases=40, seed0=1000):
    """Exact greatest fixpoint by enumerating edge subsets (m <= 14)."""
    rng = np.random.default_rng(seed0)
    done = 0
    tries = 0
    while done < cases and tries < 20 * cases:
        tries += 1
        n = int(rng.integers(3, 9))
        k = int(rng.integers(2, 6))
        p = float(rng.uniform(0.3, 0.9))
        colour, edges = _graph(seed0 + tries, n, k, p, planted=bool(rng.integers(0, 2)) and n >= k)
        if len(edges) > 14:
            continue
        done += 1
        vb, eb = refs.brute_force_gfp(n, k, colour, edges)
        r = orc.fixpoint(colour, edges, k)
        if not (np.array_equal(r["vlive"].astype(bool), vb) and np.array_equal(r["elive"].astype(bool), eb)):
            return f"brute force mismatch n={n} k={k} m={len(edges)} seed={seed0 + tries}"
    return None


def pin_k3_triangles(orc, cases=12):
    """k = 3: the kernel is the union of the triangles of G."""
    for s in range(cases):
        n = 20 + 7 * s
        colour, edges = _graph(7000 + s, n, 3, 0.08 + 0.02 * s)
        vt, et = refs.triangle_closed_form(n, edges)
        r = orc.fixpoint(colour, edges, 3)
        if not (np.array_equal(r["vlive"].astype(bool), vt) and np.array_equal(r["elive"].astype(bool), et)):
            return f"k=3 triangle closed form mismatch (case {s})"
    return None


def pin_k2(orc, cases=10):
    """k = 2: only isolated vertices go, in at most one sweep; every edge stays."""
    for s in range(cases):
        n = 10 + 5 * s
        colour, edges = _graph(8000 + s, n, 2, 0.05)
        deg = np.zeros(n, int)
        for u, v in edges:
            deg[u] += 1
            deg[v] += 1
        r = orc.fixpoint(colour, edges, 2)
        if not np.array_equal(r["vlive"].astype(bool), deg > 0):
            return "k=2 vertex survivors wrong"
        if not r["elive"].all() or r["sweeps"] > 1:
            return "k=2 edges deleted or more than one sweep"
    return None


def pin_k1(orc):
    """k = 1: no rule can fire."""
    colour = np.zeros(9, np.int32)
    r = orc.fixpoint(colour, np.zeros((0, 2), np.int32), 1)
    if not r["vlive"].all() or r["sweeps"] != 0:
        return "k=1 deleted something"
    return None


def pin_complete_kpartite(orc):
    """Complete k-partite with non-empty classes: nothing is deleted."""
    for sizes in ([1, 1, 1], [2, 3, 1, 2], [3, 3, 3, 3, 3], [1, 4, 2, 2, 1, 3]):
        colour, edges = refs.complete_kpartite(sizes)
        r = orc.fixpoint(colour, edges, len(sizes))
        if not r["vlive"].all() or not r["elive"].all() or r["sweeps"] != 0:
            return f"complete k-partite {sizes} lost elements"
    return None


def pin_empty_class(orc):
    """A colour class with no vertex: no vertex can see k-1 other colours, so
    everything goes in the first sweep."""
    for sizes in ([2, 3, 0, 2], [0, 4, 4], [3, 3, 3, 0]):
        colour, edges = refs.complete_kpartite(sizes)
        r = orc.fixpoint(colour, edges, len(sizes))
        if r["vlive"].any() or r["elive"].any() or r["sweeps"] != 1:
            return f"empty class {sizes}: survivors or sweeps={r['sweeps']}"
    return None


def pin_planted_isolated(orc):
    """A planted k-clique plus isolated vertices: exactly the clique survives."""
    rng = np.random.default_rng(5)
    for k in (3, 5, 8):
        n = 40
        colour = rng.integers(0, k, n).astype(np.int32)
        colour[:k] = np.arange(k)          # vertices 0..k-1 carry the clique
        picks = list(range(k))
        edges = synth.canonical_edges(np.array([(a, b) for i, a in enumerate(picks) for b in picks[i + 1:]]))
        r = orc.fixpoint(colour, edges, k)
        want = np.zeros(n, bool)
        want[picks] = True
        if not np.array_equal(r["vlive"].astype(bool), want) or not r["elive"].all():
            return f"planted {k}-clique with isolated noise: wrong survivors"
    return None


def pin_clique_survival(orc, cases=25):
    """No vertex or edge of a k-clique is ever deleted (Section 4.2 remarks),
    checked against exhaustive enumeration on graphs up to 40 vertices; and
    graphs with no k-clique whose kernel is empty are consistent with it."""
    rng = np.random.default_rng(77)
    for s in range(cases):
        n = int(rng.integers(8, 41))
        k = int(rng.integers(3, 7))
        p = float(rng.uniform(0.4, 0.95))
        colour, edges = _graph(9000 + s, n, k, p, planted=(s % 2 == 0))
        cl = refs.k_cliques(n, k, colour, edges)
        r = orc.fixpoint(colour, edges, k)
        eid = {tuple(e): i for i, e in enumerate(edges.tolist())}
        for q in cl:
            if not all(r["vlive"][v] for v in q):
                return f"clique vertex deleted (case {s})"
            for i in range(len(q)):
                for j in range(i + 1, len(q)):
                    if not r["elive"][eid[(q[i], q[j])]]:
                        return f"clique edge deleted (case {s})"
    return None


def pin_order_independence(orc, cases=12):
    """Random-order Gauss-Seidel and random-subset schedules reach the same
    survivors (the greatest fixpoint is unique)."""
    rng = np.random.default_rng(123)
    for s in range(cases):
        n = int(rng.integers(10, 50))
        k = int(rng.integers(3, 8))
        p = float(rng.uniform(0.2, 0.7))
        colour, edges = _graph(11000 + s, n, k, p, planted=(s % 3 == 0))
        r = orc.fixpoint(colour, edges, k)
        for mode in ("shuffled", "subset"):
            vl, el = refs.chaotic_fixpoint(n, k, colour, edges, rng, mode)
            if not (np.array_equal(vl, r["vlive"].astype(bool)) and np.array_equal(el, r["elive"].astype(bool))):
                return f"order dependence ({mode}, case {s})"
    return None


def pin_certificate(orc, cases=20):
    """The Jacobi trace deletes, in each sweep, exactly what fails on that
    sweep's snapshot, and ends closed.  Includes cascading graphs."""
    rng = np.random.default_rng(321)
    multi = 0
    for s in range(cases):
        n = int(rng.integers(10, 60))
        k = int(rng.integers(3, 9))
        p = float(rng.uniform(0.2, 0.8))
        colour, edges = _graph(12000 + s, n, k, p, planted=(s % 2 == 0))
        r = orc.fixpoint(colour, edges, k)
        msg = refs.check_certificate(n, k, colour, edges, r["v_sweep"], r["e_rule_sweep"], r["sweeps"])
        if msg:
            return f"certificate (case {s}): {msg}"
        if len(r["dv"]) != r["sweeps"] or any(r["dv"][t] != int(np.sum(r["v_sweep"] == t + 1)) for t in range(r["sweeps"])):
            return "per-sweep vertex counts disagree with the trace"
        if any(r["de"][t] != int(np.sum(r["e_rule_sweep"] == t + 1)) for t in range(r["sweeps"])):
            return "per-sweep edge counts disagree with the trace"
        multi += r["sweeps"] >= 2
    if multi == 0:
        return "no multi-sweep case exercised"
    return None


def pin_incident_edges_fail(orc, cases=20):
    """In every sweep, each live edge at a deleted vertex also fails the edge
    rule on the same snapshot: if v misses colour c, no neighbour of v has
    colour c, so no common neighbour of v and u does either (and c differs
    from col(u) because u is a neighbour of v)."""
    rng = np.random.default_rng(99)
    for s in range(cases):
        n = int(rng.integers(10, 60))
        k = int(rng.integers(2, 9))
        colour, edges = _graph(13000 + s, n, k, float(rng.uniform(0.1, 0.6)))
        r = orc.fixpoint(colour, edges, k)
        vs, es = r["v_sweep"], r["e_rule_sweep"]
        for i, (u, v) in enumerate(edges):
            for x in (u, v):
                t = vs[x]
                if t == 0:
                    continue
                other = v if x == u else u
                died_before = (0 < es[i] < t) or (0 < vs[other] < t)
                if not died_before and es[i] != t:
                    return f"edge {i} at vertex {x} deleted in sweep {t} did not fail the edge rule"
    return None


def pin_validation(orc):
    """Illegal inputs are rejected (Definition 4.2.1 needs a legal colouring)."""
    from oracle import OracleError
    bad = [
        (np.array([0, 0], np.int32), np.array([[0, 1]], np.int32), 2),   # same colour
        (np.array([0, 1], np.int32), np.array([[0, 0]], np.int32), 2),   # self loop
        (np.array([0, 2], np.int32), np.array([[0, 1]], np.int32), 2),   # colour range
        (np.array([0, 1], np.int32), np.array([[0, 5]], np.int32), 2),   # vertex range
    ]
    for colour, edges, k in bad:
        try:
            orc.fixpoint(colour, edges, k)
        except OracleError:
            continue
        return "illegal input accepted"
    return None


def pin_brute_force_q(orc, cases=30, seed0=3000):
    """Clique size q below the colour count k (thresholds q-1 and q-2, Section
    4.2 Remarks): exact greatest fixpoint by enumerating edge subsets."""
    rng = np.random.default_rng(seed0)
    done = tries = 0
    while done < cases and tries < 20 * cases:
        tries += 1
        n = int(rng.integers(3, 9))
        k = int(rng.integers(3, 7))
        q = int(rng.integers(1, k))
        p = float(rng.uniform(0.3, 0.9))
        colour, edges = _graph(seed0 + tries, n, k, p, planted=bool(rng.integers(0, 2)) and n >= k)
        if len(edges) > 14:
            continue
        done += 1
        vb, eb = refs.brute_force_gfp(n, k, colour, edges, q=q)
        r = orc.fixpoint(colour, edges, k, clique_k=q)
        if not (np.array_equal(r["vlive"].astype(bool), vb) and np.array_equal(r["elive"].astype(bool), eb)):
            return f"brute force mismatch n={n} k={k} q={q} m={len(edges)} seed={seed0 + tries}"
    return None


def pin_q_cliques_and_order(orc, cases=12):
    """Clique size q < k: every q-clique (any q colours) survives; random
    Gauss-Seidel and random-subset schedules reach the same survivors; and
    the kernel only grows as q falls (each threshold is lower)."""
    rng = np.random.default_rng(4321)
    for s in range(cases):
        n = int(rng.integers(10, 36))
        k = int(rng.integers(4, 8))
        p = float(rng.uniform(0.25, 0.7))
        colour, edges = _graph(13000 + s, n, k, p, planted=(s % 2 == 0))
        eid = {tuple(e): i for i, e in enumerate(edges.tolist())}
        prev = None
        for q in range(k, 0, -1):
            r = orc.fixpoint(colour, edges, k, clique_k=q)
            vl, el = r["vlive"].astype(bool), r["elive"].astype(bool)
            if prev is not None and not (np.all(vl >= prev[0]) and np.all(el >= prev[1])):
                return f"kernel shrank as q fell to {q} (case {s})"
            prev = (vl, el)
            if q >= 3:
                for cl in refs.q_cliques(n, q, colour, edges):
                    if not all(vl[v] for v in cl) or not all(
                            el[eid[(cl[i], cl[j])]] for i in range(q) for j in range(i + 1, q)):
                        return f"{q}-clique lost with k={k} (case {s})"
            if q in (k - 1, 2 + (k - 1) // 2):
                for mode in ("shuffled", "subset"):
                    cv, ce = refs.chaotic_fixpoint(n, k, colour, edges, rng, mode, q=q)
                    if not (np.array_equal(cv, vl) and np.array_equal(ce, el)):
                        return f"order dependence at q={q} ({mode}, case {s})"
    return None


def _live_nbrs(n, edges, vlive, elive):
    nb = [set() for _ in range(n)]
    for i, (u, v) in enumerate(np.asarray(edges).tolist()):
        if elive[i]:
            nb[u].add(v)
            nb[v].add(u)
    return nb


def pin_dominance_examples(orc):
    """Definition 4.3.1 on hand-made graphs.  (1) Twins: a path a-c-b with a,
    b of colour 0 and c of colour 1 (k = 2): N(a) = N(b) = {c}; of two
    vertices with equal neighbourhoods only the smaller key (colour, id)
    goes, so a (id 0) is deleted and b, c and their edge stay.  (2) Strict
    subsets: k = 3, a and b of colour 0, c and d of colour 1, e of colour 2,
    edges a-c, a-e, c-e, b-c, b-d, b-e, d-e.  N(a) = {c, e} lies inside
    N(b) = {c, d, e} and N(d) = {b, e} inside N(c) = {a, b, e}, so a and d
    go in one round; the triangle b-c-e remains, and nothing in it is
    dominated (its vertices are pairwise adjacent)."""
    r = orc.fixpoint_dominance(np.array([0, 0, 1], np.int32), np.array([[0, 2], [1, 2]], np.int32), 2)
    if r["vlive"].tolist() != [0, 1, 1] or r["elive"].tolist() != [0, 1] or r["rounds"] != 1:
        return f"twins: {r['vlive'].tolist()} {r['elive'].tolist()} rounds {r['rounds']}"
    colour = np.array([0, 0, 1, 1, 2], np.int32)
    edges = np.array([[0, 2], [0, 4], [2, 4], [1, 2], [1, 3], [1, 4], [3, 4]], np.int32)
    r = orc.fixpoint_dominance(colour, edges, 3)
    if r["vlive"].tolist() != [0, 1, 1, 0, 1] or r["elive"].tolist() != [0, 0, 1, 1, 0, 1, 0] or \
            r["dominated"] != 2 or r["rounds"] != 1:
        return f"strict subset: {r['vlive'].tolist()} {r['elive'].tolist()} dominated {r['dominated']}"
    # (3) No edges, q = 2: the vertex rule removes every vertex (it needs one
    # neighbour) before dominance could keep the largest of the equal twins.
    r = orc.fixpoint_dominance(np.array([0, 1, 2], np.int32), np.zeros((0, 2), np.int32), 3, clique_k=2)
    if r["vlive"].tolist() != [0, 0, 0] or r["rounds"] != 0:
        return f"edgeless q=2: {r['vlive'].tolist()} rounds {r['rounds']}"
    return None


def pin_dominance_keeps_cliques(orc, cases=16):
    """Vertex dominance keeps the clique number: a q-clique exists in the
    graph exactly when one exists in the result (checked by exhaustive
    enumeration), and the result is closed: no live vertex is dominated (two
    with equal neighbourhoods are allowed only when neither would go) and no
    element fails a colour-index rule."""
    rng = np.random.default_rng(909)
    for s in range(cases):
        n = int(rng.integers(8, 28))
        k = int(rng.integers(3, 6))
        p = float(rng.uniform(0.35, 0.85))
        colour, edges = _graph(15000 + s, n, k, p, planted=(s % 2 == 0))
        for q in (k, k - 1):
            r = orc.fixpoint_dominance(colour, edges, k, clique_k=q)
            vl, el = r["vlive"].astype(bool), r["elive"].astype(bool)
            had = bool(refs.q_cliques(n, q, colour, edges))
            kept = bool(refs.q_cliques(n, q, colour, edges[el])) if el.any() else False
            if had != kept:
                return f"q-clique existence changed (q={q}, case {s}): before {had}, after {kept}"
            nb = _live_nbrs(n, edges, vl, el)
            for i, (u, v) in enumerate(np.asarray(edges).tolist()):
                if el[i] and len({int(colour[w]) for w in nb[u] & nb[v]}) < q - 2:
                    return f"live edge fails the edge rule (case {s})"
            for a in np.flatnonzero(vl).tolist():
                if len({int(colour[w]) for w in nb[a]}) < q - 1:
                    return f"live vertex fails the vertex rule (case {s})"
                for b in np.flatnonzero(vl).tolist():
                    if b != a and nb[a] <= nb[b] and b not in nb[a]:
                        if nb[a] != nb[b] or (int(colour[b]), b) > (int(colour[a]), a):
                            return f"vertex {a} still dominated by {b} (case {s})"
    return None


def pin_edge_dominance_examples(orc):
    """Definitions 4.3.2 and 4.3.3 on hand-made graphs.  (1) Two triangles
    a-u-w and u-b-w sharing the edge u-w, a and b not adjacent (k = 3; a, b of
    colour 0, u of 1, w of 2): N(a) ∩ N(u) = {w} = N(u) ∩ N(b), so {u, b}
    dominates {a, u} and {a, u} dominates {u, b} (Definition 4.3.2).  Their
    records share vertices, so only the smaller key {a, u} goes; then a-w has
    no common neighbour left and a none of colour 1, so the colour-index rules
    remove both, and the triangle u-b-w remains.  (2) Two 4-cliques
    {x, y, c, d} and {u, v, c, d} sharing c-d, with x, u of colour 0 and y, v
    of colour 1 (k = 4): N(x) ∩ N(y) = {c, d} = N(u) ∩ N(v), and neither u nor
    v is adjacent to x or y, so {u, v} and {x, y} dominate each other
    (Definition 4.3.3) and no other edge is dominated; {x, y} (the smaller
    key) goes, x and y then see only colours 2 and 3 and leave, and the
    4-clique {u, v, c, d} remains."""
    r = orc.fixpoint_edge_dominance(np.array([0, 1, 0, 2], np.int32),
                                    np.array([[0, 1], [1, 2], [0, 3], [1, 3], [2, 3]], np.int32), 3)
    if r["vlive"].tolist() != [0, 1, 1, 1] or r["elive"].tolist() != [0, 1, 0, 1, 1] or \
            r["rounds"] != 1 or r["deleted"] != 1:
        return f"shared vertex: {r['vlive'].tolist()} {r['elive'].tolist()} rounds {r['rounds']}"
    colour = np.array([0, 1, 2, 3, 0, 1], np.int32)
    edges = np.array([[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3], [4, 5], [2, 4], [3, 4], [2, 5], [3, 5]],
                     np.int32)
    r = orc.fixpoint_edge_dominance(colour, edges, 4)
    if r["vlive"].tolist() != [0, 0, 1, 1, 1, 1] or r["elive"].tolist() != [0] * 5 + [1] * 6 or \
            r["rounds"] != 1 or r["deleted"] != 1:
        return f"disjoint edges: {r['vlive'].tolist()} {r['elive'].tolist()} rounds {r['rounds']}"
    # (3) A strict subset (k = 3): triangle x-y-c and triangles u-v-c, u-v-c'
    # (x, u of colour 0; y, v of 1; c, c' of 2; ids x..c' = 0..5).
    # N(x) ∩ N(y) = {c} lies strictly inside N(u) ∩ N(v) = {c, c'}, so {u, v}
    # dominates {x, y} but not the other way round; also {u, c} and {u, c'}
    # dominate each other (N = {v} for both), as do {v, c} and {v, c'}.
    # Round 1: the record of {x, y} is {x, y, u, v} and holds the smallest key
    # at all four vertices, while {u, c} loses u to it, so only {x, y} goes;
    # x and y then see one colour and leave.  Round 2: {u, c} (the smallest
    # key left) goes, c keeps only v and leaves.  The triangle u-v-c' remains.
    colour = np.array([0, 1, 2, 0, 1, 2], np.int32)
    edges = np.array([[0, 1], [0, 2], [1, 2], [3, 4], [2, 3], [2, 4], [3, 5], [4, 5]], np.int32)
    r = orc.fixpoint_edge_dominance(colour, edges, 3)
    if r["vlive"].tolist() != [0, 0, 0, 1, 1, 1] or r["elive"].tolist() != [0, 0, 0, 1, 0, 0, 1, 1] or \
            r["rounds"] != 2 or r["deleted"] != 2:
        return f"strict subset: {r['vlive'].tolist()} {r['elive'].tolist()} rounds {r['rounds']}"
    return None


def _dominated(nb, e, f):
    """Edge f dominates edge e (Definitions 4.3.2 and 4.3.3, written out on
    live neighbourhoods): f != e, each endpoint of f non-adjacent to an
    endpoint of e (a vertex is not adjacent to itself), and every common
    neighbour of e's endpoints a neighbour of both of f's."""
    (x, y), (u, v) = e, f
    if {x, y} == {u, v}:
        return False
    for z in (u, v):
        if z in nb[x] and z in nb[y]:
            return False
    return (nb[x] & nb[y]) <= (nb[u] & nb[v])


def pin_edge_dominance_keeps_cliques(orc, cases=14):
    """Edge dominance keeps the clique number: a q-clique exists in the graph
    exactly when one exists in the result (exhaustive enumeration), and the
    result is closed: no live edge is dominated by another live edge and no
    element fails a colour-index rule."""
    rng = np.random.default_rng(919)
    for s in range(cases):
        n = int(rng.integers(8, 24))
        k = int(rng.integers(3, 6))
        p = float(rng.uniform(0.4, 0.9))
        colour, edges = _graph(16000 + s, n, k, p, planted=(s % 2 == 0))
        for q in (k, k - 1):
            r = orc.fixpoint_edge_dominance(colour, edges, k, clique_k=q)
            vl, el = r["vlive"].astype(bool), r["elive"].astype(bool)
            had = bool(refs.q_cliques(n, q, colour, edges))
            kept = bool(refs.q_cliques(n, q, colour, edges[el])) if el.any() else False
            if had != kept:
                return f"q-clique existence changed (q={q}, case {s}): before {had}, after {kept}"
            nb = _live_nbrs(n, edges, vl, el)
            live = [tuple(e) for e, on in zip(np.asarray(edges).tolist(), el) if on]
            for e in live:
                if len({int(colour[w]) for w in nb[e[0]] & nb[e[1]]}) < q - 2:
                    return f"live edge fails the edge rule (case {s})"
                for f in live:
                    if _dominated(nb, e, f):
                        return f"edge {e} still dominated by {f} (case {s}, q={q})"
            for a in np.flatnonzero(vl).tolist():
                if len({int(colour[w]) for w in nb[a]}) < q - 1:
                    return f"live vertex fails the vertex rule (case {s})"
    return None


ALL_PINS = [pin_fig8, pin_brute_force, pin_k3_triangles, pin_k2, pin_k1, pin_complete_kpartite,
            pin_empty_class, pin_planted_isolated, pin_clique_survival, pin_order_independence,
            pin_certificate, pin_incident_edges_fail, pin_validation, pin_brute_force_q,
            pin_q_cliques_and_order, pin_dominance_examples, pin_dominance_keeps_cliques,
            pin_edge_dominance_examples, pin_edge_dominance_keeps_cliques]
