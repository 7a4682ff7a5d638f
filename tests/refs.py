"""Independent checks used to pin the oracle (test-side only).

None of these share code with ``oracle/`` or with the CUDA path.  They
characterise the result differently from the oracle's sweep loop:

* ``brute_force_gfp``: the kernel as the union of all *closed* subgraphs
  (every vertex sees every other colour, every edge has a common neighbour
  of every other colour), found by enumerating edge subsets.
* ``triangle_closed_form``: for k = 3 the kernel is the union of the
  triangles of G, computed with a library matrix product.
* ``k_cliques``: exhaustive k-clique enumeration (soundness: no vertex or
  edge of a k-clique may be deleted, Section 4.2 remarks).
* ``chaotic_fixpoint``: deletion in random orders / random subsets; the
  greatest fixpoint of monotone deletion rules is order independent.
* ``check_certificate``: replays a Jacobi trace and checks that every sweep
  deleted exactly the failing elements of its snapshot, and that the final
  state is closed.
"""
from __future__ import annotations

import itertools
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ----------------------------------------------------------------------------
# Figure 8 fixture
# ----------------------------------------------------------------------------

def load_fig8():
    names, colour, edges, ev, ee = [], [], [], [], []
    k = None
    with open(os.path.join(GOLDEN, "fig8_colour_index.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "k":
                k = int(line[1])
            elif line[0] == "vertex":
                names.append(line[1])
                colour.append(int(line[2]))
            elif line[0] == "edge":
                edges.append((names.index(line[1]), names.index(line[2])))
            elif line[0] == "expect_vertex":
                ev.append((names.index(line[1]), int(line[2])))
            elif line[0] == "expect_edge":
                ee.append((names.index(line[1]), names.index(line[2]), int(line[3])))
    return dict(k=k, names=names, colour=np.array(colour, np.int32),
                edges=np.array(edges, np.int32), expect_vertex=ev, expect_edge=ee)


# ----------------------------------------------------------------------------
# brute-force greatest closed subgraph
# ----------------------------------------------------------------------------

def brute_force_gfp(n, k, colour, edges, q=None):
    """Union of all closed subgraphs, by enumerating every edge subset.

    H = (V_H, E_H) is closed when every vertex of V_H has H-neighbours in at
    least q-1 colours other than its own, and every edge {u,v} of E_H has,
    in at least q-2 colours other than col(u), col(v), a vertex w with {u,w}
    and {v,w} in E_H (q = k: every such colour).  For q >= 2 a vertex of a
    closed H needs an incident H-edge, so V_H is the set of endpoints of E_H;
    for q = 1 there are no conditions.
    Returns (vertex_mask bool[n], edge_mask bool[m]).
    """
    q = k if q is None else q
    colour = [int(c) for c in colour]
    edges = [tuple(map(int, e)) for e in edges]
    m = len(edges)
    assert m <= 18, "brute force is exponential in m"
    if q <= 1:
        return np.ones(n, bool), np.ones(m, bool)
    eidx = {}
    for i, (u, v) in enumerate(edges):
        eidx[(u, v)] = i
        eidx[(v, u)] = i
    inc = [[0] * k for _ in range(n)]          # edges from v into colour c
    for i, (u, v) in enumerate(edges):
        inc[u][colour[v]] |= 1 << i
        inc[v][colour[u]] |= 1 << i
    wit = []                                    # per edge, per needed colour: pair masks
    for i, (u, v) in enumerate(edges):
        per = []
        for c in range(k):
            if c in (colour[u], colour[v]):
                continue
            masks = []
            for w in range(n):
                if colour[w] == c and (u, w) in eidx and (v, w) in eidx:
                    masks.append((1 << eidx[(u, w)]) | (1 << eidx[(v, w)]))
            per.append(masks)
        wit.append(per)
    union = 0
    for S in range(1 << m):
        if S & ~union == 0 and S != 0:
            continue  # cannot add anything new
        ok = True
        verts = set()
        for i in range(m):
            if S >> i & 1:
                verts.update(edges[i])
        for v in verts:
            covered = sum(1 for c in range(k) if c != colour[v] and (S & inc[v][c]))
            if covered < q - 1:
                ok = False
                break
        if ok:
            for i in range(m):
                if not (S >> i & 1):
                    continue
                covered = sum(1 for masks in wit[i] if any((S & pm) == pm for pm in masks))
                if covered < q - 2:
                    ok = False
                    break
        if ok:
            union |= S
    emask = np.array([(union >> i) & 1 == 1 for i in range(m)], bool)
    vmask = np.zeros(n, bool)
    for i in range(m):
        if emask[i]:
            vmask[edges[i][0]] = vmask[edges[i][1]] = True
    return vmask, emask


# ----------------------------------------------------------------------------
# k = 3 closed form: union of triangles
# ----------------------------------------------------------------------------

def triangle_closed_form(n, edges):
    """Edges lying on a triangle, and vertices lying on a triangle."""
    A = np.zeros((n, n), np.float64)
    if len(edges):
        e = np.asarray(edges)
        A[e[:, 0], e[:, 1]] = 1.0
        A[e[:, 1], e[:, 0]] = 1.0
    common = A @ A
    on_tri = (common > 0) & (A > 0)
    emask = np.array([on_tri[u, v] for u, v in edges], bool) if len(edges) else np.zeros(0, bool)
    vmask = on_tri.any(axis=1)
    return vmask, emask


# ----------------------------------------------------------------------------
# exhaustive k-clique enumeration
# ----------------------------------------------------------------------------

def k_cliques(n, k, colour, edges):
    """All k-cliques (as sorted vertex tuples).  Under a legal k-colouring a
    k-clique holds one vertex of every colour, so the search goes colour by
    colour."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[int(u)].add(int(v))
        adj[int(v)].add(int(u))
    by_colour = [[v for v in range(n) if colour[v] == c] for c in range(k)]
    out = []

    def rec(c, chosen, cand):
        if c == k:
            out.append(tuple(sorted(chosen)))
            return
        for v in by_colour[c]:
            if v in cand:
                rec(c + 1, chosen + [v], cand & adj[v])

    rec(0, [], set(range(n)))
    return out


def q_cliques(n, q, colour, edges):
    """All cliques of exactly q vertices (sorted tuples), by extending each
    vertex with higher-numbered common neighbours; independent of colours."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[int(u)].add(int(v))
        adj[int(v)].add(int(u))
    out = []

    def rec(chosen, cand):
        if len(chosen) == q:
            out.append(tuple(chosen))
            return
        for v in sorted(cand):
            if not chosen or v > chosen[-1]:
                rec(chosen + [v], cand & adj[v])

    if q <= 0:
        return [()]
    rec([], set(range(n)))
    return out


def has_q_clique(n, q, colour, edges):
    """Whether a clique of q vertices exists: depth-first extension that stops
    at the first one (dense graphs hold far too many to list)."""
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[int(u)].add(int(v))
        adj[int(v)].add(int(u))

    def rec(size, cand):
        if size == q:
            return True
        if size + len(cand) < q:
            return False
        for v in sorted(cand):
            if rec(size + 1, {w for w in cand & adj[v] if w > v}):
                return True
        return False

    return q <= 0 or rec(0, set(range(n)))


# ----------------------------------------------------------------------------
# random-order deletion
# ----------------------------------------------------------------------------

def _live_adj(n, edges, elive):
    adj = [dict() for _ in range(n)]
    for i, (u, v) in enumerate(edges):
        if elive[i]:
            adj[u][v] = i
            adj[v][u] = i
    return adj


def _misses_colour_v(v, colour, k, adj, q=None):
    seen = {colour[w] for w in adj[v]}
    if q is not None:
        return len(seen) < q - 1
    return any(c not in seen for c in range(k) if c != colour[v])


def _misses_colour_e(u, v, colour, k, adj, q=None):
    common = set(adj[u]) & set(adj[v])
    seen = {colour[w] for w in common}
    if q is not None:
        return len(seen) < q - 2
    return any(c not in seen for c in range(k) if c not in (colour[u], colour[v]))


def chaotic_fixpoint(n, k, colour, edges, rng, mode="shuffled", q=None):
    """Delete failing elements in a random order until nothing fails.

    A vertex fails when some colour other than its own has no live neighbour;
    an edge fails when some colour other than its endpoints' has no live
    common neighbour (these are the Section 4.2 conditions, phrased as
    "misses a colour").  ``shuffled``: Gauss-Seidel over a random order,
    deleting at once.  ``subset``: each round tests a random subset on the
    round's snapshot and deletes the failures together.  With ``q`` (the
    clique size sought) an element fails below q-1 (vertex) or q-2 (edge)
    covered colours instead.
    """
    colour = [int(c) for c in colour]
    edges = [tuple(map(int, e)) for e in edges]
    vlive = np.ones(n, bool)
    elive = np.ones(len(edges), bool)

    def kill_vertex(v, adj):
        vlive[v] = False
        for w, i in list(adj[v].items()):
            elive[i] = False
            del adj[w][v]
        adj[v].clear()

    while True:
        adj = _live_adj(n, edges, elive)
        items = [("v", v) for v in range(n) if vlive[v]] + [("e", i) for i in range(len(edges)) if elive[i]]
        order = rng.permutation(len(items))
        changed = False
        if mode == "shuffled":
            for j in order:
                kind, x = items[j]
                if kind == "v":
                    if vlive[x] and _misses_colour_v(x, colour, k, adj, q):
                        kill_vertex(x, adj)
                        changed = True
                else:
                    if elive[x]:
                        u, v = edges[x]
                        if _misses_colour_e(u, v, colour, k, adj, q):
                            elive[x] = False
                            del adj[u][v]
                            del adj[v][u]
                            changed = True
        else:
            take = [items[j] for j in order if rng.random() < 0.5]
            fv = [x for kind, x in take if kind == "v" and _misses_colour_v(x, colour, k, adj, q)]
            fe = [x for kind, x in take if kind == "e" and _misses_colour_e(*edges[x], colour, k, adj, q)]
            for x in fe:
                if elive[x]:
                    u, v = edges[x]
                    elive[x] = False
                    del adj[u][v]
                    del adj[v][u]
            for x in fv:
                kill_vertex(x, adj)
            changed = bool(fv or fe)
            if not changed:
                # certify with a full pass before stopping
                adj = _live_adj(n, edges, elive)
                changed = any(vlive[v] and _misses_colour_v(v, colour, k, adj, q) for v in range(n)) or \
                    any(elive[i] and _misses_colour_e(*edges[i], colour, k, adj, q) for i in range(len(edges)))
        if not changed:
            return vlive, elive


# ----------------------------------------------------------------------------
# Jacobi certificate
# ----------------------------------------------------------------------------

def check_certificate(n, k, colour, edges, v_sweep, e_rule_sweep, sweeps):
    """Replay a Jacobi trace.  For each productive sweep t the vertices with
    v_sweep == t and the edges with e_rule_sweep == t must be *exactly* the
    elements failing on the snapshot S_t; after the last sweep nothing may
    fail.  Returns None if the certificate holds, else a message."""
    colour = [int(c) for c in colour]
    edges = [tuple(map(int, e)) for e in edges]
    v_sweep = np.asarray(v_sweep)
    e_rule_sweep = np.asarray(e_rule_sweep)
    vlive = np.ones(n, bool)
    elive = np.ones(len(edges), bool)
    for t in range(1, sweeps + 2):
        adj = _live_adj(n, edges, elive)
        fail_v = {v for v in range(n) if vlive[v] and _misses_colour_v(v, colour, k, adj)}
        fail_e = {i for i in range(len(edges)) if elive[i] and _misses_colour_e(*edges[i], colour, k, adj)}
        if t == sweeps + 1:
            if fail_v or fail_e:
                return f"final state not closed: {len(fail_v)} vertices, {len(fail_e)} edges fail"
            return None
        want_v = {v for v in range(n) if v_sweep[v] == t}
        want_e = {i for i in range(len(edges)) if e_rule_sweep[i] == t}
        if want_v != fail_v:
            return f"sweep {t}: vertex deletions differ ({sorted(want_v ^ fail_v)[:5]})"
        if want_e != fail_e:
            return f"sweep {t}: edge deletions differ ({sorted(want_e ^ fail_e)[:5]})"
        if not fail_v and not fail_e:
            return f"sweep {t}: recorded as productive but nothing fails"
        for v in fail_v:
            vlive[v] = False
        for i, (u, v) in enumerate(edges):
            if i in fail_e or not vlive[u] or not vlive[v]:
                elive[i] = False
    return None


def complete_kpartite(sizes):
    colour = np.concatenate([np.full(s, c, np.int32) for c, s in enumerate(sizes)]) if sizes else np.zeros(0, np.int32)
    n = len(colour)
    edges = [(u, v) for u, v in itertools.combinations(range(n), 2) if colour[u] != colour[v]]
    return colour, np.array(edges, np.int32).reshape(-1, 2)
