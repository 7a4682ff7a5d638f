"""The two facts the worklist schedules rest on, checked on the oracle's own
Jacobi sweeps (CPU only; nothing here runs a kernel).

1. Frontier completeness (Section 4.2 rules, edge index).  An edge that
   fails in sweep r + 1 passed in sweep r, so every needed class it now
   lacks held a common neighbour w before sweep r, and sweep r deleted the
   edge from one of its ends to w.  Hence the pairs {a, x} with x a common
   neighbour of a deleted edge {a, b} (in the rows before that sweep), each in
   the class of b, contain every (edge, class) that fails next: the dirty
   set of the learned schedule and the re-checks of the support schedule on
   bitset rows.
2. Vertex failures imply edge failures.  Every edge at a vertex that fails
   the vertex rule in a sweep fails the edge rule in the same sweep: the
   class the vertex lacks is a class no common neighbour can have.
"""
import numpy as np
import pytest

import oracle
from paper_2212_00574_gb300 import synth


def _state(g, edges, s):
    """Live edges (bool[m]) after s productive sweeps."""
    if s == 0:
        return np.ones(len(edges), bool)
    r = oracle.fixpoint(g.colour, edges, g.k, max_sweeps=s, raise_on_limit=False)
    return r["elive"].astype(bool)


def _adj(n, edges, live):
    A = np.zeros((n, n), bool)
    e = edges[live]
    A[e[:, 0], e[:, 1]] = True
    A[e[:, 1], e[:, 0]] = True
    return A


def _cascades():
    out = []
    for seed in range(40):
        g = synth.tiny_random(3000 + seed, 120 + 7 * seed, 5 + seed % 6, 0.18 + 0.01 * (seed % 9),
                              planted=bool(seed % 2))
        orc = oracle.fixpoint(g.colour, g.get_edges(), g.k)
        if orc["sweeps"] >= 3:
            out.append((g, orc))
    return out


CASES = _cascades()


def test_enough_cascades():
    assert len(CASES) >= 8
    assert max(o["sweeps"] for _, o in CASES) >= 5


@pytest.mark.parametrize("case", range(8))
def test_failures_of_the_next_sweep_are_marked(case):
    g, orc = CASES[case]
    edges = g.get_edges()
    n, k, col = g.n, g.k, np.asarray(g.colour)
    for r in range(1, orc["sweeps"]):
        before, after, nxt = _state(g, edges, r - 1), _state(g, edges, r), _state(g, edges, r + 1)
        A0, A1 = _adj(n, edges, before), _adj(n, edges, after)
        deleted = before & ~after
        D = np.zeros((n, n), bool)   # D[x, w]: edge {x, w} deleted in sweep r
        d = edges[deleted]
        D[d[:, 0], d[:, 1]] = True
        D[d[:, 1], d[:, 0]] = True
        failing = after & ~nxt
        for (u, v) in edges[failing]:
            for c in range(k):
                if c in (col[u], col[v]):
                    continue
                members = col == c
                if (A1[u] & A1[v] & members).any():
                    continue   # class c still covered: not why the edge fails
                # the lost common neighbours of class c, each from a deleted edge
                lost = A0[u] & A0[v] & members & (D[u] | D[v])
                assert lost.any(), (r, u, v, c)
                # ... and the pair was covered in class c before sweep r
                assert (A0[u] & A0[v] & members).any()


@pytest.mark.parametrize("case", range(8))
def test_vertex_failures_take_all_their_edges_by_the_edge_rule(case):
    g, orc = CASES[case]
    edges = g.get_edges()
    vs, es = orc["v_sweep"], orc["e_rule_sweep"]
    for i, (u, v) in enumerate(edges):
        for x in (u, v):
            if vs[x] > 0:
                # the edge goes by the edge rule no later than its end goes
                assert 0 < es[i] <= vs[x], (i, u, v, vs[x], es[i])
