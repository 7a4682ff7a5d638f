"""Plausible mistakes planted in copies of the oracle must each fail a pin.

The mistakes are planted in edited copies of the oracle source compiled into
a temporary directory, on the CPU; the real oracle is untouched.
"""
import pytest

import oracle
from tests import pins

MUTANTS = {
    # vertex rule threshold off by one (index < q-2 instead of < q-1)
    "vertex_threshold": ("(vlive[v] && vertex_index(&g, elive, &s, v) < q - 1) {", "(vlive[v] && vertex_index(&g, elive, &s, v) < q - 2) {"),
    # edge rule threshold off by one
    "edge_threshold": ("edges[2 * e + 1]) < q - 2)", "edges[2 * e + 1]) < q - 3)"),
    # the clique size ignored: thresholds from the colour count
    "vertex_threshold_from_k": ("(vlive[v] && vertex_index(&g, elive, &s, v) < q - 1) {", "(vlive[v] && vertex_index(&g, elive, &s, v) < k - 1) {"),
    # the same thresholds in the dominance procedure's colour-index phases
    "dominance_vertex_threshold": ("fail_v[v] = vlive[v] && vertex_index(g, elive, s, v) < q - 1;",
                                   "fail_v[v] = vlive[v] && vertex_index(g, elive, s, v) < q - 2;"),
    "dominance_edge_threshold": ("edges[2 * e], edges[2 * e + 1]) < q - 2;", "edges[2 * e], edges[2 * e + 1]) < q - 3;"),
    "edge_threshold_from_k": ("edges[2 * e + 1]) < q - 2)", "edges[2 * e + 1]) < k - 2)"),
    # common neighbour test dropped: counts every neighbour of v
    "no_common_check": ("        if (s->nbr_mark[w] != s->stamp) continue;\n", ""),
    # (Not listed: keeping the edges of a deleted vertex live.  That edit is
    # equivalent: a vertex that misses a colour c makes each of its live
    # edges miss c as a common-neighbour colour in the same sweep, so those
    # edges fail the edge rule anyway; pin_incident_edges_fail checks this.)
    # a dead edge still counts as a witness in the edge index
    "dead_witness_edge": ("    for (int64_t i = g->off[v]; i < g->off[v + 1]; i++) {\n        if (!elive[g->eid[i]]) continue;\n        int32_t w = g->nbr[i];",
                          "    for (int64_t i = g->off[v]; i < g->off[v + 1]; i++) {\n        int32_t w = g->nbr[i];"),
    # dominance: both of two vertices with equal neighbourhoods deleted
    "dominance_no_tie_break": ("                if (deg[a] == deg[b] &&\n", "                if (0 && deg[a] == deg[b] &&\n"),
    # dominance: the dominator deleted instead of the dominated vertex
    "dominance_reversed": ("if (b == a || !vlive[b] || deg[b] < deg[a]) continue;", "if (b == a || !vlive[b] || deg[b] > deg[a]) continue;"),
    # edge dominance: every dominated edge deleted, no vertex-disjoint selection
    "edge_dominance_no_selection": ("            fail_e[e] = (uint8_t)mine;", "            fail_e[e] = 1;"),
    # edge dominance: the subset condition reversed
    "edge_dominance_reversed": ("                for (int32_t i = 0; i < nx && subset; i++)\n                    if (!(A[(size_t)u * n + common[i]] && A[(size_t)v * n + common[i]])) subset = 0;",
                                "                for (int32_t w = 0; w < n && subset; w++)\n                    if (A[(size_t)u * n + w] && A[(size_t)v * n + w] && !(A[(size_t)x * n + w] && A[(size_t)y * n + w])) subset = 0;"),
    # edge dominance: an edge counted as its own dominator
    "edge_dominance_self": ("                if (f == e || !elive[f]) continue;", "                if (!elive[f]) continue;"),
    # the sweep index recorded one too late
    "sweep_off_by_one": ("if (v_sweep) v_sweep[v] = (int32_t)sweeps;", "if (v_sweep) v_sweep[v] = (int32_t)sweeps + 1;"),
    # Gauss-Seidel instead of Jacobi: vertices leave before the edge rule runs
    "not_jacobi": ("            if (vlive[v] && vertex_index(&g, elive, &s, v) < q - 1) {\n                fail_v[v] = 1;",
                   "            if (vlive[v] && vertex_index(&g, elive, &s, v) < q - 1) {\n                fail_v[v] = 1;\n                for (int64_t i = g.off[v]; i < g.off[v + 1]; i++) elive[g.eid[i]] = 0;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = oracle.compile_variant(src.replace(old, new), str(tmp_path / f"libmut_{name}.so"))
    orc = oracle.Oracle(path)
    failures = []
    for pin in pins.ALL_PINS:
        try:
            msg = pin(orc)
        except Exception as exc:  # a crash in the mutant also counts as caught
            msg = f"raised {exc!r}"
        if msg:
            failures.append(f"{pin.__name__}: {msg}")
    assert failures, f"mutant {name} passed every pin"
