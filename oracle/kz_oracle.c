/*
 * kz_oracle.c -- CPU oracle for the colour-index kernelization.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it computes (thesis Section 4.2, "Colour indices"):
 *
 *   - Definition 4.2.1: G is legally coloured with k colours; the colour
 *     classes are c_1..c_k (here 0-based: colours 0..k-1).
 *   - Colour index of a vertex v: the number of colour classes that contain
 *     at least one vertex adjacent to v.  Remark: a vertex whose index is
 *     below k-1 is in no k-clique and may be deleted.
 *   - Colour index of an edge {u,v}: the number of colour classes that
 *     contain at least one vertex adjacent to both u and v.  Remark: an edge
 *     whose index is below k-2 is in no k-clique and may be deleted, but u
 *     and v themselves are kept.
 *
 * Readings taken where the thesis is silent (each is listed in the design
 * notes of the repository):
 *
 *   1. The two rules are applied repeatedly to the *live* graph until no rule
 *      fires (the thesis states them once).  Adjacency means a live edge
 *      between live vertices; a common neighbour w of u and v needs both
 *      {u,w} and {v,w} live.
 *   2. Sweeps are Jacobi sweeps: in sweep t both rules are evaluated on the
 *      same snapshot S_t; the vertices D_V and edges D_E that fail are then
 *      removed together, along with every edge incident to a vertex of D_V.
 *      "sweeps" counts productive sweeps (at least one deletion); a graph that
 *      is already a fixpoint reports sweeps = 0.
 *   3. Only colours other than the element's own count: c != col(v) for a
 *      vertex and c not in {col(u), col(v)} for an edge.  Under a legal
 *      colouring these classes cannot hold a neighbour anyway.
 *   4. Illegal input (colour out of range, self loop, vertex out of range, an
 *      edge inside one colour class) is rejected.
 *
 * Data structures are deliberately plain: an adjacency list with edge ids,
 * one live flag per vertex and per edge, and a per-colour "seen" array.
 *
 * Parity pins for this file live in the tests (brute-force greatest fixpoint,
 * closed forms for k = 2 and k = 3, clique survival, order independence,
 * certificate check, the Figure 8 worked example).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    KZO_OK = 0,
    KZO_ERR_ARG = -1,
    KZO_ERR_COLOUR_RANGE = -2,
    KZO_ERR_ILLEGAL_COLOURING = -3,
    KZO_ERR_SELF_LOOP = -4,
    KZO_ERR_VERTEX_RANGE = -5,
    KZO_ERR_OOM = -6,
    KZO_ERR_LIMIT = -7
};

/* Adjacency list: the neighbours of v are nbr[off[v] .. off[v+1]) and the
 * id of the edge to nbr[i] is eid[i]. */
typedef struct {
    int32_t n, k;
    const int32_t *colour;
    int64_t m;
    int64_t *off;
    int32_t *nbr;
    int64_t *eid;
} adj_t;

static void adj_free(adj_t *g)
{
    free(g->off);
    free(g->nbr);
    free(g->eid);
    g->off = NULL;
    g->nbr = NULL;
    g->eid = NULL;
}

/* Definition 4.2.1 requires a legal colouring; anything else is rejected. */
static int validate(int32_t n, int32_t k, const int32_t *colour, int64_t m,
                    const int32_t *edges)
{
    if (n < 0 || k < 1 || m < 0) return KZO_ERR_ARG;
    if ((n > 0 && !colour) || (m > 0 && !edges)) return KZO_ERR_ARG;
    for (int32_t v = 0; v < n; v++)
        if (colour[v] < 0 || colour[v] >= k) return KZO_ERR_COLOUR_RANGE;
    for (int64_t e = 0; e < m; e++) {
        int32_t u = edges[2 * e], v = edges[2 * e + 1];
        if (u < 0 || u >= n || v < 0 || v >= n) return KZO_ERR_VERTEX_RANGE;
        if (u == v) return KZO_ERR_SELF_LOOP;
        if (colour[u] == colour[v]) return KZO_ERR_ILLEGAL_COLOURING;
    }
    return KZO_OK;
}

static int adj_build(adj_t *g, int32_t n, int32_t k, const int32_t *colour,
                     int64_t m, const int32_t *edges)
{
    g->n = n;
    g->k = k;
    g->colour = colour;
    g->m = m;
    g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    g->eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    if (!g->off || !g->nbr || !g->eid) {
        adj_free(g);
        return KZO_ERR_OOM;
    }
    for (int64_t e = 0; e < m; e++) {
        g->off[edges[2 * e] + 1]++;
        g->off[edges[2 * e + 1] + 1]++;
    }
    for (int32_t v = 0; v < n; v++) g->off[v + 1] += g->off[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!fill) {
        adj_free(g);
        return KZO_ERR_OOM;
    }
    memcpy(fill, g->off, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < m; e++) {
        int32_t u = edges[2 * e], v = edges[2 * e + 1];
        g->nbr[fill[u]] = v;
        g->eid[fill[u]++] = e;
        g->nbr[fill[v]] = u;
        g->eid[fill[v]++] = e;
    }
    free(fill);
    return KZO_OK;
}

/* Scratch shared by the two index functions: a per-colour "seen" stamp and a
 * per-vertex "neighbour of u" stamp.  Stamps avoid clearing between calls. */
typedef struct {
    int64_t *colour_seen; /* k */
    int64_t *nbr_mark;    /* n */
    int64_t stamp;
} scratch_t;

static int scratch_init(scratch_t *s, int32_t n, int32_t k)
{
    s->colour_seen = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
    s->nbr_mark = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    s->stamp = 0;
    if (!s->colour_seen || !s->nbr_mark) {
        free(s->colour_seen);
        free(s->nbr_mark);
        return KZO_ERR_OOM;
    }
    return KZO_OK;
}

static void scratch_free(scratch_t *s)
{
    free(s->colour_seen);
    free(s->nbr_mark);
}

/* Colour index of vertex v on the live graph: the number of colour classes
 * other than col(v) holding at least one vertex joined to v by a live edge.
 * A live edge always has live endpoints (deleting a vertex kills its edges). */
static int32_t vertex_index(const adj_t *g, const uint8_t *elive, scratch_t *s, int32_t v)
{
    s->stamp++;
    int32_t count = 0;
    for (int64_t i = g->off[v]; i < g->off[v + 1]; i++) {
        if (!elive[g->eid[i]]) continue;
        int32_t c = g->colour[g->nbr[i]];
        if (c == g->colour[v]) continue;
        if (s->colour_seen[c] != s->stamp) {
            s->colour_seen[c] = s->stamp;
            count++;
        }
    }
    return count;
}

/* Colour index of edge {u,v} on the live graph: the number of colour classes
 * other than col(u), col(v) holding at least one vertex w with both {u,w} and
 * {v,w} live. */
static int32_t edge_index(const adj_t *g, const uint8_t *elive, scratch_t *s,
                          int32_t u, int32_t v)
{
    s->stamp++;
    for (int64_t i = g->off[u]; i < g->off[u + 1]; i++)
        if (elive[g->eid[i]]) s->nbr_mark[g->nbr[i]] = s->stamp;
    int32_t count = 0;
    for (int64_t i = g->off[v]; i < g->off[v + 1]; i++) {
        if (!elive[g->eid[i]]) continue;
        int32_t w = g->nbr[i];
        if (s->nbr_mark[w] != s->stamp) continue;
        int32_t c = g->colour[w];
        if (c == g->colour[u] || c == g->colour[v]) continue;
        if (s->colour_seen[c] != s->stamp) {
            s->colour_seen[c] = s->stamp;
            count++;
        }
    }
    return count;
}

/*
 * Jacobi fixpoint of the two Section 4.2 rules.
 *
 * Inputs: n vertices, k colours, colour[n], m edges as pairs edges[2m]
 * (no duplicates, no reversed repeats).  max_sweeps bounds the productive
 * sweeps (<= 0 means |V| + |E| + 1, which always suffices because every
 * productive sweep removes at least one element).
 *
 * Outputs (each may be NULL):
 *   vlive[n], elive[m]   1 if the element survives, 0 if deleted
 *   v_sweep[n]           productive sweep (1-based) that deleted v, 0 if kept
 *   e_rule_sweep[m]      sweep in which e failed the edge rule, 0 if never
 *                        (an edge can also die with an endpoint; that is not
 *                        recorded here)
 *   dv[cap], de[cap]     |D_V| and |D_E| of each productive sweep
 *   sweeps               number of productive sweeps
 *   tests                live edges tested, summed over all passes
 *                        (the last, unproductive pass included)
 *
 * Returns KZO_OK, KZO_ERR_LIMIT (stopped after max_sweeps productive sweeps
 * with deletions still pending), or an input error.
 *
 * kzo_fixpoint_q takes the clique size q sought (1 <= q <= k) as its own
 * argument: a vertex fails below colour index q-1, an edge below q-2.  The
 * Section 4.2 Remarks derive both thresholds from the clique size alone: a
 * vertex of a q-clique sees q-1 other clique members, all coloured
 * differently under a legal colouring, and an edge of it sees q-2 common
 * neighbours in the clique.  kzo_fixpoint is the thesis's case q = k.
 */
int kzo_fixpoint_q(int32_t n, int32_t k, int32_t q, const int32_t *colour, int64_t m,
                   const int32_t *edges, int64_t max_sweeps,
                   uint8_t *vlive_out, uint8_t *elive_out,
                   int32_t *v_sweep, int32_t *e_rule_sweep,
                   int64_t *dv, int64_t *de, int64_t cap,
                   int64_t *sweeps_out, int64_t *tests_out)
{
    if (q < 1 || q > k) return KZO_ERR_ARG;
    int rc = validate(n, k, colour, m, edges);
    if (rc != KZO_OK) return rc;
    adj_t g;
    rc = adj_build(&g, n, k, colour, m, edges);
    if (rc != KZO_OK) return rc;
    scratch_t s;
    if (scratch_init(&s, n, k) != KZO_OK) {
        adj_free(&g);
        return KZO_ERR_OOM;
    }
    uint8_t *vlive = (uint8_t *)malloc((size_t)n + 1);
    uint8_t *elive = (uint8_t *)malloc((size_t)m + 1);
    uint8_t *fail_v = (uint8_t *)malloc((size_t)n + 1);
    uint8_t *fail_e = (uint8_t *)malloc((size_t)m + 1);
    if (!vlive || !elive || !fail_v || !fail_e) {
        rc = KZO_ERR_OOM;
        goto done;
    }
    memset(vlive, 1, (size_t)n);
    memset(elive, 1, (size_t)m);
    if (v_sweep) memset(v_sweep, 0, sizeof(int32_t) * (size_t)n);
    if (e_rule_sweep) memset(e_rule_sweep, 0, sizeof(int32_t) * (size_t)m);
    if (max_sweeps <= 0) max_sweeps = (int64_t)n + m + 1;

    int64_t sweeps = 0, tests = 0;
    for (;;) {
        /* one Jacobi pass on the snapshot (vlive, elive) */
        int64_t nv = 0, ne = 0;
        for (int32_t v = 0; v < n; v++) {
            fail_v[v] = 0;
            if (vlive[v] && vertex_index(&g, elive, &s, v) < q - 1) {
                fail_v[v] = 1;
                nv++;
            }
        }
        for (int64_t e = 0; e < m; e++) {
            fail_e[e] = 0;
            if (!elive[e]) continue;
            tests++;
            if (edge_index(&g, elive, &s, edges[2 * e], edges[2 * e + 1]) < q - 2) {
                fail_e[e] = 1;
                ne++;
            }
        }
        if (nv == 0 && ne == 0) break;
        if (sweeps >= max_sweeps) {
            rc = KZO_ERR_LIMIT;
            break;
        }
        sweeps++;
        if (dv && sweeps <= cap) dv[sweeps - 1] = nv;
        if (de && sweeps <= cap) de[sweeps - 1] = ne;
        /* apply: remove D_V, D_E and the edges incident to D_V */
        for (int32_t v = 0; v < n; v++)
            if (fail_v[v]) {
                vlive[v] = 0;
                if (v_sweep) v_sweep[v] = (int32_t)sweeps;
            }
        for (int64_t e = 0; e < m; e++) {
            if (!elive[e]) continue;
            if (fail_e[e] && e_rule_sweep) e_rule_sweep[e] = (int32_t)sweeps;
            if (fail_e[e] || fail_v[edges[2 * e]] || fail_v[edges[2 * e + 1]]) elive[e] = 0;
        }
    }
    if (vlive_out) memcpy(vlive_out, vlive, (size_t)n);
    if (elive_out) memcpy(elive_out, elive, (size_t)m);
    if (sweeps_out) *sweeps_out = sweeps;
    if (tests_out) *tests_out = tests;
done:
    free(vlive);
    free(elive);
    free(fail_v);
    free(fail_e);
    scratch_free(&s);
    adj_free(&g);
    return rc;
}

int kzo_fixpoint(int32_t n, int32_t k, const int32_t *colour, int64_t m,
                 const int32_t *edges, int64_t max_sweeps,
                 uint8_t *vlive_out, uint8_t *elive_out,
                 int32_t *v_sweep, int32_t *e_rule_sweep,
                 int64_t *dv, int64_t *de, int64_t cap,
                 int64_t *sweeps_out, int64_t *tests_out)
{
    return kzo_fixpoint_q(n, k, k, colour, m, edges, max_sweeps, vlive_out, elive_out, v_sweep,
                          e_rule_sweep, dv, de, cap, sweeps_out, tests_out);
}

/*
 * The colour-index phase of the dominance procedures: kzo_fixpoint_q's
 * Jacobi sweeps for clique size q, from the current live state (vlive,
 * elive) until a sweep deletes nothing.  fail_v[n] and fail_e[m] are scratch.
 */
static void colour_index_phase(const adj_t *g, scratch_t *s, int32_t q, const int32_t *edges,
                               uint8_t *vlive, uint8_t *elive, uint8_t *fail_v, uint8_t *fail_e)
{
    const int32_t n = g->n;
    const int64_t m = g->m;
    for (;;) {
        int64_t nv = 0, ne = 0;
        for (int32_t v = 0; v < n; v++) {
            fail_v[v] = vlive[v] && vertex_index(g, elive, s, v) < q - 1;
            nv += fail_v[v];
        }
        for (int64_t e = 0; e < m; e++) {
            fail_e[e] = elive[e] && edge_index(g, elive, s, edges[2 * e], edges[2 * e + 1]) < q - 2;
            ne += fail_e[e];
        }
        if (nv == 0 && ne == 0) break;
        for (int32_t v = 0; v < n; v++)
            if (fail_v[v]) vlive[v] = 0;
        for (int64_t e = 0; e < m; e++)
            if (elive[e] && (fail_e[e] || fail_v[edges[2 * e]] || fail_v[edges[2 * e + 1]])) elive[e] = 0;
    }
}

/*
 * Colour-index fixpoint followed by rounds of vertex dominance (thesis
 * Section 4.3, Definition 4.3.1), each round followed by the colour-index
 * fixpoint again, until a dominance round deletes nothing.
 *
 * Vertex b dominates vertex a when a and b are distinct, not adjacent, and
 * N(a) is a subset of N(b) (live neighbours).  The Remarks of Definition
 * 4.3.1 allow deleting a dominated vertex: a clique through a becomes one
 * through b when a is swapped for b, so the clique number is kept (some
 * cliques may go, which is why this pass is opt-in).  Reading for the
 * parallel (Jacobi) round: every vertex dominated on the round's snapshot is
 * deleted together, except that of two vertices with equal neighbourhoods
 * only the one with the smaller key (colour, id) goes.  The dominators then
 * form a strict order, whose maximal elements survive and dominate every
 * deleted vertex of their chain, so the clique number is still kept.
 *
 * The colour-index phases are kzo_fixpoint_q's Jacobi sweeps for clique
 * size q.  Outputs: vlive[n], elive[m], the dominance rounds that deleted
 * something, and the vertices they deleted.
 */
int kzo_fixpoint_dominance(int32_t n, int32_t k, int32_t q, const int32_t *colour, int64_t m,
                           const int32_t *edges, uint8_t *vlive_out, uint8_t *elive_out,
                           int64_t *rounds_out, int64_t *dominated_out)
{
    if (q < 1 || q > k) return KZO_ERR_ARG;
    int rc = validate(n, k, colour, m, edges);
    if (rc != KZO_OK) return rc;
    adj_t g;
    rc = adj_build(&g, n, k, colour, m, edges);
    if (rc != KZO_OK) return rc;
    scratch_t s;
    if (scratch_init(&s, n, k) != KZO_OK) {
        adj_free(&g);
        return KZO_ERR_OOM;
    }
    uint8_t *vlive = (uint8_t *)malloc((size_t)n + 1);
    uint8_t *elive = (uint8_t *)malloc((size_t)m + 1);
    uint8_t *fail_v = (uint8_t *)malloc((size_t)n + 1);
    uint8_t *fail_e = (uint8_t *)malloc((size_t)m + 1);
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int64_t rounds = 0, dominated = 0;
    if (!vlive || !elive || !fail_v || !fail_e || !deg) {
        rc = KZO_ERR_OOM;
        goto done;
    }
    memset(vlive, 1, (size_t)n);
    memset(elive, 1, (size_t)m);
    for (;;) {
        colour_index_phase(&g, &s, q, edges, vlive, elive, fail_v, fail_e);
        /* one dominance round on the snapshot */
        for (int32_t v = 0; v < n; v++) {
            deg[v] = 0;
            for (int64_t i = g.off[v]; i < g.off[v + 1]; i++) deg[v] += elive[g.eid[i]];
        }
        int64_t nd = 0;
        for (int32_t a = 0; a < n; a++) {
            fail_v[a] = 0;
            if (!vlive[a]) continue;
            for (int32_t b = 0; b < n && !fail_v[a]; b++) {
                if (b == a || !vlive[b] || deg[b] < deg[a]) continue;
                /* mark the live neighbours of b; a must not be one of them */
                s.stamp++;
                for (int64_t i = g.off[b]; i < g.off[b + 1]; i++)
                    if (elive[g.eid[i]]) s.nbr_mark[g.nbr[i]] = s.stamp;
                if (s.nbr_mark[a] == s.stamp) continue;
                int subset = 1;
                for (int64_t i = g.off[a]; i < g.off[a + 1] && subset; i++)
                    if (elive[g.eid[i]] && s.nbr_mark[g.nbr[i]] != s.stamp) subset = 0;
                if (!subset) continue;
                /* equal neighbourhoods: only the smaller key (colour, id) goes */
                if (deg[a] == deg[b] &&
                    (colour[b] < colour[a] || (colour[b] == colour[a] && b < a))) continue;
                fail_v[a] = 1;
            }
            nd += fail_v[a];
        }
        if (nd == 0) break;
        rounds++;
        dominated += nd;
        for (int32_t v = 0; v < n; v++)
            if (fail_v[v]) vlive[v] = 0;
        for (int64_t e = 0; e < m; e++)
            if (elive[e] && (fail_v[edges[2 * e]] || fail_v[edges[2 * e + 1]])) elive[e] = 0;
    }
    if (vlive_out) memcpy(vlive_out, vlive, (size_t)n);
    if (elive_out) memcpy(elive_out, elive, (size_t)m);
    if (rounds_out) *rounds_out = rounds;
    if (dominated_out) *dominated_out = dominated;
done:
    free(vlive);
    free(elive);
    free(fail_v);
    free(fail_e);
    free(deg);
    scratch_free(&s);
    adj_free(&g);
    return rc;
}

/*
 * Colour-index fixpoint alternating with rounds of edge dominance (thesis
 * Section 4.3, Definitions 4.3.2 and 4.3.3), until a round deletes nothing.
 *
 * Definition 4.3.3: for four distinct vertices, edge f = {u, v} dominates
 * edge e = {x, y} when u is not adjacent to both x and y, v is not adjacent
 * to both x and y, and N(x) and N(y) have no common neighbour outside
 * N(u) and N(v): N(x) ∩ N(y) ⊆ N(u) ∩ N(v).  Definition 4.3.2 is the case of
 * two edges sharing a vertex: {u, b} dominates {a, u} when
 * N(a) ∩ N(u) ⊆ N(u) ∩ N(b) and b is not adjacent to a.  (The printed
 * condition reads "b is not in N(a) ∩ N(b)", which every b meets since no
 * vertex is its own neighbour; the reading "b is not in N(a)" is the one the
 * Remarks' swap argument needs.)  Taking "{u, x} is not an edge" as true
 * when u = x, the conditions of Definition 4.3.3 for f = {y, b} sharing y
 * with e = {x, y} are exactly those of Definition 4.3.2 with a = x, so one
 * test covers both: f != e live, u and v each non-adjacent to x or to y, and
 * the subset condition, on live neighbourhoods.
 *
 * The Remarks: a clique through e turns into one through f when x and y are
 * swapped for u and v (a for b), so deleting a dominated edge keeps the
 * clique number (some cliques may go: the pass is opt-in).
 *
 * Reading for a parallel round: on the round's snapshot every dominated live
 * edge e takes as witness the dominating edge of smallest key, the key of an
 * edge {s, t} being (min(s, t), max(s, t)) in caller ids; the record of e is
 * the set of the vertices of e and of its witness.  An edge is deleted in the
 * round when its key is the smallest among all records that share a vertex
 * with its record.  Deleted records are pairwise vertex-disjoint, so deleting
 * them together equals deleting them one at a time (a deletion changes only
 * its endpoints' neighbourhoods, which no other deleted record involves), and
 * the dominated edge of smallest key is always deleted.
 *
 * Dense adjacency matrix: n <= 4096 (KZO_ERR_ARG beyond).  Outputs: vlive[n],
 * elive[m], the dominance rounds that deleted something, the edges they
 * deleted.
 */
static uint64_t edge_key(int32_t s, int32_t t)
{
    int32_t lo = s < t ? s : t, hi = s < t ? t : s;
    return ((uint64_t)(uint32_t)lo << 32) | (uint32_t)hi;
}

int kzo_fixpoint_edge_dominance(int32_t n, int32_t k, int32_t q, const int32_t *colour, int64_t m,
                                const int32_t *edges, uint8_t *vlive_out, uint8_t *elive_out,
                                int64_t *rounds_out, int64_t *deleted_out)
{
    if (q < 1 || q > k || n > 4096) return KZO_ERR_ARG;
    int rc = validate(n, k, colour, m, edges);
    if (rc != KZO_OK) return rc;
    adj_t g;
    rc = adj_build(&g, n, k, colour, m, edges);
    if (rc != KZO_OK) return rc;
    scratch_t s;
    if (scratch_init(&s, n, k) != KZO_OK) {
        adj_free(&g);
        return KZO_ERR_OOM;
    }
    uint8_t *vlive = (uint8_t *)malloc((size_t)n + 1);
    uint8_t *elive = (uint8_t *)malloc((size_t)m + 1);
    uint8_t *fail_v = (uint8_t *)malloc((size_t)n + 1);
    uint8_t *fail_e = (uint8_t *)malloc((size_t)m + 1);
    uint8_t *A = (uint8_t *)calloc((size_t)n * (size_t)n + 1, 1);   /* live adjacency */
    int64_t *witness = (int64_t *)malloc(sizeof(int64_t) * ((size_t)m + 1));
    uint64_t *claim = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    int32_t *common = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int64_t rounds = 0, deleted = 0;
    if (!vlive || !elive || !fail_v || !fail_e || !A || !witness || !claim || !common) {
        rc = KZO_ERR_OOM;
        goto done;
    }
    memset(vlive, 1, (size_t)n);
    memset(elive, 1, (size_t)m);
    for (int64_t e = 0; e < m; e++) {
        int32_t x = edges[2 * e], y = edges[2 * e + 1];
        A[(size_t)x * n + y] = A[(size_t)y * n + x] = 1;
    }
    for (;;) {
        colour_index_phase(&g, &s, q, edges, vlive, elive, fail_v, fail_e);
        for (int64_t e = 0; e < m; e++)
            if (!elive[e]) {
                int32_t x = edges[2 * e], y = edges[2 * e + 1];
                A[(size_t)x * n + y] = A[(size_t)y * n + x] = 0;
            }
        /* one edge-dominance round on the snapshot: each dominated edge's witness */
        for (int64_t e = 0; e < m; e++) {
            witness[e] = -1;
            if (!elive[e]) continue;
            int32_t x = edges[2 * e], y = edges[2 * e + 1];
            /* the common neighbours of x and y */
            int32_t nx = 0;
            for (int32_t w = 0; w < n; w++)
                if (A[(size_t)x * n + w] && A[(size_t)y * n + w]) common[nx++] = w;
            for (int64_t f = 0; f < m; f++) {
                if (f == e || !elive[f]) continue;
                int32_t u = edges[2 * f], v = edges[2 * f + 1];
                /* u and v each non-adjacent to x or to y ({z, z} is no edge) */
                int u_ok = (u == x || u == y) || !A[(size_t)u * n + x] || !A[(size_t)u * n + y];
                int v_ok = (v == x || v == y) || !A[(size_t)v * n + x] || !A[(size_t)v * n + y];
                if (!u_ok || !v_ok) continue;
                /* every common neighbour of x and y is a neighbour of u and of v */
                int subset = 1;
                for (int32_t i = 0; i < nx && subset; i++)
                    if (!(A[(size_t)u * n + common[i]] && A[(size_t)v * n + common[i]])) subset = 0;
                if (!subset) continue;
                if (witness[e] < 0 ||
                    edge_key(u, v) < edge_key(edges[2 * witness[e]], edges[2 * witness[e] + 1]))
                    witness[e] = f;
            }
        }
        /* claims: the smallest key of a record through each vertex */
        for (int32_t z = 0; z < n; z++) claim[z] = UINT64_MAX;
        for (int64_t e = 0; e < m; e++) {
            if (witness[e] < 0) continue;
            const int32_t rec[4] = {edges[2 * e], edges[2 * e + 1], edges[2 * witness[e]],
                                    edges[2 * witness[e] + 1]};
            const uint64_t key = edge_key(edges[2 * e], edges[2 * e + 1]);
            for (int i = 0; i < 4; i++)
                if (key < claim[rec[i]]) claim[rec[i]] = key;
        }
        int64_t nd = 0;
        for (int64_t e = 0; e < m; e++) {
            fail_e[e] = 0;
            if (witness[e] < 0) continue;
            const int32_t rec[4] = {edges[2 * e], edges[2 * e + 1], edges[2 * witness[e]],
                                    edges[2 * witness[e] + 1]};
            const uint64_t key = edge_key(edges[2 * e], edges[2 * e + 1]);
            int mine = 1;
            for (int i = 0; i < 4; i++)
                if (claim[rec[i]] != key) mine = 0;
            fail_e[e] = (uint8_t)mine;
            nd += mine;
        }
        if (nd == 0) break;
        rounds++;
        deleted += nd;
        for (int64_t e = 0; e < m; e++)
            if (fail_e[e]) {
                int32_t x = edges[2 * e], y = edges[2 * e + 1];
                elive[e] = 0;
                A[(size_t)x * n + y] = A[(size_t)y * n + x] = 0;
            }
    }
    if (vlive_out) memcpy(vlive_out, vlive, (size_t)n);
    if (elive_out) memcpy(elive_out, elive, (size_t)m);
    if (rounds_out) *rounds_out = rounds;
    if (deleted_out) *deleted_out = deleted;
done:
    free(vlive);
    free(elive);
    free(fail_v);
    free(fail_e);
    free(A);
    free(witness);
    free(claim);
    free(common);
    scratch_free(&s);
    adj_free(&g);
    return rc;
}

/*
 * Colour indices of chosen elements on a given live state (vlive, elive).
 * The state must be consistent: a live edge has live endpoints.  Used for
 * the Figure 8 worked example and for sampled checks on large graphs.
 * which_v[nv] are vertex ids, which_e[ne] are edge ids; results go to
 * out_v[nv] and out_e[ne].  vlive/elive may be NULL (everything live).
 */
int kzo_indices(int32_t n, int32_t k, const int32_t *colour, int64_t m,
                const int32_t *edges, const uint8_t *vlive, const uint8_t *elive,
                const int32_t *which_v, int64_t nv, int32_t *out_v,
                const int64_t *which_e, int64_t ne, int32_t *out_e)
{
    int rc = validate(n, k, colour, m, edges);
    if (rc != KZO_OK) return rc;
    adj_t g;
    rc = adj_build(&g, n, k, colour, m, edges);
    if (rc != KZO_OK) return rc;
    scratch_t s;
    if (scratch_init(&s, n, k) != KZO_OK) {
        adj_free(&g);
        return KZO_ERR_OOM;
    }
    uint8_t *el = (uint8_t *)malloc((size_t)m + 1);
    if (!el) {
        scratch_free(&s);
        adj_free(&g);
        return KZO_ERR_OOM;
    }
    for (int64_t e = 0; e < m; e++) {
        int32_t u = edges[2 * e], v = edges[2 * e + 1];
        uint8_t live = elive ? elive[e] : 1;
        if (vlive && (!vlive[u] || !vlive[v])) live = 0;
        el[e] = live;
    }
    for (int64_t i = 0; i < nv; i++) {
        int32_t v = which_v[i];
        out_v[i] = (v >= 0 && v < n) ? vertex_index(&g, el, &s, v) : -1;
    }
    for (int64_t i = 0; i < ne; i++) {
        int64_t e = which_e[i];
        out_e[i] = (e >= 0 && e < m) ? edge_index(&g, el, &s, edges[2 * e], edges[2 * e + 1]) : -1;
    }
    free(el);
    scratch_free(&s);
    adj_free(&g);
    return KZO_OK;
}

/*
 * The same two indices read straight off a dense 0/1 adjacency matrix, for
 * graphs too large to hold as adjacency lists in a test.  bits is row-major,
 * row_words uint64 words per row, bit (j % 64) of word (j / 64) in row i set
 * iff {i,j} is an edge; vlive[n] (NULL = all live) masks dead vertices.  Edge
 * deletions are expressed by clearing bits in the matrix the caller passes.
 * pairs[2*np] are the (u,v) whose edge index is wanted (the pair need not be
 * an edge); verts[nv] the vertices whose index is wanted.
 */
static int bit_at(const uint64_t *bits, int64_t row_words, int32_t i, int32_t j)
{
    return (int)((bits[(int64_t)i * row_words + (j >> 6)] >> (j & 63)) & 1u);
}

int kzo_dense_indices(int32_t n, int32_t k, const int32_t *colour,
                      const uint64_t *bits, int64_t row_words, const uint8_t *vlive,
                      const int32_t *verts, int64_t nv, int32_t *out_v,
                      const int32_t *pairs, int64_t np, int32_t *out_e)
{
    if (n < 0 || k < 1 || row_words * 64 < n) return KZO_ERR_ARG;
    uint8_t *seen = (uint8_t *)malloc((size_t)k);
    if (!seen) return KZO_ERR_OOM;
    for (int64_t i = 0; i < nv; i++) {
        int32_t v = verts[i];
        memset(seen, 0, (size_t)k);
        int32_t count = 0;
        for (int32_t w = 0; w < n; w++) {
            if (vlive && !vlive[w]) continue;
            if (!bit_at(bits, row_words, v, w)) continue;
            int32_t c = colour[w];
            if (c == colour[v] || seen[c]) continue;
            seen[c] = 1;
            count++;
        }
        out_v[i] = count;
    }
    for (int64_t i = 0; i < np; i++) {
        int32_t u = pairs[2 * i], v = pairs[2 * i + 1];
        memset(seen, 0, (size_t)k);
        int32_t count = 0;
        for (int32_t w = 0; w < n; w++) {
            if (vlive && !vlive[w]) continue;
            if (!bit_at(bits, row_words, u, w) || !bit_at(bits, row_words, v, w)) continue;
            int32_t c = colour[w];
            if (c == colour[u] || c == colour[v] || seen[c]) continue;
            seen[c] = 1;
            count++;
        }
        out_e[i] = count;
    }
    free(seen);
    return KZO_OK;
}

/*
 * Session form of kzo_indices for repeated queries on one graph (the CPU
 * baseline times only the rule evaluations): kzo_open validates and builds
 * the adjacency list once; kzo_session_edge_index evaluates the edge colour
 * index of the given edge ids with every element live; kzo_close frees.
 */
typedef struct {
    adj_t g;
    scratch_t s;
    uint8_t *elive;
    const int32_t *edges;
} session_t;

void *kzo_open(int32_t n, int32_t k, const int32_t *colour, int64_t m, const int32_t *edges,
               int *rc_out)
{
    int rc = validate(n, k, colour, m, edges);
    session_t *ss = NULL;
    if (rc == KZO_OK) {
        ss = (session_t *)calloc(1, sizeof(session_t));
        if (!ss) rc = KZO_ERR_OOM;
    }
    if (rc == KZO_OK) rc = adj_build(&ss->g, n, k, colour, m, edges);
    if (rc == KZO_OK && scratch_init(&ss->s, n, k) != KZO_OK) {
        adj_free(&ss->g);
        rc = KZO_ERR_OOM;
    }
    if (rc == KZO_OK) {
        ss->elive = (uint8_t *)malloc((size_t)m + 1);
        if (!ss->elive) {
            scratch_free(&ss->s);
            adj_free(&ss->g);
            rc = KZO_ERR_OOM;
        } else {
            memset(ss->elive, 1, (size_t)m);
            ss->edges = edges;
        }
    }
    if (rc != KZO_OK) {
        free(ss);
        ss = NULL;
    }
    if (rc_out) *rc_out = rc;
    return ss;
}

int kzo_session_edge_index(void *session, const int64_t *which_e, int64_t ne, int32_t *out_e)
{
    session_t *ss = (session_t *)session;
    if (!ss) return KZO_ERR_ARG;
    for (int64_t i = 0; i < ne; i++) {
        int64_t e = which_e[i];
        out_e[i] = (e >= 0 && e < ss->g.m)
                       ? edge_index(&ss->g, ss->elive, &ss->s, ss->edges[2 * e], ss->edges[2 * e + 1])
                       : -1;
    }
    return KZO_OK;
}

void kzo_close(void *session)
{
    session_t *ss = (session_t *)session;
    if (!ss) return;
    free(ss->elive);
    scratch_free(&ss->s);
    adj_free(&ss->g);
    free(ss);
}
