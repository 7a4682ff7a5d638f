"""Seeded synthetic inputs: legally coloured random k-partite graphs.

This module only draws inputs. It holds none of the kernelization
arithmetic (no colour index, no rule, no fixpoint), so both the CUDA path
and the CPU oracle may consume what it produces.

A graph is returned as ``colour`` (int32[n], values in [0, k)) plus either

* ``edges``: int32[m, 2], canonical (u < v), sorted lexicographically, no
  duplicates; or
* ``bits``: uint64[n, ceil(n/64)], the symmetric 0/1 adjacency matrix with
  bit ``j % 64`` of word ``j // 64`` in row ``i`` set iff {i, j} is an edge.

Colourings are legal by construction: pairs of the same colour are never
joined (the problem of Section 4.2 assumes a legal k-colouring).

Workload recipes (seeds are fixed per workload: ``221200574 * 10 + i``):

* dense k-partite  : colour ~ U[0, k); each differently coloured pair is an
  edge with probability p; one k-clique is planted on one random vertex per
  colour (an empty class first receives a random vertex of the largest one).
* Chung-Lu sparse  : colour ~ Zipf(1.2) over k classes; expected degrees from
  a Pareto(2.3) tail capped at sqrt(sum w); edges drawn by the fast
  Chung-Lu sampler (endpoint pairs drawn with probability proportional to
  w_u * w_v), same-colour pairs and repeats dropped; 5 disjoint planted
  k-cliques.
* batch            : n = round(exp(U[ln 64, ln 4096])), k ~ U{6..32},
  p ~ U[0.3, 0.95], planted clique on even indices.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 221200574 * 10


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.uint64(seed & ((1 << 64) - 1))))


# ----------------------------------------------------------------------------
# format conversions (no method arithmetic)
# ----------------------------------------------------------------------------

def row_words(n: int) -> int:
    return (n + 63) // 64


def edges_to_bits(n: int, edges: np.ndarray) -> np.ndarray:
    """Symmetric uint64 bit matrix [n, ceil(n/64)] from an edge list."""
    W = row_words(n)
    bits = np.zeros((n, W), dtype=np.uint64)
    if len(edges):
        e = np.asarray(edges, dtype=np.int64)
        for a, b in ((e[:, 0], e[:, 1]), (e[:, 1], e[:, 0])):
            np.bitwise_or.at(bits, (a, b // 64),
                             np.left_shift(np.uint64(1), (b % 64).astype(np.uint64)))
    return bits


def bits_to_bool(bits: np.ndarray, n: int) -> np.ndarray:
    """Dense bool adjacency [n, n] from the uint64 bit matrix."""
    b8 = np.ascontiguousarray(bits).view(np.uint8)
    return np.unpackbits(b8, axis=1, bitorder="little")[:, :n].astype(bool)


def bool_to_bits(adj: np.ndarray) -> np.ndarray:
    """Pack bool rows [r, n] into uint64 words [r, ceil(n/64)]."""
    r, n = adj.shape
    W = row_words(n)
    padded = np.zeros((r, W * 64), dtype=bool)
    padded[:, :n] = adj
    return np.packbits(padded, axis=1, bitorder="little").view(np.uint64).reshape(r, W)


def bits_to_edges(bits: np.ndarray, n: int, block: int = 2048) -> np.ndarray:
    """Canonical sorted edge list (u < v) from the bit matrix."""
    out = []
    for a in range(0, n, block):
        b = min(n, a + block)
        blk = bits_to_bool(bits[a:b], n)
        iu, iv = np.nonzero(blk)
        iu = iu + a
        keep = iu < iv
        out.append(np.stack([iu[keep], iv[keep]], axis=1).astype(np.int32))
    if not out:
        return np.zeros((0, 2), dtype=np.int32)
    return np.concatenate(out, axis=0)


def canonical_edges(edges: np.ndarray) -> np.ndarray:
    """u < v, sorted, duplicates removed."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if len(e) == 0:
        return np.zeros((0, 2), dtype=np.int32)
    e = np.sort(e, axis=1)
    e = np.unique(e, axis=0)
    return e.astype(np.int32)


# ----------------------------------------------------------------------------
# colourings and planted cliques
# ----------------------------------------------------------------------------

def colours_uniform(rng: np.random.Generator, n: int, k: int) -> np.ndarray:
    return rng.integers(0, k, size=n, dtype=np.int64).astype(np.int32)


def colours_zipf(rng: np.random.Generator, n: int, k: int, s: float = 1.2) -> np.ndarray:
    q = (np.arange(1, k + 1, dtype=np.float64)) ** (-s)
    q /= q.sum()
    return rng.choice(k, size=n, p=q).astype(np.int32)


def plant_vertices(rng: np.random.Generator, colour: np.ndarray, k: int,
                   exclude: np.ndarray | None = None) -> np.ndarray:
    """One uniformly random vertex per colour (mutates ``colour`` so that an
    empty class receives a random vertex of the largest class first)."""
    n = len(colour)
    if n < k:
        raise ValueError("cannot plant a k-clique on fewer than k vertices")
    taken = np.zeros(n, dtype=bool)
    if exclude is not None:
        taken[exclude] = True
    for c in range(k):
        if not np.any((colour == c) & ~taken):
            sizes = np.bincount(colour[~taken], minlength=k)
            big = int(np.argmax(sizes))
            cand = np.nonzero((colour == big) & ~taken)[0]
            colour[int(cand[rng.integers(0, len(cand))])] = c
    picks = np.empty(k, dtype=np.int64)
    for c in range(k):
        cand = np.nonzero((colour == c) & ~taken)[0]
        picks[c] = cand[rng.integers(0, len(cand))]
        taken[picks[c]] = True
    return picks


def _clique_pairs(verts: np.ndarray) -> np.ndarray:
    iu, iv = np.triu_indices(len(verts), 1)
    return np.stack([verts[iu], verts[iv]], axis=1)


# ----------------------------------------------------------------------------
# dense random k-partite graphs
# ----------------------------------------------------------------------------

@dataclass
class Graph:
    n: int
    k: int
    colour: np.ndarray                 # int32[n]
    edges: np.ndarray | None = None    # int32[m, 2] canonical
    bits: np.ndarray | None = None     # uint64[n, W]
    planted: list | None = None        # list of int64 arrays (clique vertices)
    name: str = ""

    def get_edges(self) -> np.ndarray:
        if self.edges is None:
            self.edges = bits_to_edges(self.bits, self.n)
        return self.edges

    def get_bits(self) -> np.ndarray:
        if self.bits is None:
            self.bits = edges_to_bits(self.n, self.edges)
        return self.bits

    @property
    def m(self) -> int:
        if self.edges is not None:
            return int(len(self.edges))
        return int(sum(int(np.unpackbits(r.view(np.uint8)).sum()) for r in self.bits)) // 2


def kpartite(n: int, k: int, p: float, seed: int, planted: bool = True,
             out: str = "bits", block: int = 1024) -> Graph:
    """Random k-partite graph with uniform colours and a planted k-clique."""
    rng = _rng(seed)
    colour = colours_uniform(rng, n, k)
    picks = plant_vertices(rng, colour, k) if (planted and n >= k) else None
    W = row_words(n)
    upper = np.zeros((n, n), dtype=bool)
    p32 = np.float32(p)
    for a in range(0, n, block):
        b = min(n, a + block)
        r = rng.random((b - a, n), dtype=np.float32) < p32
        r &= colour[a:b, None] != colour[None, :]
        cols = np.arange(n)[None, :]
        rows = np.arange(a, b)[:, None]
        r &= cols > rows
        upper[a:b] = r
    if picks is not None:
        pr = _clique_pairs(np.sort(picks))
        upper[pr[:, 0], pr[:, 1]] = True
    bits = np.empty((n, W), dtype=np.uint64)
    for a in range(0, n, block):
        b = min(n, a + block)
        sym = upper[a:b] | upper[:, a:b].T
        bits[a:b] = bool_to_bits(sym)
    del upper
    g = Graph(n=n, k=k, colour=colour, bits=bits,
              planted=[np.sort(picks)] if picks is not None else [],
              name=f"kpartite(n={n},k={k},p={p},seed={seed})")
    if out == "edges":
        g.get_edges()
    return g


def tiny_random(seed: int, n: int, k: int, p: float, planted: bool = False) -> Graph:
    """Small graph as a canonical edge list (parity and pin cases)."""
    rng = _rng(seed)
    colour = colours_uniform(rng, n, k)
    pairs = []
    if n >= 2:
        iu, iv = np.triu_indices(n, 1)
        keep = (colour[iu] != colour[iv]) & (rng.random(len(iu)) < p)
        pairs.append(np.stack([iu[keep], iv[keep]], axis=1))
    plist = []
    if planted and n >= k:
        picks = plant_vertices(rng, colour, k)
        # recolouring may have made some drawn pair monochromatic: drop those
        if pairs:
            pr = pairs[0]
            pairs[0] = pr[colour[pr[:, 0]] != colour[pr[:, 1]]]
        pairs.append(_clique_pairs(np.sort(picks)))
        plist.append(np.sort(picks))
    edges = canonical_edges(np.concatenate(pairs, axis=0)) if pairs else np.zeros((0, 2), np.int32)
    return Graph(n=n, k=k, colour=colour, edges=edges, planted=plist,
                 name=f"tiny(seed={seed},n={n},k={k},p={p})")


# ----------------------------------------------------------------------------
# Chung-Lu sparse power-law graph with Zipf colour classes
# ----------------------------------------------------------------------------

def chung_lu(n: int, k: int, mean_degree: float, seed: int, gamma: float = 2.3,
             zipf_s: float = 1.2, n_planted: int = 5) -> Graph:
    rng = _rng(seed)
    colour = colours_zipf(rng, n, k, zipf_s)
    q = np.bincount(colour, minlength=k) / max(n, 1)
    inter = 1.0 - float(np.sum(q * q))
    target_m = mean_degree * n / 2.0
    # expected inter-colour edges ~ (S/2) * inter, S = sum of weights
    S_target = 2.0 * target_m / max(inter, 1e-9)
    w = (1.0 - rng.random(n)) ** (-1.0 / (gamma - 1.0))
    for _ in range(8):
        w *= S_target / w.sum()
        cap = math.sqrt(w.sum())
        w = np.minimum(w, cap)
    S = w.sum()
    n_draw = int(rng.poisson(S / 2.0))
    prob = w / S
    a = rng.choice(n, size=n_draw, p=prob)
    b = rng.choice(n, size=n_draw, p=prob)
    keep = (a != b) & (colour[a] != colour[b])
    e = np.stack([a[keep], b[keep]], axis=1)
    planted = []
    taken = np.zeros(0, dtype=np.int64)
    for _ in range(n_planted):
        picks = plant_vertices(rng, colour, k, exclude=taken)
        taken = np.concatenate([taken, picks])
        planted.append(np.sort(picks))
    # planting never recolours here unless a class is exhausted; re-filter
    e = e[colour[e[:, 0]] != colour[e[:, 1]]]
    allp = [e] + [_clique_pairs(p) for p in planted]
    edges = canonical_edges(np.concatenate(allp, axis=0))
    return Graph(n=n, k=k, colour=colour, edges=edges, planted=planted,
                 name=f"chung_lu(n={n},k={k},deg={mean_degree},seed={seed})")


# ----------------------------------------------------------------------------
# batch of graphs
# ----------------------------------------------------------------------------

def batch_specs(count: int, seed: int, n_lo: int = 64, n_hi: int = 4096,
                k_lo: int = 6, k_hi: int = 32, p_lo: float = 0.3, p_hi: float = 0.95):
    """(n, k, p, planted, graph_seed) for each graph of a batch."""
    rng = _rng(seed)
    specs = []
    for j in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        k = int(rng.integers(k_lo, k_hi + 1))
        p = float(rng.uniform(p_lo, p_hi))
        specs.append((n, k, p, j % 2 == 0, int(seed * 1000003 + j)))
    return specs


def batch(count: int, seed: int, **kw) -> list:
    return [kpartite(n, k, p, s, planted=pl) for (n, k, p, pl, s) in batch_specs(count, seed, **kw)]


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

WORKLOADS = {
    # name: (description, builder)
    "c1": "kpartite n=300 k=10 p=0.7, planted 10-clique",
    "c2": "kpartite n=4096 k=20 p=0.92, planted 20-clique",
    "c3": "chung-lu n=200000 k=12 zipf(1.2) mean degree 60, 5 planted 12-cliques",
    "c4": "batch of 1024 kpartite graphs, n log-uniform [64,4096], k U{6..32}, p U[0.3,0.95]",
    "c5": "kpartite n=32768 k=24 p=0.85, planted 24-clique",
    "c5c": "kpartite n=32768 k=24 p=0.12, planted 24-clique (the C5 size where the tensor form wins)",
    "c5s": "kpartite n=32768 k=24 p=0.07, planted 24-clique (the C5 size in the cascade regime)",
}

# the seed offset of the workloads that share a config number with another
_SEED_OFFSET = {"c5c": 10, "c5s": 20}


def workload_seed(name: str) -> int:
    """The fixed seed of a named workload: 221200574 * 10 + i for config i."""
    return SEED_BASE + int(name[1]) + _SEED_OFFSET.get(name, 0)


def workload(name: str, scale: float = 1.0):
    """Build a named workload. ``scale`` < 1 shrinks n (and the batch count)
    for small parity cases while keeping k, p and the structure."""
    seed = workload_seed(name)
    if name == "c1":
        return kpartite(max(10, int(300 * scale)), 10, 0.7, seed)
    if name == "c2":
        return kpartite(max(20, int(4096 * scale)), 20, 0.92, seed)
    if name == "c3":
        return chung_lu(max(2000, int(200_000 * scale)), 12, 60.0, seed)
    if name == "c4":
        return batch(max(2, int(1024 * scale)), seed)
    if name == "c5":
        return kpartite(max(24, int(32768 * scale)), 24, 0.85, seed)
    if name == "c5c":
        return kpartite(max(24, int(32768 * scale)), 24, 0.12, seed)
    if name == "c5s":
        return kpartite(max(24, int(32768 * scale)), 24, 0.07, seed)
    raise KeyError(name)
