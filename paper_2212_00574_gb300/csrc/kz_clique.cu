// kz_clique.cu -- the kernel's consumer: a q-clique search on the kernel and
// the maximum-clique driver that runs the kernelization for q = k, k-1, ...
// (thesis Section 4: a k-clique test run for several k answers the maximum
// clique problem; Section 4.2: the kernel for q keeps every q-clique).
//
// The search is an exact colour-ordered branch and bound on the host, over
// the kernel that the last kz_kernelize left (usually far smaller than the
// graph).  Under a legal colouring a clique holds at most one vertex per
// class, so the search picks a class, branches on its candidates (vertices
// adjacent to everything chosen so far) and on leaving the class out, and
// prunes when fewer classes with candidates remain than vertices are still
// needed.  It always branches on the class with the fewest candidates.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kz_internal.cuh"

namespace {

struct CliqueSearch {
  int nl = 0, k = 0, q = 0, W = 0;
  std::vector<uint64_t> adj;    // nl x W adjacency bitsets of the kernel
  std::vector<uint64_t> cls;    // k x W members of each class
  std::vector<int32_t> ids;     // compact index -> caller id
  std::vector<int32_t> chosen;  // compact indices
  std::vector<std::vector<uint64_t>> cand;  // candidate set per depth
  int64_t nodes = 0, limit = 0;
  bool found = false, exhausted = false;

  static int count_and(const uint64_t *a, const uint64_t *b, int W) {
    int c = 0;
    for (int w = 0; w < W; w++) c += __builtin_popcountll(a[w] & b[w]);
    return c;
  }

  // remaining: bit c set for classes not yet decided
  void rec(int depth, uint64_t remaining) {
    if ((int)chosen.size() == q) {
      found = true;
      return;
    }
    if (++nodes > limit) {
      exhausted = true;
      return;
    }
    const uint64_t *cd = cand[depth].data();
    const int need = q - (int)chosen.size();
    int usable = 0, best = -1, best_cnt = 0;
    for (uint64_t r = remaining; r; r &= r - 1) {
      const int c = __builtin_ctzll(r);
      const int cnt = count_and(cd, cls.data() + (size_t)c * W, W);
      if (cnt == 0) continue;
      usable++;
      if (best < 0 || cnt < best_cnt) {
        best = c;
        best_cnt = cnt;
      }
    }
    if (usable < need) return;
    const uint64_t *cm = cls.data() + (size_t)best * W;
    uint64_t *next = cand[depth + 1].data();
    for (int w = 0; w < W && !found && !exhausted; w++) {
      uint64_t bits = cd[w] & cm[w];
      while (bits && !found && !exhausted) {
        const int v = w * 64 + __builtin_ctzll(bits);
        bits &= bits - 1;
        const uint64_t *av = adj.data() + (size_t)v * W;
        for (int x = 0; x < W; x++) next[x] = cd[x] & av[x];
        chosen.push_back(v);
        rec(depth + 1, remaining & ~(1ull << best));  // deeper levels write cand[depth + 2 ..] only
        if (found) return;
        chosen.pop_back();
      }
    }
    if (found || exhausted) return;
    // leave the class out (possible only while enough other classes remain)
    if (usable - 1 >= need) {
      std::memcpy(cand[depth + 1].data(), cd, sizeof(uint64_t) * W);
      rec(depth + 1, remaining & ~(1ull << best));
    }
  }
};

// Kernel of g (after kz_kernelize) as compact adjacency bitsets.
kz_status build_search(kz_graph g, int32_t q, int64_t node_limit, CliqueSearch &s) {
  const int32_t n = g->n;
  std::vector<uint8_t> alive((size_t)std::max(n, 1));
  std::vector<int32_t> edges;
  int64_t m_live = 0;
  kz_stats st;
  try {
    edges.resize((size_t)std::max<int64_t>(2 * g->m, 2));
  } catch (...) {
    return KZ_ERR_OOM;
  }
  // a run stopped by its sweep limit still holds every q-clique
  kz_status rc = kz_fetch_kernel(g, alive.data(), edges.data(), g->m, &m_live, &st);
  if (rc != KZ_OK && rc != KZ_ERR_LIMIT) return rc;
  std::vector<int32_t> cidx((size_t)std::max(n, 1), -1);
  s.k = g->k;
  s.q = q;
  for (int32_t v = 0; v < n; v++)
    if (alive[v]) {
      cidx[v] = (int32_t)s.ids.size();
      s.ids.push_back(v);
    }
  s.nl = (int)s.ids.size();
  s.W = std::max(1, (s.nl + 63) / 64);
  if ((double)s.nl * s.W * 8.0 > (double)(1ull << 33)) return KZ_ERR_UNSUPPORTED;  // adjacency above 8 GB
  try {
    s.adj.assign((size_t)s.nl * s.W, 0ull);
    s.cls.assign((size_t)s.k * s.W, 0ull);
    s.cand.assign((size_t)s.k + 2, std::vector<uint64_t>((size_t)s.W, 0ull));
  } catch (...) {
    return KZ_ERR_OOM;
  }
  for (int64_t e = 0; e < m_live; e++) {
    const int32_t a = cidx[edges[2 * e]], b = cidx[edges[2 * e + 1]];
    if (a < 0 || b < 0) return KZ_ERR_INTERNAL;  // a kernel edge always has live endpoints
    s.adj[(size_t)a * s.W + b / 64] |= 1ull << (b % 64);
    s.adj[(size_t)b * s.W + a / 64] |= 1ull << (a % 64);
  }
  for (int i = 0; i < s.nl; i++) {
    // class of the caller id: relabelled ids are contiguous per class
    const int x = g->inv[s.ids[i]];
    const int c = (int)(std::upper_bound(g->coff.begin(), g->coff.end(), x) - g->coff.begin()) - 1;
    s.cls[(size_t)c * s.W + i / 64] |= 1ull << (i % 64);
  }
  for (int i = 0; i < s.nl; i++) s.cand[0][i / 64] |= 1ull << (i % 64);
  s.limit = node_limit > 0 ? node_limit : INT64_MAX;
  return KZ_OK;
}

}  // namespace

extern "C" {

kz_status kz_find_clique(kz_graph g, int32_t q, int64_t node_limit, int32_t *clique_out, int32_t *found) {
  if (!g || !found || q < 0 || q > g->k || (q > 0 && !clique_out)) return KZ_ERR_ARG;
  if (!g->kernelized) return KZ_ERR_NOT_READY;
  *found = 0;
  CliqueSearch s;
  KZ_TRY(build_search(g, q, node_limit, s));
  if (q == 0) {
    *found = 1;
    return KZ_OK;
  }
  const uint64_t all = s.k >= 64 ? ~0ull : ((1ull << s.k) - 1);
  s.rec(0, all);
  if (s.found) {
    std::vector<int32_t> out;
    for (int v : s.chosen) out.push_back(s.ids[v]);
    std::sort(out.begin(), out.end());
    std::memcpy(clique_out, out.data(), sizeof(int32_t) * q);
    *found = 1;
    return KZ_OK;
  }
  return s.exhausted ? KZ_ERR_LIMIT : KZ_OK;
}

kz_status kz_max_clique(kz_graph g, const kz_options *opt, int64_t node_limit, int32_t *q_out, int32_t *clique_out,
                        void *stream) {
  if (!g || !q_out || (g->n > 0 && !clique_out)) return KZ_ERR_ARG;
  kz_options o;
  if (opt) o = *opt;
  else kz_default_options(&o);
  *q_out = 0;
  if (g->n == 0) return KZ_OK;
  for (int32_t q = g->k; q >= 1; q--) {
    KZ_TRY(kz_reset(g, stream));
    o.clique_k = q;
    KZ_TRY(kz_kernelize(g, &o, stream));
    int32_t found = 0;
    const kz_status rc = kz_find_clique(g, q, node_limit, clique_out, &found);
    if (rc == KZ_ERR_LIMIT) {
      *q_out = q;  // the size at which the search gave up
      return KZ_ERR_LIMIT;
    }
    KZ_TRY(rc);
    if (found) {
      *q_out = q;
      return KZ_OK;
    }
  }
  return KZ_ERR_INTERNAL;  // q = 1 always finds a vertex of a non-empty graph
}

}  // extern "C"
