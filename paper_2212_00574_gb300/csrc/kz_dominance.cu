// kz_dominance.cu -- rounds of vertex dominance (thesis Section 4.3,
// Definition 4.3.1) on the bitset rows, run between colour-index fixpoints.
//
// Vertex b dominates vertex a when they are distinct, not adjacent, and the
// live neighbourhood N(a) lies inside N(b).  The definition's Remarks allow
// deleting a: a clique through a becomes one through b (b is adjacent to
// every other member), so the clique number is kept although some cliques
// go.  A round tests every live vertex on the same snapshot and deletes the
// dominated ones together; of two vertices with equal neighbourhoods only the
// one with the smaller relabelled id goes (relabelled ids order vertices by
// (colour, caller id)), so every deleted vertex keeps a surviving dominator.
//
// Kernels, all on the current ping-pong buffer:
//   position_kernel   word and bit of every vertex inside a row (once);
//   degree_kernel     live degree of every vertex (-1: deleted);
//   dominated_kernel  one warp per vertex a: the lanes filter 32 candidates
//                     b at a time (live, deg(b) >= deg(a), not in a's row),
//                     then the warp tests N(a) & ~N(b) == 0 word-parallel
//                     for each survivor; a dominated a sets its bit in a
//                     deletion mask laid out like the vertex live words;
//   apply_kernel      clears the deleted vertices' rows, their bits in every
//                     row, and their live bits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "kz_internal.cuh"

namespace kz {
namespace dom {

// Word (r * k + c) and bit of relabelled vertex x inside any row, as
// (word << 5) | bit.
__global__ void position_kernel(int32_t n, int32_t k, const int32_t *__restrict__ coff, int32_t *__restrict__ pos) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = k;  // coff[lo] <= x < coff[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (coff[mid] <= x) lo = mid;
      else hi = mid;
    }
    const int ix = (int)x - coff[lo];
    pos[x] = ((((ix >> 5) * k) + lo) << 5) | (ix & 31);
  }
}

__global__ void degree_kernel(const uint32_t *__restrict__ A, const uint32_t *__restrict__ V, int32_t n, int32_t ldw,
                              const int32_t *__restrict__ pos, int32_t *__restrict__ deg) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = warp0; x < n; x += warps) {
    const int p = pos[x];
    const bool live = (V[p >> 5] >> (p & 31)) & 1u;
    int d = 0;
    if (live) {
      const uint32_t *row = A + x * ldw;
      for (int w = lane; w < ldw; w += 32) d += __popc(row[w]);
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    }
    if (lane == 0) deg[x] = live ? d : -1;
  }
}

__global__ void dominated_kernel(const uint32_t *__restrict__ A, int32_t n, int32_t ldw,
                                 const int32_t *__restrict__ pos, const int32_t *__restrict__ deg,
                                 uint32_t *__restrict__ D, unsigned long long *__restrict__ count) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long found = 0;
  for (int64_t a = warp0; a < n; a += warps) {
    const int da = deg[a];
    if (da < 0) continue;
    const uint32_t *ra = A + a * ldw;
    bool dominated = false;
    // the lanes filter 32 candidates at a time; the warp then tests the
    // survivors' rows one by one
    for (int64_t b0 = 0; b0 < n && !dominated; b0 += 32) {
      const int64_t b = b0 + lane;
      bool cand = false;
      if (b < n && b != a) {
        const int db = deg[b];
        const int pb = pos[b];
        cand = db >= da                                 // a deleted b has deg -1 <= da
               && !((ra[pb >> 5] >> (pb & 31)) & 1u)    // adjacent: b is in N(a), never in N(b)
               && !(db == da && b < a);                 // equal neighbourhoods: only the smaller id goes
      }
      uint32_t todo = __ballot_sync(0xffffffffu, cand);
      while (todo && !dominated) {
        const int64_t bb = b0 + __ffs(todo) - 1;
        todo &= todo - 1;
        const uint32_t *rb = A + bb * ldw;
        bool outside = false;
        for (int w0 = 0; w0 < ldw && !outside; w0 += 32) {
          const int w = w0 + lane;
          const bool miss = w < ldw && (ra[w] & ~rb[w]) != 0u;
          outside = __any_sync(0xffffffffu, miss);
        }
        dominated = !outside;
      }
    }
    if (dominated && lane == 0) {
      const int pa = pos[a];
      atomicOr(&D[pa >> 5], 1u << (pa & 31));
      found++;
    }
  }
  if (lane == 0 && found) atomicAdd(count, found);
}

__global__ void apply_kernel(uint32_t *__restrict__ A, uint32_t *__restrict__ V, const uint32_t *__restrict__ D,
                             int32_t n, int32_t ldw, const int32_t *__restrict__ pos) {
  const int64_t total = (int64_t)n * ldw;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = t / ldw;
    const int w = (int)(t - y * ldw);
    const int py = pos[y];
    const bool gone = (D[py >> 5] >> (py & 31)) & 1u;
    A[t] = gone ? 0u : (A[t] & ~D[w]);
    if (y == 0) V[w] &= ~D[w];
  }
}

}  // namespace dom

// ---------------------------------------------------------------------------
// Edge dominance (thesis Section 4.3, Definitions 4.3.2 and 4.3.3).
//
// Edge f = {u, v} dominates a distinct edge e = {x, y} when every common
// neighbour of x and y is a neighbour of u and of v (X = N(x) ∩ N(y) ⊆
// N(u) ∩ N(v)) and each of u, v is non-adjacent to x or to y (a vertex is not
// adjacent to itself).  The non-adjacency conditions follow from the subset
// one: a vertex z with X ⊆ N(z) cannot lie in X, since no vertex is its own
// neighbour.  So the dominators of e are the live edges other than e inside
// C(e) = {x, y} ∪ {z : X ⊆ N(z)}, and since X is not empty after the
// colour-index fixpoint for a clique size of at least 3 (a live edge then has
// a common neighbour), the candidates z are neighbours of any one w in X.
//
// A round, on the snapshot: every dominated edge takes as witness the
// dominator of smallest key (key of an edge = its caller ids, smaller
// first); each vertex of e and of its witness receives e's key as a claim
// (the smallest claim wins); an edge whose claims it holds at all of its
// record's vertices is deleted.  The deleted records are vertex-disjoint,
// so the round equals deleting them one after another, each still
// dominated by its witness when its turn comes.
// ---------------------------------------------------------------------------
namespace edom {

struct Record {
  int32_t x, y, u, v;
  unsigned long long key;
};

__device__ __forceinline__ unsigned long long edge_key(const int32_t *__restrict__ perm, int a, int b) {
  const uint32_t pa = (uint32_t)perm[a], pb = (uint32_t)perm[b];
  const uint32_t lo = pa < pb ? pa : pb, hi = pa < pb ? pb : pa;
  return ((unsigned long long)lo << 32) | hi;
}

// Relabelled vertex of bit b of word w of a row.
__device__ __forceinline__ int vertex_of(const int32_t *__restrict__ coff, int k, int w, int b) {
  return coff[w % k] + 32 * (w / k) + b;
}

// One warp per vertex x; the warp takes x's live edges {x, y}, y > x, one at a
// time.  Per edge: X into the warp's scratch row, the first vertex w0 of X,
// the candidates z in N(w0) filtered lane-parallel (each lane runs its
// candidates' subset tests, stopping at the first word that fails), C(e) as
// a bit mask in the warp's second scratch row, then the smallest key among
// the live edges inside C(e) other than e.
__global__ void witness_kernel(const uint32_t *__restrict__ A, int32_t n, int32_t k, int32_t ldw,
                               const int32_t *__restrict__ coff, const int32_t *__restrict__ pos,
                               const int32_t *__restrict__ perm, uint32_t *__restrict__ scratch,
                               Record *__restrict__ rec, unsigned long long *__restrict__ n_rec) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t *Xs = scratch + warp0 * 2 * (int64_t)ldw;  // X of the current edge
  uint32_t *Cm = Xs + ldw;                            // C(e) as a bit mask
  for (int64_t x = warp0; x < n; x += warps) {
    const uint32_t *rx = A + x * ldw;
    for (int wy0 = 0; wy0 < ldw; wy0 += 32) {
      const int wyl = wy0 + lane;
      uint32_t ybits = wyl < ldw ? rx[wyl] : 0u;
      // the y of this chunk, one at a time across the warp
      for (;;) {
        const uint32_t have = __ballot_sync(0xffffffffu, ybits != 0u);
        if (!have) break;
        const int src = __ffs(have) - 1;
        const uint32_t wb = __shfl_sync(0xffffffffu, ybits, src);
        const int b = __ffs(wb) - 1;
        if (lane == src) ybits &= ybits - 1;
        const int y = vertex_of(coff, k, wy0 + src, b);
        if (y <= x) continue;
        const uint32_t *ry = A + (int64_t)y * ldw;
        // X and its first set word
        int first = ldw;
        for (int w = lane; w < ldw; w += 32) {
          const uint32_t xw = rx[w] & ry[w];
          Xs[w] = xw;
          Cm[w] = 0u;
          if (xw && w < first) first = w;
        }
        first = __reduce_min_sync(0xffffffffu, first);
        __syncwarp();
        if (first >= ldw) continue;  // no common neighbour (not reached for q >= 3)
        const int w0 = vertex_of(coff, k, first, __ffs(Xs[first]) - 1);
        const uint32_t *r0 = A + (int64_t)w0 * ldw;
        if (lane == 0) {
          const int px = pos[x], py = pos[y];
          atomicOr(&Cm[px >> 5], 1u << (px & 31));
          atomicOr(&Cm[py >> 5], 1u << (py & 31));
        }
        // candidates z in N(w0) other than x and y: X must lie in N(z)
        bool found = false;
        for (int w = lane; w < ldw; w += 32) {
          uint32_t zb = r0[w];
          while (zb) {
            const int bz = __ffs(zb) - 1;
            zb &= zb - 1;
            const int z = vertex_of(coff, k, w, bz);
            if (z == x || z == y) continue;
            const uint32_t *rz = A + (int64_t)z * ldw;
            bool in = true;
            for (int j = first; j < ldw && in; j++) in = (Xs[j] & ~rz[j]) == 0u;
            if (in) {
              atomicOr(&Cm[w], 1u << bz);
              found = true;
            }
          }
        }
        // no candidate: C(e) = {x, y} holds no edge but e itself
        if (!__any_sync(0xffffffffu, found)) continue;
        __syncwarp();
        // the dominator of smallest key: live edges {z1, z2} inside C(e)
        unsigned long long best = ~0ull;
        int bu = -1, bv = -1;
        for (int w = lane; w < ldw; w += 32) {
          uint32_t cb = Cm[w];
          while (cb) {
            const int b1 = __ffs(cb) - 1;
            cb &= cb - 1;
            const int z1 = vertex_of(coff, k, w, b1);
            const uint32_t *r1 = A + (int64_t)z1 * ldw;
            for (int j = 0; j < ldw; j++) {
              uint32_t pb = r1[j] & Cm[j];
              while (pb) {
                const int b2 = __ffs(pb) - 1;
                pb &= pb - 1;
                const int z2 = vertex_of(coff, k, j, b2);
                if (z2 <= z1) continue;
                if ((z1 == x && z2 == y) || (z1 == y && z2 == x)) continue;
                const unsigned long long kk = edge_key(perm, z1, z2);
                if (kk < best) {
                  best = kk;
                  bu = z1;
                  bv = z2;
                }
              }
            }
          }
        }
        unsigned long long wbest = best;
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long other = __shfl_xor_sync(0xffffffffu, wbest, o);
          wbest = other < wbest ? other : wbest;
        }
        const uint32_t holder = __ballot_sync(0xffffffffu, best == wbest && wbest != ~0ull);
        if (holder && lane == __ffs(holder) - 1) {
          const unsigned long long at = atomicAdd(n_rec, 1ull);
          Record r;
          r.x = (int32_t)x;
          r.y = y;
          r.u = bu;
          r.v = bv;
          r.key = edge_key(perm, (int)x, y);
          rec[at] = r;
        }
        __syncwarp();
      }
    }
  }
}

__global__ void claim_kernel(const Record *__restrict__ rec, const unsigned long long *__restrict__ n_rec,
                             unsigned long long *__restrict__ claim) {
  const int64_t total = (int64_t)*n_rec;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const Record r = rec[i];
    atomicMin(&claim[r.x], r.key);
    atomicMin(&claim[r.y], r.key);
    atomicMin(&claim[r.u], r.key);
    atomicMin(&claim[r.v], r.key);
  }
}

// Deletes the edges that hold every claim of their record.
__global__ void select_kernel(uint32_t *__restrict__ A, int32_t ldw, const int32_t *__restrict__ pos,
                              const Record *__restrict__ rec, const unsigned long long *__restrict__ n_rec,
                              const unsigned long long *__restrict__ claim, unsigned long long *__restrict__ count) {
  const int64_t total = (int64_t)*n_rec;
  unsigned long long mine = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const Record r = rec[i];
    if (claim[r.x] != r.key || claim[r.y] != r.key || claim[r.u] != r.key || claim[r.v] != r.key) continue;
    const int px = pos[r.x], py = pos[r.y];
    atomicAnd(&A[(int64_t)r.x * ldw + (py >> 5)], ~(1u << (py & 31)));
    atomicAnd(&A[(int64_t)r.y * ldw + (px >> 5)], ~(1u << (px & 31)));
    mine++;
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(count, mine);
}

}  // namespace edom

// Per-graph buffers of the dominance rounds (allocated on first use).
struct DominanceBufs {
  int32_t *pos = nullptr, *deg = nullptr;
  uint32_t *D = nullptr;
  unsigned long long *count = nullptr;
  // edge dominance
  unsigned long long *n_rec = nullptr;
  edom::Record *rec = nullptr;
  unsigned long long *claim = nullptr;
  uint32_t *scratch = nullptr;
  int64_t scratch_warps = 0;
};

static int sms_d() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

kz_status dominance_round(kz_graph g, int64_t *removed, cudaStream_t s) {
  *removed = 0;
  if (g->n == 0) return KZ_OK;
  if (!g->dominance_bufs) {
    DominanceBufs *b = new DominanceBufs();
    g->dominance_bufs = b;
    KZ_TRY(graph_alloc(g, &b->pos, (size_t)g->n, s));
    KZ_TRY(graph_alloc(g, &b->deg, (size_t)g->n, s));
    KZ_TRY(graph_alloc(g, &b->D, (size_t)g->ldw, s));
    KZ_TRY(graph_alloc(g, &b->count, 1, s));
    dom::position_kernel<<<4 * sms_d(), 256, 0, s>>>(g->n, g->k, g->d_coff, b->pos);
    KZ_CUDA_TRY(cudaGetLastError());
  }
  DominanceBufs &b = *static_cast<DominanceBufs *>(g->dominance_bufs);
  int32_t cur = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&cur, &g->st->cur, 4, cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  uint32_t *A = g->A[cur & 1];
  uint32_t *V = g->V[cur & 1];
  KZ_CUDA_TRY(cudaMemsetAsync(b.D, 0, (size_t)g->ldw * 4, s));
  KZ_CUDA_TRY(cudaMemsetAsync(b.count, 0, 8, s));
  const int sms = sms_d();
  dom::degree_kernel<<<8 * sms, 256, 0, s>>>(A, V, g->n, g->ldw, b.pos, b.deg);
  dom::dominated_kernel<<<8 * sms, 256, 0, s>>>(A, g->n, g->ldw, b.pos, b.deg, b.D, b.count);
  dom::apply_kernel<<<8 * sms, 256, 0, s>>>(A, V, b.D, g->n, g->ldw, b.pos);
  KZ_CUDA_TRY(cudaGetLastError());
  unsigned long long h = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&h, b.count, 8, cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  *removed = (int64_t)h;
  g->ab_synced = false;  // rows changed outside the sweep kernels
  return KZ_OK;
}

constexpr int kEdgeDomBlocksPerSm = 4;

kz_status edge_dominance_round(kz_graph g, int64_t *removed, cudaStream_t s) {
  *removed = 0;
  if (g->n == 0) return KZ_OK;
  if (!g->dominance_bufs) {
    DominanceBufs *b = new DominanceBufs();
    g->dominance_bufs = b;
    KZ_TRY(graph_alloc(g, &b->pos, (size_t)g->n, s));
    KZ_TRY(graph_alloc(g, &b->deg, (size_t)g->n, s));
    KZ_TRY(graph_alloc(g, &b->D, (size_t)g->ldw, s));
    KZ_TRY(graph_alloc(g, &b->count, 1, s));
    dom::position_kernel<<<4 * sms_d(), 256, 0, s>>>(g->n, g->k, g->d_coff, b->pos);
    KZ_CUDA_TRY(cudaGetLastError());
  }
  DominanceBufs &b = *static_cast<DominanceBufs *>(g->dominance_bufs);
  const int sms = sms_d();
  const int grid = kEdgeDomBlocksPerSm * sms;
  if (!b.rec) {
    b.scratch_warps = (int64_t)grid * (256 / 32);
    KZ_TRY(graph_alloc(g, &b.n_rec, 1, s));
    KZ_TRY(graph_alloc(g, &b.rec, (size_t)std::max<int64_t>(g->m, 1), s));
    KZ_TRY(graph_alloc(g, &b.claim, (size_t)g->n, s));
    KZ_TRY(graph_alloc(g, &b.scratch, (size_t)(b.scratch_warps * 2 * g->ldw), s));
  }
  int32_t cur = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&cur, &g->st->cur, 4, cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  uint32_t *A = g->A[cur & 1];
  KZ_CUDA_TRY(cudaMemsetAsync(b.count, 0, 8, s));
  KZ_CUDA_TRY(cudaMemsetAsync(b.claim, 0xff, (size_t)g->n * 8, s));
  unsigned long long *n_rec = b.n_rec;
  KZ_CUDA_TRY(cudaMemsetAsync(n_rec, 0, 8, s));
  edom::witness_kernel<<<grid, 256, 0, s>>>(A, g->n, g->k, g->ldw, g->d_coff, b.pos, g->d_perm, b.scratch, b.rec,
                                            n_rec);
  edom::claim_kernel<<<grid, 256, 0, s>>>(b.rec, n_rec, b.claim);
  edom::select_kernel<<<grid, 256, 0, s>>>(A, g->ldw, b.pos, b.rec, n_rec, b.claim, b.count);
  KZ_CUDA_TRY(cudaGetLastError());
  unsigned long long h = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&h, b.count, 8, cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  *removed = (int64_t)h;
  g->ab_synced = false;  // rows changed outside the sweep kernels
  return KZ_OK;
}

void dominance_release(kz_graph g) {
  delete static_cast<DominanceBufs *>(g->dominance_bufs);
  g->dominance_bufs = nullptr;
}

}  // namespace kz
