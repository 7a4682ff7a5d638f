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

// Per-graph buffers of the dominance rounds (allocated on first use).
struct DominanceBufs {
  int32_t *pos = nullptr, *deg = nullptr;
  uint32_t *D = nullptr;
  unsigned long long *count = nullptr;
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

void dominance_release(kz_graph g) {
  delete static_cast<DominanceBufs *>(g->dominance_bufs);
  g->dominance_bufs = nullptr;
}

}  // namespace kz
