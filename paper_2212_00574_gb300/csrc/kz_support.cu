// kz_support.cu -- the CSR path with incremental per-class support counts
// (schedule KZ_SCHED_SUPPORT): the same Jacobi sweeps of the thesis
// Section 4.2 rules as the plain CSR path, but each sweep re-tests only the
// elements whose counts changed.
//
// State, exact for the live graph S_t at the start of every sweep:
//   cnt_e[e][c]  live common neighbours of class c of live edge e
//                (number of live triangles (u, v, w) with col(w) = c),
//   cnt_v[v][c]  live neighbours of class c of live vertex v.
// A live edge fails the edge rule exactly when one of its needed classes
// (c != col u, col v) has count zero, a live vertex the vertex rule when one
// of the classes c != col v has count zero -- the rules of the thesis
// restated with counts (a class is covered iff its count is positive).
//
// Sweep t:
//   1. rule: every dirty element (its counts changed in the last update; all
//      live elements after a recount) is tested on the counts of S_t; the
//      failing edges are listed;
//   2. update (only when the sweep is applied): every live triangle of S_t
//      that loses an edge is visited once, from its deleted edge of smallest
//      id, and each surviving edge of it loses that witness; each deleted
//      edge decrements its endpoints' vertex counts.  The rows walked are
//      the live rows compacted at the last recount (their dead entries are
//      skipped).  After a sweep that deletes more than a quarter of the live
//      edges the counts are recounted from scratch on the compacted live
//      graph instead;
//   3. apply: the live flags drop the failing elements.
// Every edge of a failing vertex fails the edge rule in the same sweep (see
// kz_bitset.cu), so the edge list of step 1 already holds them.  Counts only
// fall, so an element whose counts did not change keeps its verdict: the
// failing sets, sweeps, per-sweep deletion counts and vertex deletion sweeps
// are those of the plain Jacobi sweeps.  The number of tests counts the
// elements actually tested.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "kz_internal.cuh"
#include "kz_rules.cuh"

namespace kz {

struct SupportBufs {
  uint32_t *cnt_e = nullptr;   // m * k
  uint32_t *cnt_v = nullptr;   // n * k
  uint8_t *edirty = nullptr;   // m
  uint8_t *vdirty = nullptr;   // n
  uint8_t *edel = nullptr;     // m: deleted in the running sweep
  uint8_t *vdel = nullptr;     // n
  int32_t *dlist = nullptr;    // m: the running sweep's deleted edges
  unsigned int *dcount = nullptr;
  size_t bytes = 0;
};

// Bytes of the support state of a graph (the schedule is refused above a
// budget: the per-class edge counts take 4 m k bytes).
static size_t support_bytes(kz_graph g) {
  const size_t n = (size_t)std::max(g->n, 1), m = (size_t)std::max<int64_t>(g->m, 1), k = (size_t)g->k;
  return 4 * m * k + 4 * n * k + 3 * m + 2 * n + 4 * m + 16;
}
constexpr size_t kSupportBudgetBytes = size_t(6) << 30;

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Vertex counts of the live graph; every live element starts dirty.
__global__ void support_init_kernel(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                                    const int32_t *__restrict__ col, const uint8_t *__restrict__ elive,
                                    const uint8_t *__restrict__ vlive, int64_t m, int32_t n, int32_t k,
                                    uint32_t *__restrict__ cnt_v, uint8_t *__restrict__ edirty,
                                    uint8_t *__restrict__ vdirty) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = tid; e < m; e += stride) {
    const uint8_t live = elive[e];
    edirty[e] = live;
    if (live) {
      const int32_t u = eu[e], v = ev[e];
      atomicAdd(&cnt_v[(int64_t)u * k + col[v]], 1u);
      atomicAdd(&cnt_v[(int64_t)v * k + col[u]], 1u);
    }
  }
  for (int64_t v = tid; v < n; v += stride) vdirty[v] = vlive[v];
}

__device__ __forceinline__ int64_t lower_bound_sorted(const int32_t *__restrict__ a, int64_t lo, int64_t hi,
                                                      int32_t x) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Edge counts of the live graph: one warp per oriented live edge u -> v;
// every live triangle is found once and adds its third vertex's class to
// each of its three edges.
__global__ void support_triangle_kernel(const int32_t *__restrict__ col, const int64_t *__restrict__ orow,
                                        const int32_t *__restrict__ oadj, const int32_t *__restrict__ oeid,
                                        const int32_t *__restrict__ osrc, const int64_t *__restrict__ n_or, int32_t k,
                                        uint32_t *__restrict__ cnt_e) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = *n_or;
  for (int64_t q = warp0; q < total; q += warps) {
    const int32_t u = osrc[q], v = oadj[q], euv = oeid[q];
    const int64_t ub = orow[u], ue = orow[u + 1];
    const int64_t vb = orow[v], ve = orow[v + 1];
    const bool walk_u = (ue - ub) <= (ve - vb);
    const int64_t wb = walk_u ? ub : vb, we = walk_u ? ue : ve;
    const int64_t sb = walk_u ? vb : ub, se = walk_u ? ve : ue;
    const int32_t cu = col[u], cv = col[v];
    for (int64_t i = wb + lane; i < we; i += 32) {
      const int32_t w = oadj[i];
      const int64_t j = lower_bound_sorted(oadj, sb, se, w);
      if (j < se && oadj[j] == w) {
        const int32_t e_walk = oeid[i], e_srch = oeid[j];
        const int32_t euw = walk_u ? e_walk : e_srch;
        const int32_t evw = walk_u ? e_srch : e_walk;
        atomicAdd(&cnt_e[(int64_t)euv * k + col[w]], 1u);
        atomicAdd(&cnt_e[(int64_t)euw * k + cv], 1u);
        atomicAdd(&cnt_e[(int64_t)evw * k + cu], 1u);
      }
    }
  }
}

// Step 1: the dirty live elements tested on the counts of the snapshot.
// Failing edges are flagged and listed; failing vertices flagged.
__global__ void support_rule_kernel(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                                    const int32_t *__restrict__ col, const uint8_t *__restrict__ elive,
                                    const uint8_t *__restrict__ vlive, int64_t m, int32_t n, int32_t k,
                                    const uint32_t *__restrict__ cnt_e, const uint32_t *__restrict__ cnt_v,
                                    uint8_t *__restrict__ edirty, uint8_t *__restrict__ vdirty,
                                    uint8_t *__restrict__ edel, uint8_t *__restrict__ vdel,
                                    int32_t *__restrict__ dlist, unsigned int *__restrict__ dcount,
                                    int32_t *__restrict__ v_sweep, DevState *st) {
  const int lane = threadIdx.x & 31;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t sweep_no = st->sweeps;
  unsigned long long tests = 0, de = 0, dv = 0;
  // the loop bound is rounded up so that whole warps take part in the list append
  const int64_t m_up = (m + 31) / 32 * 32;
  for (int64_t e = tid; e < m_up; e += stride) {
    bool fail = false;
    if (e < m) {
      if (edirty[e] && elive[e]) {
        tests++;
        const int32_t cu = col[eu[e]], cv = col[ev[e]];
        const uint32_t *ce = cnt_e + e * k;
        for (int c = 0; c < k; c++)
          if (c != cu && c != cv && ce[c] == 0u) {
            fail = true;
            break;
          }
        edirty[e] = 0;
      }
      edel[e] = fail ? 1 : 0;
    }
    const unsigned int ballot = __ballot_sync(0xffffffffu, fail);
    if (ballot) {
      unsigned int base = 0;
      if (lane == 0) base = atomicAdd(dcount, (unsigned int)__popc(ballot));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (fail) dlist[base + __popc(ballot & ((1u << lane) - 1u))] = (int32_t)e;
      de += fail ? 1 : 0;
    }
  }
  for (int64_t v = tid; v < n; v += stride) {
    bool fail = false;
    if (vdirty[v] && vlive[v]) {
      const int32_t cv = col[v];
      const uint32_t *cc = cnt_v + v * k;
      for (int c = 0; c < k; c++)
        if (c != cv && cc[c] == 0u) {
          fail = true;
          break;
        }
      vdirty[v] = 0;
    }
    vdel[v] = fail ? 1 : 0;
    if (fail) {
      dv++;
      if (v_sweep) v_sweep[v] = (int32_t)(sweep_no + 1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    tests += __shfl_down_sync(0xffffffffu, tests, o);
    de += __shfl_down_sync(0xffffffffu, de, o);
    dv += __shfl_down_sync(0xffffffffu, dv, o);
  }
  if (lane == 0) {
    if (tests) atomicAdd(&st->pass_tests, tests);
    if (de) atomicAdd(&st->pass_de, de);
    if (dv) atomicAdd(&st->pass_dv, dv);
  }
}

// Step 2: one warp per deleted edge e = (u, v).  Its endpoints lose a
// neighbour of the other's class; every live triangle (u, v, w) of the
// snapshot is handled here unless another of its edges is deleted too and has
// a smaller id; each surviving edge of the triangle loses the witness across.
__global__ void support_update_kernel(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                                      const int32_t *__restrict__ col, const int64_t *__restrict__ row,
                                      const int32_t *__restrict__ adj, const int32_t *__restrict__ eid,
                                      const uint8_t *__restrict__ elive, const uint8_t *__restrict__ edel,
                                      const int32_t *__restrict__ dlist, const unsigned int *__restrict__ dcount,
                                      int32_t k, uint32_t *__restrict__ cnt_e, uint32_t *__restrict__ cnt_v,
                                      uint8_t *__restrict__ edirty, uint8_t *__restrict__ vdirty) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = *dcount;
  for (int64_t q = warp0; q < total; q += warps) {
    const int32_t e = dlist[q];
    const int32_t u = eu[e], v = ev[e];
    const int32_t cu = col[u], cv = col[v];
    if (lane == 0) {
      atomicSub(&cnt_v[(int64_t)u * k + cv], 1u);
      atomicSub(&cnt_v[(int64_t)v * k + cu], 1u);
      vdirty[u] = 1;
      vdirty[v] = 1;
    }
    const int64_t ub = row[u], ue = row[u + 1];
    const int64_t vb = row[v], ve = row[v + 1];
    const bool walk_u = (ue - ub) <= (ve - vb);
    const int64_t wb = walk_u ? ub : vb, we = walk_u ? ue : ve;
    const int64_t sb = walk_u ? vb : ub, se = walk_u ? ve : ue;
    for (int64_t i = wb + lane; i < we; i += 32) {
      const int32_t e_walk = eid[i];
      if (!elive[e_walk]) continue;
      const int32_t w = adj[i];
      const int64_t j = lower_bound_sorted(adj, sb, se, w);
      if (j >= se || adj[j] != w) continue;
      const int32_t e_srch = eid[j];
      if (!elive[e_srch]) continue;
      const int32_t euw = walk_u ? e_walk : e_srch;  // the triangle's edge at u
      const int32_t evw = walk_u ? e_srch : e_walk;  // and at v
      const bool del_uw = edel[euw] != 0, del_vw = edel[evw] != 0;
      if ((del_uw && euw < e) || (del_vw && evw < e)) continue;  // handled from that edge
      if (!del_uw) {
        atomicSub(&cnt_e[(int64_t)euw * k + cv], 1u);
        edirty[euw] = 1;
      }
      if (!del_vw) {
        atomicSub(&cnt_e[(int64_t)evw * k + cu], 1u);
        edirty[evw] = 1;
      }
    }
  }
}

// Step 3: the applied sweep's deletions leave the live flags.
__global__ void support_apply_kernel(uint8_t *__restrict__ elive, uint8_t *__restrict__ vlive,
                                     const uint8_t *__restrict__ edel, const uint8_t *__restrict__ vdel, int64_t m,
                                     int32_t n, unsigned int *__restrict__ dcount) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = tid; e < m; e += stride)
    if (edel[e]) elive[e] = 0;
  for (int64_t v = tid; v < n; v += stride)
    if (vdel[v]) vlive[v] = 0;
  if (tid == 0) *dcount = 0;
}

__global__ void support_finish_kernel(DevState *st) {
  finish_pass(st, st->pass_dv, st->pass_de, st->pass_tests);
  st->pass_dv = st->pass_de = st->pass_tests = 0;
}

__global__ void support_begin_kernel(DevState *st, int64_t max_sweeps, int64_t passes0) {
  st->status = KZ_OK;
  st->cont = 1;
  st->sweeps = 0;
  st->passes = passes0;
  st->tests = 0;
  st->max_sweeps = max_sweeps;
  st->pass_dv = st->pass_de = st->pass_tests = 0;
  st->ticket = 0;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static int sms_of_device() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}

static kz_status support_alloc(kz_graph g, cudaStream_t s, SupportBufs *&out) {
  out = static_cast<SupportBufs *>(g->support_bufs);
  if (out) return KZ_OK;
  if (support_bytes(g) > kSupportBudgetBytes) return KZ_ERR_UNSUPPORTED;
  SupportBufs *b = new SupportBufs;
  g->support_bufs = b;  // owned by the handle from here on (freed with it)
  const size_t n = (size_t)std::max(g->n, 1), m = (size_t)std::max<int64_t>(g->m, 1), k = (size_t)g->k;
  KZ_TRY(graph_alloc(g, &b->cnt_e, m * k, s));
  KZ_TRY(graph_alloc(g, &b->cnt_v, n * k, s));
  KZ_TRY(graph_alloc(g, &b->edirty, m, s));
  KZ_TRY(graph_alloc(g, &b->vdirty, n, s));
  KZ_TRY(graph_alloc(g, &b->edel, m, s));
  KZ_TRY(graph_alloc(g, &b->vdel, n, s));
  KZ_TRY(graph_alloc(g, &b->dlist, m, s));
  KZ_TRY(graph_alloc(g, &b->dcount, 4, s));
  b->bytes = support_bytes(g);
  out = b;
  return KZ_OK;
}

void support_release(kz_graph g) {
  delete static_cast<SupportBufs *>(g->support_bufs);  // the device buffers are in g->allocs
  g->support_bufs = nullptr;
}

// Counts from scratch for the current live state: the plain path's
// compaction (the live rows, compacted, land in the other row buffer; the
// oriented CSR of the live edges beside them), then the per-class vertex and
// edge counts; every live element is marked dirty.  Returns the live edges.
static kz_status support_recount(kz_graph g, SupportBufs *b, cudaStream_t s, int64_t *live_edges) {
  const int grid = 8 * sms_of_device(), threads = 256;
  const int64_t n = g->n, m = g->m;
  const int k = g->k;
  const int c = g->sp_cur;
  uint8_t *elive = g->sp_elive[c], *vlive = g->sp_vlive[c];
  KZ_CUDA_TRY(cudaMemsetAsync(b->cnt_e, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(m, 1) * k, s));
  KZ_CUDA_TRY(cudaMemsetAsync(b->cnt_v, 0, sizeof(uint32_t) * (size_t)n * k, s));
  support_init_kernel<<<grid, threads, 0, s>>>(g->sp_eu, g->sp_ev, g->sp_col, elive, vlive, m, (int32_t)n, k,
                                               b->cnt_v, b->edirty, b->vdirty);
  KZ_TRY(sparse_orient_live(g, s));
  support_triangle_kernel<<<grid, threads, 0, s>>>(g->sp_col, g->sp_orow, g->sp_oadj, g->sp_oeid, g->sp_osrc,
                                                   g->sp_totals + 1, k, b->cnt_e);
  KZ_CUDA_TRY(cudaGetLastError());
  KZ_CUDA_TRY(cudaMemcpyAsync(live_edges, g->sp_totals + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  return KZ_OK;
}

// A sweep that deletes more than this share of the live edges is followed by
// a recount from scratch instead of the incremental update: the update
// visits every triangle a deleted edge closes (atomics on counts shared by
// hub edges), while a recount enumerates the much smaller surviving graph.
constexpr int64_t kRecountShareInv = 4;  // one quarter

kz_status sparse_kernelize_support(kz_graph g, const kz_options &opt, cudaStream_t s) {
  if (!g->has_csr) return KZ_ERR_UNSUPPORTED;
  const int64_t max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : (int64_t)g->n + g->m + 1;
  SupportBufs *b = nullptr;
  KZ_TRY(support_alloc(g, s, b));
  support_begin_kernel<<<1, 1, 0, s>>>(g->st, max_sweeps, g->n == 0 ? 1 : 0);
  KZ_CUDA_TRY(cudaGetLastError());
  if (g->n == 0) return KZ_OK;
  const int grid = 8 * sms_of_device(), threads = 256;
  const int64_t n = g->n, m = g->m;
  const int k = g->k;
  const int c = g->sp_cur;
  uint8_t *elive = g->sp_elive[c], *vlive = g->sp_vlive[c];
  KZ_CUDA_TRY(cudaMemsetAsync(b->dcount, 0, 4, s));
  // counts of the live graph; the compacted live rows (buffer c ^ 1) serve
  // the incremental updates until the next recount (dead entries skipped)
  int64_t live_edges = 0;
  KZ_TRY(support_recount(g, b, s, &live_edges));
  for (;;) {
    support_rule_kernel<<<grid, threads, 0, s>>>(g->sp_eu, g->sp_ev, g->sp_col, elive, vlive, m, (int32_t)n, k,
                                                 b->cnt_e, b->cnt_v, b->edirty, b->vdirty, b->edel, b->vdel,
                                                 b->dlist, b->dcount, g->sp_v_sweep, g->st);
    support_finish_kernel<<<1, 1, 0, s>>>(g->st);
    KZ_CUDA_TRY(cudaGetLastError());
    int32_t cont = 0;
    unsigned int deleted = 0;
    KZ_CUDA_TRY(cudaMemcpyAsync(&cont, &g->st->cont, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaMemcpyAsync(&deleted, b->dcount, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (!cont) {
      // a sweep that deleted nothing (or was refused by the limit) is not
      // applied; the counts still describe the live graph
      KZ_CUDA_TRY(cudaMemsetAsync(b->dcount, 0, 4, s));
      break;
    }
    if ((int64_t)deleted * kRecountShareInv > live_edges) {
      support_apply_kernel<<<grid, threads, 0, s>>>(elive, vlive, b->edel, b->vdel, m, (int32_t)n, b->dcount);
      KZ_CUDA_TRY(cudaGetLastError());
      KZ_TRY(support_recount(g, b, s, &live_edges));
      continue;
    }
    const int nx = c ^ 1;  // the compacted rows of the last recount
    support_update_kernel<<<grid, threads, 0, s>>>(g->sp_eu, g->sp_ev, g->sp_col, g->sp_row[nx], g->sp_adj[nx],
                                                   g->sp_eid[nx], elive, b->edel, b->dlist, b->dcount, k, b->cnt_e,
                                                   b->cnt_v, b->edirty, b->vdirty);
    support_apply_kernel<<<grid, threads, 0, s>>>(elive, vlive, b->edel, b->vdel, m, (int32_t)n, b->dcount);
    KZ_CUDA_TRY(cudaGetLastError());
    live_edges -= (int64_t)deleted;
  }
  return KZ_OK;
}

}  // namespace kz
