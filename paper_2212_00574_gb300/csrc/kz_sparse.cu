// kz_sparse.cu -- CSR path of the colour-index kernelization, for graphs too
// large or too sparse for bitset rows (thesis Section 4.2 rules).
//
// Vertices keep the caller's ids.  Each Jacobi pass:
//   1. compacts the live adjacency (CSR rows keep only live edges, order
//      preserved) and builds a degree-oriented CSR of the live edges: every
//      live edge once, from its lower-ranked to its higher-ranked endpoint;
//   2. enumerates every live triangle once (u -> v -> w in rank order, by
//      intersecting the sorted oriented rows of u and v) and ORs the third
//      vertex's colour into each edge's colour mask;
//   3. evaluates both rules on the snapshot: a live vertex fails when the
//      colours of its live neighbours number fewer than k-1; a live edge fails
//      when its mask (the colours of its live common neighbours) has fewer than
//      k-2 bits;
//   4. writes the next live flags (ping-pong) and closes the pass.
// Every edge of a failing vertex also fails the edge rule in the same pass
// (see kz_bitset.cu), so step 4 only applies the two failure sets.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kz_internal.cuh"
#include "kz_rules.cuh"

namespace kz {

// ---------------------------------------------------------------------------
// exclusive scan of int32 counts into int64 offsets (3 kernels)
// ---------------------------------------------------------------------------

constexpr int kScanBlock = 1024;

__global__ void scan_block_sums(const int32_t *__restrict__ in, int64_t n, int64_t *__restrict__ sums) {
  __shared__ int64_t s[32];
  const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  int64_t v = i < n ? in[i] : 0;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int64_t w = s[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = w;
  }
}

// Exclusive scan of the block sums in place (one CTA, any count).
__global__ void scan_sums_serial(int64_t *sums, int64_t nblocks, int64_t *total) {
  __shared__ int64_t carry;
  __shared__ int64_t warp_tot[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nblocks; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < nblocks ? sums[i] : 0;
    // inclusive warp scan
    int64_t x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
      int64_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const int64_t before = carry + (w > 0 ? warp_tot[w - 1] : 0) + x - v;
    if (i < nblocks) sums[i] = before;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void scan_apply(const int32_t *__restrict__ in, int64_t n, const int64_t *__restrict__ sums,
                           int64_t *__restrict__ out, const int64_t *__restrict__ total) {
  __shared__ int64_t warp_tot[32];
  const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  const int64_t v = i < n ? in[i] : 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t t = warp_tot[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  if (i < n) out[i] = sums[blockIdx.x] + (w > 0 ? warp_tot[w - 1] : 0) + x - v;
  if (i == n - 1) out[n] = *total;
}

// out[0..n] = exclusive prefix of in[0..n-1] (out[n] = total); sums holds
// n / kScanBlock + 1 partial sums.
kz_status scan_counts(const int32_t *in, int64_t n, int64_t *out, int64_t *sums, int64_t *total, cudaStream_t s) {
  if (n <= 0) return cuda_status(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  scan_block_sums<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, sums);
  scan_sums_serial<<<1, kScanBlock, 0, s>>>(sums, nb, total);
  scan_apply<<<(unsigned)nb, kScanBlock, 0, s>>>(in, n, sums, out, total);
  return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// pass kernels
// ---------------------------------------------------------------------------

struct SparseArgs {
  int32_t n;
  int32_t k;
  int32_t q;                // clique size sought (k for the thesis's rules)
  const int32_t *col;       // colour of each vertex
  const int32_t *rank;      // orientation rank
  const int64_t *row;       // live CSR of this pass (n + 1)
  const int32_t *adj;
  const int32_t *eid;
  const uint8_t *elive;     // snapshot flags
  const uint8_t *vlive;
  int64_t m;
};

// Per row: live entries and live entries towards higher rank.
__global__ void sparse_count_kernel(SparseArgs a, int32_t *__restrict__ cnt_live, int32_t *__restrict__ cnt_or) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp0; u < a.n; u += warps) {
    const int64_t b = a.row[u], e = a.row[u + 1];
    const int32_t ru = a.rank[u];
    int32_t cl = 0, co = 0;
    for (int64_t i = b + lane; i < e; i += 32) {
      const int32_t v = a.adj[i];
      const bool keep = a.elive[a.eid[i]] != 0;
      cl += keep;
      co += keep && a.rank[v] > ru;
    }
    for (int o = 16; o > 0; o >>= 1) {
      cl += __shfl_down_sync(0xffffffffu, cl, o);
      co += __shfl_down_sync(0xffffffffu, co, o);
    }
    if (lane == 0) {
      cnt_live[u] = cl;
      cnt_or[u] = co;
    }
  }
}

// Order-preserving compaction of each row into the next live CSR and the
// oriented CSR (rows stay sorted by neighbour id).
__global__ void sparse_fill_kernel(SparseArgs a, const int64_t *__restrict__ row_n, int32_t *__restrict__ adj_n,
                                   int32_t *__restrict__ eid_n, const int64_t *__restrict__ orow,
                                   int32_t *__restrict__ oadj, int32_t *__restrict__ oeid,
                                   int32_t *__restrict__ osrc) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp0; u < a.n; u += warps) {
    const int64_t b = a.row[u], e = a.row[u + 1];
    const int32_t ru = a.rank[u];
    int64_t pl = row_n[u], po = orow[u];
    for (int64_t base = b; base < e; base += 32) {
      const int64_t i = base + lane;
      int32_t v = 0, ed = 0;
      bool keep = false, ori = false;
      if (i < e) {
        v = a.adj[i];
        ed = a.eid[i];
        keep = a.elive[ed] != 0;
        ori = keep && a.rank[v] > ru;
      }
      const uint32_t mk = __ballot_sync(0xffffffffu, keep);
      const uint32_t mo = __ballot_sync(0xffffffffu, ori);
      if (keep) {
        const int64_t q = pl + __popc(mk & lt);
        adj_n[q] = v;
        eid_n[q] = ed;
      }
      if (ori) {
        const int64_t q = po + __popc(mo & lt);
        oadj[q] = v;
        oeid[q] = ed;
        osrc[q] = (int32_t)u;
      }
      pl += __popc(mk);
      po += __popc(mo);
    }
  }
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *__restrict__ a, int64_t lo, int64_t hi,
                                                   int32_t x) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One warp per oriented edge u -> v: the lanes walk the shorter of the two
// oriented rows and binary-search the longer one; every common w closes a
// triangle u < v < w (in rank), found exactly once.
__global__ void sparse_triangle_kernel(const int32_t *__restrict__ col, const int64_t *__restrict__ orow,
                                       const int32_t *__restrict__ oadj, const int32_t *__restrict__ oeid,
                                       const int32_t *__restrict__ osrc, const int64_t *__restrict__ n_or,
                                       unsigned long long *__restrict__ mask) {
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
    const unsigned long long bu = 1ull << col[u], bv = 1ull << col[v];
    for (int64_t i = wb + lane; i < we; i += 32) {
      const int32_t w = oadj[i];
      const int64_t j = lower_bound_i32(oadj, sb, se, w);
      if (j < se && oadj[j] == w) {
        const int32_t e_walk = oeid[i], e_srch = oeid[j];
        const int32_t euw = walk_u ? e_walk : e_srch;
        const int32_t evw = walk_u ? e_srch : e_walk;
        atomicOr(&mask[euv], 1ull << col[w]);
        atomicOr(&mask[euw], bv);
        atomicOr(&mask[evw], bu);
      }
    }
  }
}

// Both rules on the snapshot; next live flags; pass counters.
__global__ void sparse_rule_kernel(SparseArgs a, const int32_t *__restrict__ eu, const int32_t *__restrict__ ev,
                                   const unsigned long long *__restrict__ mask, uint8_t *__restrict__ elive_n,
                                   uint8_t *__restrict__ vlive_n, int32_t *__restrict__ v_sweep, DevState *st) {
  const int lane = threadIdx.x & 31;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t sweep_no = st->sweeps;
  unsigned long long tests = 0, de = 0, dv = 0;
  for (int64_t e = tid; e < a.m; e += stride) {
    uint8_t live = a.elive[e];
    if (live) {
      tests++;
      if (__popcll(mask[e]) < a.q - 2) {
        live = 0;
        de++;
      }
    }
    elive_n[e] = live;
  }
  // vertex rule: one warp per vertex over its live row
  const int64_t warp0 = tid >> 5, warps = stride >> 5;
  for (int64_t u = warp0; u < a.n; u += warps) {
    const bool lv = a.vlive[u] != 0;
    unsigned long long cm = 0;
    if (lv)
      for (int64_t i = a.row[u] + lane; i < a.row[u + 1]; i += 32) cm |= 1ull << a.col[a.adj[i]];
    for (int o = 16; o > 0; o >>= 1) cm |= __shfl_xor_sync(0xffffffffu, cm, o);
    if (lane == 0) {
      const bool fail = lv && __popcll(cm & ~(1ull << a.col[u])) < a.q - 1;
      vlive_n[u] = (lv && !fail) ? 1 : 0;
      if (fail) {
        dv++;
        if (v_sweep) v_sweep[u] = (int32_t)(sweep_no + 1);
      }
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

__global__ void sparse_finish_kernel(DevState *st) {
  const int cont = finish_pass(st, st->pass_dv, st->pass_de, st->pass_tests);
  (void)cont;
  st->pass_dv = st->pass_de = st->pass_tests = 0;
}

__global__ void sparse_begin_kernel(DevState *st, int64_t max_sweeps, int64_t passes0) {
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

static int sms_here() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}

// The CSR structures of the caller's edges (d_edges: device int32[2 m_in],
// built on the device by sparse_build_csr, kz_csr.cu), the colours and the
// pass scratch.
kz_status sparse_load(kz_graph g, const int32_t *colour, int64_t m_in, const int32_t *d_edges, bool dedup,
                      cudaStream_t s) {
  const int32_t n = g->n;
  KZ_TRY(sparse_build_csr(g, d_edges, m_in, dedup, s));
  const size_t nn = (size_t)std::max(n, 1), mm = (size_t)std::max<int64_t>(g->m, 1);
  for (int i = 0; i < 2; i++) {
    KZ_TRY(graph_alloc(g, &g->sp_row[i], nn + 1, s));
    KZ_TRY(graph_alloc(g, &g->sp_adj[i], 2 * mm, s));
    KZ_TRY(graph_alloc(g, &g->sp_eid[i], 2 * mm, s));
    KZ_TRY(graph_alloc(g, &g->sp_elive[i], mm, s));
    KZ_TRY(graph_alloc(g, &g->sp_vlive[i], nn, s));
  }
  KZ_TRY(graph_alloc(g, &g->sp_orow, nn + 1, s));
  KZ_TRY(graph_alloc(g, &g->sp_oadj, mm, s));
  KZ_TRY(graph_alloc(g, &g->sp_oeid, mm, s));
  KZ_TRY(graph_alloc(g, &g->sp_osrc, mm, s));
  KZ_TRY(graph_alloc(g, &g->sp_col, nn, s));
  KZ_TRY(graph_alloc(g, &g->sp_mask, mm, s));
  KZ_TRY(graph_alloc(g, &g->sp_cnt_live, nn, s));
  KZ_TRY(graph_alloc(g, &g->sp_cnt_or, nn, s));
  KZ_TRY(graph_alloc(g, &g->sp_sums, nn / kScanBlock + 2, s));
  KZ_TRY(graph_alloc(g, &g->sp_totals, 4, s));
  KZ_TRY(graph_alloc(g, &g->sp_v_sweep, nn, s));
  if (!g->st) {
    KZ_TRY(graph_alloc(g, &g->st, 1, s));
    KZ_CUDA_TRY(cudaMemsetAsync(g->st, 0, sizeof(DevState), s));
  }
  if (n) KZ_TRY(h2d(g->sp_col, colour, sizeof(int32_t) * n, s));
  g->has_csr = true;
  return sparse_reset(g, s);
}

kz_status sparse_reset(kz_graph g, cudaStream_t s) {
  const size_t n = (size_t)g->n, m = (size_t)g->m;
  KZ_CUDA_TRY(cudaMemsetAsync(g->sp_elive[0], 1, std::max<size_t>(m, 1), s));
  KZ_CUDA_TRY(cudaMemsetAsync(g->sp_vlive[0], 1, std::max<size_t>(n, 1), s));
  KZ_CUDA_TRY(cudaMemcpyAsync(g->sp_row[0], g->sp_row0, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
  if (m) {
    KZ_CUDA_TRY(cudaMemcpyAsync(g->sp_adj[0], g->sp_adj0, sizeof(int32_t) * 2 * m, cudaMemcpyDeviceToDevice, s));
    KZ_CUDA_TRY(cudaMemcpyAsync(g->sp_eid[0], g->sp_eid0, sizeof(int32_t) * 2 * m, cudaMemcpyDeviceToDevice, s));
  }
  if (n) KZ_CUDA_TRY(cudaMemsetAsync(g->sp_v_sweep, 0, sizeof(int32_t) * n, s));
  g->sp_cur = 0;
  return KZ_OK;
}

// Oriented CSR of the live edges of the current state (sp_orow, sp_oadj,
// sp_oeid, sp_osrc; its size in sp_totals[1]); the compacted live rows go to
// the other row buffer, which serves as scratch here.
kz_status sparse_orient_live(kz_graph g, cudaStream_t s) {
  const int c = g->sp_cur, nx = c ^ 1;
  SparseArgs a;
  a.n = g->n;
  a.k = g->k;
  a.q = g->k - g->slack;
  a.col = g->sp_col;
  a.rank = g->sp_rank;
  a.row = g->sp_row[c];
  a.adj = g->sp_adj[c];
  a.eid = g->sp_eid[c];
  a.elive = g->sp_elive[c];
  a.vlive = g->sp_vlive[c];
  a.m = g->m;
  const int grid = 8 * sms_here(), threads = 256;
  sparse_count_kernel<<<grid, threads, 0, s>>>(a, g->sp_cnt_live, g->sp_cnt_or);
  KZ_TRY(scan_counts(g->sp_cnt_live, g->n, g->sp_row[nx], g->sp_sums, g->sp_totals, s));
  KZ_TRY(scan_counts(g->sp_cnt_or, g->n, g->sp_orow, g->sp_sums, g->sp_totals + 1, s));
  sparse_fill_kernel<<<grid, threads, 0, s>>>(a, g->sp_row[nx], g->sp_adj[nx], g->sp_eid[nx], g->sp_orow,
                                              g->sp_oadj, g->sp_oeid, g->sp_osrc);
  return cuda_status(cudaGetLastError());
}

kz_status sparse_kernelize(kz_graph g, const kz_options &opt, cudaStream_t s) {
  const int64_t max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : (int64_t)g->n + g->m + 1;
  sparse_begin_kernel<<<1, 1, 0, s>>>(g->st, max_sweeps, g->n == 0 ? 1 : 0);
  KZ_CUDA_TRY(cudaGetLastError());
  if (g->n == 0) return KZ_OK;
  const int grid = 8 * sms_here();
  const int threads = 256;
  for (;;) {
    const int c = g->sp_cur, nx = c ^ 1;
    SparseArgs a;
    a.n = g->n;
    a.k = g->k;
  a.q = g->k - g->slack;
    a.col = g->sp_col;
    a.rank = g->sp_rank;
    a.row = g->sp_row[c];
    a.adj = g->sp_adj[c];
    a.eid = g->sp_eid[c];
    a.elive = g->sp_elive[c];
    a.vlive = g->sp_vlive[c];
    a.m = g->m;
    // 1. compaction of the live rows and the oriented CSR of the live edges
    sparse_count_kernel<<<grid, threads, 0, s>>>(a, g->sp_cnt_live, g->sp_cnt_or);
    KZ_TRY(scan_counts(g->sp_cnt_live, g->n, g->sp_row[nx], g->sp_sums, g->sp_totals, s));
    KZ_TRY(scan_counts(g->sp_cnt_or, g->n, g->sp_orow, g->sp_sums, g->sp_totals + 1, s));
    sparse_fill_kernel<<<grid, threads, 0, s>>>(a, g->sp_row[nx], g->sp_adj[nx], g->sp_eid[nx], g->sp_orow,
                                                g->sp_oadj, g->sp_oeid, g->sp_osrc);
    // the compacted rows are this pass's snapshot
    a.row = g->sp_row[nx];
    a.adj = g->sp_adj[nx];
    a.eid = g->sp_eid[nx];
    // 2. colour masks of the live edges from the live triangles
    KZ_CUDA_TRY(cudaMemsetAsync(g->sp_mask, 0, sizeof(unsigned long long) * std::max<int64_t>(g->m, 1), s));
    sparse_triangle_kernel<<<grid, threads, 0, s>>>(g->sp_col, g->sp_orow, g->sp_oadj, g->sp_oeid, g->sp_osrc,
                                                    g->sp_totals + 1, g->sp_mask);
    // 3.-4. rules, next flags, pass bookkeeping
    sparse_rule_kernel<<<grid, threads, 0, s>>>(a, g->sp_eu, g->sp_ev, g->sp_mask, g->sp_elive[nx],
                                                g->sp_vlive[nx], g->sp_v_sweep, g->st);
    sparse_finish_kernel<<<1, 1, 0, s>>>(g->st);
    KZ_CUDA_TRY(cudaGetLastError());
    int32_t cont = 0;
    KZ_CUDA_TRY(cudaMemcpyAsync(&cont, &g->st->cont, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (!cont) {
      // nothing applied: the state stays in buffer c; the compacted rows of
      // buffer nx describe the same live edges, keep them for the next run
      std::swap(g->sp_row[c], g->sp_row[nx]);
      std::swap(g->sp_adj[c], g->sp_adj[nx]);
      std::swap(g->sp_eid[c], g->sp_eid[nx]);
      break;
    }
    g->sp_cur = nx;
    // the live rows of the next pass are the compacted ones now in buffer nx
  }
  return KZ_OK;
}

// Survivors in caller ids: vertex flags and the sorted (u < v) edge list.
__global__ void sparse_count_live(const uint8_t *__restrict__ elive, int64_t m, unsigned long long *cnt) {
  unsigned long long c = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    c += elive[e];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

kz_status sparse_fetch(kz_graph g, uint8_t *vertex_alive, int32_t *edges_out, int64_t cap, int64_t *m_live) {
  const size_t n = (size_t)g->n, m = (size_t)g->m;
  std::vector<uint8_t> el(std::max<size_t>(m, 1)), vl(std::max<size_t>(n, 1));
  std::vector<int32_t> eu(std::max<size_t>(m, 1)), ev(std::max<size_t>(m, 1));
  const int c = g->sp_cur;
  KZ_CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (m) {
    KZ_CUDA_TRY(cudaMemcpy(el.data(), g->sp_elive[c], m, cudaMemcpyDeviceToHost));
    KZ_CUDA_TRY(cudaMemcpy(eu.data(), g->sp_eu, 4 * m, cudaMemcpyDeviceToHost));
    KZ_CUDA_TRY(cudaMemcpy(ev.data(), g->sp_ev, 4 * m, cudaMemcpyDeviceToHost));
  }
  if (n) KZ_CUDA_TRY(cudaMemcpy(vl.data(), g->sp_vlive[c], n, cudaMemcpyDeviceToHost));
  if (vertex_alive)
    for (size_t v = 0; v < n; v++) vertex_alive[v] = vl[v];
  int64_t cnt = 0;
  for (size_t e = 0; e < m; e++) {
    if (!el[e]) continue;
    if (cnt < cap && edges_out) {
      edges_out[2 * cnt] = eu[e];
      edges_out[2 * cnt + 1] = ev[e];
    }
    cnt++;
  }
  *m_live = cnt;
  return KZ_OK;
}

kz_status sparse_vertex_alive(kz_graph g, uint8_t *host_alive, int64_t *n_live) {
  const size_t n = (size_t)g->n;
  std::vector<uint8_t> vl(std::max<size_t>(n, 1));
  if (n) KZ_CUDA_TRY(cudaMemcpy(vl.data(), g->sp_vlive[g->sp_cur], n, cudaMemcpyDeviceToHost));
  int64_t live = 0;
  for (size_t v = 0; v < n; v++) {
    live += vl[v];
    if (host_alive) host_alive[v] = vl[v];
  }
  if (n_live) *n_live = live;
  return KZ_OK;
}

kz_status sparse_v_sweep(kz_graph g, int32_t *host) {
  if (g->n) KZ_CUDA_TRY(cudaMemcpy(host, g->sp_v_sweep, sizeof(int32_t) * g->n, cudaMemcpyDeviceToHost));
  return KZ_OK;
}

}  // namespace kz

namespace kz {

// ---------------------------------------------------------------------------
// moving the live state between the bitset rows and the CSR flags
// ---------------------------------------------------------------------------

__global__ void bitset_to_flags_kernel(const uint32_t *__restrict__ A, const uint32_t *__restrict__ V, int32_t ldw,
                                       int32_t k, const int32_t *__restrict__ inv, const int32_t *__restrict__ coff,
                                       const int32_t *__restrict__ col, const int32_t *__restrict__ eu,
                                       const int32_t *__restrict__ ev, int64_t m, int32_t n,
                                       uint8_t *__restrict__ elive, uint8_t *__restrict__ vlive) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = tid; e < m; e += stride) {
    const int32_t x = inv[eu[e]], v = ev[e], y = inv[v];
    const int32_t c = col[v], i = y - coff[c];
    elive[e] = (uint8_t)((A[(int64_t)x * ldw + (i >> 5) * k + c] >> (i & 31)) & 1u);
  }
  for (int64_t v = tid; v < n; v += stride) {
    const int32_t c = col[v], i = inv[v] - coff[c];
    vlive[v] = (uint8_t)((V[(i >> 5) * k + c] >> (i & 31)) & 1u);
  }
}

__global__ void flags_to_bitset_kernel(uint32_t *__restrict__ A, uint32_t *__restrict__ V, int32_t ldw, int32_t k,
                                       const int32_t *__restrict__ inv, const int32_t *__restrict__ coff,
                                       const int32_t *__restrict__ col, const int32_t *__restrict__ eu,
                                       const int32_t *__restrict__ ev, int64_t m, int32_t n,
                                       const uint8_t *__restrict__ elive, const uint8_t *__restrict__ vlive) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = tid; e < m; e += stride) {
    if (!elive[e]) continue;
    const int32_t u = eu[e], v = ev[e], x = inv[u], y = inv[v];
    const int32_t cu = col[u], cv = col[v], iu = x - coff[cu], iv = y - coff[cv];
    atomicOr(&A[(int64_t)x * ldw + (iv >> 5) * k + cv], 1u << (iv & 31));
    atomicOr(&A[(int64_t)y * ldw + (iu >> 5) * k + cu], 1u << (iu & 31));
  }
  for (int64_t v = tid; v < n; v += stride) {
    if (!vlive[v]) continue;
    const int32_t c = col[v], i = inv[v] - coff[c];
    atomicOr(&V[(i >> 5) * k + c], 1u << (i & 31));
  }
}

kz_status state_to_sparse(kz_graph g, cudaStream_t s) {
  if (g->owner == KZ_PATH_SPARSE) return KZ_OK;
  if (!g->has_csr || !g->has_bitset) return KZ_ERR_UNSUPPORTED;
  int32_t cur = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&cur, &g->st->cur, 4, cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  bitset_to_flags_kernel<<<4 * sms_here(), 256, 0, s>>>(g->A[cur & 1], g->V[cur & 1], g->ldw, g->k, g->d_inv,
                                                        g->d_coff, g->sp_col, g->sp_eu, g->sp_ev, g->m, g->n,
                                                        g->sp_elive[g->sp_cur], g->sp_vlive[g->sp_cur]);
  KZ_CUDA_TRY(cudaGetLastError());
  g->owner = KZ_PATH_SPARSE;
  return KZ_OK;
}

kz_status state_to_bitset(kz_graph g, cudaStream_t s) {
  if (g->owner == KZ_PATH_BITSET) return KZ_OK;
  if (!g->has_csr || !g->has_bitset) return KZ_ERR_UNSUPPORTED;
  int32_t cur = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&cur, &g->st->cur, 4, cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  uint32_t *A = g->A[cur & 1], *V = g->V[cur & 1];
  KZ_CUDA_TRY(cudaMemsetAsync(A, 0, (size_t)g->n * g->ldw * 4, s));
  KZ_CUDA_TRY(cudaMemsetAsync(V, 0, (size_t)g->ldw * 4, s));
  flags_to_bitset_kernel<<<4 * sms_here(), 256, 0, s>>>(A, V, g->ldw, g->k, g->d_inv, g->d_coff, g->sp_col,
                                                        g->sp_eu, g->sp_ev, g->m, g->n, g->sp_elive[g->sp_cur],
                                                        g->sp_vlive[g->sp_cur]);
  KZ_CUDA_TRY(cudaGetLastError());
  g->owner = KZ_PATH_BITSET;
  g->ab_synced = false;  // only the current buffer was rebuilt
  return KZ_OK;
}

}  // namespace kz
