// kz_csr.cu -- the CSR of an edge-list graph, built on the device.
//
// The sparse path (kz_sparse.cu) needs, for the caller's edges:
//   * the canonical edge list (u < v) sorted by (u, v), duplicates merged or
//     rejected; an edge's id is its index in that order (eu, ev);
//   * the CSR: row u holds u's lower neighbours in ascending order, then its
//     higher ones in ascending order, each with its edge id (row0, adj0, eid0);
//   * the orientation rank: vertices ordered by degree, ties by id.
// Two stable LSD radix sorts do the work: the keys (u, v) for the edge order
// and the upper halves of the rows, and the keys (v, u) carrying edge ids for
// the lower halves; a third, over (degree, vertex), gives the rank.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "kz_internal.cuh"

namespace kz {

namespace {

constexpr int kRadixThreads = 256;  // one bin per thread
constexpr int kRadixItems = 8;      // keys per thread per tile
constexpr int kRadixTile = kRadixThreads * kRadixItems;
constexpr int kRadixWarps = kRadixThreads / 32;

int sms_csr() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}

int bits_for(uint64_t x) {  // bits needed to hold every value up to x
  int b = 1;
  while (b < 63 && (x >> b) != 0) b++;
  return b;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of 64-bit keys (optionally with int32 values), 8 bits
// a pass.  A tile is kRadixTile consecutive keys, taken in kRadixItems rounds
// of kRadixThreads consecutive keys; the scatter ranks every key among the
// equal digits before it in that order, so each pass is stable.
// ---------------------------------------------------------------------------

__global__ void radix_hist_kernel(const uint64_t *__restrict__ keys, int64_t m, int shift,
                                  int32_t *__restrict__ hist, int64_t tiles) {
  __shared__ int32_t h[256];
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = t * kRadixTile;
#pragma unroll
    for (int r = 0; r < kRadixItems; r++) {
      const int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
      if (i < m) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + t] = h[threadIdx.x];  // bin-major
    __syncthreads();
  }
}

__global__ void radix_scatter_kernel(const uint64_t *__restrict__ keys, const int32_t *__restrict__ vals, int64_t m,
                                     int shift, const int64_t *__restrict__ off, int64_t tiles,
                                     uint64_t *__restrict__ okeys, int32_t *__restrict__ ovals) {
  __shared__ int32_t run[256];                 // keys of each digit placed so far in this tile
  __shared__ int32_t wcnt[kRadixWarps][256];   // per-warp counts of a round, then warp prefixes
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    run[threadIdx.x] = 0;
    const int64_t base = t * kRadixTile;
    for (int r = 0; r < kRadixItems; r++) {
      for (int b = threadIdx.x; b < kRadixWarps * 256; b += kRadixThreads) (&wcnt[0][0])[b] = 0;
      __syncthreads();
      const int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
      const bool valid = i < m;
      const uint64_t key = valid ? keys[i] : 0ull;
      const int d = valid ? (int)((key >> shift) & 255u) : 256;  // 256: no bin
      const unsigned same = __match_any_sync(0xffffffffu, d);
      const int rank = __popc(same & lt);
      if (valid && rank == 0) wcnt[warp][d] = __popc(same);
      __syncthreads();
      // thread b: prefix of bin b over the warps, and the round's total
      int total = 0;
      for (int w = 0; w < kRadixWarps; w++) {
        const int c = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = total;
        total += c;
      }
      __syncthreads();
      if (valid) {
        const int64_t pos = off[(int64_t)d * tiles + t] + run[d] + wcnt[warp][d] + rank;
        okeys[pos] = key;
        if (ovals) ovals[pos] = vals[i];
      }
      __syncthreads();
      run[threadIdx.x] += total;
    }
    __syncthreads();
  }
}

// Sorts keys[0..m) (and vals when given) on their low `bits` bits; the result
// ends in keys / vals (the other buffers are scratch of the same sizes).
kz_status radix_sort(uint64_t *keys, uint64_t *keys_tmp, int32_t *vals, int32_t *vals_tmp, int64_t m, int bits,
                     int32_t *hist, int64_t *off, int64_t *sums, int64_t *total, cudaStream_t s) {
  if (m <= 1) return KZ_OK;
  const int64_t tiles = (m + kRadixTile - 1) / kRadixTile;
  const int grid = (int)std::min<int64_t>(tiles, 8 * sms_csr());
  uint64_t *ka = keys, *kb = keys_tmp;
  int32_t *va = vals, *vb = vals_tmp;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<<<grid, kRadixThreads, 0, s>>>(ka, m, shift, hist, tiles);
    KZ_TRY(scan_counts(hist, 256 * tiles, off, sums, total, s));
    radix_scatter_kernel<<<grid, kRadixThreads, 0, s>>>(ka, va, m, shift, off, tiles, kb, vb);
    KZ_CUDA_TRY(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    KZ_CUDA_TRY(cudaMemcpyAsync(keys, ka, (size_t)m * 8, cudaMemcpyDeviceToDevice, s));
    if (vals) KZ_CUDA_TRY(cudaMemcpyAsync(vals, va, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
  }
  return KZ_OK;
}

// ---------------------------------------------------------------------------
// the CSR steps
// ---------------------------------------------------------------------------

__global__ void canon_kernel(const int32_t *__restrict__ edges, int64_t m, int B, uint64_t *__restrict__ keys) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t u = (uint32_t)edges[2 * e], v = (uint32_t)edges[2 * e + 1];
    if (u > v) {
      const uint32_t t = u;
      u = v;
      v = t;
    }
    keys[e] = ((uint64_t)u << B) | v;
  }
}

// keep[i] = 1 for the first of equal sorted keys; *dup = 1 when any repeats
__global__ void first_of_kernel(const uint64_t *__restrict__ keys, int64_t m, int32_t *__restrict__ keep,
                                int32_t *dup) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const bool first = i == 0 || keys[i] != keys[i - 1];
    keep[i] = first ? 1 : 0;
    if (!first) *dup = 1;
  }
}

__global__ void compact_kernel(const uint64_t *__restrict__ keys, const int32_t *__restrict__ keep,
                               const int64_t *__restrict__ pos, int64_t m, uint64_t *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    if (keep[i]) out[pos[i]] = keys[i];
}

// endpoints, per-vertex counts, and the (v, u) keys carrying the edge ids
__global__ void split_kernel(const uint64_t *__restrict__ keys, int64_t m, int B, int32_t *__restrict__ eu,
                             int32_t *__restrict__ ev, int32_t *__restrict__ up_cnt, int32_t *__restrict__ low_cnt,
                             uint64_t *__restrict__ keys2, int32_t *__restrict__ vals2) {
  const uint64_t mask = (1ull << B) - 1ull;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys[e];
    const int32_t u = (int32_t)(key >> B), v = (int32_t)(key & mask);
    eu[e] = u;
    ev[e] = v;
    atomicAdd(&up_cnt[u], 1);
    atomicAdd(&low_cnt[v], 1);
    keys2[e] = ((uint64_t)v << B) | (uint64_t)u;
    vals2[e] = (int32_t)e;
  }
}

__global__ void add_kernel(const int32_t *__restrict__ a, const int32_t *__restrict__ b, int64_t n,
                           int32_t *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] + b[i];
}

// the higher neighbours of u, after its lower ones: edge e is the
// (e - up_off[u])-th of u's edges in the sorted order
__global__ void fill_upper_kernel(const int32_t *__restrict__ eu, const int32_t *__restrict__ ev, int64_t m,
                                  const int64_t *__restrict__ row, const int32_t *__restrict__ low_cnt,
                                  const int64_t *__restrict__ up_off, int32_t *__restrict__ adj,
                                  int32_t *__restrict__ eid) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = eu[e];
    const int64_t p = row[u] + low_cnt[u] + (e - up_off[u]);
    adj[p] = ev[e];
    eid[p] = (int32_t)e;
  }
}

// the lower neighbours of v, from the keys sorted by (v, u)
__global__ void fill_lower_kernel(const uint64_t *__restrict__ keys2, const int32_t *__restrict__ vals2, int64_t m,
                                  int B, const int64_t *__restrict__ row, const int64_t *__restrict__ low_off,
                                  int32_t *__restrict__ adj, int32_t *__restrict__ eid) {
  const uint64_t mask = (1ull << B) - 1ull;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys2[j];
    const int32_t v = (int32_t)(key >> B), u = (int32_t)(key & mask);
    const int64_t p = row[v] + (j - low_off[v]);
    adj[p] = u;
    eid[p] = vals2[j];
  }
}

__global__ void degree_keys_kernel(const int64_t *__restrict__ row, int32_t n, int B, uint64_t *__restrict__ keys) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    keys[x] = ((uint64_t)(row[x + 1] - row[x]) << B) | (uint64_t)x;
}

__global__ void rank_kernel(const uint64_t *__restrict__ keys, int32_t n, int B, int32_t *__restrict__ rank) {
  const uint64_t mask = (1ull << B) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    rank[keys[i] & mask] = (int32_t)i;
}

// Device scratch of one build, released when it goes out of scope.
struct Scratch {
  cudaStream_t s;
  std::vector<std::pair<void *, size_t>> held;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (auto &h : held) dev_free(h.first, h.second, s);
  }
  template <class T>
  T *get(size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    void *p = dev_alloc(bytes, s);
    if (p) held.emplace_back(p, bytes);
    return static_cast<T *>(p);
  }
};

}  // namespace

kz_status sparse_build_csr(kz_graph g, const int32_t *d_edges, int64_t m_in, bool dedup, cudaStream_t s) {
  const int32_t n = g->n;
  const int B = bits_for((uint64_t)std::max(n - 1, 1));
  const int grid = 8 * sms_csr(), threads = 256;
  const int64_t mm_in = std::max<int64_t>(m_in, 1);
  const int64_t keys_len = std::max<int64_t>(mm_in, n);  // the edge keys, then the vertex keys
  const int64_t tiles = (keys_len + kRadixTile - 1) / kRadixTile;
  const int64_t max_len = std::max<int64_t>(256 * tiles, keys_len);  // longest scan
  Scratch sc(s);
  uint64_t *k0 = sc.get<uint64_t>(keys_len), *k1 = sc.get<uint64_t>(keys_len);
  int32_t *hist = sc.get<int32_t>(256 * tiles + 1);
  int64_t *off = sc.get<int64_t>(max_len + 1);
  int64_t *sums = sc.get<int64_t>(max_len / 1024 + 2), *total = sc.get<int64_t>(2);
  int32_t *flag = sc.get<int32_t>(mm_in);
  int32_t *dup = sc.get<int32_t>(1);
  if (!k0 || !k1 || !hist || !off || !sums || !total || !flag || !dup) return KZ_ERR_OOM;

  // (u, v) keys, sorted; duplicates merged or rejected
  int64_t m = 0;
  if (m_in > 0) {
    canon_kernel<<<grid, threads, 0, s>>>(d_edges, m_in, B, k0);
    KZ_TRY(radix_sort(k0, k1, nullptr, nullptr, m_in, 2 * B, hist, off, sums, total, s));
    KZ_CUDA_TRY(cudaMemsetAsync(dup, 0, sizeof(int32_t), s));
    first_of_kernel<<<grid, threads, 0, s>>>(k0, m_in, flag, dup);
    KZ_TRY(scan_counts(flag, m_in, off, sums, total, s));
    compact_kernel<<<grid, threads, 0, s>>>(k0, flag, off, m_in, k1);
    KZ_CUDA_TRY(cudaGetLastError());
    int32_t h_dup = 0;
    KZ_CUDA_TRY(cudaMemcpyAsync(&h_dup, dup, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaMemcpyAsync(&m, total, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_dup && !dedup) return KZ_ERR_DUPLICATE_EDGE;
  }
  g->m = m;
  const size_t nn = (size_t)std::max(n, 1), mm = (size_t)std::max<int64_t>(m, 1);
  KZ_TRY(graph_alloc(g, &g->sp_row0, nn + 1, s));
  KZ_TRY(graph_alloc(g, &g->sp_adj0, 2 * mm, s));
  KZ_TRY(graph_alloc(g, &g->sp_eid0, 2 * mm, s));
  KZ_TRY(graph_alloc(g, &g->sp_eu, mm, s));
  KZ_TRY(graph_alloc(g, &g->sp_ev, mm, s));
  KZ_TRY(graph_alloc(g, &g->sp_rank, nn, s));
  int32_t *up_cnt = sc.get<int32_t>(nn), *low_cnt = sc.get<int32_t>(nn), *deg = sc.get<int32_t>(nn);
  int64_t *up_off = sc.get<int64_t>(nn + 1), *low_off = sc.get<int64_t>(nn + 1);
  int32_t *vals = sc.get<int32_t>(mm), *vals_tmp = sc.get<int32_t>(mm);
  if (!up_cnt || !low_cnt || !deg || !up_off || !low_off || !vals || !vals_tmp) return KZ_ERR_OOM;
  KZ_CUDA_TRY(cudaMemsetAsync(up_cnt, 0, nn * 4, s));
  KZ_CUDA_TRY(cudaMemsetAsync(low_cnt, 0, nn * 4, s));
  uint64_t *keys2 = k0, *keys = k1;  // k1 holds the unique (u, v) keys
  if (m > 0) split_kernel<<<grid, threads, 0, s>>>(keys, m, B, g->sp_eu, g->sp_ev, up_cnt, low_cnt, keys2, vals);
  add_kernel<<<grid, threads, 0, s>>>(up_cnt, low_cnt, n, deg);
  KZ_CUDA_TRY(cudaGetLastError());
  if (n > 0) {
    KZ_TRY(scan_counts(deg, n, g->sp_row0, sums, total, s));
    KZ_TRY(scan_counts(up_cnt, n, up_off, sums, total, s));
    KZ_TRY(scan_counts(low_cnt, n, low_off, sums, total, s));
  } else {
    KZ_CUDA_TRY(cudaMemsetAsync(g->sp_row0, 0, sizeof(int64_t), s));
  }
  if (m > 0) {
    fill_upper_kernel<<<grid, threads, 0, s>>>(g->sp_eu, g->sp_ev, m, g->sp_row0, low_cnt, up_off, g->sp_adj0,
                                               g->sp_eid0);
    KZ_TRY(radix_sort(keys2, keys, vals, vals_tmp, m, 2 * B, hist, off, sums, total, s));
    fill_lower_kernel<<<grid, threads, 0, s>>>(keys2, vals, m, B, g->sp_row0, low_off, g->sp_adj0, g->sp_eid0);
    KZ_CUDA_TRY(cudaGetLastError());
  }
  // orientation rank: degree order, ties by id (degrees below 2m + 1)
  if (n > 0) {
    degree_keys_kernel<<<grid, threads, 0, s>>>(g->sp_row0, n, B, k0);
    KZ_TRY(radix_sort(k0, k1, nullptr, nullptr, n, B + bits_for((uint64_t)(2 * m + 1)), hist, off, sums, total, s));
    rank_kernel<<<grid, threads, 0, s>>>(k0, n, B, g->sp_rank);
    KZ_CUDA_TRY(cudaGetLastError());
  }
  // the scratch is released on the stream after this work
  return KZ_OK;
}

}  // namespace kz
