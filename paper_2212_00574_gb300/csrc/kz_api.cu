// kz_api.cu -- the C ABI declared in include/kz.h: argument checking,
// colour-sorted relabelling, device allocation, and dispatch to the paths.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "kz_internal.cuh"

namespace {

std::mutex g_alloc_mu;
kz_allocator g_alloc = {nullptr, nullptr, nullptr};
std::atomic<uint64_t> g_next_uid{1};

}  // namespace

namespace kz {

void *dev_alloc(size_t bytes, cudaStream_t s) {
  kz_allocator a;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
  }
  if (a.alloc) return a.alloc(bytes, (void *)s, a.ctx);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  kz_allocator a;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc;
  }
  if (a.free) {
    a.free(p, bytes, (void *)s, a.ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

// The pinned staging arena of the loaders (see LoadStage): one per process,
// grown when a load needs more, used by one load at a time.
namespace {
std::mutex g_stage_mu;
char *g_stage = nullptr;
size_t g_stage_cap = 0, g_stage_off = 0;
thread_local LoadStage *t_stage = nullptr;
constexpr size_t kStageMinBytes = size_t(4) << 20;
}  // namespace

LoadStage::LoadStage(cudaStream_t s) : stream(s) {
  g_stage_mu.lock();
  g_stage_off = 0;
  t_stage = this;
}

LoadStage::~LoadStage() {
  // every staged copy of this load has landed before the arena is reused
  cudaStreamSynchronize(stream);
  cudaGetLastError();
  t_stage = nullptr;
  g_stage_mu.unlock();
}

kz_status h2d(void *dst, const void *src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return KZ_OK;
  LoadStage *st = t_stage;
  if (!st || st->stream != s) return cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
  const size_t need = (bytes + 255) & ~size_t(255);
  if (g_stage_off + need > g_stage_cap) {
    // the arena is full: wait for the copies in flight, then reuse or grow it
    KZ_CUDA_TRY(cudaStreamSynchronize(s));
    g_stage_off = 0;
    if (need > g_stage_cap) {
      if (g_stage) cudaFreeHost(g_stage);
      g_stage = nullptr;
      g_stage_cap = 0;
      const size_t cap = std::max(need, kStageMinBytes);
      char *p = nullptr;
      if (cudaMallocHost(&p, cap) != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
      }
      g_stage = p;
      g_stage_cap = cap;
    }
  }
  char *slot = g_stage + g_stage_off;
  memcpy(slot, src, bytes);
  g_stage_off += need;
  return cuda_status(cudaMemcpyAsync(dst, slot, bytes, cudaMemcpyHostToDevice, s));
}

}  // namespace kz

using namespace kz;

namespace {

// Definition 4.2.1 requires a legal colouring; the checks that need no
// device run here, before any CUDA call.
kz_status check_colours(int32_t n, int32_t k, const int32_t *colour) {
  if (n < 0 || k < 1 || k > 64) return KZ_ERR_ARG;
  if (n > 0 && !colour) return KZ_ERR_ARG;
  for (int32_t v = 0; v < n; v++)
    if (colour[v] < 0 || colour[v] >= k) return KZ_ERR_COLOUR_RANGE;
  return KZ_OK;
}

kz_status check_edges(int32_t n, const int32_t *colour, int64_t m, const int32_t *edges) {
  if (m < 0) return KZ_ERR_ARG;
  if (m > 0 && !edges) return KZ_ERR_ARG;
  for (int64_t e = 0; e < m; e++) {
    const int32_t u = edges[2 * e], v = edges[2 * e + 1];
    if (u < 0 || u >= n || v < 0 || v >= n) return KZ_ERR_VERTEX_RANGE;
    if (u == v) return KZ_ERR_SELF_LOOP;
    if (colour[u] == colour[v]) return KZ_ERR_ILLEGAL_COLOURING;
  }
  return KZ_OK;
}

// Counting sort by colour, stable in the caller's id order.
void relabel(kz_graph g, const int32_t *colour) {
  const int n = g->n, k = g->k;
  g->coff.assign(k + 1, 0);
  for (int v = 0; v < n; v++) g->coff[colour[v] + 1]++;
  for (int c = 0; c < k; c++) g->coff[c + 1] += g->coff[c];
  std::vector<int32_t> fill(g->coff.begin(), g->coff.end() - 1);
  g->perm.assign(n, 0);
  g->inv.assign(n, 0);
  for (int v = 0; v < n; v++) {
    const int x = fill[colour[v]]++;
    g->perm[x] = v;
    g->inv[v] = x;
  }
}

void release(kz_graph g) {
  if (!g) return;
  cudaStream_t s = g->stream;
  // the graph's last work must be finished before its memory is handed back
  cudaStreamSynchronize(s);
  if (g->loop_exec) cudaGraphExecDestroy(g->loop_exec);
  if (g->run_exec) cudaGraphExecDestroy(g->run_exec);
  learned_release(g);
  tensor_release(g);
  dominance_release(g);
  support_release(g);
  for (auto &a : g->allocs) dev_free(a.p, a.bytes, s);
  g->allocs.clear();
  cudaStreamSynchronize(s);
  delete g;
}

// Bitset rows are built when their three copies fit this budget; larger
// graphs (or graphs with very uneven colour classes) use the CSR path only.
constexpr size_t kBitsetBudgetBytes = size_t(8) << 30;

// Common tail of both loaders: relabelling, bitset layout and packing (when
// the rows fit), CSR structures (edge-list input), buffers.
template <class Pack, class Csr>
kz_status load_common(int32_t n, int32_t k, const int32_t *colour, void *stream, kz_graph *out,
                      Pack pack, Csr csr, bool want_csr) {
  // no device, no fallback
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return KZ_ERR_CUDA;
  }
  kz_graph g = new (std::nothrow) kz_graph_s();
  if (!g) return KZ_ERR_OOM;
  g->n = n;
  g->k = k;
  g->uid = g_next_uid.fetch_add(1);
  g->stream = (cudaStream_t)stream;
  cudaGetDevice(&g->device);
  LoadStage stage(g->stream);  // small host tables travel through one pinned arena
  relabel(g, colour);
  kz_status st = KZ_OK;
  if (want_csr) st = csr(g);  // host-side duplicate check comes first
  const kz_status lay = bitset_build_layout(g);
  const size_t bitset_bytes = (size_t)3 * g->n * g->ldw * 4;
  const bool want_bitset = lay == KZ_OK && bitset_bytes <= kBitsetBudgetBytes;
  if (st == KZ_OK && want_bitset) {
    st = graph_alloc(g, &g->d_perm, (size_t)std::max(n, 1), g->stream);
    if (st == KZ_OK) st = graph_alloc(g, &g->d_inv, (size_t)std::max(n, 1), g->stream);
    if (st == KZ_OK) st = graph_alloc(g, &g->d_cpos, (size_t)std::max(n, 1), g->stream);
    if (st == KZ_OK && n > 0)
      st = h2d(g->d_perm, g->perm.data(), sizeof(int32_t) * n, g->stream);
    if (st == KZ_OK && n > 0)
      st = h2d(g->d_inv, g->inv.data(), sizeof(int32_t) * n, g->stream);
    if (st == KZ_OK && n > 0) {
      // position of every caller vertex inside a row of the block-plane layout
      std::vector<int32_t> cpos((size_t)n);
      for (int c = 0; c < k; c++)
        for (int x = g->coff[c]; x < g->coff[c + 1]; x++) {
          const int ix = x - g->coff[c];
          cpos[g->perm[x]] = ((((ix >> 5) * k) + c) << 5) | (ix & 31);
        }
      st = h2d(g->d_cpos, cpos.data(), sizeof(int32_t) * n, g->stream);
    }
    if (st == KZ_OK) st = pack(g);
    if (st == KZ_OK) st = bitset_finish_load(g, g->stream);
    if (st == KZ_OK) g->has_bitset = true;
  }
  if (st == KZ_OK && !g->has_bitset && !g->has_csr) st = KZ_ERR_UNSUPPORTED;
  if (st == KZ_OK) st = cuda_status(cudaStreamSynchronize(g->stream));
  if (st != KZ_OK) {
    release(g);
    return st;
  }
  g->owner = g->has_bitset ? KZ_PATH_BITSET : KZ_PATH_SPARSE;
  *out = g;
  return KZ_OK;
}

}  // namespace

extern "C" {

void kz_default_options(kz_options *opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->path = KZ_PATH_AUTO;
  opt->schedule = KZ_SCHED_PLAIN;
  opt->max_sweeps = 0;
  opt->use_graph = 1;
}

kz_status kz_set_allocator(const kz_allocator *allocator) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  if (!allocator) {
    g_alloc = {nullptr, nullptr, nullptr};
    return KZ_OK;
  }
  if (!allocator->alloc || !allocator->free) return KZ_ERR_ARG;
  g_alloc = *allocator;
  return KZ_OK;
}

kz_status kz_load_graph(int32_t n, int32_t k, const int32_t *colour, int64_t m,
                        const int32_t *edges, uint32_t flags, void *stream, kz_graph *out) {
  if (!out) return KZ_ERR_ARG;
  *out = nullptr;
  if (flags & ~KZ_DEDUP) return KZ_ERR_ARG;
  KZ_TRY(check_colours(n, k, colour));
  KZ_TRY(check_edges(n, colour, m, edges));
  const bool dedup = (flags & KZ_DEDUP) != 0;
  // the caller's edges go to the device once; both builders read them there
  int32_t *d_edges = nullptr;
  const size_t ebytes = (size_t)m * 8;
  auto upload = [&](kz_graph g) -> kz_status {
    if (d_edges || m == 0) return KZ_OK;
    d_edges = (int32_t *)dev_alloc(ebytes, g->stream);
    if (!d_edges) return KZ_ERR_OOM;
    return cuda_status(cudaMemcpyAsync(d_edges, edges, ebytes, cudaMemcpyHostToDevice, g->stream));
  };
  auto pack = [&](kz_graph g) -> kz_status {
    if (m == 0) return bitset_pack_edges(g, nullptr, 0, true, g->stream);
    KZ_TRY(upload(g));
    return bitset_pack_edges(g, d_edges, m, dedup, g->stream);
  };
  auto csr = [&](kz_graph g) -> kz_status {
    KZ_TRY(upload(g));
    return sparse_load(g, colour, m, d_edges, dedup, g->stream);
  };
  const kz_status st = load_common(n, k, colour, stream, out, pack, csr, true);
  // load_common has waited for the stream (or released the graph, which waits)
  if (d_edges) dev_free(d_edges, ebytes, (cudaStream_t)stream);
  return st;
}

kz_status kz_load_graph_dense(int32_t n, int32_t k, const int32_t *colour,
                              const uint64_t *adj_bits, int64_t row_words, uint32_t flags,
                              void *stream, kz_graph *out) {
  if (!out) return KZ_ERR_ARG;
  *out = nullptr;
  if (flags & ~KZ_DEDUP) return KZ_ERR_ARG;
  KZ_TRY(check_colours(n, k, colour));
  if (row_words < (int64_t)((n + 63) / 64) || (n > 0 && !adj_bits)) return KZ_ERR_ARG;
  auto no_csr = [](kz_graph) -> kz_status { return KZ_OK; };
  return load_common(n, k, colour, stream, out, [&](kz_graph g) -> kz_status {
    const size_t bytes = (size_t)n * row_words * 8;
    if (bytes == 0) return bitset_pack_edges(g, nullptr, 0, true, g->stream);
    return bitset_pack_dense(g, adj_bits, row_words, g->stream);
  }, no_csr, false);
}

static kz_status read_options(const kz_options *opt, kz_options &o) {
  if (opt) {
    o = *opt;
    for (int i = 0; i < 4; i++)
      if (o.reserved[i]) return KZ_ERR_ARG;
  } else {
    kz_default_options(&o);
  }
  if (o.path < KZ_PATH_AUTO || o.path > KZ_PATH_TENSOR) return KZ_ERR_ARG;
  if (o.schedule != KZ_SCHED_PLAIN && o.schedule != KZ_SCHED_LEARNED && o.schedule != KZ_SCHED_SUPPORT)
    return KZ_ERR_ARG;
  if (o.plane0 < KZ_PLANE0_AUTO || o.plane0 > KZ_PLANE0_TWO) return KZ_ERR_ARG;
  if (o.batch < KZ_BATCH_CONCURRENT || o.batch > KZ_BATCH_FUSED) return KZ_ERR_ARG;
  if (o.clique_k < 0) return KZ_ERR_ARG;
  if (o.dominance < 0 || o.dominance > 2) return KZ_ERR_ARG;
  if (o.tensor_precision < 0 || o.tensor_precision > 1) return KZ_ERR_ARG;
  return KZ_OK;
}

// The clique size q of this run, as slack = k - q (0: the thesis's rules).
static kz_status set_clique(kz_graph g, const kz_options &o) {
  const int q = o.clique_k ? o.clique_k : g->k;
  if (q < 1 || q > g->k) return KZ_ERR_ARG;
  g->slack = g->k - q;
  if (g->slack != 0 && o.schedule != KZ_SCHED_PLAIN) return KZ_ERR_UNSUPPORTED;
  return KZ_OK;
}

// The path a graph takes when the options leave the choice to the library:
// bitset rows when they exist, else the CSR path.  A graph of at most 64
// vertices runs inside one CTA from shared memory (a multi-CTA pass would be
// all launch and barrier); anything larger is spread over the GPU.
constexpr int kSmallAutoMaxN = 64;

// Bitset sweep or tensor-core form for a graph held as bitset rows, from a
// table measured on GB300 by the autotuner (paper_2212_00574_gb300/autotune.py:
// time to fixpoint of both paths on seeded k-partite graphs with a planted
// clique, n in {2048, 4096, 8192, 16384}, k in {12, 24}, density in {0.05,
// 0.1, 0.2, 0.3, 0.45}, and over the batch workload's range, n in {64, 256,
// 1024, 2048, 4096}, k in {6, 12, 24, 32}, density in {0.3, 0.45, 0.6, 0.8,
// 0.95}; its measurements are in autotune_grid.json beside it): 1 where the
// tensor form was faster over the bin's measured graphs.
// The bitset sweep settles most pairs from the first word of each class when
// common neighbours are plentiful (dense graphs); the tensor form does the
// same work whatever the density, so it wins where pairs need many words or
// sweeps (sparser graphs, larger n).
constexpr int kTensorTable[4][2][5] = {
    // density bins: < 0.075, < 0.15, < 0.25, < 0.375, >= 0.375
    {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}},  // n < 3072 (k < 18, k >= 18)
    {{0, 1, 1, 0, 0}, {0, 0, 1, 0, 0}},  // n < 6144
    {{1, 1, 1, 0, 0}, {0, 1, 1, 0, 0}},  // n < 12288
    {{1, 1, 0, 0, 0}, {1, 1, 1, 0, 0}},  // larger
};

static bool tensor_preferred(kz_graph g) {
  if (g->k > 64 || g->k < 3) return false;
  const int nb = g->n < 3072 ? 0 : g->n < 6144 ? 1 : g->n < 12288 ? 2 : 3;
  const int kb = g->k < 18 ? 0 : 1;
  const double d = g->density;
  const int db = d < 0.075 ? 0 : d < 0.15 ? 1 : d < 0.25 ? 2 : d < 0.375 ? 3 : 4;
  return kTensorTable[nb][kb][db] != 0;
}

static int auto_path(kz_graph g) {
  if (!g->has_bitset) return KZ_PATH_SPARSE;
  if (g->n <= kSmallAutoMaxN && cta_fits_shared(g)) return KZ_PATH_SMALL;
  return tensor_preferred(g) ? KZ_PATH_TENSOR : KZ_PATH_BITSET;
}

static kz_status run_one(kz_graph g, const kz_options &o, int path) {
  if (path == KZ_PATH_SPARSE) {
    if (!g->has_csr) return KZ_ERR_UNSUPPORTED;
    KZ_TRY(state_to_sparse(g, g->stream));
    KZ_TRY(sparse_kernelize(g, o, g->stream));
  } else {
    if (!g->has_bitset) return KZ_ERR_UNSUPPORTED;
    KZ_TRY(state_to_bitset(g, g->stream));
    // only the multi-CTA sweep kernels keep the two row buffers in step
    if (path != KZ_PATH_BITSET) g->ab_synced = false;
    if (path == KZ_PATH_SMALL) KZ_TRY(cta_kernelize_one(g, o, g->stream));
    else if (path == KZ_PATH_TENSOR) KZ_TRY(tensor_kernelize(g, o, g->stream));
    else KZ_TRY(bitset_kernelize(g, o, g->stream));
  }
  g->kernelized = true;
  g->path_ran = path;
  return KZ_OK;
}

kz_status kz_kernelize(kz_graph g, const kz_options *opt, void *stream) {
  if (!g) return KZ_ERR_ARG;
  kz_options o;
  KZ_TRY(read_options(opt, o));
  KZ_TRY(set_clique(g, o));
  g->stream = (cudaStream_t)stream;
  g->dom_rounds = 0;
  g->dom_removed = 0;
  if (o.dominance && (o.schedule != KZ_SCHED_PLAIN || !g->has_bitset)) return KZ_ERR_UNSUPPORTED;
  if (o.schedule == KZ_SCHED_LEARNED) {
    // learned worklist rounds on the bitset rows, certified by full passes of
    // the path AUTO would take (the bitset sweep or the tensor form)
    if (!g->has_bitset || !g->model) return KZ_ERR_UNSUPPORTED;
    if (o.path != KZ_PATH_AUTO && o.path != KZ_PATH_BITSET && o.path != KZ_PATH_TENSOR) return KZ_ERR_UNSUPPORTED;
    const int full = o.path == KZ_PATH_AUTO ? (tensor_preferred(g) ? KZ_PATH_TENSOR : KZ_PATH_BITSET) : o.path;
    KZ_TRY(state_to_bitset(g, g->stream));
    g->ab_synced = false;
    KZ_TRY(learned_kernelize(g, o, full, g->stream));
    g->kernelized = true;
    g->path_ran = full;
    return KZ_OK;
  }
  if (o.schedule == KZ_SCHED_SUPPORT) {
    if (g->has_csr && (o.path == KZ_PATH_AUTO || o.path == KZ_PATH_SPARSE)) {
      // incremental support counts on the CSR state
      KZ_TRY(state_to_sparse(g, g->stream));
      KZ_TRY(sparse_kernelize_support(g, o, g->stream));
      g->kernelized = true;
      g->path_ran = KZ_PATH_SPARSE;
      return KZ_OK;
    }
    // re-check sweeps on the bitset rows, the first sweep on the path AUTO
    // would take (the bitset sweep or the tensor form)
    if (!g->has_bitset) return KZ_ERR_UNSUPPORTED;
    if (o.path != KZ_PATH_AUTO && o.path != KZ_PATH_BITSET && o.path != KZ_PATH_TENSOR) return KZ_ERR_UNSUPPORTED;
    const int full = o.path == KZ_PATH_AUTO ? (tensor_preferred(g) ? KZ_PATH_TENSOR : KZ_PATH_BITSET) : o.path;
    KZ_TRY(state_to_bitset(g, g->stream));
    g->ab_synced = false;
    KZ_TRY(recheck_kernelize(g, o, full, g->stream));
    g->kernelized = true;
    g->path_ran = full;
    return KZ_OK;
  }
  const int path = o.path == KZ_PATH_AUTO ? auto_path(g) : o.path;
  if (o.dominance && path == KZ_PATH_SPARSE) return KZ_ERR_UNSUPPORTED;
  // edge dominance relies on every live edge having a common neighbour
  if (o.dominance == 2 && g->k - g->slack < 3) return KZ_ERR_UNSUPPORTED;
  KZ_TRY(run_one(g, o, path));
  if (!o.dominance) return KZ_OK;
  // rounds of vertex (1) or edge (2) dominance, each followed by the
  // colour-index fixpoint
  for (;;) {
    int32_t status = 0;
    KZ_CUDA_TRY(cudaMemcpyAsync(&status, &g->st->status, 4, cudaMemcpyDeviceToHost, g->stream));
    KZ_CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (status != KZ_OK) return KZ_OK;  // a sweep limit or timeout ends the run; fetch reports it
    int64_t removed = 0;
    if (o.dominance == 2) KZ_TRY(edge_dominance_round(g, &removed, g->stream));
    else KZ_TRY(dominance_round(g, &removed, g->stream));
    if (removed == 0) return KZ_OK;
    g->dom_rounds++;
    g->dom_removed += removed;
    KZ_TRY(run_one(g, o, path));
  }
}

}  // extern "C"

namespace {

// Streams (and their events) on which kz_kernelize_batch spreads graphs,
// created once per device.
constexpr int kBatchStreams = 16;

struct StreamPool {
  std::mutex mu;  // one batch enqueues on the pool at a time
  cudaStream_t streams[kBatchStreams];
  cudaEvent_t done[kBatchStreams];
  cudaEvent_t fork;
};

std::mutex g_pools_mu;
std::map<int, StreamPool *> g_pools;

kz_status stream_pool(StreamPool *&out) {
  int dev = 0;
  KZ_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_pools_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) {
    out = it->second;
    return KZ_OK;
  }
  StreamPool *p = new (std::nothrow) StreamPool;
  if (!p) return KZ_ERR_OOM;
  for (int i = 0; i < kBatchStreams; i++) {
    KZ_CUDA_TRY(cudaStreamCreateWithFlags(&p->streams[i], cudaStreamNonBlocking));
    KZ_CUDA_TRY(cudaEventCreateWithFlags(&p->done[i], cudaEventDisableTiming));
  }
  KZ_CUDA_TRY(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
  g_pools[dev] = p;  // kept until the process exits
  out = p;
  return KZ_OK;
}

// Estimated work of one pass of a graph: tested pairs (dense graphs) or
// stored edges, whichever representation it has.
double pass_cost(kz_graph g) {
  if (g->has_bitset) return (double)g->n * (double)g->n * (double)std::max(g->k, 1) + 1e5;
  return (double)g->m * 16.0 + 1e5;
}

// Each graph on its own path, on the pool's streams: longest first, each to
// the stream with the least estimated work so far; the caller's stream then
// waits for all of them.
kz_status batch_concurrent(kz_graph *graphs, int32_t count, const kz_options &o, cudaStream_t s) {
  StreamPool *pool = nullptr;
  KZ_TRY(stream_pool(pool));
  std::lock_guard<std::mutex> lk(pool->mu);
  std::vector<int32_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> cost(count);
  for (int32_t i = 0; i < count; i++) cost[i] = pass_cost(graphs[i]);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  const int used = std::min<int>(kBatchStreams, std::max(count, 1));
  KZ_CUDA_TRY(cudaEventRecord(pool->fork, s));
  for (int i = 0; i < used; i++) KZ_CUDA_TRY(cudaStreamWaitEvent(pool->streams[i], pool->fork, 0));
  std::vector<double> load(used, 0.0);
  kz_status st = KZ_OK;
  for (int32_t j = 0; j < count && st == KZ_OK; j++) {
    kz_graph g = graphs[order[j]];
    const int i = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[i] += cost[order[j]];
    g->stream = pool->streams[i];
    st = run_one(g, o, o.path == KZ_PATH_AUTO ? auto_path(g) : o.path);
  }
  // join every stream that may hold work, even after a failure
  for (int i = 0; i < used; i++) {
    cudaError_t e = cudaEventRecord(pool->done[i], pool->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, pool->done[i], 0);
    if (e != cudaSuccess && st == KZ_OK) st = kz::cuda_status(e);
  }
  for (int32_t j = 0; j < count; j++) graphs[j]->stream = s;
  return st;
}

// One launch for all graphs (after the CSR-only graphs, one by one).
kz_status batch_fused(kz_graph *graphs, int32_t count, const kz_options &o, cudaStream_t s) {
  std::vector<kz_graph> rows;
  for (int32_t i = 0; i < count; i++) {
    if (!graphs[i]->has_bitset) {
      KZ_TRY(run_one(graphs[i], o, KZ_PATH_SPARSE));
      continue;
    }
    KZ_TRY(state_to_bitset(graphs[i], s));
    graphs[i]->ab_synced = false;
    rows.push_back(graphs[i]);
  }
  std::vector<kz_graph> loop, cta;
  for (kz_graph g : rows) {
    // SMALL: every graph in the in-CTA persistent launch; otherwise the
    // batched Jacobi kernel for k <= 32, the in-CTA launch for more colours
    if (o.path == KZ_PATH_SMALL || g->k > 32) cta.push_back(g);
    else loop.push_back(g);
  }
  if (!loop.empty()) KZ_TRY(batch_kernelize(loop.data(), (int)loop.size(), o, s));
  if (!cta.empty()) KZ_TRY(cta_kernelize(cta.data(), (int)cta.size(), o, s, 1));
  for (kz_graph g : loop) {
    g->kernelized = true;
    g->path_ran = KZ_PATH_BITSET;
  }
  for (kz_graph g : cta) {
    g->kernelized = true;
    g->path_ran = KZ_PATH_SMALL;
  }
  return KZ_OK;
}

}  // namespace

extern "C" {

kz_status kz_kernelize_batch(kz_graph *graphs, int32_t count, const kz_options *opt, void *stream) {
  if (count < 0 || (count > 0 && !graphs)) return KZ_ERR_ARG;
  for (int32_t i = 0; i < count; i++)
    if (!graphs[i]) return KZ_ERR_ARG;
  kz_options o;
  KZ_TRY(read_options(opt, o));
  if (o.dominance) return KZ_ERR_UNSUPPORTED;
  if (o.schedule != KZ_SCHED_PLAIN) {
    for (int32_t i = 0; i < count; i++) KZ_TRY(kz_kernelize(graphs[i], &o, stream));
    return KZ_OK;
  }
  bool any_slack = false;
  for (int32_t i = 0; i < count; i++) {
    KZ_TRY(set_clique(graphs[i], o));
    any_slack |= graphs[i]->slack != 0;
  }
  cudaStream_t s = (cudaStream_t)stream;
  for (int32_t i = 0; i < count; i++) graphs[i]->stream = s;
  if (count == 0) return KZ_OK;
  if (o.batch == KZ_BATCH_FUSED) {
    if (o.path == KZ_PATH_BITSET || o.path == KZ_PATH_SPARSE || o.path == KZ_PATH_TENSOR) return KZ_ERR_ARG;
    if (any_slack) return KZ_ERR_UNSUPPORTED;
    return batch_fused(graphs, count, o, s);
  }
  if (o.batch == KZ_BATCH_SEQUENTIAL) {
    for (int32_t i = 0; i < count; i++) {
      kz_graph g = graphs[i];
      KZ_TRY(run_one(g, o, o.path == KZ_PATH_AUTO ? auto_path(g) : o.path));
    }
    return KZ_OK;
  }
  return batch_concurrent(graphs, count, o, s);
}

// Vertices alive, from whichever representation holds the state.
static kz_status owner_vertex_alive(kz_graph g, uint8_t *alive, int64_t *n_live) {
  if (g->owner == KZ_PATH_SPARSE) return sparse_vertex_alive(g, alive, n_live);
  return bitset_vertex_alive(g, alive, n_live);
}

kz_status kz_fetch_stats(kz_graph g, kz_stats *stats) {
  if (!g) return KZ_ERR_ARG;
  if (!g->kernelized) return KZ_ERR_NOT_READY;
  KZ_CUDA_TRY(cudaStreamSynchronize(g->stream));
  DevState hs;
  KZ_CUDA_TRY(cudaMemcpy(&hs, g->st, offsetof(DevState, trace_dv), cudaMemcpyDeviceToHost));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->n = g->n;
    stats->m = g->m;
    stats->sweeps = hs.sweeps;
    stats->passes = hs.passes;
    stats->edge_tests = hs.tests;
    stats->path = g->path_ran;
    stats->status = hs.status;
    stats->k = g->k;
    stats->clique_k = g->k - g->slack;
    stats->dominance_rounds = g->dom_rounds;
    stats->dominated = (int32_t)g->dom_removed;
    KZ_TRY(owner_vertex_alive(g, nullptr, &stats->n_live));
    stats->m_live = -1;  // filled by the fetch calls that count edges
  }
  return (kz_status)hs.status;
}

kz_status kz_fetch_kernel_dense(kz_graph g, uint8_t *vertex_alive, uint64_t *adj_bits,
                                int64_t row_words, kz_stats *stats) {
  if (!g) return KZ_ERR_ARG;
  if (!g->kernelized) return KZ_ERR_NOT_READY;
  if (row_words < (int64_t)((g->n + 63) / 64) || (g->n > 0 && !adj_bits)) return KZ_ERR_ARG;
  if (g->owner == KZ_PATH_SPARSE) {
    KZ_CUDA_TRY(cudaStreamSynchronize(g->stream));
    std::vector<int32_t> e;
    int64_t ml = 0;
    KZ_TRY(sparse_fetch(g, vertex_alive, nullptr, 0, &ml));
    try {
      e.resize((size_t)std::max<int64_t>(2 * ml, 2));
    } catch (...) {
      return KZ_ERR_OOM;
    }
    KZ_TRY(sparse_fetch(g, nullptr, e.data(), ml, &ml));
    memset(adj_bits, 0, (size_t)g->n * row_words * 8);
    for (int64_t i = 0; i < ml; i++) {
      const int32_t u = e[2 * i], v = e[2 * i + 1];
      adj_bits[(size_t)u * row_words + (v >> 6)] |= 1ull << (v & 63);
      adj_bits[(size_t)v * row_words + (u >> 6)] |= 1ull << (u & 63);
    }
    kz_stats tmp;
    kz_status dev_status = kz_fetch_stats(g, &tmp);
    tmp.m_live = ml;
    if (stats) *stats = tmp;
    return dev_status;
  }
  // everything on the stream, one wait at the end: the caller-ordered rows
  // and vertex flags (gathered on the device), the bit count, the run record
  const size_t aux = 16 + (size_t)g->n;
  uint8_t *d_aux = (uint8_t *)dev_alloc(aux, g->stream);
  kz_status st = d_aux ? KZ_OK : KZ_ERR_OOM;
  unsigned long long cnt = 0;
  std::vector<uint8_t> alive((size_t)std::max(g->n, 1));
  DevState hs;
  unsigned long long *d_cnt = reinterpret_cast<unsigned long long *>(d_aux);
  if (st == KZ_OK) st = bitset_fetch_dense(g, adj_bits, row_words, d_aux + 16, d_cnt, g->stream);
  if (st == KZ_OK && g->n)
    st = cuda_status(cudaMemcpyAsync(alive.data(), d_aux + 16, (size_t)g->n, cudaMemcpyDeviceToHost, g->stream));
  if (st == KZ_OK)
    st = cuda_status(cudaMemcpyAsync(&cnt, d_cnt, 8, cudaMemcpyDeviceToHost, g->stream));
  if (st == KZ_OK)
    st = cuda_status(cudaMemcpyAsync(&hs, g->st, offsetof(DevState, trace_dv), cudaMemcpyDeviceToHost, g->stream));
  if (st == KZ_OK) st = cuda_status(cudaStreamSynchronize(g->stream));
  if (d_aux) dev_free(d_aux, aux, g->stream);
  if (st != KZ_OK) return st;
  int64_t n_live = 0;
  for (int32_t v = 0; v < g->n; v++) n_live += alive[v];
  if (vertex_alive && g->n) memcpy(vertex_alive, alive.data(), (size_t)g->n);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->n = g->n;
    stats->m = g->m;
    stats->sweeps = hs.sweeps;
    stats->passes = hs.passes;
    stats->edge_tests = hs.tests;
    stats->path = g->path_ran;
    stats->status = hs.status;
    stats->k = g->k;
    stats->clique_k = g->k - g->slack;
    stats->dominance_rounds = g->dom_rounds;
    stats->dominated = (int32_t)g->dom_removed;
    stats->n_live = n_live;
    stats->m_live = (int64_t)(cnt / 2);
  }
  return (kz_status)hs.status;
}

kz_status kz_fetch_kernel(kz_graph g, uint8_t *vertex_alive, int32_t *edges_out, int64_t cap,
                          int64_t *m_out, kz_stats *stats) {
  if (!g || !m_out || cap < 0 || (cap > 0 && !edges_out)) return KZ_ERR_ARG;
  if (!g->kernelized) return KZ_ERR_NOT_READY;
  if (g->owner == KZ_PATH_SPARSE) {
    kz_stats tmp;
    kz_status dev_status = kz_fetch_stats(g, &tmp);
    if (dev_status != KZ_OK && dev_status != KZ_ERR_LIMIT) return dev_status;
    int64_t ml = 0;
    KZ_TRY(sparse_fetch(g, vertex_alive, edges_out, cap, &ml));
    *m_out = ml;
    tmp.m_live = ml;
    if (stats) *stats = tmp;
    if (ml > cap) return KZ_ERR_BUFFER;
    return dev_status;
  }
  const int64_t rw = (g->n + 63) / 64;
  std::vector<uint64_t> bits;
  try {
    bits.resize((size_t)g->n * rw);
  } catch (...) {
    return KZ_ERR_OOM;
  }
  kz_stats tmp;
  kz_status st = kz_fetch_kernel_dense(g, vertex_alive, bits.data(), rw, &tmp);
  if (st != KZ_OK && st != KZ_ERR_LIMIT) return st;
  // row-major scan of the upper triangle yields (u < v) in lexicographic order
  int64_t cnt = 0;
  for (int32_t u = 0; u < g->n; u++) {
    const uint64_t *row = bits.data() + (size_t)u * rw;
    for (int64_t w = (u + 1) / 64; w < rw; w++) {
      uint64_t word = row[w];
      if (w == (u + 1) / 64) word &= ~0ull << ((u + 1) % 64);
      while (word) {
        const int b = __builtin_ctzll(word);
        word &= word - 1;
        if (cnt < cap) {
          edges_out[2 * cnt] = u;
          edges_out[2 * cnt + 1] = (int32_t)(w * 64 + b);
        }
        cnt++;
      }
    }
  }
  *m_out = cnt;
  if (stats) *stats = tmp;
  if (cnt > cap) return KZ_ERR_BUFFER;
  return st;
}

kz_status kz_fetch_trace(kz_graph g, int64_t *dv, int64_t *de, int64_t cap, int32_t *v_sweep) {
  if (!g || cap < 0 || (cap > 0 && (!dv || !de))) return KZ_ERR_ARG;
  if (!g->kernelized) return KZ_ERR_NOT_READY;
  KZ_CUDA_TRY(cudaStreamSynchronize(g->stream));
  DevState hs;
  KZ_CUDA_TRY(cudaMemcpy(&hs, g->st, offsetof(DevState, trace_dv), cudaMemcpyDeviceToHost));
  const int64_t have = std::min<int64_t>(hs.sweeps, kTraceCap);
  const int64_t ncopy = std::min<int64_t>(have, cap);
  if (ncopy > 0) {
    KZ_CUDA_TRY(cudaMemcpy(dv, g->st->trace_dv, sizeof(int64_t) * ncopy, cudaMemcpyDeviceToHost));
    KZ_CUDA_TRY(cudaMemcpy(de, g->st->trace_de, sizeof(int64_t) * ncopy, cudaMemcpyDeviceToHost));
  }
  if (v_sweep && g->n > 0) {
    std::vector<int32_t> vs((size_t)g->n);
    if (g->owner == KZ_PATH_SPARSE) {
      KZ_TRY(sparse_v_sweep(g, vs.data()));
      for (int32_t v = 0; v < g->n; v++) v_sweep[v] = vs[v] > hs.sweeps ? 0 : vs[v];
    } else {
      KZ_CUDA_TRY(cudaMemcpy(vs.data(), g->v_sweep, sizeof(int32_t) * g->n, cudaMemcpyDeviceToHost));
      for (int32_t x = 0; x < g->n; x++) {
        // a pass stopped by the sweep limit is never applied
        v_sweep[g->perm[x]] = vs[x] > hs.sweeps ? 0 : vs[x];
      }
    }
  }
  return KZ_OK;
}

kz_status kz_reset(kz_graph g, void *stream) {
  if (!g) return KZ_ERR_ARG;
  g->stream = (cudaStream_t)stream;
  if (g->has_bitset) KZ_TRY(bitset_reset(g, g->stream));
  if (g->has_csr) KZ_TRY(sparse_reset(g, g->stream));
  g->owner = g->has_bitset ? KZ_PATH_BITSET : KZ_PATH_SPARSE;
  g->kernelized = false;
  return KZ_OK;
}

void kz_free_graph(kz_graph g) { release(g); }

const char *kz_status_string(kz_status s) {
  switch (s) {
    case KZ_OK: return "ok";
    case KZ_ERR_ARG: return "invalid argument";
    case KZ_ERR_COLOUR_RANGE: return "colour outside [0, k)";
    case KZ_ERR_ILLEGAL_COLOURING: return "edge inside one colour class (colouring not legal)";
    case KZ_ERR_SELF_LOOP: return "self loop";
    case KZ_ERR_VERTEX_RANGE: return "vertex id outside [0, n)";
    case KZ_ERR_DUPLICATE_EDGE: return "duplicate edge";
    case KZ_ERR_OOM: return "device out of memory";
    case KZ_ERR_CUDA: return "CUDA runtime error";
    case KZ_ERR_LIMIT: return "sweep limit reached before the fixpoint";
    case KZ_ERR_TIMEOUT: return "bounded device wait timed out";
    case KZ_ERR_NOT_READY: return "graph not kernelized yet";
    case KZ_ERR_BUFFER: return "output buffer too small";
    case KZ_ERR_UNSUPPORTED: return "path or schedule not available for this graph";
    case KZ_ERR_INTERNAL: return "internal consistency check failed";
  }
  return "unknown status";
}

int32_t kz_version(void) { return 100; }

kz_status kz_probe_barrier_timeout(kz_graph g, uint32_t spin_limit, void *stream) {
  if (!g || spin_limit == 0) return KZ_ERR_ARG;
  if (!g->has_bitset) return KZ_ERR_UNSUPPORTED;
  g->stream = (cudaStream_t)stream;
  g->slack = 0;
  KZ_TRY(state_to_bitset(g, g->stream));
  KZ_TRY(bitset_barrier_timeout_probe(g, spin_limit, g->stream));
  g->kernelized = true;
  g->path_ran = KZ_PATH_BITSET;
  return KZ_OK;
}

}  // extern "C"
