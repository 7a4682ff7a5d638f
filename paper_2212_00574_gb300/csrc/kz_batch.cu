// kz_batch.cu -- batched Jacobi loop: many graphs, one pass of every
// unconverged graph per launch of a multi-graph sweep kernel, launches
// repeated by a CUDA-graph while node until no graph changes.
//
// Each graph keeps its own Jacobi state (thesis Section 4.2 rules, ping-pong
// buffers, counters) exactly as a single-graph kernelize does.  A work item
// is (graph, block x, blocks [y0, y1)); the last item of a graph to finish
// closes that graph's pass, and the last warp of the launch sets the loop
// condition.  Nothing ever waits on another CTA.  Per-graph item sizes come
// from a cost model so that a batch of uneven graphs fills the GPU evenly.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kz_internal.cuh"
#include "kz_rules.cuh"

namespace kz {

struct BatchGraph {
  uint32_t *A0, *A1, *V0, *V1;
  int32_t *v_sweep;
  DevState *st;
  const BlockDesc *blocks;
  const int32_t *rounds;
  int32_t k, ldw;
  int32_t n_items;
  int32_t n;
  int64_t max_sweeps;
};

struct BatchItem {
  int32_t g;
  int32_t x;
  int32_t y0;
  int32_t y1v;  // y1 | (vflag << 31)
};

struct BatchCtl {
  unsigned int ticket;     // warps finished in this launch
  int32_t any_cont;        // some graph needs another pass
};

struct BatchArgs {
  const BatchGraph *graphs;
  const BatchItem *items;
  int32_t n_items;
  BatchCtl *ctl;
  cudaGraphConditionalHandle cond;
  int32_t use_cond;
};

constexpr int kBatchWarps = 4;

template <int KMAX>
__global__ void __launch_bounds__(kBatchWarps * 32) batch_sweep_kernel(BatchArgs p) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint32_t *sv = smem + wib * 32 * KMAX;
  const int warps_total = gridDim.x * kBatchWarps;
  for (int it = blockIdx.x * kBatchWarps + wib; it < p.n_items; it += warps_total) {
    const BatchItem item = p.items[it];
    const BatchGraph &G = p.graphs[item.g];
    DevState *st = G.st;
    if (!*((volatile int32_t *)&st->cont)) continue;  // converged: its items are skipped
    const int cur = *((volatile int32_t *)&st->cur);
    const int64_t sweep_no = *((volatile int64_t *)&st->sweeps);
    const uint32_t *__restrict__ A = cur ? G.A1 : G.A0;
    uint32_t *__restrict__ An = cur ? G.A0 : G.A1;
    const uint32_t *__restrict__ Vc = cur ? G.V1 : G.V0;
    uint32_t *__restrict__ Vn = cur ? G.V0 : G.V1;
    const int k = G.k, ldw = G.ldw;
    const int y1 = item.y1v & 0x7fffffff;
    const bool vflag = (item.y1v >> 31) & 1;
    const BlockDesc X = G.blocks[item.x];
    const int cu = X.c;
    const bool valid_u = lane < X.size;
    const int u = X.base + lane;
    const uint32_t *rowu = A + (int64_t)(valid_u ? u : X.base) * ldw;
    uint32_t Fu[KMAX];
    load_plane0<KMAX>(Fu, rowu, k, valid_u);
    unsigned long long my_tests = 0, my_de = 0, my_dv = 0;
    if (vflag) {
      const int wx = X.r * k + cu;
      const uint32_t vword = Vc[wx];
      const bool live = valid_u && ((vword >> lane) & 1u);
      int cnt = plane0_vertex_cover<KMAX>(Fu, k, cu);
      if (live && cnt < k - 1) cnt = exact_vertex_cover_row(rowu, k, G.rounds, cu);
      const bool fail = live && cnt < k - 1;
      const uint32_t failmask = __ballot_sync(0xffffffffu, fail);
      if (lane == 0) {
        Vn[wx] = vword & ~failmask;
        my_dv += __popc(failmask);
      }
      if (fail && G.v_sweep) G.v_sweep[u] = (int32_t)(sweep_no + 1);
    }
    uint32_t P[KMAX];
    int prev_cv = -1;
    for (int y = item.y0; y < y1; y++) {
      const BlockDesc Y = G.blocks[y];
      const int cv = Y.c;
      if (cv != prev_cv) {
        pair_mask<KMAX>(P, k, cu, cv);
        prev_cv = cv;
      }
      __syncwarp();
      const int kq = (k + 3) & ~3;  // columns the test reads
      for (int idx = lane; idx < 32 * kq; idx += 32) {
        const int b = idx / kq;
        const int c = idx - b * kq;
        sv[b * KMAX + c] = (b < Y.size && c < k) ? A[(int64_t)(Y.base + b) * ldw + c] : 0u;
      }
      __syncwarp();
      const int wy = Y.r * k + cv;
      const uint32_t adjw = valid_u ? A[(int64_t)u * ldw + wy] : 0u;
      my_tests += __popc(adjw);
      const uint32_t del = edge_rule_block<KMAX>(
          Fu, P, rowu, adjw, k, G.rounds, cu, cv,
          [&](int b) { return (const uint32_t *)(sv + b * KMAX); },
          [&](int b) { return A + (int64_t)(Y.base + b) * ldw; });
      if (valid_u) An[(int64_t)u * ldw + wy] = adjw & ~del;
      my_de += __popc(del);
      const uint32_t delT = transpose_deletions(del);
      if (lane < Y.size) {
        const int64_t wi = (int64_t)(Y.base + lane) * ldw + X.r * k + cu;
        An[wi] = A[wi] & ~delT;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      my_tests += __shfl_down_sync(0xffffffffu, my_tests, o);
      my_de += __shfl_down_sync(0xffffffffu, my_de, o);
      my_dv += __shfl_down_sync(0xffffffffu, my_dv, o);
    }
    if (lane == 0) {
      if (my_tests) atomicAdd(&st->pass_tests, my_tests);
      if (my_de) atomicAdd(&st->pass_de, my_de);
      if (my_dv) atomicAdd(&st->pass_dv, my_dv);
      __threadfence();
      const unsigned int t = atomicAdd(&st->ticket, 1u);
      if (t == (unsigned int)G.n_items - 1u) {
        // last item of this graph's pass
        __threadfence();
        const unsigned long long dv = atomicAdd(&st->pass_dv, 0ull);
        const unsigned long long de = atomicAdd(&st->pass_de, 0ull);
        const unsigned long long tests = atomicAdd(&st->pass_tests, 0ull);
        const int cont = finish_pass(st, dv, de, tests);
        st->pass_dv = 0;
        st->pass_de = 0;
        st->pass_tests = 0;
        st->ticket = 0;
        if (cont) atomicOr(&p.ctl->any_cont, 1);
        __threadfence();
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(&p.ctl->ticket, 1u);
    if (t == (unsigned int)warps_total - 1u) {
      __threadfence();
      const int cont = atomicExch(&p.ctl->any_cont, 0);
      p.ctl->ticket = 0;
      __threadfence();
      if (p.use_cond) cudaGraphSetConditional(p.cond, cont ? 1u : 0u);
    }
  }
}

// Run start for every graph of the batch: counters zero, every graph active.
__global__ void batch_begin_kernel(const BatchGraph *graphs, int count, BatchCtl *ctl) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < count; g += gridDim.x * blockDim.x) {
    DevState *st = graphs[g].st;
    st->status = KZ_OK;
    st->sweeps = 0;
    st->passes = graphs[g].n == 0 ? 1 : 0;
    st->tests = 0;
    st->max_sweeps = graphs[g].max_sweeps;
    st->pass_dv = st->pass_de = st->pass_tests = 0;
    st->ticket = 0;
    st->cont = graphs[g].n_items > 0 ? 1 : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->ticket = 0;
    ctl->any_cont = 0;
  }
}

// ---------------------------------------------------------------------------
// host side: cost model, item lists, the loop graph
// ---------------------------------------------------------------------------

// Cost of one block pair (x, y): 32 pair tests of ~k class words each.
static inline double pair_cost(int k) { return 32.0 * (double)std::max(k, 1); }

static int sm_count_here() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}

// The autotuner: picks each graph's item length (block pairs per item) so that
// items cost about the same across the batch and there are ~16 warps' worth of
// items per SM scheduler.
static void build_batch_items(kz_graph *gs, int count, std::vector<BatchItem> &items,
                              std::vector<int32_t> &per_graph) {
  double total = 0;
  for (int i = 0; i < count; i++) total += (double)gs[i]->n_pairs * pair_cost(gs[i]->k);
  const double target_items = 16.0 * 4 * sm_count_here();
  const double item_cost = std::max(total / target_items, pair_cost(8));
  per_graph.assign(count, 0);
  for (int i = 0; i < count; i++) {
    kz_graph g = gs[i];
    const int nb = (int)g->blocks.size();
    const int64_t S = std::max<int64_t>(1, (int64_t)(item_cost / pair_cost(g->k)));
    for (int x = 0; x < nb; x++) {
      const int yb = g->boff[g->blocks[x].c + 1];
      if (yb >= nb) {
        items.push_back({i, x, nb, (int32_t)(nb | (1u << 31))});
        per_graph[i]++;
        continue;
      }
      bool first = true;
      for (int64_t y = yb; y < nb; y += S) {
        const int32_t y1 = (int32_t)std::min<int64_t>(nb, y + S);
        items.push_back({i, x, (int32_t)y, (int32_t)(y1 | (first ? (1u << 31) : 0u))});
        per_graph[i]++;
        first = false;
      }
    }
  }
}

kz_status batch_kernelize(kz_graph *gs, int count, const kz_options &opt, cudaStream_t s) {
  if (count <= 0) return KZ_OK;
  for (int i = 0; i < count; i++)
    if (gs[i]->k > 32) return KZ_ERR_UNSUPPORTED;  // caller routes k > 32 elsewhere
  std::vector<BatchItem> items;
  std::vector<int32_t> per_graph;
  build_batch_items(gs, count, items, per_graph);
  std::vector<BatchGraph> desc((size_t)count);
  for (int i = 0; i < count; i++) {
    kz_graph g = gs[i];
    BatchGraph &d = desc[i];
    memset(&d, 0, sizeof(d));
    d.A0 = g->A[0];
    d.A1 = g->A[1];
    d.V0 = g->V[0];
    d.V1 = g->V[1];
    d.v_sweep = g->v_sweep;
    d.st = g->st;
    d.blocks = g->d_blocks;
    d.rounds = g->d_rounds;
    d.k = g->k;
    d.ldw = g->ldw;
    d.n_items = per_graph[i];
    d.n = g->n;
    d.max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : (int64_t)g->n + g->m + 1;
  }
  const size_t bytes_g = sizeof(BatchGraph) * count;
  const size_t bytes_i = sizeof(BatchItem) * std::max<size_t>(items.size(), 1);
  BatchGraph *d_desc = (BatchGraph *)dev_alloc(bytes_g, s);
  BatchItem *d_items = (BatchItem *)dev_alloc(bytes_i, s);
  BatchCtl *d_ctl = (BatchCtl *)dev_alloc(sizeof(BatchCtl), s);
  kz_status st = (d_desc && d_items && d_ctl) ? KZ_OK : KZ_ERR_OOM;
  if (st == KZ_OK)
    st = cuda_status(cudaMemcpyAsync(d_desc, desc.data(), bytes_g, cudaMemcpyHostToDevice, s));
  if (st == KZ_OK && !items.empty())
    st = cuda_status(cudaMemcpyAsync(d_items, items.data(), sizeof(BatchItem) * items.size(),
                                     cudaMemcpyHostToDevice, s));
  if (st == KZ_OK) {
    batch_begin_kernel<<<(count + 255) / 256, 256, 0, s>>>(d_desc, count, d_ctl);
    st = cuda_status(cudaGetLastError());
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (st == KZ_OK && !items.empty()) {
    const int kmax = 32;
    auto fn = batch_sweep_kernel<32>;
    const size_t smem = (size_t)kBatchWarps * 32 * kmax * 4;
    int per_sm = 0;
    st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn,
                                                                   kBatchWarps * 32, smem));
    const int want = (int)((items.size() + kBatchWarps - 1) / kBatchWarps);
    const int grid = std::max(1, std::min(want, std::max(per_sm, 1) * sm_count_here()));
    if (st == KZ_OK) st = cuda_status(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    if (st == KZ_OK)
      st = cuda_status(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
    cudaGraphNode_t wnode;
    if (st == KZ_OK) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      st = cuda_status(cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &cp));
    }
    if (st == KZ_OK) {
      BatchArgs a;
      a.graphs = d_desc;
      a.items = d_items;
      a.n_items = (int32_t)items.size();
      a.ctl = d_ctl;
      a.cond = handle;
      a.use_cond = 1;
      void *kargs[] = {&a};
      cudaKernelNodeParams kp;
      memset((void *)&kp, 0, sizeof(kp));
      kp.func = (void *)fn;
      kp.gridDim = dim3(grid);
      kp.blockDim = dim3(kBatchWarps * 32);
      kp.sharedMemBytes = (unsigned)smem;
      kp.kernelParams = kargs;
      cudaGraphNode_t knode;
      st = cuda_status(cudaGraphAddKernelNode(&knode, cp.conditional.phGraph_out[0], nullptr, 0, &kp));
    }
    if (st == KZ_OK) st = cuda_status(cudaGraphInstantiate(&exec, graph, 0));
    if (st == KZ_OK) st = cuda_status(cudaGraphLaunch(exec, s));
  }
  if (exec) cudaGraphExecDestroy(exec);  // safe: destruction waits for nothing, launch keeps its copy
  if (graph) cudaGraphDestroy(graph);
  if (d_desc) dev_free(d_desc, bytes_g, s);
  if (d_items) dev_free(d_items, bytes_i, s);
  if (d_ctl) dev_free(d_ctl, sizeof(BatchCtl), s);
  return st;
}

}  // namespace kz
