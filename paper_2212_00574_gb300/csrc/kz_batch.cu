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
#include <mutex>
#include <vector>

#include "kz_internal.cuh"
#include "kz_rules.cuh"
#include "kz_sweep.cuh"

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

struct PersistCtl {
  unsigned int bar_count;
  unsigned int bar_gen;
  int32_t any_cont;
  int32_t go;
  int32_t abort;
  int32_t pad;
};

constexpr uint32_t kBatchSpinLimit = 1u << 25;

// Every pass of every graph in one cooperative launch.  A pass of the batch
// processes the items of all unconverged graphs; the last item of a graph
// closes that graph's pass; a bounded grid barrier separates the batch's
// passes, and the last CTA to arrive decides whether another follows.
template <int KMAX>
__global__ void __launch_bounds__(kBatchWarps * 32) batch_persistent_kernel(BatchArgs p, PersistCtl *ctl) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_go;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint32_t *buf0 = smem + wib * 2 * 32 * KMAX;
  uint32_t *buf1 = buf0 + 32 * KMAX;
  const int warps_total = gridDim.x * kBatchWarps;
  for (;;) {
    for (int it = blockIdx.x * kBatchWarps + wib; it < p.n_items; it += warps_total) {
      const BatchItem bi = p.items[it];
      const BatchGraph &B = p.graphs[bi.g];
      DevState *st = B.st;
      if (!*((volatile int32_t *)&st->cont)) continue;
      const int cur = *((volatile int32_t *)&st->cur);
      const int64_t sweep_no = *((volatile int64_t *)&st->sweeps);
      GraphView G;
      G.blocks = B.blocks;
      G.rounds = B.rounds;
      G.A0 = B.A0;
      G.A1 = B.A1;
      G.V0 = B.V0;
      G.V1 = B.V1;
      G.v_sweep = B.v_sweep;
      G.k = B.k;
      G.ldw = B.ldw;
      WorkItem wi;
      wi.x = bi.x;
      wi.y0 = bi.y0;
      wi.y1 = bi.y1v & 0x7fffffff;
      wi.vflag = (bi.y1v >> 31) & 1;
      PassCounters pc;
      sweep_item<KMAX>(G, wi, cur, sweep_no, buf0, buf1, pc);
      for (int o = 16; o > 0; o >>= 1) {
        pc.tests += __shfl_down_sync(0xffffffffu, pc.tests, o);
        pc.de += __shfl_down_sync(0xffffffffu, pc.de, o);
        pc.dv += __shfl_down_sync(0xffffffffu, pc.dv, o);
      }
      if (lane == 0) {
        if (pc.tests) atomicAdd(&st->pass_tests, pc.tests);
        if (pc.de) atomicAdd(&st->pass_de, pc.de);
        if (pc.dv) atomicAdd(&st->pass_dv, pc.dv);
        __threadfence();
        if (atomicAdd(&st->ticket, 1u) == (unsigned int)B.n_items - 1u) {
          __threadfence();
          const unsigned long long dv = atomicAdd(&st->pass_dv, 0ull);
          const unsigned long long de = atomicAdd(&st->pass_de, 0ull);
          const unsigned long long tests = atomicAdd(&st->pass_tests, 0ull);
          const int cont = finish_pass(st, dv, de, tests);
          st->pass_dv = st->pass_de = st->pass_tests = 0;
          st->ticket = 0;
          if (cont) atomicOr(&ctl->any_cont, 1);
          __threadfence();
        }
      }
      __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned int gen = *((volatile unsigned int *)&ctl->bar_gen);
      if (atomicAdd(&ctl->bar_count, 1u) == gridDim.x - 1u) {
        __threadfence();
        ctl->go = atomicExch(&ctl->any_cont, 0);
        ctl->bar_count = 0;
        __threadfence();
        atomicExch(&ctl->bar_gen, gen + 1u);
      } else {
        uint32_t spins = 0;
        while (*((volatile unsigned int *)&ctl->bar_gen) == gen) {
          if (*((volatile int32_t *)&ctl->abort)) break;
          __nanosleep(64);
          if (++spins > kBatchSpinLimit) {
            atomicExch(&ctl->abort, 1);
            break;
          }
        }
      }
      __threadfence();
      s_go = *((volatile int32_t *)&ctl->go) && !*((volatile int32_t *)&ctl->abort);
    }
    __syncthreads();
    if (!s_go) break;
  }
}

// After a batch: graphs whose barrier wait ran out are marked.
__global__ void batch_timeout_kernel(const BatchGraph *graphs, int count, const PersistCtl *ctl) {
  if (!ctl->abort) return;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < count; g += gridDim.x * blockDim.x)
    atomicCAS(&graphs[g].st->status, (int32_t)KZ_OK, (int32_t)KZ_ERR_TIMEOUT);
}

__global__ void persist_ctl_reset_kernel(PersistCtl *ctl) {
  ctl->bar_count = 0;
  ctl->bar_gen = 0;
  ctl->any_cont = 0;
  ctl->go = 0;
  ctl->abort = 0;
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
  if (ctl && blockIdx.x == 0 && threadIdx.x == 0) {
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

// The plan of the last batch (descriptors, items, control block), kept on
// the device so that running the same batch again does no host work.  A plan
// is identified by the graphs' load identities and the sweep limit.
struct BatchPlan {
  std::vector<uint64_t> key;
  BatchGraph *desc = nullptr;
  BatchItem *items = nullptr;
  PersistCtl *ctl = nullptr;
  size_t desc_bytes = 0, item_bytes = 0;
  int32_t n_items = 0;
  int device = -1;
};

static std::mutex g_plan_mu;
static BatchPlan g_plan;

static void plan_release(BatchPlan &pl) {
  if (pl.desc) cudaFree(pl.desc);
  if (pl.items) cudaFree(pl.items);
  if (pl.ctl) cudaFree(pl.ctl);
  pl = BatchPlan();
}

kz_status batch_kernelize(kz_graph *gs, int count, const kz_options &opt, cudaStream_t s) {
  if (count <= 0) return KZ_OK;
  for (int i = 0; i < count; i++)
    if (gs[i]->k > 32) return KZ_ERR_UNSUPPORTED;  // caller routes k > 32 elsewhere
  std::vector<uint64_t> key;
  key.reserve((size_t)count + 1);
  for (int i = 0; i < count; i++) key.push_back(gs[i]->uid);
  key.push_back((uint64_t)opt.max_sweeps);
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_plan_mu);
  if (g_plan.key != key || g_plan.device != dev) {
    // the plan must not be freed while an earlier launch may still read it
    if (g_plan.desc) KZ_CUDA_TRY(cudaDeviceSynchronize());
    plan_release(g_plan);
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
    BatchPlan pl;
    pl.key = key;
    pl.device = dev;
    pl.desc_bytes = sizeof(BatchGraph) * count;
    pl.item_bytes = sizeof(BatchItem) * std::max<size_t>(items.size(), 1);
    pl.n_items = (int32_t)items.size();
    cudaError_t e = cudaMalloc(&pl.desc, pl.desc_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&pl.items, pl.item_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&pl.ctl, sizeof(PersistCtl));
    if (e == cudaSuccess) e = cudaMemcpy(pl.desc, desc.data(), pl.desc_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !items.empty())
      e = cudaMemcpy(pl.items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      plan_release(pl);
      return cuda_status(e);
    }
    g_plan = pl;
  }
  BatchPlan &pl = g_plan;
  batch_begin_kernel<<<(count + 255) / 256, 256, 0, s>>>(pl.desc, count, nullptr);
  persist_ctl_reset_kernel<<<1, 1, 0, s>>>(pl.ctl);
  KZ_CUDA_TRY(cudaGetLastError());
  if (pl.n_items == 0) return KZ_OK;
  auto fn = batch_persistent_kernel<32>;
  const size_t smem = (size_t)kBatchWarps * 2 * 32 * 32 * 4;
  KZ_CUDA_TRY(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  KZ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, kBatchWarps * 32, smem));
  const int want = (pl.n_items + kBatchWarps - 1) / kBatchWarps;
  const int grid = std::max(1, std::min(want, std::max(per_sm, 1) * sm_count_here()));
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.graphs = pl.desc;
  a.items = pl.items;
  a.n_items = pl.n_items;
  a.ctl = nullptr;
  a.use_cond = 0;
  PersistCtl *ctl = pl.ctl;
  void *kargs[] = {&a, &ctl};
  KZ_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(kBatchWarps * 32), kargs, smem, s));
  batch_timeout_kernel<<<(count + 255) / 256, 256, 0, s>>>(pl.desc, count, pl.ctl);
  KZ_CUDA_TRY(cudaGetLastError());
  return KZ_OK;
}

}  // namespace kz
