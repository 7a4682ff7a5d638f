// kz_batch.cu -- the fused batch: many graphs kernelized in one persistent
// cooperative launch, captured once per batch into a CUDA graph and replayed.
//
// Each graph keeps its own Jacobi state (thesis Section 4.2 rules, ping-pong
// buffers, counters) exactly as a single-graph kernelize does.  The launch's
// CTAs form groups: a group of c_g CTAs owns graph g from its first pass to
// its fixpoint, then its CTAs move on.  Graphs are claimed from a queue in
// order of estimated cost, largest first; the queue holds one entry per
// (graph, member), and a CTA that takes an entry joins that graph's group.
// Inside a group a pass is split into work items (block X against a run of
// higher-class blocks Y) that the group's warps take in turn; the warp that
// finishes a graph's last item closes the pass; a barrier among the group's
// CTAs (one CTA: __syncthreads) separates passes, and its last arriver
// decides for the whole group whether another pass follows.  So a graph's rows stay in
// L2 across its passes, no CTA waits for graphs it does not work on, and
// small graphs (one CTA each) never pay a grid-wide barrier.
//
// Why no deadlock: the cooperative launch makes every CTA resident, and the
// queue is taken in order, so when some CTA waits for the members of graph g
// every graph before g already has all its members, and those finish.
//
// The per-graph group sizes and item lengths come from a cost model (the
// batch autotuner, paper_2212_00574_gb300/autotune.py, measured its scale).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
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
  int32_t item0, n_items;  // this graph's items: [item0, item0 + n_items)
  int32_t n;
  int32_t pad;
  int64_t max_sweeps;
};

struct BatchItem {
  int32_t x;
  int32_t y0;
  int32_t y1v;  // y1 | (vflag << 31)
};

struct GroupEntry {
  int32_t g;        // graph
  int32_t member;   // this CTA's index in the graph's group
  int32_t members;  // group size
};

struct BatchCtl {
  unsigned int next;  // queue head: next entry to take
  int32_t abort;      // a bounded wait ran out
};

struct BatchArgs {
  const BatchGraph *graphs;
  const BatchItem *items;
  const GroupEntry *entries;
  int32_t n_entries;
  BatchCtl *ctl;
};

constexpr int kBatchWarps = 4;
constexpr uint64_t kGroupWaitNs = 30ull * 1000 * 1000 * 1000;  // 30 s of wall clock per barrier wait

__device__ __forceinline__ uint64_t batch_clock() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier of a group's CTAs (thread 0 of each), bounded by the wall clock.
// The last to arrive reads whether the graph needs another pass and publishes
// it in the top bit of the barrier word together with the next generation
// (low 31 bits); the others wait for the generation to move and read the
// decision from the word.  Returns the decision (0 also after an abort).
__device__ __forceinline__ int group_sync(DevState *st, BatchCtl *ctl, int members, uint32_t gen) {
  constexpr uint32_t kGenMask = 0x7fffffffu;
  __threadfence();
  if (atomicAdd(&st->bar_count, 1u) == (unsigned int)members - 1u) {
    st->bar_count = 0;
    __threadfence();
    const int go = *((volatile int32_t *)&st->cont) && !*((volatile int32_t *)&ctl->abort);
    atomicExch(&st->bar_gen, ((gen + 1u) & kGenMask) | (go ? 0x80000000u : 0u));
    return go;
  }
  const uint64_t t0 = batch_clock();
  for (;;) {
    const uint32_t w = *((volatile unsigned int *)&st->bar_gen);
    if ((w & kGenMask) != (gen & kGenMask)) {
      __threadfence();
      return (int)(w >> 31) && !*((volatile int32_t *)&ctl->abort);
    }
    if (*((volatile int32_t *)&ctl->abort)) return 0;
    __nanosleep(128);
    if (batch_clock() - t0 > kGroupWaitNs) {
      atomicExch(&ctl->abort, 1);
      atomicCAS(&st->status, (int32_t)KZ_OK, (int32_t)KZ_ERR_TIMEOUT);
      return 0;
    }
  }
}

// One work item at class-word width KMAX, kept out of line so that the four
// widths the kernel dispatches between do not add up their registers.
template <int KMAX>
__device__ __noinline__ void batch_item(const GraphView &G, const WorkItem wi, int cur, int64_t sweep_no,
                                        uint32_t *buf0, uint32_t *buf1, PassCounters &pc) {
  sweep_item<KMAX>(G, wi, cur, sweep_no, buf0, buf1, pc);
}

template <int KMAX>
__global__ void __launch_bounds__(kBatchWarps * 32, 4) batch_group_kernel(BatchArgs p) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_entry;
  __shared__ int s_go;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint32_t *buf0 = smem + wib * 2 * 32 * KMAX;
  uint32_t *buf1 = buf0 + 32 * KMAX;
  BatchCtl *ctl = p.ctl;
  for (;;) {
    if (threadIdx.x == 0) s_entry = (int)atomicAdd(&ctl->next, 1u);
    __syncthreads();
    const int e = s_entry;
    if (e >= p.n_entries || *((volatile int32_t *)&ctl->abort)) break;
    const GroupEntry E = p.entries[e];
    const BatchGraph &B = p.graphs[E.g];
    DevState *st = B.st;
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
    uint32_t gen = 0;  // the group barrier's generations this CTA has passed
    for (;;) {
      // Whether the graph needs another pass.  A group decides it at its
      // barrier: every member arrives (once before the first pass, then after
      // each pass), and the last to arrive -- after every item of the pass, so
      // after the pass was closed -- publishes the decision with the new
      // generation.  A member must not read the graph's state on its own: one
      // with no items in a pass could read it after the others closed the pass
      // and leave without arriving.
      if (threadIdx.x == 0) {
        if (E.members > 1) s_go = group_sync(st, ctl, E.members, gen);
        else s_go = *((volatile int32_t *)&st->cont) && !*((volatile int32_t *)&ctl->abort);
      }
      gen++;
      __syncthreads();
      if (!s_go) break;
      const int cur = *((volatile int32_t *)&st->cur);
      const int64_t sweep_no = *((volatile int64_t *)&st->sweeps);
      const int step = E.members * kBatchWarps;
      for (int it = E.member * kBatchWarps + wib; it < B.n_items; it += step) {
        const BatchItem bi = p.items[B.item0 + it];
        WorkItem wi;
        wi.x = bi.x;
        wi.y0 = bi.y0;
        wi.y1 = bi.y1v & 0x7fffffff;
        wi.vflag = (bi.y1v >> 31) & 1;
        PassCounters pc;
        // the narrowest class-word width that holds the graph's k
        if (B.k <= 8) batch_item<8>(G, wi, cur, sweep_no, buf0, buf1, pc);
        else if (B.k <= 16) batch_item<16>(G, wi, cur, sweep_no, buf0, buf1, pc);
        else if (B.k <= 24) batch_item<24>(G, wi, cur, sweep_no, buf0, buf1, pc);
        else batch_item<KMAX>(G, wi, cur, sweep_no, buf0, buf1, pc);
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
            // the last item of the pass: close it
            __threadfence();
            const unsigned long long dv = atomicAdd(&st->pass_dv, 0ull);
            const unsigned long long de = atomicAdd(&st->pass_de, 0ull);
            const unsigned long long tests = atomicAdd(&st->pass_tests, 0ull);
            finish_pass(st, dv, de, tests);
            st->pass_dv = st->pass_de = st->pass_tests = 0;
            st->ticket = 0;
            __threadfence();
          }
        }
        __syncwarp();
      }
      __syncthreads();
    }
  }
}

// After a batch whose wait ran out: every unfinished graph is marked.
__global__ void batch_timeout_kernel(const BatchGraph *graphs, int count, const BatchCtl *ctl) {
  if (!ctl->abort) return;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < count; g += gridDim.x * blockDim.x)
    if (graphs[g].st->cont) atomicCAS(&graphs[g].st->status, (int32_t)KZ_OK, (int32_t)KZ_ERR_TIMEOUT);
}

// Run start for every graph of the batch: counters zero, every graph with
// work active, the group barriers and the queue reset.
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
    st->bar_count = 0;
    st->bar_gen = 0;
    st->cont = graphs[g].n_items > 0 ? 1 : 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->next = 0;
    ctl->abort = 0;
  }
}

// ---------------------------------------------------------------------------
// host side: cost model, the plan, the captured graph
// ---------------------------------------------------------------------------

// Cost of one block pair (x, y): 32 pair tests of ~k class words each.
static inline double pair_cost(int k) { return 32.0 * (double)std::max(k, 1); }

static int sm_count_here() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}

// The batch cost model.  A graph's pass costs its block pairs times k; its
// group gets c_g = clamp(cost / unit, 1, kMaxGroup) CTAs, where unit is the
// batch's total cost divided by kGroupSpread times the grid (so that, if all
// graphs ran at once, they would ask for kGroupSpread grids' worth of CTAs),
// and its items hold about kItemsPerWarp items per warp of the group.
// The three constants are the batch autotuner's fastest setting on the
// 1024-graph workload (paper_2212_00574_gb300/autotune_batch.json): large
// groups win, because a graph's passes are latency-bound chains of work items
// and cascading graphs need many of them.
constexpr int kMaxGroup = 64;
constexpr double kGroupSpread = 128.0;
constexpr int kItemsPerWarp = 4;

struct BatchTuning {
  double group_spread = kGroupSpread;
  int32_t items_per_warp = kItemsPerWarp;
  int32_t max_group = kMaxGroup;
};
static BatchTuning g_tuning;  // guarded by g_plan_mu

static void build_plan(kz_graph *gs, int count, int grid, std::vector<BatchItem> &items,
                       std::vector<BatchGraph> &desc, std::vector<GroupEntry> &entries,
                       const kz_options &opt, const BatchTuning &tune) {
  std::vector<double> cost(count);
  double total = 0;
  for (int i = 0; i < count; i++) {
    cost[i] = (double)gs[i]->n_pairs * pair_cost(gs[i]->k) + 1.0;
    total += cost[i];
  }
  const double unit = std::max(total / (tune.group_spread * grid), 1.0);
  std::vector<int32_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
  desc.assign(count, BatchGraph());
  for (int oi = 0; oi < count; oi++) {
    const int i = order[oi];
    kz_graph g = gs[i];
    const int nb = (int)g->blocks.size();
    const int members = (int)std::min<double>(tune.max_group, std::max(1.0, std::ceil(cost[i] / unit)));
    // block pairs per item: spread the pass over ~kItemsPerWarp items per warp
    const double pairs = std::max<double>((double)g->n_pairs, 1.0);
    const int64_t S =
        std::max<int64_t>(1, (int64_t)(pairs / ((double)members * kBatchWarps * tune.items_per_warp)));
    BatchGraph &d = desc[i];
    memset(&d, 0, sizeof(d));
    d.item0 = (int32_t)items.size();
    for (int x = 0; x < nb; x++) {
      const int yb = g->boff[g->blocks[x].c + 1];
      if (yb >= nb) {
        items.push_back({x, nb, (int32_t)(nb | (1u << 31))});
        continue;
      }
      bool first = true;
      for (int64_t y = yb; y < nb; y += S) {
        const int32_t y1 = (int32_t)std::min<int64_t>(nb, y + S);
        items.push_back({x, (int32_t)y, (int32_t)(y1 | (first ? (1u << 31) : 0u))});
        first = false;
      }
    }
    d.n_items = (int32_t)items.size() - d.item0;
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
    d.n = g->n;
    d.max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : (int64_t)g->n + g->m + 1;
    if (d.n_items == 0) continue;  // nothing to test: no entry
    const int m = std::min(members, std::max(1, grid));
    for (int j = 0; j < m; j++) entries.push_back({i, j, m});
  }
}

// The plan of the last batch (descriptors, items, queue entries, control
// block) and its captured launch, kept on the device so that running the same
// batch again is one graph launch.  A plan is identified by the graphs' load
// identities and the sweep limit.
struct BatchPlan {
  std::vector<uint64_t> key;
  BatchGraph *desc = nullptr;
  BatchItem *items = nullptr;
  GroupEntry *entries = nullptr;
  BatchCtl *ctl = nullptr;
  int32_t n_entries = 0, count = 0, grid = 0;
  size_t smem = 0;
  int device = -1;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;
};

static std::mutex g_plan_mu;
static BatchPlan g_plan;

static void plan_release(BatchPlan &pl) {
  if (pl.exec) cudaGraphExecDestroy(pl.exec);
  if (pl.desc) cudaFree(pl.desc);
  if (pl.items) cudaFree(pl.items);
  if (pl.entries) cudaFree(pl.entries);
  if (pl.ctl) cudaFree(pl.ctl);
  cudaStream_t cap = pl.capture;
  pl = BatchPlan();
  pl.capture = cap;  // the capture stream is kept for the next plan
}

// The batch's launches: run start, the persistent launch, the timeout marks.
static kz_status enqueue_batch(const BatchPlan &pl, cudaStream_t s) {
  batch_begin_kernel<<<(pl.count + 255) / 256, 256, 0, s>>>(pl.desc, pl.count, pl.ctl);
  KZ_CUDA_TRY(cudaGetLastError());
  if (pl.n_entries == 0) return KZ_OK;
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.graphs = pl.desc;
  a.items = pl.items;
  a.entries = pl.entries;
  a.n_entries = pl.n_entries;
  a.ctl = pl.ctl;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(pl.grid);
  cfg.blockDim = dim3(kBatchWarps * 32);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  KZ_CUDA_TRY(cudaLaunchKernelEx(&cfg, batch_group_kernel<32>, a));
  batch_timeout_kernel<<<(pl.count + 255) / 256, 256, 0, s>>>(pl.desc, pl.count, pl.ctl);
  KZ_CUDA_TRY(cudaGetLastError());
  return KZ_OK;
}

// Capture the batch's launches into a graph (once per plan).  If the capture
// is refused, the plan keeps no graph and the launches are enqueued directly.
static void capture_plan(BatchPlan &pl) {
  if (!pl.capture && cudaStreamCreateWithFlags(&pl.capture, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    pl.capture = nullptr;
    return;
  }
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(pl.capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const kz_status st = enqueue_batch(pl, pl.capture);
  const cudaError_t e = cudaStreamEndCapture(pl.capture, &graph);
  if (st == KZ_OK && e == cudaSuccess && graph) {
    if (cudaGraphInstantiate(&pl.exec, graph, 0) != cudaSuccess) pl.exec = nullptr;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
}

kz_status batch_kernelize(kz_graph *gs, int count, const kz_options &opt, cudaStream_t s) {
  if (count <= 0) return KZ_OK;
  for (int i = 0; i < count; i++)
    if (gs[i]->k > 32) return KZ_ERR_UNSUPPORTED;  // the caller routes k > 32 elsewhere
  std::vector<uint64_t> key;
  key.reserve((size_t)count + 1);
  for (int i = 0; i < count; i++) key.push_back(gs[i]->uid);
  key.push_back((uint64_t)opt.max_sweeps);
  int dev = 0;
  KZ_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_plan_mu);
  uint64_t spread_bits = 0;
  memcpy(&spread_bits, &g_tuning.group_spread, sizeof(spread_bits));
  key.push_back(spread_bits);
  key.push_back(((uint64_t)(uint32_t)g_tuning.items_per_warp << 32) | (uint32_t)g_tuning.max_group);
  if (g_plan.key != key || g_plan.device != dev) {
    // the plan must not be freed while an earlier launch may still read it
    if (g_plan.desc) KZ_CUDA_TRY(cudaDeviceSynchronize());
    plan_release(g_plan);
    auto fn = batch_group_kernel<32>;
    const size_t smem = (size_t)kBatchWarps * 2 * 32 * 32 * 4;
    KZ_CUDA_TRY(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    KZ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, kBatchWarps * 32, smem));
    const int grid = std::max(1, per_sm) * sm_count_here();
    std::vector<BatchItem> items;
    std::vector<BatchGraph> desc;
    std::vector<GroupEntry> entries;
    build_plan(gs, count, grid, items, desc, entries, opt, g_tuning);
    BatchPlan pl;
    pl.capture = g_plan.capture;
    pl.key = key;
    pl.device = dev;
    pl.count = count;
    pl.grid = std::max(1, std::min<int>(grid, (int)entries.size()));
    pl.smem = smem;
    pl.n_entries = (int32_t)entries.size();
    cudaError_t e = cudaMalloc(&pl.desc, sizeof(BatchGraph) * count);
    if (e == cudaSuccess) e = cudaMalloc(&pl.items, sizeof(BatchItem) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&pl.entries, sizeof(GroupEntry) * std::max<size_t>(entries.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&pl.ctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMemcpy(pl.desc, desc.data(), sizeof(BatchGraph) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !items.empty())
      e = cudaMemcpy(pl.items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !entries.empty())
      e = cudaMemcpy(pl.entries, entries.data(), sizeof(GroupEntry) * entries.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      plan_release(pl);
      g_plan.capture = pl.capture;
      return cuda_status(e);
    }
    capture_plan(pl);
    g_plan = pl;
  }
  if (g_plan.exec) {
    KZ_CUDA_TRY(cudaGraphLaunch(g_plan.exec, s));
    return KZ_OK;
  }
  return enqueue_batch(g_plan, s);
}

}  // namespace kz

extern "C" kz_status kz_set_batch_tuning(double group_spread, int32_t items_per_warp, int32_t max_group) {
  if (!(group_spread == group_spread)) return KZ_ERR_ARG;  // NaN
  std::lock_guard<std::mutex> lk(kz::g_plan_mu);
  kz::g_tuning.group_spread = group_spread > 0 ? group_spread : kz::kGroupSpread;
  kz::g_tuning.items_per_warp = items_per_warp > 0 ? items_per_warp : kz::kItemsPerWarp;
  kz::g_tuning.max_group = max_group > 0 ? max_group : kz::kMaxGroup;
  return KZ_OK;
}
