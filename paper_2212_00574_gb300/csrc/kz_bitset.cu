// kz_bitset.cu -- bitset path of the colour-index kernelization.
//
// Rules (thesis Section 4.2, the remarks after the colour index of a node and
// of an edge): a live vertex v is deleted when its live neighbours cover
// fewer than k-1 colour classes; a live edge {u,v} is deleted when the live
// common neighbours of u and v cover fewer than k-2 colour classes.  Both
// rules read the same snapshot (Jacobi sweep) and the sweep repeats until
// nothing is deleted.
//
// A fact the kernels rely on: if a vertex v fails the vertex rule because no
// neighbour has colour c, then every live edge {v,u} fails the edge rule in
// the same sweep, since no common neighbour of v and u can have colour c
// either (and c differs from col(u), u being a neighbour of v).  So deleting
// the failing edges already removes every edge of a failing vertex: the
// adjacency rows never need masking with the vertex live set.
//
// Sweep kernel design (one launch per pass, warp-granular work items):
//   * A warp owns a block X of 32 vertices u (lane = u) of class cu and holds
//     plane 0 of their rows (k words) in registers.
//   * It walks blocks Y of higher classes cv > cu.  For each Y it stages plane
//     0 of the 32 rows v in shared memory, and for every v tests all lanes'
//     pairs (u, v) at once: the pair is covered in class c when
//     row_u[c] & row_v[c] != 0.  The classes cu and cv are forced to "covered"
//     on both sides, so "every class covered" is one min-reduction over the
//     k word-ANDs.  A live edge whose plane-0 test fails is recounted exactly
//     over all planes (rare on dense graphs).
//   * Results go to the other ping-pong buffer: the warp writes row u's word
//     for block Y and (transposed with ballots) row v's word for block X.
//     Every (X, Y) pair with class(X) < class(Y) belongs to exactly one work
//     item, so every word of the next state is written exactly once.
//   * The last warp to finish (atomic ticket) records the pass counters,
//     flips the buffers when something was deleted and sets the CUDA-graph
//     while-condition.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kz_internal.cuh"
#include "kz_rules.cuh"
#include "kz_sweep.cuh"

namespace kz {

// ---------------------------------------------------------------------------
// layout (host)
// ---------------------------------------------------------------------------

kz_status bitset_build_layout(kz_graph g) {
  const int k = g->k;
  g->rounds.assign(k, 0);
  g->boff.assign(k + 1, 0);
  g->blocks.clear();
  int R = 0;
  for (int c = 0; c < k; c++) {
    const int sz = g->coff[c + 1] - g->coff[c];
    g->rounds[c] = (sz + 31) / 32;
    R = std::max(R, g->rounds[c]);
    g->boff[c + 1] = g->boff[c] + g->rounds[c];
    for (int r = 0; r < g->rounds[c]; r++) {
      BlockDesc b;
      b.c = c;
      b.r = r;
      b.base = g->coff[c] + 32 * r;
      b.size = std::min(32, sz - 32 * r);
      g->blocks.push_back(b);
    }
  }
  g->R = std::max(R, 1);
  const int64_t rk = (int64_t)g->R * k;
  const int64_t ldw = (rk + 3) / 4 * 4;
  if (ldw > (1 << 30)) return KZ_ERR_UNSUPPORTED;
  g->ldw = (int32_t)ldw;
  g->row_bytes = (size_t)ldw * 4;
  return KZ_OK;
}

// Work list: each block x against the blocks of higher classes, cut into
// pieces so that there are enough warps to fill the GPU.
static void build_items(kz_graph g, int target_items, std::vector<WorkItem> &items) {
  const int nb = (int)g->blocks.size();
  int64_t pairs = 0;
  for (int x = 0; x < nb; x++) pairs += nb - g->boff[g->blocks[x].c + 1];
  int64_t S = std::max<int64_t>(1, (pairs + target_items - 1) / std::max(1, target_items));
  items.clear();
  for (int x = 0; x < nb; x++) {
    const int y_begin = g->boff[g->blocks[x].c + 1];
    if (y_begin >= nb) {
      items.push_back({x, nb, nb, 1});
      continue;
    }
    bool first = true;
    for (int64_t y = y_begin; y < nb; y += S) {
      items.push_back({x, (int32_t)y, (int32_t)std::min<int64_t>(nb, y + S), first ? 1 : 0});
      first = false;
    }
  }
}

// ---------------------------------------------------------------------------
// packing kernels
// ---------------------------------------------------------------------------

struct PackArgs {
  uint32_t *A;
  int32_t ldw, k;
  const int32_t *inv;     // caller -> relabelled
  const int32_t *col;     // relabelled colour
  const int32_t *coff;    // k + 1
  unsigned long long *edge_count;
  int32_t *error;         // first error code seen (0 = none)
};

__global__ void pack_edges_kernel(PackArgs a, const int32_t *__restrict__ edges, int64_t m,
                                  int dedup) {
  unsigned long long mine = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t x = a.inv[edges[2 * e]], y = a.inv[edges[2 * e + 1]];
    if (x > y) {
      int32_t t = x;
      x = y;
      y = t;
    }
    const int32_t cx = a.col[x], cy = a.col[y];
    const int32_t ix = x - a.coff[cx], iy = y - a.coff[cy];
    const uint32_t bx = 1u << (ix & 31), by = 1u << (iy & 31);
    const int64_t wxy = (int64_t)x * a.ldw + (iy >> 5) * a.k + cy;
    const int64_t wyx = (int64_t)y * a.ldw + (ix >> 5) * a.k + cx;
    const uint32_t old = atomicOr(&a.A[wxy], by);
    if (old & by) {
      if (!dedup) atomicCAS(a.error, 0, (int32_t)KZ_ERR_DUPLICATE_EDGE);
      continue;
    }
    atomicOr(&a.A[wyx], bx);
    mine++;
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(a.edge_count, mine);
}

// Dense caller-id bit matrix: only bits j > i are read.
__global__ void pack_dense_kernel(PackArgs a, const uint64_t *__restrict__ bits, int64_t row_words,
                                  int32_t n, const int32_t *__restrict__ colour_caller) {
  unsigned long long mine = 0;
  const int64_t total = (int64_t)n * row_words;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = (int32_t)(t / row_words);
    const int64_t w = t - (int64_t)i * row_words;
    uint64_t word = bits[t];
    const int64_t j0 = w * 64;
    if (j0 + 63 <= i || j0 >= n) continue;
    // keep bits j with i < j < n
    if (j0 <= i) {
      const int sh = i - (int)j0 + 1;  // 1..64
      word = sh >= 64 ? 0 : (word >> sh) << sh;
    }
    if (j0 + 64 > n) {
      const int keep = n - (int)j0;  // 1..63
      word &= (keep >= 64) ? ~0ull : ((1ull << keep) - 1);
    }
    if (!word) continue;
    const int32_t ci = colour_caller[i];
    const int32_t x = a.inv[i];
    const int32_t ix = x - a.coff[ci];
    const uint32_t bx = 1u << (ix & 31);
    while (word) {
      const int b = __ffsll((long long)word) - 1;
      word &= word - 1;
      const int32_t j = (int32_t)j0 + b;
      const int32_t cj = colour_caller[j];
      if (cj == ci) {
        atomicCAS(a.error, 0, (int32_t)KZ_ERR_ILLEGAL_COLOURING);
        continue;
      }
      const int32_t y = a.inv[j];
      const int32_t iy = y - a.coff[cj];
      atomicOr(&a.A[(int64_t)x * a.ldw + (iy >> 5) * a.k + cj], 1u << (iy & 31));
      atomicOr(&a.A[(int64_t)y * a.ldw + (ix >> 5) * a.k + ci], bx);
      mine++;
    }
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(a.edge_count, mine);
}

__global__ void init_vlive_kernel(uint32_t *V, const BlockDesc *blocks, int nb, int k) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
    const BlockDesc d = blocks[b];
    V[d.r * k + d.c] = d.size >= 32 ? 0xffffffffu : ((1u << d.size) - 1u);
  }
}

// ---------------------------------------------------------------------------
// sweep kernel
// ---------------------------------------------------------------------------

struct SweepArgs {
  const BlockDesc *blocks;
  const WorkItem *items;
  int32_t n_items;
  int32_t k, ldw;
  const int32_t *rounds;  // blocks per class
  uint32_t *A0, *A1;      // ping-pong adjacency
  uint32_t *V0, *V1;      // ping-pong vertex live words
  int32_t *v_sweep;       // relabelled ids, may be null
  DevState *st;
  cudaGraphConditionalHandle cond;
  int32_t use_cond;
  uint32_t bar_extra;    // arrivals the grid barrier waits for beyond the grid (0; tests use 1)
  uint32_t spin_limit;   // polls before a barrier wait gives up
};

constexpr int kSweepWarps = 4;

template <int KMAX>
__device__ __forceinline__ void sweep_items(const SweepArgs &p, int cur, int64_t sweep_no, uint32_t *buf0,
                                            uint32_t *buf1, int first_item, int item_stride, PassCounters &pc) {
  GraphView G;
  G.blocks = p.blocks;
  G.rounds = p.rounds;
  G.A0 = p.A0;
  G.A1 = p.A1;
  G.V0 = p.V0;
  G.V1 = p.V1;
  G.v_sweep = p.v_sweep;
  G.k = p.k;
  G.ldw = p.ldw;
  for (int it = first_item; it < p.n_items; it += item_stride)
    sweep_item<KMAX>(G, p.items[it], cur, sweep_no, buf0, buf1, pc);
}

template <int KMAX>
__device__ __forceinline__ void reduce_counters(PassCounters &pc) {
  for (int o = 16; o > 0; o >>= 1) {
    pc.tests += __shfl_down_sync(0xffffffffu, pc.tests, o);
    pc.de += __shfl_down_sync(0xffffffffu, pc.de, o);
    pc.dv += __shfl_down_sync(0xffffffffu, pc.dv, o);
  }
}

// One Jacobi pass per launch (the CUDA-graph loop and the host-driven loop).
template <int KMAX>
__global__ void __launch_bounds__(kSweepWarps * 32)
    bitset_sweep_kernel(SweepArgs p) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint32_t *buf0 = smem + wib * 2 * 32 * KMAX;
  uint32_t *buf1 = buf0 + 32 * KMAX;
  DevState *st = p.st;
  const int cur = *((volatile int32_t *)&st->cur);
  const int64_t sweep_no = *((volatile int64_t *)&st->sweeps);
  const int warps_total = gridDim.x * kSweepWarps;
  PassCounters pc;
  sweep_items<KMAX>(p, cur, sweep_no, buf0, buf1, blockIdx.x * kSweepWarps + wib, warps_total, pc);
  reduce_counters<KMAX>(pc);
  if (lane == 0) {
    if (pc.tests) atomicAdd(&st->pass_tests, pc.tests);
    if (pc.de) atomicAdd(&st->pass_de, pc.de);
    if (pc.dv) atomicAdd(&st->pass_dv, pc.dv);
    __threadfence();
    const unsigned int t = atomicAdd(&st->ticket, 1u);
    if (t == (unsigned int)warps_total - 1u) {
      __threadfence();
      const unsigned long long dv = atomicAdd(&st->pass_dv, 0ull);
      const unsigned long long de = atomicAdd(&st->pass_de, 0ull);
      const unsigned long long tests = atomicAdd(&st->pass_tests, 0ull);
      const int cont = finish_pass(st, dv, de, tests);
      st->pass_dv = 0;
      st->pass_de = 0;
      st->pass_tests = 0;
      st->ticket = 0;
      __threadfence();
      if (p.use_cond) cudaGraphSetConditional(p.cond, cont ? 1u : 0u);
    }
  }
}

constexpr uint32_t kBarrierSpinLimit = 1u << 25;

// Every pass of the fixpoint in one cooperative launch (all CTAs resident):
// after its share of a pass each CTA arrives at a grid barrier; the last one
// closes the pass (counters, buffer flip) and releases the others.  Every
// barrier wait is bounded: one that runs out records KZ_ERR_TIMEOUT and all
// CTAs leave.
template <int KMAX>
__global__ void __launch_bounds__(kSweepWarps * 32)
    bitset_persistent_kernel(SweepArgs p) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_go;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  uint32_t *buf0 = smem + wib * 2 * 32 * KMAX;
  uint32_t *buf1 = buf0 + 32 * KMAX;
  DevState *st = p.st;
  const int warps_total = gridDim.x * kSweepWarps;
  for (;;) {
    const int cur = *((volatile int32_t *)&st->cur);
    const int64_t sweep_no = *((volatile int64_t *)&st->sweeps);
    PassCounters pc;
    sweep_items<KMAX>(p, cur, sweep_no, buf0, buf1, blockIdx.x * kSweepWarps + wib, warps_total, pc);
    reduce_counters<KMAX>(pc);
    if (lane == 0) {
      if (pc.tests) atomicAdd(&st->pass_tests, pc.tests);
      if (pc.de) atomicAdd(&st->pass_de, pc.de);
      if (pc.dv) atomicAdd(&st->pass_dv, pc.dv);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned int gen = *((volatile unsigned int *)&st->bar_gen);
      if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1u + p.bar_extra) {
        __threadfence();
        const unsigned long long dv = atomicAdd(&st->pass_dv, 0ull);
        const unsigned long long de = atomicAdd(&st->pass_de, 0ull);
        const unsigned long long tests = atomicAdd(&st->pass_tests, 0ull);
        finish_pass(st, dv, de, tests);
        st->pass_dv = 0;
        st->pass_de = 0;
        st->pass_tests = 0;
        st->bar_count = 0;
        __threadfence();
        atomicExch(&st->bar_gen, gen + 1u);
      } else {
        uint32_t spins = 0;
        while (*((volatile unsigned int *)&st->bar_gen) == gen) {
          if (*((volatile int32_t *)&st->bar_abort)) break;
          __nanosleep(64);
          if (++spins > p.spin_limit) {
            atomicCAS(&st->status, (int32_t)KZ_OK, (int32_t)KZ_ERR_TIMEOUT);
            atomicExch(&st->bar_abort, 1);
            break;
          }
        }
      }
      __threadfence();
      s_go = *((volatile int32_t *)&st->cont) && !*((volatile int32_t *)&st->bar_abort);
    }
    __syncthreads();
    if (!s_go) break;
  }
}

__global__ void begin_run_kernel(DevState *st, int64_t max_sweeps, int64_t passes0) {
  st->bar_count = 0;
  st->bar_gen = 0;
  st->bar_abort = 0;
  st->status = KZ_OK;
  st->cont = 1;
  st->sweeps = 0;
  st->passes = passes0;
  st->tests = 0;
  st->max_sweeps = max_sweeps;
  st->pass_dv = st->pass_de = st->pass_tests = 0;
  st->ticket = 0;
}

__global__ void reset_state_kernel(DevState *st) {
  st->cur = 0;
  st->status = KZ_OK;
  st->cont = 0;
  st->sweeps = st->passes = st->tests = 0;
  st->pass_dv = st->pass_de = st->pass_tests = 0;
  st->ticket = 0;
}

// ---------------------------------------------------------------------------
// kernel selection
// ---------------------------------------------------------------------------

typedef void (*SweepFn)(SweepArgs);

static SweepFn pick_sweep(int k, int &kmax) {
#define KZ_CASE(K)                        \
  if (k <= K) {                           \
    kmax = K;                             \
    return bitset_sweep_kernel<K>;        \
  }
  KZ_CASE(4)
  KZ_CASE(8)
  KZ_CASE(12)
  KZ_CASE(16)
  KZ_CASE(20)
  KZ_CASE(24)
  KZ_CASE(28)
  KZ_CASE(32)
  KZ_CASE(48)
  KZ_CASE(64)
#undef KZ_CASE
  kmax = 0;
  return nullptr;
}

static SweepFn pick_persistent(int k, int &kmax) {
#define KZ_CASE(K)                           \
  if (k <= K) {                              \
    kmax = K;                                \
    return bitset_persistent_kernel<K>;      \
  }
  KZ_CASE(4)
  KZ_CASE(8)
  KZ_CASE(12)
  KZ_CASE(16)
  KZ_CASE(20)
  KZ_CASE(24)
  KZ_CASE(28)
  KZ_CASE(32)
  KZ_CASE(48)
  KZ_CASE(64)
#undef KZ_CASE
  kmax = 0;
  return nullptr;
}

// ---------------------------------------------------------------------------
// host entry points of the path
// ---------------------------------------------------------------------------

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

kz_status bitset_finish_load(kz_graph g, cudaStream_t s) {
  const int nb = (int)g->blocks.size();
  KZ_TRY(graph_alloc(g, &g->V0, (size_t)g->ldw, s));
  KZ_TRY(graph_alloc(g, &g->V[0], (size_t)g->ldw, s));
  KZ_TRY(graph_alloc(g, &g->V[1], (size_t)g->ldw, s));
  KZ_CUDA_TRY(cudaMemsetAsync(g->V0, 0, (size_t)g->ldw * 4, s));
  KZ_TRY(graph_alloc(g, &g->d_blocks, (size_t)std::max(nb, 1), s));
  if (nb) {
    KZ_CUDA_TRY(cudaMemcpyAsync(g->d_blocks, g->blocks.data(), sizeof(BlockDesc) * nb,
                                cudaMemcpyHostToDevice, s));
    init_vlive_kernel<<<(nb + 255) / 256, 256, 0, s>>>(g->V0, g->d_blocks, nb, g->k);
    KZ_CUDA_TRY(cudaGetLastError());
  }
  KZ_TRY(graph_alloc(g, &g->d_coff, (size_t)g->k + 1, s));
  KZ_CUDA_TRY(cudaMemcpyAsync(g->d_coff, g->coff.data(), sizeof(int32_t) * (g->k + 1),
                              cudaMemcpyHostToDevice, s));
  KZ_TRY(graph_alloc(g, &g->d_rounds, (size_t)g->k, s));
  KZ_CUDA_TRY(cudaMemcpyAsync(g->d_rounds, g->rounds.data(), sizeof(int32_t) * g->k,
                              cudaMemcpyHostToDevice, s));
  // work items: aim for ~16 warps per SM scheduler
  std::vector<WorkItem> items;
  build_items(g, 16 * 4 * sm_count(), items);
  g->n_items = (int32_t)items.size();
  KZ_TRY(graph_alloc(g, &g->d_items, std::max<size_t>(items.size(), 1), s));
  if (!items.empty())
    KZ_CUDA_TRY(cudaMemcpyAsync(g->d_items, items.data(), sizeof(WorkItem) * items.size(),
                                cudaMemcpyHostToDevice, s));
  KZ_TRY(graph_alloc(g, &g->A[0], (size_t)g->n * g->ldw, s));
  KZ_TRY(graph_alloc(g, &g->A[1], (size_t)g->n * g->ldw, s));
  KZ_TRY(graph_alloc(g, &g->v_sweep, (size_t)std::max(g->n, 1), s));
  if (!g->st) {
    KZ_TRY(graph_alloc(g, &g->st, 1, s));
    KZ_CUDA_TRY(cudaMemsetAsync(g->st, 0, sizeof(DevState), s));
  }
  KZ_TRY(cta_prepare(g, s));
  KZ_TRY(cta_upload_descriptor(g, s));
  return bitset_reset(g, s);
}

kz_status bitset_reset(kz_graph g, cudaStream_t s) {
  const size_t abytes = (size_t)g->n * g->ldw * 4;
  if (abytes) {
    KZ_CUDA_TRY(cudaMemcpyAsync(g->A[0], g->A0, abytes, cudaMemcpyDeviceToDevice, s));
    KZ_CUDA_TRY(cudaMemcpyAsync(g->A[1], g->A0, abytes, cudaMemcpyDeviceToDevice, s));
  }
  KZ_CUDA_TRY(cudaMemcpyAsync(g->V[0], g->V0, (size_t)g->ldw * 4, cudaMemcpyDeviceToDevice, s));
  KZ_CUDA_TRY(cudaMemcpyAsync(g->V[1], g->V0, (size_t)g->ldw * 4, cudaMemcpyDeviceToDevice, s));
  if (g->n) KZ_CUDA_TRY(cudaMemsetAsync(g->v_sweep, 0, sizeof(int32_t) * g->n, s));
  reset_state_kernel<<<1, 1, 0, s>>>(g->st);
  KZ_CUDA_TRY(cudaGetLastError());
  g->kernelized = false;
  return KZ_OK;
}

static kz_status launch_config(kz_graph g, SweepFn fn, int kmax, int &grid, size_t &smem) {
  smem = (size_t)kSweepWarps * 2 * 32 * kmax * 4;
  // always raise the limit: the kernels' static shared memory comes on top
  KZ_CUDA_TRY(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  KZ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn,
                                                            kSweepWarps * 32, smem));
  per_sm = std::max(per_sm, 1);
  const int want = (g->n_items + kSweepWarps - 1) / kSweepWarps;
  grid = std::max(1, std::min(want, per_sm * sm_count()));
  return KZ_OK;
}

static SweepArgs make_args(kz_graph g) {
  SweepArgs a;
  a.blocks = g->d_blocks;
  a.items = g->d_items;
  a.n_items = g->n_items;
  a.k = g->k;
  a.ldw = g->ldw;
  a.rounds = g->d_rounds;
  a.A0 = g->A[0];
  a.A1 = g->A[1];
  a.V0 = g->V[0];
  a.V1 = g->V[1];
  a.v_sweep = g->v_sweep;
  a.st = g->st;
  a.cond = 0;
  a.use_cond = 0;
  a.bar_extra = 0;
  a.spin_limit = kBarrierSpinLimit;
  return a;
}

// Builds (once per graph) an executable CUDA graph whose while-node runs one
// sweep-kernel launch per pass until the kernel clears the condition.
static kz_status build_loop_graph(kz_graph g, int64_t max_sweeps) {
  int kmax = 0;
  SweepFn fn = pick_sweep(g->k, kmax);
  if (!fn) return KZ_ERR_ARG;
  int grid = 0;
  size_t smem = 0;
  KZ_TRY(launch_config(g, fn, kmax, grid, smem));
  cudaGraph_t graph = nullptr;
  KZ_CUDA_TRY(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle;
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_status(e);
  }
  // the params struct holds a union with deleted default constructors
  alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
  memset(cp_raw, 0, sizeof(cp_raw));
  cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  // run-start kernel, then the while node
  cudaGraphNode_t bnode;
  {
    DevState *stp = g->st;
    int64_t ms = max_sweeps, p0 = 0;
    void *bargs[] = {&stp, &ms, &p0};
    cudaKernelNodeParams bp;
    memset((void *)&bp, 0, sizeof(bp));
    bp.func = (void *)begin_run_kernel;
    bp.gridDim = dim3(1);
    bp.blockDim = dim3(1);
    bp.kernelParams = bargs;
    e = cudaGraphAddKernelNode(&bnode, graph, nullptr, 0, &bp);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return cuda_status(e);
    }
  }
  cudaGraphNode_t wnode;
  e = cudaGraphAddNode(&wnode, graph, &bnode, nullptr, 1, &cp);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_status(e);
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  SweepArgs args = make_args(g);
  args.cond = handle;
  args.use_cond = 1;
  void *kargs[] = {&args};
  cudaKernelNodeParams kp;
  memset((void *)&kp, 0, sizeof(kp));
  kp.func = (void *)fn;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(kSweepWarps * 32);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = kargs;
  cudaGraphNode_t knode;
  e = cudaGraphAddKernelNode(&knode, body, nullptr, 0, &kp);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return cuda_status(e);
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_status(e);
  g->loop_exec = exec;
  g->loop_grid = grid;
  g->loop_max_sweeps = max_sweeps;
  return KZ_OK;
}

kz_status bitset_kernelize(kz_graph g, const kz_options &opt, cudaStream_t s) {
  int64_t max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : (int64_t)g->n + g->m + 1;
  if (g->n > 0 && opt.use_graph == 1) {
    // every pass in one cooperative launch (grid sized to be fully resident)
    begin_run_kernel<<<1, 1, 0, s>>>(g->st, max_sweeps, 0);
    KZ_CUDA_TRY(cudaGetLastError());
    int kmax = 0;
    SweepFn fn = pick_persistent(g->k, kmax);
    if (!fn) return KZ_ERR_ARG;
    int grid = 0;
    size_t smem = 0;
    KZ_TRY(launch_config(g, fn, kmax, grid, smem));
    SweepArgs args = make_args(g);
    void *kargs[] = {&args};
    KZ_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(kSweepWarps * 32), kargs, smem, s));
    return KZ_OK;
  }
  if (g->n > 0 && opt.use_graph == 2) {
    // one graph launch: run-start kernel, then the while node of sweep passes
    if (g->loop_exec && g->loop_max_sweeps != max_sweeps) {
      cudaGraphExecDestroy(g->loop_exec);
      g->loop_exec = nullptr;
    }
    if (!g->loop_exec) KZ_TRY(build_loop_graph(g, max_sweeps));
    KZ_CUDA_TRY(cudaGraphLaunch(g->loop_exec, s));
    return KZ_OK;
  }
  begin_run_kernel<<<1, 1, 0, s>>>(g->st, max_sweeps, g->n == 0 ? 1 : 0);
  KZ_CUDA_TRY(cudaGetLastError());
  if (g->n == 0) {
    // nothing to test: one empty pass
    return KZ_OK;
  }
  // host-driven loop: one launch per pass, the host reads the continue flag
  int kmax = 0;
  SweepFn fn = pick_sweep(g->k, kmax);
  if (!fn) return KZ_ERR_ARG;
  int grid = 0;
  size_t smem = 0;
  KZ_TRY(launch_config(g, fn, kmax, grid, smem));
  SweepArgs args = make_args(g);
  for (;;) {
    fn<<<grid, kSweepWarps * 32, smem, s>>>(args);
    KZ_CUDA_TRY(cudaGetLastError());
    int32_t cont = 0;
    KZ_CUDA_TRY(cudaMemcpyAsync(&cont, &g->st->cont, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (!cont) break;
  }
  return KZ_OK;
}

kz_status bitset_begin_run(kz_graph g, int64_t max_sweeps, cudaStream_t s) {
  begin_run_kernel<<<1, 1, 0, s>>>(g->st, max_sweeps, g->n == 0 ? 1 : 0);
  return cuda_status(cudaGetLastError());
}

kz_status bitset_one_pass(kz_graph g, cudaStream_t s, int *cont) {
  *cont = 0;
  if (g->n == 0) return KZ_OK;
  int kmax = 0;
  SweepFn fn = pick_sweep(g->k, kmax);
  if (!fn) return KZ_ERR_ARG;
  int grid = 0;
  size_t smem = 0;
  KZ_TRY(launch_config(g, fn, kmax, grid, smem));
  SweepArgs args = make_args(g);
  fn<<<grid, kSweepWarps * 32, smem, s>>>(args);
  KZ_CUDA_TRY(cudaGetLastError());
  int32_t c = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&c, &g->st->cont, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  *cont = c;
  return KZ_OK;
}

// Runs the persistent sweep kernel with a grid barrier that waits for one
// arrival more than the grid has, so every bounded wait runs out: the kernel
// must record KZ_ERR_TIMEOUT and return.  For tests of the failure path.
kz_status bitset_barrier_timeout_probe(kz_graph g, uint32_t spin_limit, cudaStream_t s) {
  if (g->n == 0) return KZ_ERR_ARG;
  begin_run_kernel<<<1, 1, 0, s>>>(g->st, (int64_t)g->n + g->m + 1, 0);
  KZ_CUDA_TRY(cudaGetLastError());
  int kmax = 0;
  SweepFn fn = pick_persistent(g->k, kmax);
  if (!fn) return KZ_ERR_ARG;
  int grid = 0;
  size_t smem = 0;
  KZ_TRY(launch_config(g, fn, kmax, grid, smem));
  SweepArgs args = make_args(g);
  args.bar_extra = 1;
  args.spin_limit = spin_limit;
  void *kargs[] = {&args};
  KZ_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(kSweepWarps * 32), kargs, smem, s));
  return KZ_OK;
}

// ---------------------------------------------------------------------------
// unpacking to caller ids
// ---------------------------------------------------------------------------

__global__ void unpack_dense_kernel(const uint32_t *__restrict__ A, int32_t n, int32_t ldw, int32_t k,
                                    int32_t rk, const int32_t *__restrict__ coff,
                                    const int32_t *__restrict__ perm, uint64_t *out,
                                    int64_t row_words, unsigned long long *edge_count) {
  unsigned long long mine = 0;
  const int64_t total = (int64_t)n * rk;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = (int32_t)(t / rk);
    const int32_t w = (int32_t)(t - (int64_t)x * rk);
    uint32_t word = A[(int64_t)x * ldw + w];
    if (!word) continue;
    const int32_t c = w % k, r = w / k;
    const int32_t ox = perm[x];
    mine += __popc(word);
    while (word) {
      const int b = __ffs(word) - 1;
      word &= word - 1;
      const int32_t y = coff[c] + 32 * r + b;
      const int32_t oy = perm[y];
      atomicOr(reinterpret_cast<unsigned long long *>(&out[(int64_t)ox * row_words + (oy >> 6)]),
               1ull << (oy & 63));
    }
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(edge_count, mine);
}

kz_status bitset_unpack_dense(kz_graph g, uint64_t *d_out, int64_t row_words,
                              unsigned long long *d_edge_count, cudaStream_t s) {
  KZ_CUDA_TRY(cudaMemsetAsync(d_out, 0, (size_t)g->n * row_words * 8, s));
  KZ_CUDA_TRY(cudaMemsetAsync(d_edge_count, 0, sizeof(unsigned long long), s));
  if (g->n == 0) return KZ_OK;
  // the current buffer index lives on the device; read it (the stream is
  // synchronous with the caller here)
  int32_t cur = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&cur, &g->st->cur, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  const int32_t rk = g->R * g->k;
  const int64_t total = (int64_t)g->n * rk;
  const int threads = 256;
  const int grid = (int)std::min<int64_t>((total + threads - 1) / threads, 32 * sm_count());
  unpack_dense_kernel<<<std::max(grid, 1), threads, 0, s>>>(g->A[cur & 1], g->n, g->ldw, g->k, rk,
                                                           g->d_coff, g->d_perm, d_out, row_words,
                                                           d_edge_count);
  KZ_CUDA_TRY(cudaGetLastError());
  return KZ_OK;
}

kz_status bitset_vertex_alive(kz_graph g, uint8_t *host_alive, int64_t *n_live) {
  int32_t cur = 0;
  KZ_CUDA_TRY(cudaMemcpy(&cur, &g->st->cur, sizeof(int32_t), cudaMemcpyDeviceToHost));
  std::vector<uint32_t> V((size_t)g->ldw);
  KZ_CUDA_TRY(cudaMemcpy(V.data(), g->V[cur & 1], (size_t)g->ldw * 4, cudaMemcpyDeviceToHost));
  int64_t live = 0;
  for (int32_t x = 0; x < g->n; x++) {
    // class of x: coff is sorted
    const int c = (int)(std::upper_bound(g->coff.begin(), g->coff.end(), x) - g->coff.begin()) - 1;
    const int i = x - g->coff[c];
    const bool a = (V[(size_t)(i >> 5) * g->k + c] >> (i & 31)) & 1u;
    live += a;
    if (host_alive) host_alive[g->perm[x]] = a ? 1 : 0;
  }
  if (n_live) *n_live = live;
  return KZ_OK;
}

// Shared set-up of the two packers: relabelling tables on the device and the
// zeroed pristine adjacency.  Returns the temporaries to free after the sync.
static kz_status pack_setup(kz_graph g, cudaStream_t s, PackArgs &a, std::vector<void *> &tmp) {
  KZ_TRY(graph_alloc(g, &g->A0, (size_t)g->n * g->ldw, s));
  if (g->n > 0 && g->ldw > 0)
    KZ_CUDA_TRY(cudaMemsetAsync(g->A0, 0, (size_t)g->n * g->ldw * 4, s));
  std::vector<int32_t> col_new((size_t)g->n);
  for (int c = 0; c < g->k; c++)
    for (int x = g->coff[c]; x < g->coff[c + 1]; x++) col_new[x] = c;
  int32_t *d_inv = nullptr, *d_col = nullptr, *d_coff = nullptr, *d_err = nullptr;
  unsigned long long *d_cnt = nullptr;
  const size_t nn = (size_t)std::max(g->n, 1);
  d_inv = (int32_t *)dev_alloc(nn * 4, s);
  d_col = (int32_t *)dev_alloc(nn * 4, s);
  d_coff = (int32_t *)dev_alloc(((size_t)g->k + 1) * 4, s);
  d_err = (int32_t *)dev_alloc(16, s);
  d_cnt = (unsigned long long *)dev_alloc(16, s);
  tmp = {d_inv, d_col, d_coff, d_err, d_cnt};
  for (void *q : tmp)
    if (!q) return KZ_ERR_OOM;
  if (g->n) {
    KZ_CUDA_TRY(cudaMemcpyAsync(d_inv, g->inv.data(), (size_t)g->n * 4, cudaMemcpyHostToDevice, s));
    KZ_CUDA_TRY(cudaMemcpyAsync(d_col, col_new.data(), (size_t)g->n * 4, cudaMemcpyHostToDevice, s));
  }
  KZ_CUDA_TRY(cudaMemcpyAsync(d_coff, g->coff.data(), ((size_t)g->k + 1) * 4, cudaMemcpyHostToDevice, s));
  KZ_CUDA_TRY(cudaMemsetAsync(d_err, 0, 16, s));
  KZ_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 16, s));
  a.A = g->A0;
  a.ldw = g->ldw;
  a.k = g->k;
  a.inv = d_inv;
  a.col = d_col;
  a.coff = d_coff;
  a.edge_count = d_cnt;
  a.error = d_err;
  return KZ_OK;
}

static kz_status pack_finish(kz_graph g, cudaStream_t s, PackArgs &a, std::vector<void *> &tmp) {
  int32_t err = 0;
  unsigned long long cnt = 0;
  cudaError_t e1 = cudaMemcpyAsync(&err, a.error, 4, cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaMemcpyAsync(&cnt, a.edge_count, 8, cudaMemcpyDeviceToHost, s);
  cudaError_t e3 = cudaStreamSynchronize(s);
  for (void *q : tmp)
    if (q) dev_free(q, 0, s);
  tmp.clear();
  if (e1 != cudaSuccess) return cuda_status(e1);
  if (e2 != cudaSuccess) return cuda_status(e2);
  if (e3 != cudaSuccess) return cuda_status(e3);
  if (err) return (kz_status)err;
  g->m = (int64_t)cnt;
  return KZ_OK;
}

kz_status bitset_pack_edges(kz_graph g, const int32_t *d_edges, int64_t m, bool dedup,
                            cudaStream_t s) {
  PackArgs a;
  std::vector<void *> tmp;
  kz_status st = pack_setup(g, s, a, tmp);
  if (st == KZ_OK && m > 0) {
    const int threads = 256;
    const int grid = (int)std::min<int64_t>((m + threads - 1) / threads, 64 * sm_count());
    pack_edges_kernel<<<grid, threads, 0, s>>>(a, d_edges, m, dedup ? 1 : 0);
    st = cuda_status(cudaGetLastError());
  }
  kz_status st2 = tmp.empty() ? KZ_OK : pack_finish(g, s, a, tmp);
  return st != KZ_OK ? st : st2;
}

kz_status bitset_pack_dense(kz_graph g, const uint64_t *d_bits, int64_t row_words,
                            const int32_t *d_colour_caller, cudaStream_t s) {
  PackArgs a;
  std::vector<void *> tmp;
  kz_status st = pack_setup(g, s, a, tmp);
  const int64_t total = (int64_t)g->n * row_words;
  if (st == KZ_OK && total > 0) {
    const int threads = 256;
    const int grid = (int)std::min<int64_t>((total + threads - 1) / threads, 64 * sm_count());
    pack_dense_kernel<<<grid, threads, 0, s>>>(a, d_bits, row_words, g->n, d_colour_caller);
    st = cuda_status(cudaGetLastError());
  }
  kz_status st2 = tmp.empty() ? KZ_OK : pack_finish(g, s, a, tmp);
  return st != KZ_OK ? st : st2;
}

}  // namespace kz
