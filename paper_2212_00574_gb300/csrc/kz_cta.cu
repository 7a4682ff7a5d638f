// kz_cta.cu -- whole-fixpoint-in-one-CTA kernel: the small-graph path and
// the batched persistent launch.
//
// One CTA runs every Jacobi pass of one graph (thesis Section 4.2 rules, see
// kz_rules.cuh) with __syncthreads() between passes, so no pass needs a new
// launch and no CTA ever waits on another.  A persistent grid (one CTA per
// SM) pulls graphs from an atomic queue in longest-first order.  A graph
// whose two ping-pong copies fit in shared memory is copied in once and
// swept there ("shared" mode); a larger one is swept in place in its global
// ping-pong buffers ("global" mode, L2-resident for the sizes of a batch).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "kz_internal.cuh"
#include "kz_rules.cuh"

namespace kz {

constexpr int kCtaThreads = 512;
constexpr int kCtaWarps = kCtaThreads / 32;

struct CtaArgs {
  const CtaGraph *graphs;
  const int32_t *order;   // queue order (longest first)
  int32_t count;
  unsigned int *queue;    // next queue slot; null: CTA b takes order[b] only
  int32_t smem_words;     // dynamic shared memory available, in words
  int32_t slack;          // colours minus the clique size sought, every graph (0: the thesis's rules)
  int64_t max_sweeps;     // option value; <= 0 means n + m + 1 per graph
};

// First pair index of the warp's share, then the block X holding it.
__device__ __forceinline__ int find_x(const int32_t *__restrict__ pair_off, int nb, int64_t p) {
  int lo = 0, hi = nb;  // pair_off[lo] <= p < pair_off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pair_off[mid] <= p) lo = mid;
    else hi = mid;
  }
  return lo;
}

// The running record of one graph's fixpoint, kept in shared memory while
// its CTA works on it and written to the graph's DevState at the end.
struct CtaRun {
  int64_t sweeps, passes, tests, max_sweeps;
  int32_t cur, status;
};

template <int KMAX, bool SHARED>
__device__ void cta_fixpoint(const CtaGraph &G, int64_t max_sweeps, int slack, uint32_t *smem, unsigned long long *s_cnt,
                             int *s_flag, int32_t *s_rounds, CtaRun *run) {
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int k = G.k, ldw = G.ldw, nb = G.nb;
  DevState *st = G.st;
  int cur = st->cur;
  const size_t words = (size_t)G.n * ldw;

  uint32_t *Ac, *An, *Vc, *Vn;
  if (SHARED) {
    Ac = smem;
    An = smem + words;
    Vc = An + words;
    Vn = Vc + ldw;
    const uint32_t *src = cur ? G.A1 : G.A0;
    const uint32_t *vsrc = cur ? G.V1 : G.V0;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *a4 = reinterpret_cast<uint4 *>(Ac);
    uint4 *n4 = reinterpret_cast<uint4 *>(An);
    for (size_t i = tid; i < words / 4; i += kCtaThreads) {
      const uint4 w = s4[i];
      a4[i] = w;
      n4[i] = w;
    }
    for (int i = tid; i < ldw; i += kCtaThreads) {
      Vc[i] = vsrc[i];
      Vn[i] = vsrc[i];
    }
  } else {
    Ac = cur ? G.A1 : G.A0;
    An = cur ? G.A0 : G.A1;
    Vc = cur ? G.V1 : G.V0;
    Vn = cur ? G.V0 : G.V1;
  }
  for (int c = tid; c < k; c += kCtaThreads) s_rounds[c] = G.rounds[c];
  if (tid == 0) {
    run->sweeps = 0;
    run->passes = G.n == 0 ? 1 : 0;
    run->tests = 0;
    run->max_sweeps = max_sweeps > 0 ? max_sweeps : (int64_t)G.n + G.m + 1;
    run->cur = cur;
    run->status = KZ_OK;
    s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
  }
  __syncthreads();

  const int64_t npairs = G.pair_off[nb];
  const int64_t share = (npairs + kCtaWarps - 1) / kCtaWarps;
  for (; G.n > 0;) {
    const int64_t sweep_no = run->sweeps;
    unsigned long long my_tests = 0, my_de = 0, my_dv = 0;
    // vertex rule, one warp per block
    for (int x = warp; x < nb; x += kCtaWarps) {
      const BlockDesc X = G.blocks[x];
      const bool valid_u = lane < X.size;
      const int u = X.base + lane;
      const uint32_t *rowu = Ac + (size_t)(valid_u ? u : X.base) * ldw;
      uint32_t Fu[KMAX];
      load_plane0<KMAX>(Fu, rowu, k, valid_u);
      const int wx = X.r * k + X.c;
      const uint32_t vword = Vc[wx];
      const bool live = valid_u && ((vword >> lane) & 1u);
      const uint64_t miss0 = plane0_vertex_missing<KMAX>(Fu, k, X.c);
      int cnt = (k - 1) - __popcll(miss0);
      if (live && cnt < k - 1 - slack) cnt += vertex_cover_beyond_plane0(rowu, k, s_rounds, miss0);
      const bool fail = live && cnt < k - 1 - slack;
      const uint32_t failmask = __ballot_sync(0xffffffffu, fail);
      if (lane == 0) {
        Vn[wx] = vword & ~failmask;
        my_dv += __popc(failmask);
      }
      if (fail && G.v_sweep) G.v_sweep[u] = (int32_t)(sweep_no + 1);
    }
    // edge rule over the warp's contiguous share of block pairs
    const int64_t p0 = (int64_t)warp * share;
    const int64_t p1 = min(npairs, p0 + share);
    if (p0 < p1) {
      int x = find_x(G.pair_off, nb, p0);
      BlockDesc X = G.blocks[x];
      int ybeg = G.boff[X.c + 1];
      bool valid_u = lane < X.size;
      int u = X.base + lane;
      const uint32_t *rowu = Ac + (size_t)(valid_u ? u : X.base) * ldw;
      uint32_t Fu[KMAX], P[KMAX];
      load_plane0<KMAX>(Fu, rowu, k, valid_u);
      int prev_cv = -1;
      for (int64_t p = p0; p < p1; p++) {
        while (p >= G.pair_off[x + 1]) {
          x++;
          X = G.blocks[x];
          ybeg = G.boff[X.c + 1];
          valid_u = lane < X.size;
          u = X.base + lane;
          rowu = Ac + (size_t)(valid_u ? u : X.base) * ldw;
          load_plane0<KMAX>(Fu, rowu, k, valid_u);
          prev_cv = -1;
        }
        const BlockDesc Y = G.blocks[ybeg + (int)(p - G.pair_off[x])];
        if (Y.c != prev_cv) {
          pair_mask<KMAX>(P, k, X.c, Y.c);
          prev_cv = Y.c;
        }
        const int wy = Y.r * k + Y.c;
        const uint32_t adjw = valid_u ? rowu[wy] : 0u;
        my_tests += __popc(adjw);
        const uint32_t *Ybase = Ac + (size_t)Y.base * ldw;
        const uint32_t del = edge_rule_block<KMAX>(
            Fu, P, rowu, adjw, k, slack, s_rounds, X.c, Y.c,
            [&](int b) { return Ybase + (size_t)b * ldw; },
            [&](int b) { return Ybase + (size_t)b * ldw; });
        if (valid_u) An[(size_t)u * ldw + wy] = adjw & ~del;
        my_de += __popc(del);
        const uint32_t delT = transpose_deletions(del);
        if (lane < Y.size) {
          const size_t wi = (size_t)(Y.base + lane) * ldw + X.r * k + X.c;
          An[wi] = Ac[wi] & ~delT;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      my_tests += __shfl_down_sync(0xffffffffu, my_tests, o);
      my_de += __shfl_down_sync(0xffffffffu, my_de, o);
      my_dv += __shfl_down_sync(0xffffffffu, my_dv, o);
    }
    if (lane == 0) {
      if (my_tests) atomicAdd(&s_cnt[0], my_tests);
      if (my_de) atomicAdd(&s_cnt[1], my_de);
      if (my_dv) atomicAdd(&s_cnt[2], my_dv);
    }
    __syncthreads();
    if (tid == 0) {  // close the pass in shared memory (the trace goes straight out)
      const unsigned long long dv = s_cnt[2], de = s_cnt[1];
      run->passes += 1;
      run->tests += (int64_t)s_cnt[0];
      int cont = 0;
      if (dv + de > 0) {
        if (run->sweeps >= run->max_sweeps) {
          run->status = KZ_ERR_LIMIT;
        } else {
          if (run->sweeps < kTraceCap) {
            st->trace_dv[run->sweeps] = (int64_t)dv;
            st->trace_de[run->sweeps] = (int64_t)de;
          }
          run->sweeps += 1;
          run->cur ^= 1;
          cont = 1;
        }
      }
      *s_flag = cont;
      s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
    }
    __syncthreads();
    if (!*s_flag) break;
    uint32_t *t = Ac;
    Ac = An;
    An = t;
    t = Vc;
    Vc = Vn;
    Vn = t;
    __syncthreads();
  }
  if (SHARED && G.n > 0) {
    // hand the final state back through buffer 0
    uint4 *d4 = reinterpret_cast<uint4 *>(G.A0);
    const uint4 *a4 = reinterpret_cast<const uint4 *>(Ac);
    for (size_t i = tid; i < words / 4; i += kCtaThreads) d4[i] = a4[i];
    for (int i = tid; i < ldw; i += kCtaThreads) G.V0[i] = Vc[i];
  }
  if (tid == 0) {  // the run's record (global mode: the live buffer is run->cur)
    st->sweeps = run->sweeps;
    st->passes = run->passes;
    st->tests = run->tests;
    st->max_sweeps = run->max_sweeps;
    st->status = run->status;
    st->cont = 0;
    st->cur = SHARED ? 0 : run->cur;
  }
  __syncthreads();
}

template <int KMAX>
__global__ void __launch_bounds__(kCtaThreads, 1) cta_fixpoint_kernel(CtaArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long s_cnt[3];
  __shared__ int s_flag;
  __shared__ int s_g;
  __shared__ int32_t s_rounds[KMAX];
  __shared__ CtaRun s_run;
  for (int round = 0;; round++) {
    if (threadIdx.x == 0) s_g = a.queue ? (int)atomicAdd(a.queue, 1u) : (round == 0 ? (int)blockIdx.x : a.count);
    __syncthreads();
    const int g = s_g;
    __syncthreads();
    if (g >= a.count) break;
    const CtaGraph G = a.graphs[a.order[g]];
    if (G.k > KMAX) continue;  // never scheduled: the host groups graphs by KMAX
    if (G.smem_words > 0 && G.smem_words <= a.smem_words)
      cta_fixpoint<KMAX, true>(G, a.max_sweeps, a.slack, smem, s_cnt, &s_flag, s_rounds, &s_run);
    else
      cta_fixpoint<KMAX, false>(G, a.max_sweeps, a.slack, smem, s_cnt, &s_flag, s_rounds, &s_run);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

typedef void (*CtaFn)(CtaArgs);

static CtaFn pick_cta(int k, int &kmax) {
  if (k <= 8) { kmax = 8; return cta_fixpoint_kernel<8>; }
  if (k <= 16) { kmax = 16; return cta_fixpoint_kernel<16>; }
  if (k <= 32) { kmax = 32; return cta_fixpoint_kernel<32>; }
  kmax = 64;
  return cta_fixpoint_kernel<64>;
}

static int device_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// Shared memory words a graph needs for the shared mode (two copies of the
// rows and of the live words).
size_t cta_smem_words(kz_graph g) { return 2 * ((size_t)g->n * g->ldw + (size_t)g->ldw); }

kz_status cta_prepare(kz_graph g, cudaStream_t s) {
  // prefix of the block pairs (x, y) with class(x) < class(y)
  const int nb = (int)g->blocks.size();
  std::vector<int32_t> poff((size_t)nb + 1, 0);
  for (int x = 0; x < nb; x++) poff[x + 1] = poff[x] + (nb - g->boff[g->blocks[x].c + 1]);
  KZ_TRY(graph_alloc(g, &g->d_pair_off, (size_t)nb + 1, s));
  KZ_TRY(h2d(g->d_pair_off, poff.data(), sizeof(int32_t) * (nb + 1), s));
  KZ_TRY(graph_alloc(g, &g->d_boff, (size_t)g->k + 1, s));
  KZ_TRY(h2d(g->d_boff, g->boff.data(), sizeof(int32_t) * (g->k + 1), s));
  g->n_pairs = poff[nb];
  return KZ_OK;
}

static CtaGraph describe(kz_graph g, int64_t max_sweeps);

// Descriptor of the graph for single-graph in-CTA launches (needs every
// buffer of the graph allocated).
kz_status cta_upload_descriptor(kz_graph g, cudaStream_t s) {
  CtaGraph *d = nullptr;
  KZ_TRY(graph_alloc(g, &d, 1, s));
  g->d_cta_desc = d;
  KZ_TRY(graph_alloc(g, &g->d_zero, 4, s));
  KZ_CUDA_TRY(cudaMemsetAsync(g->d_zero, 0, 16, s));
  CtaGraph h = describe(g, 0);
  // staged (or, outside a load, a copy from pageable memory, which has left
  // the local by the time the call returns)
  KZ_TRY(h2d(d, &h, sizeof(h), s));
  return KZ_OK;
}

static CtaGraph describe(kz_graph g, int64_t max_sweeps) {
  CtaGraph d;
  memset(&d, 0, sizeof(d));
  d.A0 = g->A[0];
  d.A1 = g->A[1];
  d.V0 = g->V[0];
  d.V1 = g->V[1];
  d.v_sweep = g->v_sweep;
  d.st = g->st;
  d.blocks = g->d_blocks;
  d.rounds = g->d_rounds;
  d.pair_off = g->d_pair_off;
  d.boff = g->d_boff;
  d.n = g->n;
  d.k = g->k;
  d.ldw = g->ldw;
  d.nb = (int32_t)g->blocks.size();
  const size_t sw = cta_smem_words(g);
  d.smem_words = sw > (size_t)INT32_MAX ? -1 : (int32_t)sw;
  (void)max_sweeps;
  d.m = g->m;
  // cost estimate for the queue order: block pairs x class words
  d.cost = (int64_t)g->n_pairs * 32 * g->k + (int64_t)g->blocks.size() * g->k;
  return d;
}

bool cta_fits_shared(kz_graph g) {
  const size_t limit = (size_t)(device_smem_optin() / 4);
  return cta_smem_words(g) * 4 + 64 <= limit * 4;
}

// Kernelizes `count` graphs with persistent launches, one per KMAX group
// (one launch when every k <= 32, as in a batch of k-partite graphs).
kz_status cta_kernelize(kz_graph *gs, int count, const kz_options &opt, cudaStream_t s,
                        int force_mode) {
  if (count <= 0) return KZ_OK;
  const int optin = device_smem_optin();
  std::vector<CtaGraph> desc((size_t)count);
  for (int i = 0; i < count; i++) {
    desc[i] = describe(gs[i], opt.max_sweeps);
    if (force_mode == 0) desc[i].smem_words = -1;  // global mode everywhere
  }
  // group by KMAX, longest first inside a group
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  CtaGraph *d_desc = (CtaGraph *)dev_alloc(sizeof(CtaGraph) * count, s);
  int32_t *d_order = (int32_t *)dev_alloc(sizeof(int32_t) * count, s);
  unsigned int *d_queue = (unsigned int *)dev_alloc(64, s);
  kz_status st = (d_desc && d_order && d_queue) ? KZ_OK : KZ_ERR_OOM;
  if (st == KZ_OK)
    st = cuda_status(cudaMemcpyAsync(d_desc, desc.data(), sizeof(CtaGraph) * count,
                                     cudaMemcpyHostToDevice, s));
  if (st == KZ_OK) st = cuda_status(cudaMemsetAsync(d_queue, 0, 64, s));
  std::vector<int32_t> order;
  int group = 0;
  for (int kmax_want : {8, 16, 32, 64}) {
    if (st != KZ_OK) break;
    std::vector<int32_t> idx;
    for (int i = 0; i < count; i++) {
      int km = 0;
      pick_cta(desc[i].k, km);
      if (km == kmax_want) idx.push_back(i);
    }
    if (idx.empty()) continue;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return desc[a].cost > desc[b].cost; });
    const size_t off = order.size();
    order.insert(order.end(), idx.begin(), idx.end());
    int km = 0;
    CtaFn fn = pick_cta(desc[idx[0]].k, km);
    const int smem_bytes = std::max(0, optin - 1024);  // static shared memory of the kernel
    st = cuda_status(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          smem_bytes));
    if (st != KZ_OK) break;
    CtaArgs a;
    a.graphs = d_desc;
    a.order = d_order + off;
    a.count = (int32_t)idx.size();
    a.queue = d_queue + 4 * group;  // each group its own 16-byte counter
    a.smem_words = smem_bytes / 4;
    a.slack = 0;  // the fused batch runs the thesis's rules only
    a.max_sweeps = opt.max_sweeps;
    const int grid = std::max(1, std::min<int>((int)idx.size(), sms));
    // order slice must be on the device before the launch
    st = cuda_status(cudaMemcpyAsync(d_order + off, order.data() + off, sizeof(int32_t) * idx.size(),
                                     cudaMemcpyHostToDevice, s));
    if (st != KZ_OK) break;
    fn<<<grid, kCtaThreads, smem_bytes, s>>>(a);
    st = cuda_status(cudaGetLastError());
    group++;
  }
  // (pageable host-to-device copies return once the source is staged, so
  // the host vectors may go out of scope here)
  if (d_desc) dev_free(d_desc, sizeof(CtaGraph) * count, s);
  if (d_order) dev_free(d_order, sizeof(int32_t) * count, s);
  if (d_queue) dev_free(d_queue, 64, s);
  return st;
}

static bool configure_once(CtaFn fn, int kmax, int bytes) {
  static bool done[4] = {false, false, false, false};
  const int slot = kmax == 8 ? 0 : kmax == 16 ? 1 : kmax == 32 ? 2 : 3;
  if (done[slot]) return true;
  if (cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) !=
      cudaSuccess)
    return false;
  done[slot] = true;
  return true;
}

kz_status cta_kernelize_one(kz_graph g, const kz_options &opt, cudaStream_t s) {
  int km = 0;
  CtaFn fn = pick_cta(g->k, km);
  const int max_bytes = std::max(0, device_smem_optin() - 1024);
  if (!configure_once(fn, km, max_bytes)) return KZ_ERR_CUDA;
  // ask only for what this graph's shared mode needs (a small graph should
  // not force the largest shared-memory carve-out)
  const size_t need = cta_smem_words(g) * 4;
  const int smem_bytes = need <= (size_t)max_bytes ? (int)((need + 15) / 16 * 16) : 0;
  CtaArgs a;
  a.graphs = g->d_cta_desc;
  a.order = g->d_zero;
  a.count = 1;
  a.queue = nullptr;
  a.smem_words = smem_bytes / 4;
  a.slack = g->slack;
  a.max_sweeps = opt.max_sweeps;
  fn<<<1, kCtaThreads, smem_bytes, s>>>(a);
  return cuda_status(cudaGetLastError());
}

}  // namespace kz

// ---------------------------------------------------------------------------
// kz_kernelize_dense_noalloc: one graph, start to finish, with no memory
// allocation at all.  Every intermediate lives in one file-scope device array
// (g_noalloc_scratch below) that each GPU loading the library keeps until the
// process exits; the caller passes device buffers for inputs and outputs.
// The fixpoint itself is the in-CTA kernel above, reading its descriptor from
// that array.
// ---------------------------------------------------------------------------

namespace kz {
namespace noalloc {

constexpr int kMaxN = KZ_NOALLOC_MAX_N;
constexpr int kMaxWords = KZ_NOALLOC_MAX_WORDS;  // words per adjacency buffer
constexpr int kMaxLdw = 4096;                    // words per row
constexpr int kMaxBlocks = 256;

struct Header {
  CtaGraph desc;
  int32_t status;
  int32_t pad;
  unsigned long long m;
  int32_t coff[65];
  int32_t boff[65];
  int32_t rounds[64];
  int32_t fill[64];
  int32_t pair_off[kMaxBlocks + 1];
  BlockDesc blocks[kMaxBlocks];
};

struct Scratch {
  alignas(256) Header h;
  alignas(256) DevState st;
  alignas(256) uint32_t A0[kMaxWords];
  alignas(256) uint32_t A1[kMaxWords];
  alignas(256) uint32_t V0[kMaxLdw];
  alignas(256) uint32_t V1[kMaxLdw];
  alignas(256) int32_t perm[kMaxN];
  alignas(256) int32_t inv[kMaxN];
  alignas(256) int32_t v_sweep[kMaxN];
};

}  // namespace noalloc
}  // namespace kz

// The scratch of kz_kernelize_dense_noalloc (about 9 MiB per device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(kz::noalloc::Scratch)];

namespace kz {
namespace noalloc {

// First index i in [0, len) with a[i] > x (a sorted ascending).
__device__ __forceinline__ int upper_bound_int(const int32_t *a, int len, int32_t x) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Layout of the caller's graph: colour classes, blocks, block pairs, the
// descriptor of the in-CTA kernel.  One CTA.
__global__ void setup_kernel(Scratch *s, int32_t n, int32_t k, const int32_t *__restrict__ colour) {
  Header &h = s->h;
  __shared__ int cnt[64];
  __shared__ int bad;
  __shared__ int status;
  const int tid = threadIdx.x;
  if (tid < 64) cnt[tid] = 0;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int v = tid; v < n; v += blockDim.x) {
    const int c = colour[v];
    if (c < 0 || c >= k) atomicExch(&bad, (int)KZ_ERR_COLOUR_RANGE);
    else atomicAdd(&cnt[c], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int st = bad;
    int R = 1, nb = 0;
    h.coff[0] = 0;
    for (int c = 0; c < k; c++) {
      h.coff[c + 1] = h.coff[c] + cnt[c];
      h.rounds[c] = (cnt[c] + 31) / 32;
      R = max(R, h.rounds[c]);
      nb += h.rounds[c];
    }
    const int64_t ldw = ((int64_t)R * k + 3) / 4 * 4;
    if (!st && (ldw > kMaxLdw || (int64_t)n * ldw > kMaxWords || nb > kMaxBlocks)) st = KZ_ERR_UNSUPPORTED;
    if (!st) {
      h.boff[0] = 0;
      int b = 0;
      for (int c = 0; c < k; c++) {
        h.boff[c + 1] = h.boff[c] + h.rounds[c];
        for (int r = 0; r < h.rounds[c]; r++, b++) {
          h.blocks[b].c = c;
          h.blocks[b].r = r;
          h.blocks[b].base = h.coff[c] + 32 * r;
          h.blocks[b].size = min(32, cnt[c] - 32 * r);
        }
        h.fill[c] = h.coff[c];
      }
      h.pair_off[0] = 0;
      for (int x = 0; x < nb; x++) h.pair_off[x + 1] = h.pair_off[x] + (nb - h.boff[h.blocks[x].c + 1]);
      CtaGraph &d = h.desc;
      d.A0 = s->A0;
      d.A1 = s->A1;
      d.V0 = s->V0;
      d.V1 = s->V1;
      d.v_sweep = s->v_sweep;
      d.st = &s->st;
      d.blocks = h.blocks;
      d.rounds = h.rounds;
      d.pair_off = h.pair_off;
      d.boff = h.boff;
      d.n = n;
      d.k = k;
      d.ldw = (int32_t)ldw;
      d.nb = nb;
      d.smem_words = (int32_t)(2 * ((int64_t)n * ldw + ldw));
      d.m = 0;
      d.cost = 0;
      h.m = 0;
      DevState &ds = s->st;
      ds.cur = 0;
      ds.status = KZ_OK;
      ds.cont = 0;
      ds.sweeps = ds.passes = ds.tests = 0;
      ds.pass_dv = ds.pass_de = ds.pass_tests = 0;
      ds.ticket = 0;
    }
    h.status = st;
    status = st;
  }
  __syncthreads();
  if (status) return;
  // relabel: every class a contiguous id range (order inside a class is free:
  // the fixpoint and every count reported do not depend on it)
  for (int v = tid; v < n; v += blockDim.x) {
    const int x = atomicAdd(&h.fill[colour[v]], 1);
    s->inv[v] = x;
    s->perm[x] = v;
  }
}

// Zeroed rows, live words of every block, zeroed deletion sweeps.
__global__ void clear_kernel(Scratch *s) {
  if (s->h.status) return;
  const CtaGraph &d = s->h.desc;
  const int64_t words = (int64_t)d.n * d.ldw;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < words; i += stride) s->A0[i] = 0u;
  for (int64_t i = tid; i < d.ldw; i += stride) s->V0[i] = 0u;
  for (int64_t i = tid; i < d.n; i += stride) s->v_sweep[i] = 0;
}

__global__ void live_words_kernel(Scratch *s) {
  if (s->h.status) return;
  const CtaGraph &d = s->h.desc;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < d.nb; b += gridDim.x * blockDim.x) {
    const BlockDesc bd = s->h.blocks[b];
    s->V0[bd.r * d.k + bd.c] = bd.size >= 32 ? 0xffffffffu : ((1u << bd.size) - 1u);
  }
}

// Caller's dense bit matrix (strict upper triangle) into the block-plane rows.
__global__ void pack_kernel(Scratch *s, const uint64_t *__restrict__ bits, int64_t row_words,
                            const int32_t *__restrict__ colour) {
  Header &h = s->h;
  if (h.status) return;
  const int n = h.desc.n, k = h.desc.k, ldw = h.desc.ldw;
  unsigned long long mine = 0;
  const int64_t total = (int64_t)n * row_words;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = (int32_t)(t / row_words);
    const int64_t w = t - (int64_t)i * row_words;
    const int64_t j0 = w * 64;
    if (j0 + 63 <= i || j0 >= n) continue;
    uint64_t word = bits[t];
    if (j0 <= i) {
      const int sh = i - (int)j0 + 1;
      word = sh >= 64 ? 0 : (word >> sh) << sh;
    }
    if (j0 + 64 > n) word &= (1ull << (n - (int)j0)) - 1;
    if (!word) continue;
    const int32_t ci = colour[i];
    const int32_t x = s->inv[i];
    const int32_t ix = x - h.coff[ci];
    while (word) {
      const int b = __ffsll((long long)word) - 1;
      word &= word - 1;
      const int32_t j = (int32_t)j0 + b;
      const int32_t cj = colour[j];
      if (cj == ci) {
        atomicCAS(&h.status, 0, (int32_t)KZ_ERR_ILLEGAL_COLOURING);
        continue;
      }
      const int32_t y = s->inv[j];
      const int32_t iy = y - h.coff[cj];
      atomicOr(&s->A0[(int64_t)x * ldw + (iy >> 5) * k + cj], 1u << (iy & 31));
      atomicOr(&s->A0[(int64_t)y * ldw + (ix >> 5) * k + ci], 1u << (ix & 31));
      mine++;
    }
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&h.m, mine);
}

// Both ping-pong copies start from the packed rows (own-class words zero).
__global__ void mirror_kernel(Scratch *s) {
  if (s->h.status) return;
  const CtaGraph &d = s->h.desc;
  const int64_t words = (int64_t)d.n * d.ldw;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < words; i += stride) s->A1[i] = s->A0[i];
  for (int64_t i = tid; i < d.ldw; i += stride) s->V1[i] = s->V0[i];
  if (tid == 0) s->h.desc.m = (int64_t)s->h.m;
}

// The in-CTA fixpoint on the scratch descriptor (k <= 32).
__global__ void __launch_bounds__(kCtaThreads, 1) fixpoint_kernel(Scratch *s, int64_t max_sweeps,
                                                                        int32_t smem_words) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long s_cnt[3];
  __shared__ int s_flag;
  __shared__ int32_t s_rounds[32];
  __shared__ CtaRun s_run;
  if (s->h.status) return;
  const CtaGraph G = s->h.desc;
  if (G.smem_words > 0 && G.smem_words <= smem_words)
    cta_fixpoint<32, true>(G, max_sweeps, 0, smem, s_cnt, &s_flag, s_rounds, &s_run);
  else
    cta_fixpoint<32, false>(G, max_sweeps, 0, smem, s_cnt, &s_flag, s_rounds, &s_run);
}

__global__ void zero_out_kernel(uint64_t *__restrict__ out, int64_t words) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 0ull;
}

// Kernel rows back to caller ids: the symmetric bit matrix, the live
// vertices, and (sweeps, passes, edge tests, status).
__global__ void unpack_kernel(Scratch *s, int32_t n_in, uint64_t *__restrict__ out, int64_t row_words,
                              uint8_t *__restrict__ alive, int64_t *__restrict__ counts) {
  const Header &h = s->h;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (h.status) {
    // a rejected input leaves defined outputs: no vertex, no edge (the bit
    // matrix was zeroed before this kernel), zero counts and the status
    for (int64_t v = tid; v < n_in; v += stride) alive[v] = 0;
    if (tid == 0) {
      counts[0] = counts[1] = counts[2] = 0;
      counts[3] = h.status;
    }
    return;
  }
  const CtaGraph &d = h.desc;
  const int cur = s->st.cur;
  const uint32_t *A = cur ? s->A1 : s->A0;
  const uint32_t *V = cur ? s->V1 : s->V0;
  const int n = d.n, k = d.k, ldw = d.ldw;
  const int rk = ldw;  // rows are scanned over their padded length; padding words are zero
  for (int64_t t = tid; t < (int64_t)n * rk; t += stride) {
    const int32_t x = (int32_t)(t / rk);
    const int32_t w = (int32_t)(t - (int64_t)x * rk);
    uint32_t word = A[(int64_t)x * ldw + w];
    if (!word) continue;
    const int32_t c = w % k, r = w / k;
    const int32_t ox = s->perm[x];
    while (word) {
      const int b = __ffs(word) - 1;
      word &= word - 1;
      const int32_t oy = s->perm[h.coff[c] + 32 * r + b];
      atomicOr(reinterpret_cast<unsigned long long *>(&out[(int64_t)ox * row_words + (oy >> 6)]),
               1ull << (oy & 63));
    }
  }
  for (int64_t v = tid; v < n; v += stride) {
    const int32_t x = s->inv[v];
    const int32_t c = (int32_t)(upper_bound_int(h.coff, k + 1, x) - 1);
    const int32_t i = x - h.coff[c];
    alive[v] = (uint8_t)((V[(i >> 5) * k + c] >> (i & 31)) & 1u);
  }
  if (tid == 0) {
    counts[0] = s->st.sweeps;
    counts[1] = s->st.passes;
    counts[2] = s->st.tests;
    counts[3] = s->st.status;
  }
}

}  // namespace noalloc
}  // namespace kz

namespace {

// Device address of the scratch array, looked up once per device (host code
// cannot use the array's name as a device pointer).
std::mutex g_noalloc_mu;
void *g_noalloc_addr[64] = {nullptr};

kz_status noalloc_scratch(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return KZ_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return KZ_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return KZ_OK;
}

}  // namespace

extern "C" kz_status kz_kernelize_dense_noalloc(int32_t n, int32_t k, const int32_t *colour,
                                                const uint64_t *adj_bits, int64_t row_words,
                                                int64_t max_sweeps, uint8_t *vertex_alive,
                                                uint64_t *adj_out, int64_t *counts, void *stream) {
  using namespace kz::noalloc;
  if (n < 0 || k < 1 || k > 32) return KZ_ERR_ARG;
  if (n > kMaxN) return KZ_ERR_UNSUPPORTED;
  if (row_words < (int64_t)((n + 63) / 64) || !counts) return KZ_ERR_ARG;
  if (n > 0 && (!colour || !adj_bits || !vertex_alive || !adj_out)) return KZ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  void *scratch = nullptr;
  KZ_TRY(noalloc_scratch(&scratch));  // device address of the array on this device
  Scratch *sp = static_cast<Scratch *>(scratch);
  int dev = 0, sms = 1, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int smem_bytes = std::max(0, optin - 1024);
  {
    static std::mutex mu;
    static bool configured[64] = {false};
    std::lock_guard<std::mutex> lk(mu);
    if (!configured[dev]) {
      KZ_CUDA_TRY(cudaFuncSetAttribute((const void *)fixpoint_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes));
      configured[dev] = true;
    }
  }
  const int grid = 2 * std::max(sms, 1);
  setup_kernel<<<1, 1024, 0, s>>>(sp, n, k, colour);
  clear_kernel<<<grid, 256, 0, s>>>(sp);
  live_words_kernel<<<1, 256, 0, s>>>(sp);
  if ((int64_t)n * row_words > 0) pack_kernel<<<grid, 256, 0, s>>>(sp, adj_bits, row_words, colour);
  mirror_kernel<<<grid, 256, 0, s>>>(sp);
  fixpoint_kernel<<<1, kz::kCtaThreads, smem_bytes, s>>>(sp, max_sweeps, smem_bytes / 4);
  if ((int64_t)n * row_words > 0) zero_out_kernel<<<grid, 256, 0, s>>>(adj_out, (int64_t)n * row_words);
  unpack_kernel<<<grid, 256, 0, s>>>(sp, n, adj_out, row_words, vertex_alive, counts);
  KZ_CUDA_TRY(cudaGetLastError());
  // synchronous: the device status decides the return value
  int64_t status = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&status, counts + 3, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  return (kz_status)status;
}
