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
// Sweep kernel design:
//   * The work of a pass is a sequence of units (X, Y): a block X of 32
//     vertices u (lane = u) of class cu against one block Y of a higher class
//     cv > cu.  The host cuts the sequence into one range of about equal cost
//     per warp, so every warp of the grid ends its pass at about the same time.
//   * A warp holds plane 0 of its X rows (k words per lane) in registers.  For
//     each unit it stages plane 0 of the 32 rows v of Y in shared memory (the
//     next unit's copy is in flight meanwhile) and for every v tests all
//     lanes' pairs (u, v) at once: the pair is covered in class c when
//     row_u[c] & row_v[c] != 0.  The classes cu and cv are forced to "covered"
//     on both sides, so "every class covered" is one min-reduction over the
//     k word-ANDs.  A live edge whose plane-0 test fails is recounted exactly
//     over all planes (rare on dense graphs).
//   * The two words a unit owns (row u's word for Y, and row v's word for X,
//     the warp transpose of the first) go to the other ping-pong buffer only
//     when they change in this pass or changed in the previous one: the other
//     buffer already holds every other word.  A per-unit tag records the sweep
//     of the last change.  After another path has written the rows, one pass
//     writes every word.
//   * The last CTA (persistent kernel) or warp (one-pass kernel) to finish
//     records the pass counters, flips the buffers when something was deleted
//     and, in the CUDA-graph loop, sets the while-condition.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
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

// Work of the sweep kernels: the units of a pass in order (x ascending; for
// each x the blocks y of higher classes, or one vertex-only unit y = nb for a
// block of the last class), listed as (x, y) pairs and cut into `ctas`
// consecutive ranges of about equal estimated cost.  A CTA owns one range and
// its warps take the range's units one at a time, so every warp of the CTA
// stays busy until the CTA's share is done.  A unit costs the members of Y it
// tests plus a fixed part for staging and bookkeeping; the first unit of each
// x also evaluates the vertex rule.
//
// The list is laid out block by block: block x's units are (x, y) for every
// block y of a higher class (one unit (x, nb) when there is none), starting at
// unit_off[x].  The host computes unit_off and the CTA ranges from per-block
// sums in O(blocks) (binary searches inside a block's run of units); the
// list itself is filled on the device (fill_units_kernel).
static void plan_units(kz_graph g, int ctas, std::vector<int32_t> &unit_off, std::vector<int32_t> &cta_begin) {
  constexpr int64_t kUnitFixed = 8, kVertexCost = 8;
  const int nb = (int)g->blocks.size();
  auto ybegin = [&](int x) { return std::min(g->boff[g->blocks[x].c + 1], nb); };
  // size_pre[y] = sizes of blocks 0..y-1
  std::vector<int64_t> size_pre((size_t)nb + 1, 0);
  for (int y = 0; y < nb; y++) size_pre[y + 1] = size_pre[y] + g->blocks[y].size;
  // cost of the first i units of block x (y = yb .. yb + i - 1)
  auto run_cost = [&](int x, int64_t i) -> int64_t {
    const int yb = ybegin(x);
    if (i <= 0) return 0;
    if (yb >= nb) return kUnitFixed + kVertexCost;  // the single unit (x, nb)
    return size_pre[yb + i] - size_pre[yb] + kUnitFixed * i + kVertexCost;
  };
  unit_off.assign((size_t)nb + 1, 0);
  std::vector<int64_t> cost_off((size_t)nb + 1, 0);
  for (int x = 0; x < nb; x++) {
    const int yb = ybegin(x);
    const int64_t cnt = yb >= nb ? 1 : nb - yb;
    unit_off[x + 1] = unit_off[x] + (int32_t)cnt;
    cost_off[x + 1] = cost_off[x] + run_cost(x, cnt);
  }
  const int64_t total = cost_off[nb];
  // CTA c takes the units whose running cost ends in (c, c + 1] * total / ctas
  cta_begin.assign((size_t)ctas + 1, unit_off[nb]);
  cta_begin[0] = 0;
  int x = 0;
  for (int c = 1; c < ctas; c++) {
    // the first unit whose running cost * ctas exceeds c * total
    while (x < nb && cost_off[x + 1] * ctas <= (int64_t)c * total) x++;
    if (x >= nb) {
      cta_begin[(size_t)c] = unit_off[nb];
      continue;
    }
    const int64_t cnt = unit_off[x + 1] - unit_off[x];
    int64_t lo = 0, hi = cnt;  // units i < lo end at or below the cut
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if ((cost_off[x] + run_cost(x, mid + 1)) * ctas <= (int64_t)c * total) lo = mid + 1;
      else hi = mid;
    }
    cta_begin[(size_t)c] = unit_off[x] + (int32_t)lo;
  }
}

// The unit list from the per-block offsets: unit u of block x is (x, y) with
// y = ybegin(x) + (u - unit_off[x]), or (x, nb) when x has no partner.
__global__ void fill_units_kernel(int2 *__restrict__ units, const int32_t *__restrict__ unit_off,
                                  const BlockDesc *__restrict__ blocks, const int32_t *__restrict__ boff, int32_t nb) {
  const int64_t total = unit_off[nb];
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < total; u += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nb;  // the last x with unit_off[x] <= u
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (unit_off[mid] <= u) lo = mid;
      else hi = mid;
    }
    const int yb = min(boff[blocks[lo].c + 1], nb);
    units[u] = make_int2(lo, yb >= nb ? nb : yb + (int32_t)(u - unit_off[lo]));
  }
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
  const int2 *units;        // (x, y) of every unit of a pass
  const int32_t *cta_begin; // first unit of each CTA's range (grid + 1)
  int32_t nb;               // blocks
  int32_t k, ldw;
  const int32_t *rounds;  // blocks per class
  const int32_t *boff;    // first block of each class, k + 1
  uint32_t *A0, *A1;      // ping-pong adjacency
  uint32_t *V0, *V1;      // ping-pong vertex live words
  int32_t *v_sweep;       // relabelled ids, may be null
  uint8_t *changed;       // per unit: low byte of the sweep that last changed its words
  int32_t fast_half;      // half-word form: try the whole-block fold first (very dense graphs)
  int32_t slack;          // colours minus the clique size sought (0: the thesis's rules)
  DevState *st;
  cudaGraphConditionalHandle cond;
  int32_t use_cond;
  uint32_t bar_extra;    // arrivals the grid barrier waits for beyond the grid (0; tests use 1)
  uint32_t spin_limit;   // polls before a barrier wait gives up
};

// First test of a pair in the sweep kernels (the FORM template argument).
constexpr int kFormFull = 0;  // plane 0: the first 32 members of each class, one word per class
constexpr int kFormHalf = 1;  // the first 16 members, two classes per word (dense graphs)
constexpr int kFormTwo = 2;   // planes 0 and 1: the first 64 members (sparser graphs)
// density (edges / pairs of vertices in different classes) from which the
// sweep kernels use the half-word plane-0 test
constexpr double kHalfDensity = 0.8;
// density below which a graph of at least two planes (and k <= 32) tests the
// first 64 members of each class first
constexpr double kTwoPlaneDensity = 0.42;
// density from which a whole block is first folded without per-pair results
// (almost every 32 x 32 block then has every pair covered); below it the
// half-word form (when forced) tests pair by pair
constexpr double kFastHalfDensity = 0.8;
// Warps of a sweep CTA (one CTA per SM): as many as the registers of the
// form allow -- 20 for the half-word form up to k = 24 (96 registers), 16 at
// up to 128 registers, 8 for the widest kernels.
__host__ __device__ constexpr int cta_warps(int kmax, int form) {
  return form == kFormHalf ? (kmax <= 24 ? 20 : (kmax <= 32 ? 16 : 8))
         : form == kFormTwo ? (kmax <= 24 ? 16 : 8)
                            : (kmax <= 32 ? 16 : 8);
}
// Shared memory of one warp: two staging buffers of plane-0 rows (KMAX words
// each) and, in the half-word form, the converted rows of the current unit.
template <int KMAX, int FORM>
__host__ __device__ constexpr int warp_smem_words() {
  return FORM == kFormTwo ? 2 * 32 * 2 * KMAX : 2 * 32 * KMAX + (FORM == kFormHalf ? 32 * half_stride<KMAX>() : 0);
}

__device__ __forceinline__ void prefetch_l1(const uint32_t *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// One warp's share of one Jacobi pass: units taken one at a time from its
// CTA's range [u_begin, u_end) through the shared counter *s_next, so the
// CTA's warps stay busy until its whole range is done.  `cur` is the current
// ping-pong buffer, `sweep_no` the productive sweeps so far, `full` asks for
// every owned word to be written.  FORM selects the first test of a pair
// (kFormFull, kFormHalf, kFormTwo).
template <int KMAX, int FORM>
__device__ __forceinline__ void sweep_cta(const SweepArgs &p, int u_begin, int u_end, unsigned int *s_next,
                                          int cur, int64_t sweep_no, bool full, uint32_t *buf0, uint32_t *buf1,
                                          uint32_t *bufh, const int32_t *rounds, PassCounters &pc) {
  const int lane = threadIdx.x & 31;
  const uint32_t *__restrict__ A = cur ? p.A1 : p.A0;
  uint32_t *__restrict__ An = cur ? p.A0 : p.A1;
  const uint32_t *__restrict__ Vc = cur ? p.V1 : p.V0;
  uint32_t *__restrict__ Vn = cur ? p.V0 : p.V1;
  constexpr bool HALF = FORM == kFormHalf;
  constexpr bool TWO = FORM == kFormTwo;
  const int k = p.k, ldw = p.ldw, nb = p.nb, slack = p.slack;
  const int kq4 = TWO ? (2 * k + 3) >> 2 : (k + 3) >> 2;  // 16-byte chunks staged per row
  const uint8_t tag_now = (uint8_t)(sweep_no & 0xff);
  const uint8_t tag_next = (uint8_t)((sweep_no + 1) & 0xff);

  // cursor (x, y, unit): the next unit to stage.  Its adjacency word, change
  // tag and live word are loaded one unit ahead.
  int unit = u_begin + (int)__shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(s_next, 1u) : 0u, 0);
  if (unit >= u_end) return;
  int2 e = p.units[unit];
  int x = e.x, y = e.y;
  BlockDesc X = p.blocks[x];
  int ybeg = min(p.boff[X.c + 1], nb);
  BlockDesc Y = X;
  if (y < nb) {
    Y = p.blocks[y];
    if constexpr (TWO) stage_block2<KMAX>(A, ldw, Y, kq4, buf0, lane);
    else stage_block<KMAX>(A, ldw, Y, kq4, buf0, lane);
  }
  cp_async_commit();
  uint32_t adj_n = (y < nb && lane < X.size) ? A[(int64_t)(X.base + lane) * ldw + Y.r * k + Y.c] : 0u;
  uint8_t chg_n = y < nb ? p.changed[unit] : (uint8_t)0;
  uint32_t vw_n = y == ybeg ? Vc[X.r * k + X.c] : 0u;

  constexpr int KH = KMAX / 2;
  constexpr int KW = HALF ? KH : KMAX;
  uint32_t F[KW], P[KW];  // plane 0 of the lanes' rows (full or half-word form), forced classes
  uint32_t F1[TWO ? KMAX : 1];  // plane 1 (two-plane form)
  int fu_x = -1, prev_cv = -1, vcnt = 0;
  uint64_t vmiss = 0;  // classes plane 0 leaves uncovered for the lane's vertex
  for (int i = 0;; i++) {
    const int xc = x, yc = y, uc_unit = unit;
    const BlockDesc Xc = X, Yc = Y;
    const bool vflag = yc == ybeg;
    const uint32_t adjw = adj_n, vword = vw_n;
    const uint8_t chg = chg_n;
    uint32_t *sv = (i & 1) ? buf1 : buf0;
    // take the next unit and stage it
    unit = u_begin + (int)__shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(s_next, 1u) : 0u, 0);
    const bool more = unit < u_end;
    if (more) {
      e = p.units[unit];
      x = e.x;
      y = e.y;
      if (x != xc) {
        X = p.blocks[x];
        ybeg = min(p.boff[X.c + 1], nb);
        if (lane < X.size) {  // warm L1 with plane 0 of the next block's rows
          const uint32_t *row = A + (int64_t)(X.base + lane) * ldw;
          prefetch_l1(row);
          prefetch_l1(row + k - 1);
        }
      }
      if (y < nb) {
        Y = p.blocks[y];
        if constexpr (TWO) stage_block2<KMAX>(A, ldw, Y, kq4, (i & 1) ? buf0 : buf1, lane);
        else stage_block<KMAX>(A, ldw, Y, kq4, (i & 1) ? buf0 : buf1, lane);
      }
      adj_n = (y < nb && lane < X.size) ? A[(int64_t)(X.base + lane) * ldw + Y.r * k + Y.c] : 0u;
      chg_n = y < nb ? p.changed[unit] : (uint8_t)0;
      vw_n = y == ybeg ? Vc[X.r * k + X.c] : 0u;
    }
    cp_async_commit();
    cp_async_wait<1>();
    __syncwarp();

    const int cu = Xc.c;
    const bool valid = lane < Xc.size;
    const int u = Xc.base + lane;
    const uint32_t *rowu = A + (int64_t)(valid ? u : Xc.base) * ldw;
    if (xc != fu_x) {  // always true at a vertex-rule unit (the first unit of its block)
      if constexpr (HALF) {
        uint32_t Fu[KMAX];
        load_plane0<KMAX>(Fu, rowu, k, valid);
        vmiss = plane0_vertex_missing<KMAX>(Fu, k, cu);
        halve_plane0<KMAX, KH>(F, Fu);
        if (!valid) {  // no vertex: never uncovered, so the fast fold is not disturbed
#pragma unroll
          for (int j = 0; j < KH; j++) F[j] = 0xffffffffu;
        }
      } else {
        load_plane0<KMAX>(F, rowu, k, valid);
        vmiss = plane0_vertex_missing<KMAX>(F, k, cu);
        if constexpr (TWO) load_plane1<KMAX>(F1, rowu, k, valid);
      }
      vcnt = (k - 1) - __popcll(vmiss);
      fu_x = xc;
      prev_cv = -1;
    }
    if (vflag) {
      const bool live = valid && ((vword >> lane) & 1u);
      int cnt = vcnt;
      if (live && cnt < k - 1 - slack) cnt += vertex_cover_beyond_plane0(rowu, k, rounds, vmiss);
      const bool fail = live && cnt < k - 1 - slack;
      const uint32_t failmask = __ballot_sync(0xffffffffu, fail);
      if (lane == 0) {
        Vn[Xc.r * k + cu] = vword & ~failmask;
        pc.dv += __popc(failmask);
      }
      if (fail && p.v_sweep) p.v_sweep[u] = (int32_t)(sweep_no + 1);
    }
    if (yc < nb) {
      const int cv = Yc.c;
      if (cv != prev_cv) {
        if constexpr (HALF) half_mask<KH>(P, k, cu, cv);
        else pair_mask<KMAX>(P, k, cu, cv);
        prev_cv = cv;
      }
      pc.tests += __popc(adjw);
      const uint32_t *ybase = A + (int64_t)Yc.base * ldw;
      uint32_t open, del = 0;
      if constexpr (HALF) {
        halve_staged_rows<KMAX>(sv, bufh, Yc.size, lane);
        __syncwarp();
        open = half_unsettled<KMAX, KH>(F, P, bufh, adjw, p.fast_half != 0);
        // the recount starts from the full staged plane 0
        if (open) del = recount_unsettled(rowu, sv, KMAX, ybase, ldw, open, k, cu, cv, rounds, slack);
      } else if constexpr (TWO) {
        spread_plane1<KMAX>(sv, Yc.size, k, lane);
        __syncwarp();
        open = two_unsettled<KMAX>(F, F1, P, sv, adjw, k);
        // the recount starts from plane 0 of the staged rows, then reads the rows
        if (open) del = recount_unsettled(rowu, sv, 2 * KMAX, ybase, ldw, open, k, cu, cv, rounds, slack);
      } else {
        open = plane0_unsettled<KMAX>(F, P, sv, adjw, k);
        if (open) del = recount_unsettled(rowu, sv, KMAX, ybase, ldw, open, k, cu, cv, rounds, slack);
      }
      const bool anydel = __any_sync(0xffffffffu, del != 0u);
      if (anydel || full || chg == tag_now) {
        const uint32_t keep = adjw & ~del;
        if (valid) An[(int64_t)u * ldw + Yc.r * k + cv] = keep;
        const uint32_t col = transpose32(keep);
        if (lane < Yc.size) An[(int64_t)(Yc.base + lane) * ldw + Xc.r * k + cu] = col;
        if (anydel && lane == 0) p.changed[uc_unit] = tag_next;
        pc.de += __popc(del);
      }
    }
    __syncwarp();
    if (!more) break;
  }
  cp_async_wait<0>();
  __syncwarp();
}

// The CTA's pass counters, summed over its warps and added to the running
// pass totals cnt[0..2] = (tests, deleted edges, deleted vertices) with one
// atomic per counter (thread 0, which also gets whether the CTA deleted
// anything).  Ends with the CTA synchronised.
template <int WARPS>
__device__ __forceinline__ bool add_cta_counters(PassCounters pc, unsigned long long *cnt) {
  __shared__ unsigned long long s_pc[WARPS][3];
  for (int o = 16; o > 0; o >>= 1) {
    pc.tests += __shfl_down_sync(0xffffffffu, pc.tests, o);
    pc.de += __shfl_down_sync(0xffffffffu, pc.de, o);
    pc.dv += __shfl_down_sync(0xffffffffu, pc.dv, o);
  }
  const int wib = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_pc[wib][0] = pc.tests;
    s_pc[wib][1] = pc.de;
    s_pc[wib][2] = pc.dv;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0, de = 0, dv = 0;
    for (int w = 0; w < WARPS; w++) {
      t += s_pc[w][0];
      de += s_pc[w][1];
      dv += s_pc[w][2];
    }
    if (t) atomicAdd(&cnt[0], t);
    if (de) atomicAdd(&cnt[1], de);
    if (dv) atomicAdd(&cnt[2], dv);
    return de + dv > 0;
  }
  return false;
}

// One Jacobi pass per launch (the CUDA-graph loop and the host-driven loop).
template <int KMAX, int FORM>
__global__ void __launch_bounds__(cta_warps(KMAX, FORM) * 32, 1)
    bitset_sweep_kernel(SweepArgs p) {
  constexpr int W = cta_warps(KMAX, FORM);
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned int s_next;
  const int wib = threadIdx.x >> 5;
  constexpr int kRow = FORM == kFormTwo ? 2 * KMAX : KMAX;  // staged row stride
  uint32_t *buf0 = smem + wib * warp_smem_words<KMAX, FORM>();
  uint32_t *buf1 = buf0 + 32 * kRow;
  uint32_t *bufh = buf1 + 32 * kRow;  // half-word rows (half-word form only)
  __shared__ int32_t s_rounds[KMAX];
  for (int c = threadIdx.x; c < p.k; c += blockDim.x) s_rounds[c] = p.rounds[c];
  if (threadIdx.x == 0) s_next = 0;
  __syncthreads();
  DevState *st = p.st;
  const int cur = *((volatile int32_t *)&st->cur);
  const int64_t sweep_no = *((volatile int64_t *)&st->sweeps);
  const bool full = *((volatile int32_t *)&st->full_write) != 0;
  PassCounters pc;
  sweep_cta<KMAX, FORM>(p, p.cta_begin[blockIdx.x], p.cta_begin[blockIdx.x + 1], &s_next, cur, sweep_no, full, buf0,
                        buf1, bufh, s_rounds, pc);
  add_cta_counters<W>(pc, st->ppass[0]);
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(&st->ticket, 1u);
    if (t == gridDim.x - 1u) {  // the last CTA closes the pass
      __threadfence();
      unsigned long long *c = st->ppass[0];
      const unsigned long long tests = atomicAdd(&c[0], 0ull);
      const unsigned long long de = atomicAdd(&c[1], 0ull);
      const unsigned long long dv = atomicAdd(&c[2], 0ull);
      const int cont = finish_pass(st, dv, de, tests);
      c[0] = c[1] = c[2] = 0;
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
template <int KMAX, int FORM>
__global__ void __launch_bounds__(cta_warps(KMAX, FORM) * 32, 1)
    bitset_persistent_kernel(SweepArgs p) {
  constexpr int W = cta_warps(KMAX, FORM);
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ unsigned long long s_word;
  __shared__ unsigned int s_next;
  const int wib = threadIdx.x >> 5;
  constexpr int kRow = FORM == kFormTwo ? 2 * KMAX : KMAX;  // staged row stride
  uint32_t *buf0 = smem + wib * warp_smem_words<KMAX, FORM>();
  uint32_t *buf1 = buf0 + 32 * kRow;
  uint32_t *bufh = buf1 + 32 * kRow;  // half-word rows (half-word form only)
  __shared__ int32_t s_rounds[KMAX];
  for (int c = threadIdx.x; c < p.k; c += blockDim.x) s_rounds[c] = p.rounds[c];
  __syncthreads();
  DevState *st = p.st;
  // the first pass reads the run's start state; every later one takes it from
  // the word the pass-closing CTA publishes with the barrier release
  int cur = *((volatile int32_t *)&st->cur);
  int64_t sweep_no = *((volatile int64_t *)&st->sweeps);
  bool full = *((volatile int32_t *)&st->full_write) != 0;
  const int64_t max_sweeps = *((volatile int64_t *)&st->max_sweeps);
  const int u_begin = p.cta_begin[blockIdx.x], u_end = p.cta_begin[blockIdx.x + 1];
  for (int pass = 0;; pass++) {
    if (threadIdx.x == 0) s_next = 0;
    __syncthreads();
    PassCounters pc;
    sweep_cta<KMAX, FORM>(p, u_begin, u_end, &s_next, cur, sweep_no, full, buf0, buf1, bufh, s_rounds, pc);
    // counters by pass parity: the closing CTA reads this pass's after the
    // release, while the next pass adds to the other set
    unsigned long long *cnt = st->ppass[pass & 1];
    const bool deleted = add_cta_counters<W>(pc, cnt);
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned long long w0 = *((volatile unsigned long long *)&st->pass_word);
      unsigned long long w = w0;
      bool abort = false;
      // arrival count in the low 20 bits, CTAs that deleted something above
      const unsigned int old = atomicAdd(&st->bar_count, 1u | (deleted ? 1u << 20 : 0u));
      if ((old & 0xfffffu) == gridDim.x - 1u + p.bar_extra) {
        // the pass closes: decide and release first, book-keep after
        const bool productive = deleted || (old >> 20) != 0u;
        const int cont = productive && sweep_no < max_sweeps ? 1 : 0;
        st->bar_count = 0;
        w = pass_word(pass_word_gen(w0) + 1u, cont, cont ? cur ^ 1 : cur, cont ? sweep_no + 1 : sweep_no);
        __threadfence();
        atomicExch(&st->pass_word, w);
        __threadfence();
        const unsigned long long tests = atomicAdd(&cnt[0], 0ull);
        const unsigned long long de = atomicAdd(&cnt[1], 0ull);
        const unsigned long long dv = atomicAdd(&cnt[2], 0ull);
        finish_pass(st, dv, de, tests);  // the same decision, from the same counts
        cnt[0] = cnt[1] = cnt[2] = 0;
      } else {
        uint32_t spins = 0;
        for (;;) {
          w = *((volatile unsigned long long *)&st->pass_word);
          if (pass_word_gen(w) != pass_word_gen(w0)) break;
          if (*((volatile int32_t *)&st->bar_abort)) {
            abort = true;
            break;
          }
          __nanosleep(64);
          if (++spins > p.spin_limit) {
            atomicCAS(&st->status, (int32_t)KZ_OK, (int32_t)KZ_ERR_TIMEOUT);
            atomicExch(&st->bar_abort, 1);
            abort = true;
            break;
          }
        }
      }
      __threadfence();
      s_word = abort ? 0ull : w;  // a cleared continue bit ends the kernel
    }
    __syncthreads();
    const unsigned long long w = s_word;
    if (!pass_word_cont(w)) break;
    cur = pass_word_cur(w);
    sweep_no = pass_word_sweeps(w);
    full = false;  // a finished pass leaves the buffers in step
  }
}

__global__ void begin_run_kernel(DevState *st, int64_t max_sweeps, int64_t passes0) {
  st->bar_count = 0;
  st->bar_gen = 0;
  st->pass_word = 0;
  st->bar_abort = 0;
  st->status = KZ_OK;
  st->cont = 1;
  st->sweeps = 0;
  st->passes = passes0;
  st->tests = 0;
  st->max_sweeps = max_sweeps;
  st->pass_dv = st->pass_de = st->pass_tests = 0;
  for (int i = 0; i < 2; i++) st->ppass[i][0] = st->ppass[i][1] = st->ppass[i][2] = 0;
  st->ticket = 0;
}

__global__ void reset_state_kernel(DevState *st) {
  st->cur = 0;
  st->status = KZ_OK;
  st->cont = 0;
  st->sweeps = st->passes = st->tests = 0;
  st->pass_dv = st->pass_de = st->pass_tests = 0;
  for (int i = 0; i < 2; i++) st->ppass[i][0] = st->ppass[i][1] = st->ppass[i][2] = 0;
  st->ticket = 0;
}

// ---------------------------------------------------------------------------
// kernel selection
// ---------------------------------------------------------------------------

typedef void (*SweepFn)(SweepArgs);

#define KZ_KMAX_LIST(X) X(4) X(8) X(12) X(16) X(20) X(24) X(28) X(32) X(48) X(64)

// One-pass and persistent kernels for k colours and a form (kmax receives the
// template width).  The two-plane form exists for k <= 32.
static SweepFn pick_sweep(int k, int form, int &kmax) {
#define KZ_CASE(K)                                                                              \
  if (k <= K) {                                                                                 \
    kmax = K;                                                                                   \
    if (form == kFormHalf) return bitset_sweep_kernel<K, kFormHalf>;                            \
    if (form == kFormTwo) return K <= 32 ? bitset_sweep_kernel<(K <= 32 ? K : 32), kFormTwo> : nullptr; \
    return bitset_sweep_kernel<K, kFormFull>;                                                   \
  }
  KZ_KMAX_LIST(KZ_CASE)
#undef KZ_CASE
  kmax = 0;
  return nullptr;
}

static SweepFn pick_persistent(int k, int form, int &kmax) {
#define KZ_CASE(K)                                                                                   \
  if (k <= K) {                                                                                      \
    kmax = K;                                                                                        \
    if (form == kFormHalf) return bitset_persistent_kernel<K, kFormHalf>;                            \
    if (form == kFormTwo) return K <= 32 ? bitset_persistent_kernel<(K <= 32 ? K : 32), kFormTwo> : nullptr; \
    return bitset_persistent_kernel<K, kFormFull>;                                                   \
  }
  KZ_KMAX_LIST(KZ_CASE)
#undef KZ_CASE
  kmax = 0;
  return nullptr;
}

// ---------------------------------------------------------------------------
// host entry points of the path
// ---------------------------------------------------------------------------

static int sm_count() {
  static std::mutex mu;
  static std::map<int, int> counts;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  const auto it = counts.find(dev);
  if (it != counts.end()) return it->second;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sms = sms > 0 ? sms : 1;
  counts[dev] = sms;
  return sms;
}

static kz_status ensure_plan(kz_graph g, int form, cudaStream_t s);

kz_status bitset_finish_load(kz_graph g, cudaStream_t s) {
  const int nb = (int)g->blocks.size();
  KZ_TRY(graph_alloc(g, &g->V0, (size_t)g->ldw, s));
  KZ_TRY(graph_alloc(g, &g->V[0], (size_t)g->ldw, s));
  KZ_TRY(graph_alloc(g, &g->V[1], (size_t)g->ldw, s));
  KZ_CUDA_TRY(cudaMemsetAsync(g->V0, 0, (size_t)g->ldw * 4, s));
  KZ_TRY(graph_alloc(g, &g->d_blocks, (size_t)std::max(nb, 1), s));
  if (nb) {
    KZ_TRY(h2d(g->d_blocks, g->blocks.data(), sizeof(BlockDesc) * nb, s));
    init_vlive_kernel<<<(nb + 255) / 256, 256, 0, s>>>(g->V0, g->d_blocks, nb, g->k);
    KZ_CUDA_TRY(cudaGetLastError());
  }
  KZ_TRY(graph_alloc(g, &g->d_coff, (size_t)g->k + 1, s));
  KZ_TRY(h2d(g->d_coff, g->coff.data(), sizeof(int32_t) * (g->k + 1), s));
  KZ_TRY(graph_alloc(g, &g->d_rounds, (size_t)g->k, s));
  KZ_TRY(h2d(g->d_rounds, g->rounds.data(), sizeof(int32_t) * g->k, s));
  KZ_TRY(cta_prepare(g, s));  // block-pair offsets and class block offsets (the unit list needs them)
  // the half-word plane-0 test pays off when 16 members of a class almost
  // always hold a common neighbour: dense graphs
  {
    double cross = 0, tot = 0;
    for (int c = 0; c < g->k; c++) {
      const double sz = g->coff[c + 1] - g->coff[c];
      cross += tot * sz;
      tot += sz;
    }
    const double density = cross > 0 ? (double)g->m / cross : 0.0;
    g->density = density;
    g->fast_half = density >= kFastHalfDensity;
    g->form = density >= kHalfDensity ? kFormHalf
              : (density < kTwoPlaneDensity && g->R >= 2 && g->k <= 32) ? kFormTwo
                                                                        : kFormFull;
  }
  // per-unit change tags, and the work split of the form the density picks
  if (g->k <= 64) {
    g->n_units = 0;
    for (int x = 0; x < nb; x++) g->n_units += std::max(1, nb - std::min(g->boff[g->blocks[x].c + 1], nb));
    if (g->n_units > INT32_MAX) return KZ_ERR_UNSUPPORTED;
    KZ_TRY(graph_alloc(g, &g->d_changed, (size_t)std::max<int64_t>(g->n_units, 1), s));
    KZ_CUDA_TRY(cudaMemsetAsync(g->d_changed, 0xff, (size_t)std::max<int64_t>(g->n_units, 1), s));
    KZ_TRY(ensure_plan(g, g->form, s));
  }
  KZ_TRY(graph_alloc(g, &g->A[0], (size_t)g->n * g->ldw, s));
  KZ_TRY(graph_alloc(g, &g->A[1], (size_t)g->n * g->ldw, s));
  KZ_TRY(graph_alloc(g, &g->v_sweep, (size_t)std::max(g->n, 1), s));
  if (!g->st) {
    KZ_TRY(graph_alloc(g, &g->st, 1, s));
    KZ_CUDA_TRY(cudaMemsetAsync(g->st, 0, sizeof(DevState), s));
  }
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
  g->ab_synced = true;  // both row buffers now equal the loaded graph
  return KZ_OK;
}

// Shared memory of a sweep kernel and its resident CTAs per SM.
// (Set up and queried once per kernel and device: the attribute persists.)
static kz_status kernel_fit(SweepFn fn, int kmax, int form, size_t &smem, int &per_sm) {
  static std::mutex mu;
  static std::map<std::tuple<const void *, int>, int> fitted;  // (kernel, device) -> CTAs per SM
  const int half_stride_words = (kmax / 2 + 3) / 4 * 4;
  const size_t warp_words = form == kFormTwo ? 2 * 32 * 2 * (size_t)kmax
                                              : 2 * 32 * (size_t)kmax + (form == kFormHalf ? 32 * half_stride_words : 0);
  smem = (size_t)cta_warps(kmax, form) * 4 * warp_words;
  int dev = 0;
  KZ_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_tuple((const void *)fn, dev);
  const auto it = fitted.find(key);
  if (it != fitted.end()) {
    per_sm = it->second;
    return KZ_OK;
  }
  // always raise the limit: the kernels' static shared memory comes on top
  KZ_CUDA_TRY(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  per_sm = 0;
  KZ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn,
                                                            cta_warps(kmax, form) * 32, smem));
  fitted[key] = per_sm;
  return KZ_OK;
}

// The grid of both sweep kernels of one form: one CTA per SM (every CTA
// resident at once, as the persistent kernel's grid barrier needs), and no
// more warps than units.
static kz_status sweep_grid_size(kz_graph g, int form, int &grid) {
  int kmax = 0, kmax2 = 0, per_a = 0, per_b = 0;
  size_t smem = 0;
  SweepFn fa = pick_persistent(g->k, form, kmax), fb = pick_sweep(g->k, form, kmax2);
  if (!fa || !fb) return KZ_ERR_ARG;
  KZ_TRY(kernel_fit(fa, kmax, form, smem, per_a));
  KZ_TRY(kernel_fit(fb, kmax2, form, smem, per_b));
  if (std::min(per_a, per_b) < 1) return KZ_ERR_UNSUPPORTED;
  const int w = cta_warps(kmax, form);
  const int64_t want = (std::max<int64_t>(g->n_units, 1) + w - 1) / w;
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count()));
  return KZ_OK;
}

// Builds the grid and the CTAs' unit ranges of one form, once per graph (the
// unit list itself is shared by the forms).
static kz_status ensure_plan(kz_graph g, int form, cudaStream_t s) {
  SweepPlan &pl = g->plan[form];
  if (pl.grid > 0) return KZ_OK;
  int grid = 0;
  KZ_TRY(sweep_grid_size(g, form, grid));
  std::vector<int32_t> unit_off, cta_begin;
  plan_units(g, grid, unit_off, cta_begin);
  const int nb = (int)g->blocks.size();
  if ((int64_t)unit_off[nb] != g->n_units) return KZ_ERR_INTERNAL;
  if (!g->d_units) {
    KZ_TRY(graph_alloc(g, &g->d_units, std::max<size_t>((size_t)g->n_units, 1), s));
    if (g->n_units > 0) {
      int32_t *d_off = nullptr;
      KZ_TRY(graph_alloc(g, &d_off, (size_t)nb + 1, s));
      KZ_TRY(h2d(d_off, unit_off.data(), sizeof(int32_t) * (nb + 1), s));
      const int ugrid = (int)std::min<int64_t>((g->n_units + 255) / 256, 8 * sm_count());
      fill_units_kernel<<<std::max(ugrid, 1), 256, 0, s>>>(g->d_units, d_off, g->d_blocks, g->d_boff, nb);
      KZ_CUDA_TRY(cudaGetLastError());
    }
  }
  KZ_TRY(graph_alloc(g, &pl.d_cta_begin, cta_begin.size(), s));
  KZ_TRY(h2d(pl.d_cta_begin, cta_begin.data(), sizeof(int32_t) * cta_begin.size(), s));
  pl.grid = grid;
  return KZ_OK;
}

static kz_status launch_config(kz_graph g, SweepFn fn, int kmax, int form, int &grid, size_t &smem,
                               int &threads) {
  int per_sm = 0;
  KZ_TRY(kernel_fit(fn, kmax, form, smem, per_sm));
  grid = g->plan[form].grid;
  threads = cta_warps(kmax, form) * 32;
  if (grid <= 0 || grid > std::max(per_sm, 1) * sm_count()) return KZ_ERR_INTERNAL;
  return KZ_OK;
}

static SweepArgs make_args(kz_graph g, int form) {
  const SweepPlan &pl = g->plan[form];
  SweepArgs a;
  a.blocks = g->d_blocks;
  a.units = g->d_units;
  a.cta_begin = pl.d_cta_begin;
  a.nb = (int32_t)g->blocks.size();
  a.k = g->k;
  a.ldw = g->ldw;
  a.rounds = g->d_rounds;
  a.boff = g->d_boff;
  a.changed = g->d_changed;
  a.fast_half = g->fast_half ? 1 : 0;
  a.slack = g->slack;
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
static kz_status build_loop_graph(kz_graph g, int64_t max_sweeps, int form) {
  int kmax = 0;
  SweepFn fn = pick_sweep(g->k, form, kmax);
  if (!fn) return KZ_ERR_ARG;
  int grid = 0, threads = 0;
  size_t smem = 0;
  KZ_TRY(launch_config(g, fn, kmax, form, grid, smem, threads));
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
  SweepArgs args = make_args(g, form);
  args.cond = handle;
  args.use_cond = 1;
  void *kargs[] = {&args};
  cudaKernelNodeParams kp;
  memset((void *)&kp, 0, sizeof(kp));
  kp.func = (void *)fn;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(threads);
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
  g->loop_form = form;
  g->loop_slack = g->slack;
  return KZ_OK;
}

// Builds (once per graph, form and sweep limit) an executable CUDA graph of
// one persistent run: the run-start kernel, then the cooperative sweep
// kernel.  One graph launch costs less than the two launches.
static kz_status build_run_graph(kz_graph g, int64_t max_sweeps, int form) {
  int kmax = 0;
  SweepFn fn = pick_persistent(g->k, form, kmax);
  if (!fn) return KZ_ERR_ARG;
  int grid = 0, threads = 0;
  size_t smem = 0;
  KZ_TRY(launch_config(g, fn, kmax, form, grid, smem, threads));
  cudaGraph_t graph = nullptr;
  KZ_CUDA_TRY(cudaGraphCreate(&graph, 0));
  cudaGraphNode_t bnode, knode;
  DevState *stp = g->st;
  int64_t ms = max_sweeps, p0 = 0;
  void *bargs[] = {&stp, &ms, &p0};
  cudaKernelNodeParams bp;
  memset((void *)&bp, 0, sizeof(bp));
  bp.func = (void *)begin_run_kernel;
  bp.gridDim = dim3(1);
  bp.blockDim = dim3(1);
  bp.kernelParams = bargs;
  cudaError_t e = cudaGraphAddKernelNode(&bnode, graph, nullptr, 0, &bp);
  SweepArgs args = make_args(g, form);
  void *kargs[] = {&args};
  cudaKernelNodeParams kp;
  memset((void *)&kp, 0, sizeof(kp));
  kp.func = (void *)fn;
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(threads);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = kargs;
  if (e == cudaSuccess) e = cudaGraphAddKernelNode(&knode, graph, &bnode, 1, &kp);
  if (e == cudaSuccess) {
    cudaLaunchAttributeValue v;
    memset((void *)&v, 0, sizeof(v));
    v.cooperative = 1;
    e = cudaGraphKernelNodeSetAttribute(knode, cudaLaunchAttributeCooperative, &v);
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  g->run_exec = exec;
  g->run_max_sweeps = max_sweeps;
  g->run_form = form;
  g->run_slack = g->slack;
  return KZ_OK;
}

// Asks the next pass to write every word of the next buffer (after anything
// but a sweep kernel wrote the rows).
static kz_status request_full_write(kz_graph g, cudaStream_t s) {
  KZ_CUDA_TRY(cudaMemsetAsync(&g->st->full_write, 1, sizeof(int32_t), s));
  return KZ_OK;
}

kz_status bitset_kernelize(kz_graph g, const kz_options &opt, cudaStream_t s) {
  int64_t max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : (int64_t)g->n + g->m + 1;
  int form = g->form;
  if (opt.plane0 == KZ_PLANE0_FULL) form = kFormFull;
  if (opt.plane0 == KZ_PLANE0_HALF) form = kFormHalf;
  if (opt.plane0 == KZ_PLANE0_TWO) form = g->R >= 2 && g->k <= 32 ? kFormTwo : kFormFull;
  if (g->n > 0) KZ_TRY(ensure_plan(g, form, s));
  if (!g->ab_synced) {
    KZ_TRY(request_full_write(g, s));
    g->ab_synced = true;
  }
  if (g->n > 0 && opt.use_graph == 1) {
    // every pass in one cooperative launch (grid fully resident) after the
    // run-start kernel.  A graph that fills the GPU launches both as one CUDA
    // graph (measured 2 us less on C2); a small one launches them directly
    // (a graph launch was slower there).
    if (g->plan[form].grid >= sm_count()) {
      if (g->run_exec && (g->run_max_sweeps != max_sweeps || g->run_form != form || g->run_slack != g->slack)) {
        cudaGraphExecDestroy(g->run_exec);
        g->run_exec = nullptr;
      }
      if (!g->run_exec) KZ_TRY(build_run_graph(g, max_sweeps, form));
      KZ_CUDA_TRY(cudaGraphLaunch(g->run_exec, s));
      return KZ_OK;
    }
    begin_run_kernel<<<1, 1, 0, s>>>(g->st, max_sweeps, 0);
    KZ_CUDA_TRY(cudaGetLastError());
    int kmax = 0;
    SweepFn fn = pick_persistent(g->k, form, kmax);
    if (!fn) return KZ_ERR_ARG;
    int grid = 0, threads = 0;
    size_t smem = 0;
    KZ_TRY(launch_config(g, fn, kmax, form, grid, smem, threads));
    SweepArgs args = make_args(g, form);
    void *kargs[] = {&args};
    KZ_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(threads), kargs, smem, s));
    return KZ_OK;
  }
  if (g->n > 0 && opt.use_graph == 2) {
    // one graph launch: run-start kernel, then the while node of sweep passes
    if (g->loop_exec && (g->loop_max_sweeps != max_sweeps || g->loop_form != form || g->loop_slack != g->slack)) {
      cudaGraphExecDestroy(g->loop_exec);
      g->loop_exec = nullptr;
    }
    if (!g->loop_exec) KZ_TRY(build_loop_graph(g, max_sweeps, form));
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
  SweepFn fn = pick_sweep(g->k, form, kmax);
  if (!fn) return KZ_ERR_ARG;
  int grid = 0, threads = 0;
  size_t smem = 0;
  KZ_TRY(launch_config(g, fn, kmax, form, grid, smem, threads));
  SweepArgs args = make_args(g, form);
  for (;;) {
    fn<<<grid, threads, smem, s>>>(args);
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
  // the caller may have changed the rows in place between passes
  KZ_TRY(request_full_write(g, s));
  g->ab_synced = false;
  int kmax = 0;
  SweepFn fn = pick_sweep(g->k, g->form, kmax);
  if (!fn) return KZ_ERR_ARG;
  int grid = 0, threads = 0;
  size_t smem = 0;
  KZ_TRY(launch_config(g, fn, kmax, g->form, grid, smem, threads));
  SweepArgs args = make_args(g, g->form);
  fn<<<grid, threads, smem, s>>>(args);
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
  SweepFn fn = pick_persistent(g->k, g->form, kmax);
  if (!fn) return KZ_ERR_ARG;
  int grid = 0, threads = 0;
  size_t smem = 0;
  KZ_TRY(launch_config(g, fn, kmax, g->form, grid, smem, threads));
  SweepArgs args = make_args(g, g->form);
  args.bar_extra = 1;
  args.spin_limit = spin_limit;
  void *kargs[] = {&args};
  KZ_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)fn, dim3(grid), dim3(threads), kargs, smem, s));
  return KZ_OK;
}

}  // namespace kz
