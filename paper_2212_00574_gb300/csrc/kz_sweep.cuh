// kz_sweep.cuh -- one work item of a Jacobi pass on the bitset rows (block X
// against a run of blocks Y of higher classes), shared by the single-graph
// sweep kernels and the batched persistent kernel.  Plane 0 of the Y rows is
// staged through a per-warp double buffer of asynchronous copies, so the next
// block's loads overlap the current block's tests; the hot loop only collects
// pairs that plane 0 leaves open, and those are recounted afterwards.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kz_internal.cuh"
#include "kz_rules.cuh"

namespace kz {

// What a work item needs to know about its graph.
struct GraphView {
  const BlockDesc *blocks;
  const int32_t *rounds;
  uint32_t *A0, *A1;  // ping-pong rows
  uint32_t *V0, *V1;  // ping-pong live words
  int32_t *v_sweep;
  int32_t k, ldw;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage plane 0 of the member rows of block Y (round_up(k, 4) words each,
// KMAX words apart) with asynchronous 16-byte copies.  Lane l copies chunk
// l % (KMAX / 4) of rows l / (KMAX / 4), l / (KMAX / 4) + 32 / (KMAX / 4), ...
// (compile-time divisions only).
template <int KMAX>
__device__ __forceinline__ void stage_block(const uint32_t *__restrict__ A, int ldw, const BlockDesc &Y, int kq4,
                                            uint32_t *buf, int lane) {
  constexpr int C = KMAX / 4;   // 16-byte chunks per staged row
  constexpr int RPI = 32 / C;   // rows per round of the warp
  const int rr = lane / C, q = lane - rr * C;
  if (rr < RPI && q < kq4) {
    const uint32_t *src = A + (int64_t)Y.base * ldw + 4 * q;
    uint32_t *dst = buf + 4 * q;
    for (int b = rr; b < Y.size; b += RPI) cp_async16(dst + b * KMAX, src + (int64_t)b * ldw);
  }
}

// Stage planes 0 and 1 of the member rows of block Y: the first
// round_up(2k, 4) words of each row at their own offsets, rows 2 KMAX words
// apart (the rows hold at least two planes).
template <int KMAX>
__device__ __forceinline__ void stage_block2(const uint32_t *__restrict__ A, int ldw, const BlockDesc &Y, int kq8,
                                             uint32_t *buf, int lane) {
  constexpr int C = KMAX / 2;   // 16-byte chunks per staged row
  constexpr int RPI = 32 / C;   // rows per round of the warp
  const int rr = lane / C, q = lane - rr * C;
  if (rr < RPI && q < kq8) {
    const uint32_t *src = A + (int64_t)Y.base * ldw + 4 * q;
    uint32_t *dst = buf + 4 * q;
    for (int b = rr; b < Y.size; b += RPI) cp_async16(dst + b * 2 * KMAX, src + (int64_t)b * ldw);
  }
}

struct PassCounters {
  unsigned long long tests = 0, de = 0, dv = 0;
};

// One work item of one Jacobi pass, executed by one warp.  `cur` is the
// graph's current ping-pong buffer, `sweep_no` its productive sweeps so far.
template <int KMAX>
__device__ __forceinline__ void sweep_item(const GraphView &p, const WorkItem item, int cur, int64_t sweep_no,
                                           uint32_t *buf0, uint32_t *buf1, PassCounters &pc) {
  const int lane = threadIdx.x & 31;
  const uint32_t *__restrict__ A = cur ? p.A1 : p.A0;
  uint32_t *__restrict__ An = cur ? p.A0 : p.A1;
  const uint32_t *__restrict__ Vc = cur ? p.V1 : p.V0;
  uint32_t *__restrict__ Vn = cur ? p.V0 : p.V1;
  const int k = p.k, ldw = p.ldw;
  const int kq4 = (k + 3) >> 2;
  {
    const BlockDesc X = p.blocks[item.x];
    const int cu = X.c;
    const bool valid_u = lane < X.size;
    const int u = X.base + lane;
    const uint32_t *rowu = A + (int64_t)(valid_u ? u : X.base) * ldw;
    // start staging the first Y block before anything else
    const int yn = item.y1 - item.y0;
    BlockDesc Yn;
    if (yn > 0) {
      Yn = p.blocks[item.y0];
      stage_block<KMAX>(A, ldw, Yn, kq4, buf0, lane);
    }
    cp_async_commit();
    uint32_t Fu[KMAX];
    load_plane0<KMAX>(Fu, rowu, k, valid_u);
    if (item.vflag) {
      const int wx = X.r * k + cu;
      const uint32_t vword = Vc[wx];
      const bool live = valid_u && ((vword >> lane) & 1u);
      int cnt = plane0_vertex_cover<KMAX>(Fu, k, cu);
      if (live && cnt < k - 1) cnt = exact_vertex_cover_row(rowu, k, p.rounds, cu);
      const bool fail = live && cnt < k - 1;
      const uint32_t failmask = __ballot_sync(0xffffffffu, fail);
      if (lane == 0) {
        Vn[wx] = vword & ~failmask;
        pc.dv += __popc(failmask);
      }
      if (fail && p.v_sweep) p.v_sweep[u] = (int32_t)(sweep_no + 1);
    }
    uint32_t P[KMAX];
    int prev_cv = -1;
    uint32_t adj_next = (yn > 0 && valid_u) ? A[(int64_t)u * ldw + Yn.r * k + Yn.c] : 0u;
    uint32_t col_next = (yn > 0 && lane < Yn.size) ? A[(int64_t)(Yn.base + lane) * ldw + X.r * k + cu] : 0u;
    for (int i = 0; i < yn; i++) {
      const BlockDesc Y = Yn;
      const uint32_t adjw = adj_next, colw = col_next;
      uint32_t *sv = (i & 1) ? buf1 : buf0;
      if (i + 1 < yn) {
        Yn = p.blocks[item.y0 + i + 1];
        stage_block<KMAX>(A, ldw, Yn, kq4, (i & 1) ? buf0 : buf1, lane);
        adj_next = valid_u ? A[(int64_t)u * ldw + Yn.r * k + Yn.c] : 0u;
        col_next = lane < Yn.size ? A[(int64_t)(Yn.base + lane) * ldw + X.r * k + cu] : 0u;
      }
      cp_async_commit();
      cp_async_wait<1>();
      __syncwarp();
      const int cv = Y.c;
      if (cv != prev_cv) {
        pair_mask<KMAX>(P, k, cu, cv);
        prev_cv = cv;
      }
      pc.tests += __popc(adjw);
      const uint32_t open = plane0_unsettled<KMAX>(Fu, P, sv, adjw, k);
      uint32_t del = 0;
      if (open)
        del = recount_unsettled(rowu, sv, KMAX, A + (int64_t)Y.base * ldw, ldw, open, k, cu, cv, p.rounds, 0);
      const int wy = Y.r * k + cv;
      if (valid_u) An[(int64_t)u * ldw + wy] = adjw & ~del;
      pc.de += __popc(del);
      const uint32_t delT = transpose_deletions(del);
      if (lane < Y.size) An[(int64_t)(Y.base + lane) * ldw + X.r * k + cu] = colw & ~delT;
      __syncwarp();
    }
    cp_async_wait<0>();
    __syncwarp();
  }
}


}  // namespace kz
