// kz_tensor.cu -- tensor-core form of the edge rule (thesis Section 4.2).
//
// For every colour class c, S_c = A[:, C_c] * A[:, C_c]^T counts the common
// neighbours of every vertex pair inside class c.  The edge rule asks, per
// live edge {u,v}, how many classes have S_c(u,v) > 0 (classes col(u) and
// col(v) always give 0: no neighbour of u has u's colour).  An edge fails when
// fewer than q-2 classes do (q: the clique size sought, k in the thesis).
//
// Operand layout: the live bitset rows are expanded into an E4M3 0/1 byte
// matrix with one 32-byte K-step per 32-bit block word (class c is the run of
// K-steps of its blocks, so S_c is a K-loop over those steps only).  The
// matrix is stored half-step-major: M[h][x][0..15] holds bits 16(h%2) ..
// 16(h%2)+15 of block word h/2 of row x (0x38 = E4M3 1.0 for a set bit), so
// the 128 rows of a tile form one contiguous 2048-byte run per half-step.
// A BF16 variant (kind::f16, 0x3F80 = 1.0) spends two bytes per vertex: one
// MMA step then covers 16 vertices (half a block word) in the same 32 bytes
// per row, so the layout, boxes and descriptors are the same and a class
// takes twice the steps.
// One A-operand TMA box (8 half-steps x 2048 bytes, read as 8-byte elements so that
// the box's inner extent is the whole contiguous run) then lands in shared
// memory as four consecutive canonical no-swizzle K-major MMA operands:
// 8-row x 16-byte core matrices 128 bytes apart along M/N and 2048 bytes
// apart along K, one K-step every 4096 bytes.  The B operand's box spans two
// such tiles, so its 256 rows lie at one uniform stride (K halves 4096 bytes
// apart).  Large boxes matter: the TMA probe measures 35 bytes per clock and
// SM for 4 KB boxes against 66 for 16 KB boxes with the same bytes in flight.
//
// Kernel (one CTA per SM, persistent over tiles of 128 A rows x 256 B rows;
// the MMA probe measures one CTA's M = 128, N = 256 stream at the full fp8
// rate, an N = 128 stream at half of it):
//   warp 0      TMA producer: fills a ring of pipeline stages (four K-steps
//               of both operands, one box each; a class's last partial stage
//               one box per K-step) as soon as the MMAs free them;
//   warp 1      MMA issuer: one thread issues tcgen05.mma.kind::f8f6f4
//               (kind::f16 for BF16; M = 128, N = 256, 32 bytes of K per
//               row, fp32 accumulation in TMEM, exact for 0/1 products)
//               over a class's K-steps, alternating
//               between two TMEM accumulators (all 512 columns) so that the
//               next class runs while the previous one is read;
//   warps 2-9   epilogue: tcgen05.ld of the class's counts, one 8-bit
//               counter per pair of classes with a non-zero count; after the
//               tile's last class, live edges below q-2 are marked in a
//               deletion bitmap.
// A row kernel then applies the vertex rule and the edge deletions.  Every
// mbarrier wait is bounded (wall clock); a wait that runs out records
// KZ_ERR_TIMEOUT, the other roles stop at their next wait, the producer and
// the MMA issuer wait (bounded) for their copies and MMAs in flight, and the
// CTA frees its tensor memory before it returns.
#include <cuda.h>  // CUtensorMap and its enums (the encoder comes from the runtime's entry-point query)
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kz_internal.cuh"
#include "kz_rules.cuh"

namespace kz {
namespace tensor {

constexpr int kTile = 128;                       // A rows per tile (MMA M)
constexpr int kTileN = 256;                      // B rows per tile (MMA N)
constexpr int kStep = 32;                        // bytes (E4M3 elements) per K-step
constexpr int kStepA = kTile * kStep;            // A operand, one K-step: 4 KB
constexpr int kStepB = kTileN * kStep;           // B operand, one K-step: 8 KB
constexpr int kStageSteps = 4;                   // K-steps per pipeline stage (class runs are chunked)
constexpr int kStages = 4;                       // pipeline depth
constexpr int kABytes = kStageSteps * kStepA;    // 16 KB
constexpr int kStageBytes = kStageSteps * (kStepA + kStepB);  // 48 KB
constexpr int kEpiWarps = 8;                     // two per TMEM lane quarter, 128 columns each
constexpr int kThreads = (2 + kEpiWarps) * 32;
constexpr uint32_t kAccCols = kTileN;            // fp32 columns per accumulator
constexpr uint32_t kTmemCols = 2 * kAccCols;     // double-buffered accumulator: all 512 columns
constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + 1024;  // + alignment slack
constexpr uint64_t kWaitNs = 4000000000ull;      // 4 s per wait before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor of one K-step of a K-major, no-swizzle
// operand as the TMA boxes lay it out: core matrices (8 rows x 16 bytes) 128
// bytes apart along M/N (stride byte offset) and rows x 16 bytes apart along
// K (leading byte offset: the second 16-byte half of the K-step follows all
// rows of the first).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t rows) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
  d |= (uint64_t)((rows * 16u) >> 4) << 16;         // leading byte offset (K direction)
  d |= (uint64_t)(128u >> 4) << 32;                 // stride byte offset (8-row groups)
  d |= (uint64_t)1 << 46;                           // descriptor version
  // base offset 0, relative LBO mode, no swizzle (bits 61-63 = 0)
  return d;
}

// Instruction descriptor: dense, D = f32, both operands K-major, N = 256,
// M = 128; A = B = E4M3 (kind::f8f6f4, format code 0) or A = B = BF16
// (kind::f16, format code 1).
template <bool BF16>
__device__ __forceinline__ uint32_t make_idesc() {
  const uint32_t fmt = BF16 ? 1u : 0u;
  uint32_t d = 0;
  d |= 1u << 4;                        // D format f32
  d |= fmt << 7;                       // A format
  d |= fmt << 10;                      // B format
  d |= ((uint32_t)kTileN >> 3) << 17;  // N >> 3
  d |= ((uint32_t)kTile >> 4) << 24;   // M >> 4
  return d;
}

__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// The same MMA on BF16 0/1 operands: K = 16 elements, the same 32 bytes per
// operand row as one E4M3 K-step.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Arrive on `mbar` once every tcgen05 operation this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// Arrive and announce `bytes` of asynchronous copies that complete this phase.
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// try_wait with a suspend-time hint: a waiting thread sleeps in hardware until
// the phase completes (or 1 ms passes) instead of polling shared memory.
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000000;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// TMA loads of the byte matrix (x counts 8-byte elements: 2 per row).
// A operand: 2-D map {2 n_pad, 2 ksteps}; box of 128 rows and 2 or 8
// half-steps (one K-step or a whole stage).  Half-steps past the end of the
// matrix read as zero; those of the next class are loaded but not used.
__device__ __forceinline__ void tma_load_a(uint32_t dst, const CUtensorMap *map, uint32_t mbar, int32_t row0,
                                           int32_t half0) {
  const int32_t x = row0 * 2;
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar), "r"(x), "r"(half0)
      : "memory");
}
// B operand: 3-D map {256 elements (one 128-row tile), n_pad / 128 tiles,
// 2 ksteps}; box of 2 tiles (256 rows, contiguous in shared memory) and 2 or
// 8 half-steps.
__device__ __forceinline__ void tma_load_b(uint32_t dst, const CUtensorMap *map, uint32_t mbar, int32_t tile0,
                                           int32_t half0) {
  const int32_t x = 0;
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar), "r"(x), "r"(tile0), "r"(half0)
      : "memory");
}

// Whole-warp wait for the completion of the phase of parity `parity`.  Every
// lane polls; the decision to give up is lane 0's, so the warp stays
// converged.  Returns false when another role has given up, or after kWaitNs
// (then records KZ_ERR_TIMEOUT and raises the CTA's abort flag).
__device__ __noinline__ bool warp_wait(uint32_t mbar, uint32_t parity, volatile int *abort_flag, int32_t *status) {
  const uint64_t t0 = globaltimer();
  for (uint32_t i = 0;; i++) {
    const bool ok = mbar_try_wait_hint(mbar, parity);
    if (__all_sync(0xffffffffu, ok)) return true;
    if ((i & 15u) == 15u) {
      int stop = 0;
      if ((threadIdx.x & 31) == 0) {
        if (*abort_flag) {
          stop = 1;
        } else if (globaltimer() - t0 > kWaitNs || i > (1u << 30)) {
          *abort_flag = 1;
          if (status) atomicCAS(status, 0, (int32_t)KZ_ERR_TIMEOUT);
          stop = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    }
  }
}

// Single-thread bounded wait used when draining work in flight on the way
// out (ignores the abort flag: copies and MMAs already issued must land
// before the CTA's shared and tensor memory go away).
__device__ __noinline__ void drain_wait(uint32_t mbar, uint32_t parity, int32_t *status) {
  const uint64_t t0 = globaltimer();
  for (uint32_t i = 0; !mbar_try_wait(mbar, parity); i++) {
    if ((i & 15u) == 15u && (globaltimer() - t0 > kWaitNs || i > (1u << 30))) {
      if (status) atomicCAS(status, 0, (int32_t)KZ_ERR_TIMEOUT);
      return;
    }
  }
}

// 32 consecutive fp32 columns of this thread's TMEM lane (no wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

struct TensorArgs {
  int32_t n, k;
  int32_t q;               // clique size sought (k for the thesis's rules)
  const int32_t *cls_step; // k + 1: first K-step of each class
  const uint32_t *A;       // current rows (adjacency bits)
  int32_t ldw;
  const int32_t *vinfo;    // n_pad: (word << 5 | bit) of vertex x in any row, -1 past n
  uint32_t *Edel;          // deletion bitmap, rows x ldw (zeroed)
  const int2 *tiles;       // (I, J): A rows 128 I .., B rows 256 J .., 2 J + 1 >= I
  int32_t n_tiles;
  unsigned long long *counts;  // [0] failing edges [1] live edges tested
  int32_t *status;
};

// Accumulate the non-zero flags of 32 fp32 counts into 8-bit counters: a
// count is a non-negative float, so its bit pattern is non-zero exactly when
// the count is.
__device__ __forceinline__ void count_nonzero(const uint32_t (&r)[32], uint32_t *cnt) {
#pragma unroll
  for (int j = 0; j < 32; j++) cnt[j >> 2] += min(r[j], 1u) << ((j & 3) * 8);
}

// The tensor maps of the byte matrix: a whole stage or one K-step, per operand.
struct TensorMaps {
  CUtensorMap a_stage, a_step, b_stage, b_step;
};

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) tensor_edge_kernel(const __grid_constant__ TensorMaps maps,
                                                                  TensorArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[2 * kStages + 5];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag_s;
  volatile int *abort_flag = &abort_flag_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = smem_u32(bars);
  // barrier addresses: full[s], empty[s], acc_full[b], acc_empty[b], drain
  const uint32_t full0 = bar0, empty0 = bar0 + 8 * kStages, accf0 = bar0 + 16 * kStages;
  const uint32_t acce0 = accf0 + 16, drain = accf0 + 32;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; s++) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, kEpiWarps);
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag_s = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    int stage = 0;
    uint32_t ph = 0;
    uint32_t filled = 0, fill_parity = 0;  // per stage: issued at least once / parity of its last fill
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
      const int I = a.tiles[t].x, J = a.tiles[t].y;
      for (int c = 0; c < a.k; c++) {
        const int sb = a.cls_step[c], se = a.cls_step[c + 1];
        for (int s0 = sb; s0 < se; s0 += kStageSteps) {
          const int ns = min(kStageSteps, se - s0);
          if (!warp_wait(empty0 + 8 * stage, ph ^ 1u, abort_flag, a.status)) goto producer_done;
          if (lane == 0) {
            const uint32_t fb = full0 + 8 * stage;
            const uint32_t sA = sbase + stage * kStageBytes, sB = sA + kABytes;
            if (ns == kStageSteps) {
              mbar_expect_tx(fb, (uint32_t)kStageBytes);
              tma_load_a(sA, &maps.a_stage, fb, I * kTile, 2 * s0);
              tma_load_b(sB, &maps.b_stage, fb, 2 * J, 2 * s0);
            } else {  // a class's last, partial stage: one box per K-step
              mbar_expect_tx(fb, (uint32_t)(ns * (kStepA + kStepB)));
              for (int j = 0; j < ns; j++) {
                tma_load_a(sA + j * kStepA, &maps.a_step, fb, I * kTile, 2 * (s0 + j));
                tma_load_b(sB + j * kStepB, &maps.b_step, fb, 2 * J, 2 * (s0 + j));
              }
            }
          }
          __syncwarp();
          filled |= 1u << stage;
          fill_parity = (fill_parity & ~(1u << stage)) | (ph << stage);
          if (++stage == kStages) {
            stage = 0;
            ph ^= 1u;
          }
        }
      }
    }
  producer_done:
    // every fill issued must land before the shared memory is released
    if (lane == 0)
      for (int s = 0; s < kStages; s++)
        if ((filled >> s) & 1u) drain_wait(full0 + 8 * s, (fill_parity >> s) & 1u, a.status);
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = make_idesc<BF16>();
    int stage = 0, abuf = 0;
    uint32_t ph = 0, empty_ph = 0;  // bit b: parity of accumulator b's next release
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
      for (int c = 0; c < a.k; c++) {
        const int sb = a.cls_step[c], se = a.cls_step[c + 1];
        if (se <= sb) continue;
        // the epilogue must have read this accumulator's previous class
        if (!warp_wait(acce0 + 8 * abuf, ((empty_ph >> abuf) & 1u) ^ 1u, abort_flag, a.status)) goto mma_done;
        tc_fence_after();
        for (int s0 = sb; s0 < se; s0 += kStageSteps) {
          const int ns = min(kStageSteps, se - s0);
          if (!warp_wait(full0 + 8 * stage, ph, abort_flag, a.status)) goto mma_done;
          tc_fence_after();
          if (lane == 0) {
            const uint32_t sA = sbase + stage * kStageBytes, sB = sA + kABytes;
            for (int j = 0; j < ns; j++) {
              const uint64_t da = make_desc(sA + j * kStepA, kTile), db = make_desc(sB + j * kStepB, kTileN);
              const uint32_t acc = (s0 > sb || j > 0) ? 1u : 0u;
              if constexpr (BF16) mma_bf16(tmem + (uint32_t)abuf * kAccCols, da, db, idesc, acc);
              else mma_f8(tmem + (uint32_t)abuf * kAccCols, da, db, idesc, acc);
            }
            mma_commit(empty0 + 8 * stage);  // stage free once these MMAs have read it
          }
          __syncwarp();
          if (++stage == kStages) {
            stage = 0;
            ph ^= 1u;
          }
        }
        if (lane == 0) mma_commit(accf0 + 8 * abuf);  // class complete in this accumulator
        __syncwarp();
        empty_ph ^= 1u << abuf;
        abuf ^= 1;
      }
    }
  mma_done:
    // every MMA issued must finish before the tensor memory is released
    if (lane == 0) {
      mma_commit(drain);
      drain_wait(drain, 0u, a.status);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue ----------------
    const int q = warp & 3;              // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;    // 128-column half of the tile
    const int row = q * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
    int abuf = 0;
    uint32_t full_ph = 0;  // bit b: parity of accumulator b's next class
    unsigned long long my_fail = 0, my_tests = 0;
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
      const int I = a.tiles[t].x, J = a.tiles[t].y;
      uint32_t cnt[32];  // 128 column counters, 8 bits each
#pragma unroll
      for (int i = 0; i < 32; i++) cnt[i] = 0;
      for (int c = 0; c < a.k; c++) {
        const int sb = a.cls_step[c], se = a.cls_step[c + 1];
        if (se <= sb) continue;
        if (!warp_wait(accf0 + 8 * abuf, (full_ph >> abuf) & 1u, abort_flag, a.status)) goto epilogue_done;
        tc_fence_after();
        const uint32_t col0 = (uint32_t)abuf * kAccCols + (uint32_t)(half * 128);
        uint32_t r0[32], r1[32];
        tmem_ld32(tmem + lane_addr + col0, r0);
        tmem_ld32(tmem + lane_addr + col0 + 32, r1);
        tmem_wait_ld();
        count_nonzero(r0, cnt);
        count_nonzero(r1, cnt + 8);
        tmem_ld32(tmem + lane_addr + col0 + 64, r0);
        tmem_ld32(tmem + lane_addr + col0 + 96, r1);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acce0 + 8 * abuf);  // accumulator free for the class after next
        full_ph ^= 1u << abuf;
        abuf ^= 1;
        count_nonzero(r0, cnt + 16);
        count_nonzero(r1, cnt + 24);
      }
      // live edges (u, v) of this thread's row and column half, u < v, in two
      // groups of 64 columns: the adjacency bits are gathered with independent
      // loads (the position of every column vertex in a row comes from one
      // table), then the tests and failures are whole-mask operations
      const int u = I * kTile + row;
      if (u < a.n) {
        const uint32_t *rowu = a.A + (int64_t)u * a.ldw;
        const int wu = a.vinfo[u];
#pragma unroll
        for (int g = 0; g < 2; g++) {
          // columns whose pair covers fewer than q-2 classes
          uint64_t low = 0;
#pragma unroll
          for (int j = 0; j < 64; j++)
            low |= (uint64_t)((int)((cnt[16 * g + (j >> 2)] >> ((j & 3) * 8)) & 0xFFu) < a.q - 2) << j;
          const int base = J * kTileN + half * 128 + g * 64;
          const int4 *vi4 = reinterpret_cast<const int4 *>(a.vinfo + base);
          uint64_t adj = 0;
#pragma unroll
          for (int q4 = 0; q4 < 16; q4++) {
            const int4 w4 = vi4[q4];
            const int w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int e = 0; e < 4; e++)
              if (w[e] >= 0) adj |= (uint64_t)((rowu[w[e] >> 5] >> (w[e] & 31)) & 1u) << (4 * q4 + e);
          }
          const uint64_t upper = u < base ? ~0ull : (u - base >= 63 ? 0ull : ~0ull << (u - base + 1));
          const uint64_t live = adj & upper;
          my_tests += (unsigned long long)__popcll(live);
          uint64_t fail = live & low;
          my_fail += (unsigned long long)__popcll(fail);
          while (fail) {
            const int j = __ffsll((long long)fail) - 1;
            fail &= fail - 1;
            const int v = base + j;
            const int wv = a.vinfo[v];
            atomicOr(&a.Edel[(int64_t)u * a.ldw + (wv >> 5)], 1u << (wv & 31));
            atomicOr(&a.Edel[(int64_t)v * a.ldw + (wu >> 5)], 1u << (wu & 31));
          }
        }
      }
    }
  epilogue_done:
    for (int o = 16; o > 0; o >>= 1) {
      my_fail += __shfl_down_sync(0xffffffffu, my_fail, o);
      my_tests += __shfl_down_sync(0xffffffffu, my_tests, o);
    }
    if (lane == 0) {
      if (my_fail) atomicAdd(&a.counts[0], my_fail);
      if (my_tests) atomicAdd(&a.counts[1], my_tests);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Operand matrix from the current rows, half-step-major (see the top of this
// file): thread t writes both 16-byte halves of MMA step s = t / n_pad of row
// x = t % n_pad, so a warp's stores are contiguous.  E4M3: one step is a
// whole 32-bit block word, step_word[s] = its index r * k + c in the row,
// one byte per vertex (0x38 = 1.0).  BF16: one step is half a block word,
// step_word[s] = 2 (r * k + c) + half, two bytes per vertex (0x3F80 = 1.0).
template <bool BF16>
__global__ void expand_kernel(const uint32_t *__restrict__ A, int32_t n, int32_t n_pad, int32_t ldw,
                              const int32_t *__restrict__ step_word, int32_t ksteps, uint8_t *__restrict__ M) {
  const int64_t total = (int64_t)n_pad * ksteps;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = (int32_t)(t / n_pad);
    const int32_t x = (int32_t)(t - (int64_t)s * n_pad);
    const int32_t sw = step_word[s];
    const int32_t wi = BF16 ? (sw >> 1) : sw;
    const uint32_t word = x < n ? __ldg(A + (int64_t)x * ldw + wi) : 0u;
    uint32_t out[8];
    if constexpr (BF16) {
      const uint32_t bits = (sw & 1) ? (word >> 16) : (word & 0xFFFFu);
#pragma unroll
      for (int q = 0; q < 8; q++)
        out[q] = (((bits >> (2 * q)) & 1u) ? 0x3F80u : 0u) | (((bits >> (2 * q + 1)) & 1u) ? 0x3F800000u : 0u);
    } else {
#pragma unroll
      for (int q = 0; q < 8; q++) {
        // bits 4q .. 4q+3 to bytes: bit j of the nibble lands on bit 8j of the product
        const uint32_t nib = (word >> (4 * q)) & 0xFu;
        out[q] = ((nib * 0x00204081u) & 0x01010101u) * 0x38u;
      }
    }
    uint4 *lo = reinterpret_cast<uint4 *>(M + ((int64_t)(2 * s) * n_pad + x) * 16);
    uint4 *hi = reinterpret_cast<uint4 *>(M + ((int64_t)(2 * s + 1) * n_pad + x) * 16);
    *lo = make_uint4(out[0], out[1], out[2], out[3]);
    *hi = make_uint4(out[4], out[5], out[6], out[7]);
  }
}

// Vertex rule and application of the marked edge deletions: next rows =
// current rows minus the deletion bitmap; next live words; pass counters.
__global__ void tensor_commit_kernel(const uint32_t *__restrict__ A, uint32_t *__restrict__ An,
                                     uint32_t *__restrict__ Edel, const uint32_t *__restrict__ V,
                                     uint32_t *__restrict__ Vn, int32_t n, int32_t ldw, int32_t k, int32_t q,
                                     int32_t R,
                                     const int32_t *__restrict__ col, const int32_t *__restrict__ coff,
                                     const int32_t *__restrict__ rounds, const BlockDesc *__restrict__ blocks,
                                     int32_t nb, int32_t *__restrict__ v_sweep, DevState *st,
                                     unsigned long long *counts) {
  const int lane = threadIdx.x & 31;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t sweep_no = st->sweeps;
  for (int64_t t = tid; t < (int64_t)n * ldw; t += stride) {
    const uint32_t d = Edel[t];
    An[t] = A[t] & ~d;
    if (d) Edel[t] = 0u;
  }
  // vertex rule: one warp per block of 32 vertices
  const int64_t warp0 = tid >> 5, warps = stride >> 5;
  unsigned long long dv = 0;
  for (int64_t x = warp0; x < nb; x += warps) {
    const BlockDesc X = blocks[x];
    const int wx = X.r * k + X.c;
    const uint32_t vword = V[wx];
    const bool valid = lane < X.size;
    const int u = X.base + lane;
    const bool live = valid && ((vword >> lane) & 1u);
    int cnt = live ? exact_vertex_cover_row(A + (int64_t)u * ldw, k, rounds, X.c) : 0;
    const bool fail = live && cnt < q - 1;
    const uint32_t failmask = __ballot_sync(0xffffffffu, fail);
    if (lane == 0) {
      Vn[wx] = vword & ~failmask;
      dv += __popc(failmask);
    }
    if (fail && v_sweep) v_sweep[u] = (int32_t)(sweep_no + 1);
  }
  for (int o = 16; o > 0; o >>= 1) dv += __shfl_down_sync(0xffffffffu, dv, o);
  if (lane == 0 && dv) atomicAdd(&counts[2], dv);
}

__global__ void tensor_finish_kernel(DevState *st, unsigned long long *counts) {
  finish_pass(st, counts[2], counts[0], counts[1]);
  counts[0] = counts[1] = counts[2] = 0;
}

}  // namespace tensor

using namespace tensor;

static int sms_t() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}

// The driver's tensor-map encoder, found once through the runtime (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

void *tensor_map_encoder() {
  static void *fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = p;
  }
  return fn;
}

static EncodeTiledFn encode_tiled() { return reinterpret_cast<EncodeTiledFn>(tensor_map_encoder()); }

// Per-graph buffers of the tensor path (allocated on first use).
struct TensorBufs {
  uint8_t *M = nullptr;
  int32_t n_pad = 0, ksteps = 0;
  int32_t *cls_step = nullptr;
  int32_t *step_word = nullptr;
  int32_t *col = nullptr;
  int32_t *vinfo = nullptr;
  uint32_t *Edel = nullptr;
  int2 *tiles = nullptr;
  int32_t n_tiles = 0;
  unsigned long long *counts = nullptr;
  TensorMaps maps;
};

// Buffers per operand precision (0 E4M3, 1 BF16), built on first use.
struct TensorState {
  TensorBufs *by[2] = {nullptr, nullptr};
};

static kz_status tensor_prepare(kz_graph g, TensorBufs &b, bool bf16, cudaStream_t s) {
  b.n_pad = (g->n + kTileN - 1) / kTileN * kTileN;
  // MMA steps per class: one per block word (E4M3), two (BF16: 16 vertices
  // of two bytes fill the 32 bytes per row of one MMA)
  const int per = bf16 ? 2 : 1;
  std::vector<int32_t> cs((size_t)g->k + 1, 0);
  for (int c = 0; c < g->k; c++) cs[c + 1] = cs[c] + per * g->rounds[c];
  b.ksteps = std::max(cs[g->k], 1);
  std::vector<int32_t> sw((size_t)b.ksteps, 0);
  for (int c = 0; c < g->k; c++)
    for (int r = 0; r < g->rounds[c]; r++)
      for (int h = 0; h < per; h++) sw[cs[c] + per * r + h] = bf16 ? 2 * (r * g->k + c) + h : r * g->k + c;
  const size_t mbytes = (size_t)b.n_pad * b.ksteps * kStep;
  KZ_TRY(graph_alloc(g, &b.M, mbytes, s));
  if (reinterpret_cast<uintptr_t>(b.M) % 16 != 0) return KZ_ERR_CUDA;  // TMA needs a 16-byte aligned base
  KZ_TRY(graph_alloc(g, &b.cls_step, (size_t)g->k + 1, s));
  KZ_CUDA_TRY(cudaMemcpyAsync(b.cls_step, cs.data(), sizeof(int32_t) * (g->k + 1), cudaMemcpyHostToDevice, s));
  KZ_TRY(graph_alloc(g, &b.step_word, sw.size(), s));
  KZ_CUDA_TRY(cudaMemcpyAsync(b.step_word, sw.data(), sizeof(int32_t) * sw.size(), cudaMemcpyHostToDevice, s));
  std::vector<int32_t> col_new((size_t)std::max(g->n, 1));
  for (int c = 0; c < g->k; c++)
    for (int x = g->coff[c]; x < g->coff[c + 1]; x++) col_new[x] = c;
  KZ_TRY(graph_alloc(g, &b.col, col_new.size(), s));
  KZ_CUDA_TRY(cudaMemcpyAsync(b.col, col_new.data(), sizeof(int32_t) * col_new.size(), cudaMemcpyHostToDevice, s));
  std::vector<int32_t> vinfo((size_t)b.n_pad, -1);
  for (int c = 0; c < g->k; c++)
    for (int x = g->coff[c]; x < g->coff[c + 1]; x++) {
      const int ix = x - g->coff[c];
      vinfo[x] = (((ix >> 5) * g->k + c) << 5) | (ix & 31);
    }
  KZ_TRY(graph_alloc(g, &b.vinfo, vinfo.size(), s));
  KZ_CUDA_TRY(cudaMemcpyAsync(b.vinfo, vinfo.data(), sizeof(int32_t) * vinfo.size(), cudaMemcpyHostToDevice, s));
  KZ_TRY(graph_alloc(g, &b.Edel, (size_t)g->n * g->ldw, s));
  KZ_CUDA_TRY(cudaMemsetAsync(b.Edel, 0, (size_t)g->n * g->ldw * 4, s));
  // Tiles (I, J): A rows 128 I .. 128 I + 127 against B rows 256 J ..
  // 256 J + 255, for every J that holds a column above row 128 I (2 J + 1 >=
  // I).  They run in super-blocks of 2S x S tiles (2 S^2 about the number of
  // SMs): CTA b takes tiles b, b + grid, ..., so the tiles in flight at one
  // time lie in about one super-block, whose rows' K-steps are read from HBM
  // once and then shared through L2 by the CTAs that stream the same K-steps
  // at about the same time.
  const int TI = b.n_pad / kTile, TJ = b.n_pad / kTileN;
  int S = 1;
  while (2 * (S + 1) * (S + 1) <= sms_t()) S++;
  std::vector<int2> tiles;
  for (int P = 0; P < TI; P += 2 * S)
    for (int Q = P / 2 / S * S; Q < TJ; Q += S)
      for (int i = P; i < std::min(P + 2 * S, TI); i++)
        for (int j = std::max(i / 2, Q); j < std::min(Q + S, TJ); j++) tiles.push_back(make_int2(i, j));
  b.n_tiles = (int32_t)tiles.size();
  KZ_TRY(graph_alloc(g, &b.tiles, std::max<size_t>(tiles.size(), 1), s));
  if (!tiles.empty())
    KZ_CUDA_TRY(cudaMemcpyAsync(b.tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, s));
  KZ_TRY(graph_alloc(g, &b.counts, 4, s));
  KZ_CUDA_TRY(cudaMemsetAsync(b.counts, 0, 32, s));
  // M as 8-byte elements.  A operand: 2-D {2 n_pad per half-step plane,
  // 2 ksteps planes}, boxes of 128 rows.  B operand: 3-D {256 elements (a
  // 128-row tile), n_pad / 128 tiles, 2 ksteps planes}, boxes of two tiles,
  // so 256 rows land contiguously.  Stage boxes hold 8 half-steps (large
  // boxes keep the TMA unit's per-copy cost small), step boxes 2.
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return KZ_ERR_UNSUPPORTED;
  std::memset(&b.maps, 0, sizeof(b.maps));
  const cuuint64_t dims_a[2] = {(cuuint64_t)2 * b.n_pad, (cuuint64_t)2 * b.ksteps};
  const cuuint64_t strides_a[1] = {(cuuint64_t)b.n_pad * 16};
  const cuuint64_t dims_b[3] = {(cuuint64_t)2 * kTile, (cuuint64_t)b.n_pad / kTile, (cuuint64_t)2 * b.ksteps};
  const cuuint64_t strides_b[2] = {(cuuint64_t)2 * kTile * 8, (cuuint64_t)b.n_pad * 16};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int w = 0; w < 2; w++) {
    const cuuint32_t halves = w == 0 ? 2 * kStageSteps : 2;
    const cuuint32_t box_a[2] = {2 * kTile, halves};
    const cuuint32_t box_b[3] = {2 * kTile, kTileN / kTile, halves};
    CUtensorMap *ma = w == 0 ? &b.maps.a_stage : &b.maps.a_step;
    CUtensorMap *mb = w == 0 ? &b.maps.b_stage : &b.maps.b_step;
    if (enc(ma, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, b.M, dims_a, strides_a, box_a, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS ||
        enc(mb, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, b.M, dims_b, strides_b, box_b, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
      return KZ_ERR_CUDA;
  }
  KZ_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors die here
  return KZ_OK;
}

// The buffers of the tensor form for this graph and precision (built on
// first use) and the kernels' shared-memory opt-in.
static kz_status tensor_buffers(kz_graph g, bool bf16, cudaStream_t s, TensorBufs **out) {
  if (g->k > 64) return KZ_ERR_UNSUPPORTED;
  if (!g->tensor_bufs) g->tensor_bufs = new TensorState();
  TensorState &ts = *static_cast<TensorState *>(g->tensor_bufs);
  if (!ts.by[bf16]) {
    TensorBufs *nb = new TensorBufs();
    kz_status st = tensor_prepare(g, *nb, bf16, s);
    if (st != KZ_OK) {
      delete nb;
      return st;
    }
    ts.by[bf16] = nb;
  }
  int dev = 0;
  KZ_CUDA_TRY(cudaGetDevice(&dev));
  static bool configured[64][2] = {};
  if (dev < 64 && !configured[dev][bf16]) {
    const void *fn = bf16 ? (const void *)tensor_edge_kernel<true> : (const void *)tensor_edge_kernel<false>;
    KZ_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
    configured[dev][bf16] = true;
  }
  *out = ts.by[bf16];
  return KZ_OK;
}

// One pass of the tensor form on the current rows: expand them into the
// operand matrix, count every class's common neighbours of every pair on the
// tensor cores and mark the failing live edges, then apply those deletions
// and the vertex rule into the other row buffer.  The run's counters must
// have been started (bitset_begin_run).  *cont receives 1 when the pass
// deleted something and the run may go on (no sweep limit or error).
kz_status tensor_one_pass(kz_graph g, const kz_options &opt, cudaStream_t s, int *cont) {
  *cont = 0;
  if (g->n == 0) return KZ_OK;
  const bool bf16 = opt.tensor_precision == 1;
  TensorBufs *bp = nullptr;
  KZ_TRY(tensor_buffers(g, bf16, s, &bp));
  TensorBufs &b = *bp;
  const int sms = sms_t();
  int32_t cur = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&cur, &g->st->cur, 4, cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  const uint32_t *A = g->A[cur & 1];
  uint32_t *An = g->A[(cur & 1) ^ 1];
  if (bf16) expand_kernel<true><<<8 * sms, 256, 0, s>>>(A, g->n, b.n_pad, g->ldw, b.step_word, b.ksteps, b.M);
  else expand_kernel<false><<<8 * sms, 256, 0, s>>>(A, g->n, b.n_pad, g->ldw, b.step_word, b.ksteps, b.M);
  TensorArgs a;
  a.n = g->n;
  a.k = g->k;
  a.q = g->k - g->slack;
  a.cls_step = b.cls_step;
  a.A = A;
  a.ldw = g->ldw;
  a.vinfo = b.vinfo;
  a.Edel = b.Edel;
  a.tiles = b.tiles;
  a.n_tiles = b.n_tiles;
  a.counts = b.counts;
  a.status = &g->st->status;
  const int grid = std::max(1, std::min(b.n_tiles, sms));
  if (bf16) tensor_edge_kernel<true><<<grid, kThreads, kSmemBytes, s>>>(b.maps, a);
  else tensor_edge_kernel<false><<<grid, kThreads, kSmemBytes, s>>>(b.maps, a);
  tensor_commit_kernel<<<8 * sms, 256, 0, s>>>(A, An, b.Edel, g->V[cur & 1], g->V[(cur & 1) ^ 1], g->n, g->ldw,
                                               g->k, g->k - g->slack, g->R, b.col, g->d_coff, g->d_rounds, g->d_blocks,
                                               (int32_t)g->blocks.size(), g->v_sweep, g->st, b.counts);
  tensor_finish_kernel<<<1, 1, 0, s>>>(g->st, b.counts);
  KZ_CUDA_TRY(cudaGetLastError());
  int32_t c = 0, status = 0;
  KZ_CUDA_TRY(cudaMemcpyAsync(&c, &g->st->cont, 4, cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaMemcpyAsync(&status, &g->st->status, 4, cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  *cont = (c && status == KZ_OK) ? 1 : 0;
  return KZ_OK;
}

kz_status tensor_kernelize(kz_graph g, const kz_options &opt, cudaStream_t s) {
  if (g->k > 64) return KZ_ERR_UNSUPPORTED;
  TensorBufs *bp = nullptr;
  KZ_TRY(tensor_buffers(g, opt.tensor_precision == 1, s, &bp));
  const int64_t max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : (int64_t)g->n + g->m + 1;
  KZ_TRY(bitset_begin_run(g, max_sweeps, s));
  if (g->n == 0) return KZ_OK;
  for (;;) {
    int cont = 0;
    KZ_TRY(tensor_one_pass(g, opt, s, &cont));
    if (!cont) break;
  }
  return KZ_OK;
}

void tensor_release(kz_graph g) {
  TensorState *ts = static_cast<TensorState *>(g->tensor_bufs);
  if (ts) {
    delete ts->by[0];
    delete ts->by[1];
  }
  delete ts;
  g->tensor_bufs = nullptr;
}

}  // namespace kz
