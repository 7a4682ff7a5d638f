// kz_tensor.cu -- tensor-core form of the edge rule (thesis Section 4.2).
//
// For every colour class c, S_c = A[:, C_c] * A[:, C_c]^T counts the common
// neighbours of every vertex pair inside class c.  The edge rule asks, per
// live edge {u,v}, how many classes have S_c(u,v) > 0 (classes col(u) and
// col(v) always give 0: no neighbour of u has u's colour).  An edge fails when
// fewer than k-2 classes do.
//
// Layout: the live bitset rows are expanded into a byte matrix M (rows in the
// relabelled order, padded to a multiple of 128) with one 32-byte K-step per
// 32-bit block word: byte 32*j + b of row x is E4M3 1.0 (0x38) when bit b of
// block word j of row x is set, else 0.  Class c is the run of K-steps of its
// blocks, so S_c is a K-loop over those steps only.
//
// Kernel: one CTA (4 warps) per upper-triangle tile (I, J) of 128 x 128
// pairs.  For each class: the K-steps of rows I and J are copied into shared
// memory in the canonical no-swizzle K-major layout (8-row x 16-byte core
// matrices), one thread issues tcgen05.mma.kind::f8f6f4 (M = N = 128, K = 32
// per step, fp32 accumulation in TMEM, exact for 0/1 products), and the four
// warps read the accumulator back with tcgen05.ld and count, per pair, the
// classes with a non-zero entry (8-bit counters packed four to a register).
// After the last class the live edges of the tile below k-2 are marked in a
// deletion bitmap; a row kernel then applies the vertex rule and the edge
// deletions to produce the next state.  Waits on the MMA mbarrier are
// bounded: a wait that runs out records KZ_ERR_TIMEOUT and the CTA returns
// after freeing its tensor memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kz_internal.cuh"
#include "kz_rules.cuh"

namespace kz {
namespace tensor {

constexpr int kTile = 128;          // rows per tile side (MMA M = N = 128)
constexpr int kStep = 32;           // bytes (E4M3 elements) per K-step
constexpr int kThreads = 128;       // 4 warps: one TMEM lane quarter each
constexpr int kMaxStepsPerStage = 16;  // K-steps staged at once (class runs are looped in chunks)
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, no swizzle.  A K-step of 128 rows
// x 32 bytes is 16 groups of 8 rows; each group holds two 8x16-byte core
// matrices (K halves) 128 bytes apart (leading byte offset), groups are 256
// bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
  d |= (uint64_t)(128u >> 4) << 16;                 // leading byte offset (K direction)
  d |= (uint64_t)(256u >> 4) << 32;                 // stride byte offset (8-row groups)
  d |= (uint64_t)1 << 46;                           // descriptor version
  // base offset 0, relative LBO mode, no swizzle (bits 61-63 = 0)
  return d;
}

// Instruction descriptor: dense, D = f32, A = B = E4M3, both K-major,
// N = 128, M = 128.
__device__ __forceinline__ uint32_t make_idesc() {
  uint32_t d = 0;
  d |= 1u << 4;              // D format f32
  d |= 0u << 7;              // A format E4M3
  d |= 0u << 10;             // B format E4M3
  d |= (128u >> 3) << 17;    // N >> 3
  d |= (128u >> 4) << 24;    // M >> 4
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

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
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

// 32 consecutive fp32 columns of this thread's TMEM lane.
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
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TensorArgs {
  const uint8_t *M;        // byte matrix [n_pad][ksteps * 32]
  int32_t n, n_pad, ksteps;
  const int32_t *cls_step; // k + 1: first K-step of each class
  const uint32_t *A;       // current rows (adjacency bits)
  int32_t ldw, k;
  const int32_t *col;      // relabelled colour
  const int32_t *coff;     // k + 1
  uint32_t *Edel;          // deletion bitmap, rows x ldw (zeroed)
  const int2 *tiles;       // (I, J) tile pairs, I <= J
  int32_t n_tiles;
  unsigned long long *counts;  // [0] failing edges [1] live edges tested
  int32_t *status;
};

// Copy K-steps [s0, s0 + ns) of the 128 rows starting at `row0` into the
// canonical layout: step s occupies 4096 bytes; inside it, row r, byte b sits
// at (r / 8) * 256 + (b / 16) * 128 + (r % 8) * 16 + (b % 16).
__device__ __forceinline__ void stage_rows(const TensorArgs &a, int row0, int s0, int ns, uint8_t *dst) {
  const int64_t ld = (int64_t)a.ksteps * kStep;
  // one 16-byte chunk per thread-iteration: (step, row, half)
  const int chunks = ns * kTile * 2;
  for (int q = threadIdx.x; q < chunks; q += kThreads) {
    const int s = q / (kTile * 2);
    const int rem = q - s * kTile * 2;
    const int r = rem >> 1, h = rem & 1;
    const uint4 v = *reinterpret_cast<const uint4 *>(a.M + (int64_t)(row0 + r) * ld + (int64_t)(s0 + s) * kStep + h * 16);
    *reinterpret_cast<uint4 *>(dst + s * 4096 + (r >> 3) * 256 + h * 128 + (r & 7) * 16) = v;
  }
}

__global__ void __launch_bounds__(kThreads, 1) tensor_edge_kernel(TensorArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *sA = smem;                                   // kMaxStepsPerStage x 4096
  uint8_t *sB = smem + kMaxStepsPerStage * 4096;        // kMaxStepsPerStage x 4096
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(128u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t mb = smem_u32(&mbar);
  const uint32_t idesc = make_idesc();
  uint32_t phase = 0;
  unsigned long long my_fail = 0, my_tests = 0;

  for (int t = blockIdx.x; t < a.n_tiles && !abort_flag; t += gridDim.x) {
    const int I = a.tiles[t].x, J = a.tiles[t].y;
    const int u = I * kTile + tid;  // this thread's TMEM lane = row u of the tile
    uint32_t cnt[32];               // 128 column counters, 8 bits each
#pragma unroll
    for (int i = 0; i < 32; i++) cnt[i] = 0;
    for (int c = 0; c < a.k && !abort_flag; c++) {
      const int sb = a.cls_step[c], se = a.cls_step[c + 1];
      if (se <= sb) continue;
      for (int s0 = sb; s0 < se && !abort_flag; s0 += kMaxStepsPerStage) {
        const int ns = min(kMaxStepsPerStage, se - s0);
        stage_rows(a, I * kTile, s0, ns, sA);
        stage_rows(a, J * kTile, s0, ns, sB);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
          for (int s = 0; s < ns; s++) {
            const uint64_t da = make_desc(smem_u32(sA + s * 4096));
            const uint64_t db = make_desc(smem_u32(sB + s * 4096));
            mma_f8(tmem, da, db, idesc, (s0 > sb || s > 0) ? 1u : 0u);
          }
          mma_commit(mb);
        }
        // every thread waits for the MMAs of this stage (bounded)
        uint32_t spins = 0;
        while (!mbar_try_wait(mb, phase)) {
          if (++spins > kSpinLimit) {
            atomicExch(&abort_flag, 1);
            if (a.status) atomicCAS(a.status, 0, (int32_t)KZ_ERR_TIMEOUT);
            break;
          }
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();  // shared operands free again
      }
      if (abort_flag) break;
      // class c done: count the non-zero entries of this thread's row
#pragma unroll
      for (int q = 0; q < 4; q++) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * 32), r);
#pragma unroll
        for (int j = 0; j < 32; j++) {
          const uint32_t nz = __uint_as_float(r[j]) > 0.f ? 1u : 0u;
          cnt[q * 8 + (j >> 2)] += nz << ((j & 3) * 8);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();  // accumulator read before the next class overwrites it
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (abort_flag) break;
    // live edges of the tile row u: (u, v) with v in tile J, u < v
    if (u < a.n) {
      const int cu = a.col[u];
      const uint32_t *row = a.A + (int64_t)u * a.ldw;
      for (int j = 0; j < kTile; j++) {
        const int v = J * kTile + j;
        if (v >= a.n || v <= u) continue;
        const int cv = a.col[v];
        if (cv == cu) continue;
        const int iv = v - a.coff[cv];
        const int wv = (iv >> 5) * a.k + cv;
        if (!((row[wv] >> (iv & 31)) & 1u)) continue;
        my_tests++;
        const int cover = (int)((cnt[j >> 2] >> ((j & 3) * 8)) & 0xFFu);
        if (cover < a.k - 2) {
          my_fail++;
          const int iu = u - a.coff[cu];
          atomicOr(&a.Edel[(int64_t)u * a.ldw + wv], 1u << (iv & 31));
          atomicOr(&a.Edel[(int64_t)v * a.ldw + (iu >> 5) * a.k + cu], 1u << (iu & 31));
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    my_fail += __shfl_down_sync(0xffffffffu, my_fail, o);
    my_tests += __shfl_down_sync(0xffffffffu, my_tests, o);
  }
  if (lane == 0) {
    if (my_fail) atomicAdd(&a.counts[0], my_fail);
    if (my_tests) atomicAdd(&a.counts[1], my_tests);
  }
  if (abort_flag && tid == 0) {
    // a wait ran out: give the MMAs in flight one more bounded wait before the
    // tensor memory they write is released
    uint32_t spins = 0;
    while (!mbar_try_wait(mb, phase) && ++spins < kSpinLimit) {
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u));
}

// Byte matrix from the current rows: block word j of row x -> bytes
// 32j .. 32j+31 (0x38 = E4M3 1.0 for a set bit).  Rows are laid out by
// K-step order: word (c, r) -> step cls_step[c] + r.
__global__ void expand_kernel(const uint32_t *__restrict__ A, int32_t n, int32_t n_pad, int32_t ldw, int32_t k,
                              int32_t R, const int32_t *__restrict__ rounds, const int32_t *__restrict__ cls_step,
                              int32_t ksteps, uint8_t *__restrict__ M) {
  const int64_t ld = (int64_t)ksteps * kStep;
  const int64_t total = (int64_t)n_pad * ksteps;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = (int32_t)(t / ksteps);
    const int32_t s = (int32_t)(t - (int64_t)x * ksteps);
    // class of step s
    int c = 0;
    while (c + 1 <= k && cls_step[c + 1] <= s) c++;
    const int r = s - cls_step[c];
    const uint32_t word = (x < n && r < rounds[c]) ? A[(int64_t)x * ldw + r * k + c] : 0u;
    uint32_t out[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      uint32_t v = 0;
#pragma unroll
      for (int b = 0; b < 4; b++) v |= ((word >> (q * 4 + b)) & 1u) ? (0x38u << (8 * b)) : 0u;
      out[q] = v;
    }
    uint4 *dst = reinterpret_cast<uint4 *>(M + (int64_t)x * ld + (int64_t)s * kStep);
    dst[0] = make_uint4(out[0], out[1], out[2], out[3]);
    dst[1] = make_uint4(out[4], out[5], out[6], out[7]);
  }
}

// Vertex rule and application of the marked edge deletions: next rows =
// current rows minus the deletion bitmap; next live words; pass counters.
__global__ void tensor_commit_kernel(const uint32_t *__restrict__ A, uint32_t *__restrict__ An,
                                     uint32_t *__restrict__ Edel, const uint32_t *__restrict__ V,
                                     uint32_t *__restrict__ Vn, int32_t n, int32_t ldw, int32_t k, int32_t R,
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
    const bool fail = live && cnt < k - 1;
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

// Per-graph buffers of the tensor path (allocated on first use).
struct TensorBufs {
  uint8_t *M = nullptr;
  int32_t n_pad = 0, ksteps = 0;
  int32_t *cls_step = nullptr;
  int32_t *col = nullptr;
  uint32_t *Edel = nullptr;
  int2 *tiles = nullptr;
  int32_t n_tiles = 0;
  unsigned long long *counts = nullptr;
};

static kz_status tensor_prepare(kz_graph g, TensorBufs &b, cudaStream_t s) {
  b.n_pad = (g->n + kTile - 1) / kTile * kTile;
  std::vector<int32_t> cs((size_t)g->k + 1, 0);
  for (int c = 0; c < g->k; c++) cs[c + 1] = cs[c] + g->rounds[c];
  b.ksteps = std::max(cs[g->k], 1);
  const size_t mbytes = (size_t)b.n_pad * b.ksteps * kStep;
  KZ_TRY(graph_alloc(g, &b.M, mbytes, s));
  KZ_TRY(graph_alloc(g, &b.cls_step, (size_t)g->k + 1, s));
  KZ_CUDA_TRY(cudaMemcpyAsync(b.cls_step, cs.data(), sizeof(int32_t) * (g->k + 1), cudaMemcpyHostToDevice, s));
  std::vector<int32_t> col_new((size_t)std::max(g->n, 1));
  for (int c = 0; c < g->k; c++)
    for (int x = g->coff[c]; x < g->coff[c + 1]; x++) col_new[x] = c;
  KZ_TRY(graph_alloc(g, &b.col, col_new.size(), s));
  KZ_CUDA_TRY(cudaMemcpyAsync(b.col, col_new.data(), sizeof(int32_t) * col_new.size(), cudaMemcpyHostToDevice, s));
  KZ_TRY(graph_alloc(g, &b.Edel, (size_t)g->n * g->ldw, s));
  KZ_CUDA_TRY(cudaMemsetAsync(b.Edel, 0, (size_t)g->n * g->ldw * 4, s));
  const int T = b.n_pad / kTile;
  std::vector<int2> tiles;
  for (int i = 0; i < T; i++)
    for (int j = i; j < T; j++) tiles.push_back(make_int2(i, j));
  b.n_tiles = (int32_t)tiles.size();
  KZ_TRY(graph_alloc(g, &b.tiles, std::max<size_t>(tiles.size(), 1), s));
  if (!tiles.empty())
    KZ_CUDA_TRY(cudaMemcpyAsync(b.tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, s));
  KZ_TRY(graph_alloc(g, &b.counts, 4, s));
  KZ_CUDA_TRY(cudaMemsetAsync(b.counts, 0, 32, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors die here
  return KZ_OK;
}

kz_status tensor_kernelize(kz_graph g, const kz_options &opt, cudaStream_t s) {
  if (g->k > 64) return KZ_ERR_UNSUPPORTED;
  if (!g->tensor_bufs) {
    TensorBufs *b = new TensorBufs();
    kz_status st = tensor_prepare(g, *b, s);
    if (st != KZ_OK) {
      delete b;
      return st;
    }
    g->tensor_bufs = b;
  }
  TensorBufs &b = *static_cast<TensorBufs *>(g->tensor_bufs);
  const int64_t max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : (int64_t)g->n + g->m + 1;
  KZ_TRY(bitset_begin_run(g, max_sweeps, s));
  if (g->n == 0) return KZ_OK;
  const size_t smem = (size_t)2 * kMaxStepsPerStage * 4096;
  static bool configured = false;
  if (!configured) {
    KZ_CUDA_TRY(cudaFuncSetAttribute((const void *)tensor_edge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    configured = true;
  }
  const int sms = sms_t();
  for (;;) {
    int32_t cur = 0;
    KZ_CUDA_TRY(cudaMemcpyAsync(&cur, &g->st->cur, 4, cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaStreamSynchronize(s));
    const uint32_t *A = g->A[cur & 1];
    uint32_t *An = g->A[(cur & 1) ^ 1];
    expand_kernel<<<8 * sms, 256, 0, s>>>(A, g->n, b.n_pad, g->ldw, g->k, g->R, g->d_rounds, b.cls_step, b.ksteps,
                                          b.M);
    TensorArgs a;
    a.M = b.M;
    a.n = g->n;
    a.n_pad = b.n_pad;
    a.ksteps = b.ksteps;
    a.cls_step = b.cls_step;
    a.A = A;
    a.ldw = g->ldw;
    a.k = g->k;
    a.col = b.col;
    a.coff = g->d_coff;
    a.Edel = b.Edel;
    a.tiles = b.tiles;
    a.n_tiles = b.n_tiles;
    a.counts = b.counts;
    a.status = &g->st->status;
    const int grid = std::max(1, std::min(b.n_tiles, sms));
    tensor_edge_kernel<<<grid, kThreads, smem, s>>>(a);
    tensor_commit_kernel<<<8 * sms, 256, 0, s>>>(A, An, b.Edel, g->V[cur & 1], g->V[(cur & 1) ^ 1], g->n, g->ldw,
                                                 g->k, g->R, b.col, g->d_coff, g->d_rounds, g->d_blocks,
                                                 (int32_t)g->blocks.size(), g->v_sweep, g->st, b.counts);
    tensor_finish_kernel<<<1, 1, 0, s>>>(g->st, b.counts);
    KZ_CUDA_TRY(cudaGetLastError());
    int32_t cont = 0, status = 0;
    KZ_CUDA_TRY(cudaMemcpyAsync(&cont, &g->st->cont, 4, cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaMemcpyAsync(&status, &g->st->status, 4, cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaStreamSynchronize(s));
    if (!cont || status != KZ_OK) break;
  }
  return KZ_OK;
}

void tensor_release(kz_graph g) {
  delete static_cast<TensorBufs *>(g->tensor_bufs);
  g->tensor_bufs = nullptr;
}

}  // namespace kz
