// kz_probe.cu -- hardware probes (include/kz_probe.h): integer throughput,
// tcgen05 fp8 MMA throughput and TMA load throughput.
#include <cuda.h>  // CUtensorMap and its enums
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/kz_probe.h"
#include "kz_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__device__ __forceinline__ uint32_t lop3_and_or(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0xEA;" : "=r"(d) : "r"(a), "r"(b), "r"(c));  // (a & b) | c
  return d;
}

__device__ __forceinline__ uint32_t umin_asm(uint32_t a, uint32_t b) {
  uint32_t d;
  asm volatile("min.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

template <int KIND>
__global__ void int_probe_kernel(uint32_t seed, uint32_t *out) {
  uint32_t x[kChains];
  uint32_t m[kChains];
#pragma unroll
  for (int i = 0; i < kChains; i++) {
    x[i] = seed * (threadIdx.x + 7 * i + 1);
    m[i] = 0xffffffffu - (uint32_t)i;
  }
  const uint32_t y = seed ^ blockIdx.x, z = seed + 3u;
  for (int it = 0; it < kIters; it++) {
#pragma unroll
    for (int i = 0; i < kChains; i++) {
      if (KIND == 0) x[i] = lop3_and_or(x[i], y, z);
      if (KIND == 1) x[i] = umin_asm(x[i], y + (uint32_t)i);
      if (KIND == 2) x[i] = __vimin3_u32(x[i], y, z + (uint32_t)i);
      if (KIND == 3) {  // one logic op feeding one two-input min
        x[i] = lop3_and_or(x[i], y, z);
        m[i] = umin_asm(m[i], x[i]);
      }
      if (KIND == 4) {  // two logic ops feeding one three-input min
        const uint32_t a = lop3_and_or(x[i], y, z), b = lop3_and_or(x[i], z, y);
        m[i] = __vimin3_u32(m[i], a, b);
        x[i] = a;
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kChains; i++) acc ^= x[i] ^ m[i];
  if (acc == 0x9e3779b9u) out[0] = acc;  // keeps the chains live
}

constexpr int kMmaKSteps = 4;  // K-steps of 32 bytes held in shared memory (one 128-byte row per operand row)

__device__ __forceinline__ uint32_t probe_smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory descriptor of K-step j of an operand of `rows` rows.
//   layout 0: no swizzle, each K-step 32 bytes x rows, its two 16-byte K
//             halves rows * 16 bytes apart, 8-row groups 128 bytes apart;
//   layout 1: no swizzle, K halves 128 bytes apart, 8-row groups 256 apart;
//   layout 2: 128-byte swizzle, K-major: one 128-byte row per operand row
//             (all four K-steps), 8-row groups 1024 bytes apart, K-step j at
//             byte 32 j of the row.
__device__ __forceinline__ uint64_t probe_desc(uint32_t base, int layout, int rows, int j) {
  uint64_t d = 0;
  uint32_t start, lbo, sbo, swz;
  if (layout == 0) {
    start = base + j * rows * 32;
    lbo = rows * 16;
    sbo = 128;
    swz = 0;
  } else if (layout == 1) {
    start = base + j * rows * 32;
    lbo = 128;
    sbo = 256;
    swz = 0;
  } else {
    start = base + j * 32;
    lbo = 16;
    sbo = 1024;
    swz = 2;  // 128-byte swizzle
  }
  d |= (uint64_t)((start & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)swz << 61;
  return d;
}

// One CTA issues iters x 4 MMAs (M = 128, N = n, K = 32, E4M3 -> f32) on
// operands already in shared memory and waits (bounded) for them.
__global__ void __launch_bounds__(128) mma_probe_kernel(int layout, int n, int iters, int32_t *status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  uint8_t *smem = smem_raw + ((1024u - (probe_smem_u32(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x;
  uint32_t *w = reinterpret_cast<uint32_t *>(smem);
  for (int i = tid; i < (128 + 256) * 128 / 4; i += blockDim.x) w[i] = 0x38383838u * (uint32_t)((i * 7) & 1);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(probe_smem_u32(&tmem_base)),
                 "r"(256u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const uint32_t mb = probe_smem_u32(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t sA = probe_smem_u32(smem), sB = sA + 128 * 128;
  if (tid == 0) {
    uint32_t idesc = 0;
    idesc |= 1u << 4;                          // D f32, A = B = E4M3, K-major
    idesc |= ((uint32_t)n >> 3) << 17;         // N >> 3
    idesc |= (128u >> 4) << 24;                // M >> 4
    for (int it = 0; it < iters; it++) {
#pragma unroll
      for (int j = 0; j < kMmaKSteps; j++) {
        const uint64_t da = probe_desc(sA, layout, 128, j), db = probe_desc(sB, layout, n, j);
        const uint32_t acc = (it | j) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
  }
  // bounded wait (wall clock) for the MMAs
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t i = 0;; i++) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mb)
        : "memory");
    if (ok) break;
    uint64_t t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (t1 - t0 > 4000000000ull || i > (1u << 30)) {
      if (tid == 0) atomicCAS(status, 0, (int32_t)KZ_ERR_TIMEOUT);
      break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u));
}

constexpr int kTmaStages = 6;
constexpr int kTmaStageBytes = 16384;
constexpr int kTmaBoxes = 4;  // boxes of 4 KB per stage (one 16 KB box in mode 3)

__device__ __forceinline__ bool probe_try_wait(uint32_t mb, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mb), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool probe_wait(uint32_t mb, uint32_t parity, int32_t *status) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t i = 0; !probe_try_wait(mb, parity); i++) {
    uint64_t t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (t1 - t0 > 4000000000ull || i > (1u << 30)) {
      atomicCAS(status, 0, (int32_t)KZ_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// One thread streams iters stages of 16 KB from an L2-resident 32 MB source
// into a ring of shared-memory stages, re-issuing each stage as soon as its
// previous load has landed (no consumer).
//   mode 0: 2-D map of 8-byte elements {8192, 512}, box {256, 2} (4 KB: two
//           contiguous 2 KB runs; the tensor path's operand box);
//   mode 1: 2-D map of bytes {8192, 4096}, box {128, 32} with 128-byte swizzle;
//   mode 2: untiled bulk copies of 4 KB;
//   mode 3: the map of mode 0 with box {256, 8} (16 KB).
__global__ void __launch_bounds__(32) tma_probe_kernel(const __grid_constant__ CUtensorMap map, int mode,
                                                       const uint8_t *src, int iters, int32_t *status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kTmaStages];
  uint8_t *smem = smem_raw + ((1024u - (probe_smem_u32(smem_raw) & 1023u)) & 1023u);
  if (threadIdx.x != 0) return;
  const uint32_t s0 = probe_smem_u32(smem), b0 = probe_smem_u32(full);
  for (int s = 0; s < kTmaStages; s++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0 + 8 * s));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const uint64_t mp = reinterpret_cast<uint64_t>(&map);
  bool ok = true;
  for (int it = 0; it < iters && ok; it++) {
    const int st = it % kTmaStages;
    const uint32_t fb = b0 + 8 * st, dst = s0 + st * kTmaStageBytes;
    if (it >= kTmaStages) ok = probe_wait(fb, (uint32_t)((it / kTmaStages - 1) & 1), status);
    if (!ok) break;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kTmaStageBytes) : "memory");
    const int r = it + 7 * (int)blockIdx.x;
    if (mode == 3) {
      const int x = 256 * (r % 32), y = 8 * (r % 64);
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
              "r"(dst),
          "l"(mp), "r"(fb), "r"(x), "r"(y)
          : "memory");
      continue;
    }
    for (int b = 0; b < kTmaBoxes; b++) {
      const uint32_t d = dst + b * 4096;
      const int q = r * kTmaBoxes + b;
      if (mode == 0) {
        const int x = 256 * (q % 32), y = 2 * (q % 256);
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
                "r"(d),
            "l"(mp), "r"(fb), "r"(x), "r"(y)
            : "memory");
      } else if (mode == 1) {
        const int x = 128 * (q % 64), y = 32 * (q % 128);
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
                "r"(d),
            "l"(mp), "r"(fb), "r"(x), "r"(y)
            : "memory");
      } else {
        const uint8_t *g = src + (int64_t)(q % 8192) * 4096;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 4096, [%2];" ::"r"(d),
            "l"(g), "r"(fb)
            : "memory");
      }
    }
  }
  // every load issued lands before the shared memory goes away
  const int issued = iters < kTmaStages ? iters : kTmaStages;
  for (int s = 0; s < issued; s++) {
    const int last = (iters - 1 - s) / kTmaStages * kTmaStages + s;  // last iteration that used stage s
    probe_wait(b0 + 8 * s, (uint32_t)((last / kTmaStages) & 1), status);
  }
}

}  // namespace

extern "C" kz_status kz_probe_tma_throughput(int32_t mode, int32_t ctas_per_sm, double *bytes_per_s, double *ms,
                                             void *stream) {
  if (!bytes_per_s || !ms || mode < 0 || mode > 3 || ctas_per_sm < 1 || ctas_per_sm > 2) return KZ_ERR_ARG;
  typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                               const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  EncodeFn enc = reinterpret_cast<EncodeFn>(kz::tensor_map_encoder());
  if (!enc) return KZ_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KZ_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t src_bytes = (size_t)32 << 20;
  uint8_t *src = nullptr;
  int32_t *status = nullptr;
  if (cudaMalloc(&src, src_bytes) != cudaSuccess) return KZ_ERR_CUDA;
  if (cudaMalloc(&status, 4) != cudaSuccess) {
    cudaFree(src);
    return KZ_ERR_CUDA;
  }
  cudaMemsetAsync(src, 0x38, src_bytes, s);
  cudaMemsetAsync(status, 0, 4, s);
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  CUresult r;
  if (mode == 1) {
    const cuuint64_t dims[2] = {8192, 4096};
    const cuuint64_t strides[1] = {8192};
    const cuuint32_t box[2] = {128, 32}, es[2] = {1, 1};
    r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, src, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    const cuuint64_t dims[2] = {8192, 512};
    const cuuint64_t strides[1] = {8192 * 8};
    const cuuint32_t box[2] = {256, mode == 3 ? 8u : 2u}, es[2] = {1, 1};
    r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, src, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  kz_status out = KZ_OK;
  const size_t smem = (size_t)kTmaStages * kTmaStageBytes + 1024;
  if (r != CUDA_SUCCESS ||
      cudaFuncSetAttribute((const void *)tma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    out = KZ_ERR_CUDA;
  } else {
    const int iters = 2048, blocks = sms * ctas_per_sm;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    tma_probe_kernel<<<blocks, 32, smem, s>>>(map, mode, src, 64, status);  // warm-up (fills L2)
    cudaEventRecord(e0, s);
    tma_probe_kernel<<<blocks, 32, smem, s>>>(map, mode, src, iters, status);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    int32_t st = 0;
    cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      out = KZ_ERR_CUDA;
    } else if (st != 0) {
      out = (kz_status)st;
    } else {
      *ms = t;
      *bytes_per_s = (double)kTmaStageBytes * iters * blocks / (t * 1e-3);
    }
  }
  cudaFree(src);
  cudaFree(status);
  return out;
}

extern "C" kz_status kz_probe_mma_throughput(int32_t layout, int32_t n, int32_t ctas_per_sm, double *flops_per_s,
                                             double *ms, void *stream) {
  if (!flops_per_s || !ms || layout < 0 || layout > 2 || (n != 128 && n != 256) || ctas_per_sm < 1 ||
      ctas_per_sm > 2)
    return KZ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KZ_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = (size_t)(128 + 256) * 128 + 1024;
  if (cudaFuncSetAttribute((const void *)mma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return KZ_ERR_CUDA;
  int32_t *status = nullptr;
  if (cudaMallocAsync(&status, 4, s) != cudaSuccess) return KZ_ERR_CUDA;
  cudaMemsetAsync(status, 0, 4, s);
  const int iters = 4096, blocks = sms * ctas_per_sm;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  mma_probe_kernel<<<blocks, 128, smem, s>>>(layout, n, 64, status);  // warm-up
  cudaEventRecord(e0, s);
  mma_probe_kernel<<<blocks, 128, smem, s>>>(layout, n, iters, status);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  int32_t st = 0;
  cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(status, s);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return KZ_ERR_CUDA;
  if (st != 0) return (kz_status)st;
  const double flops = 2.0 * 128.0 * n * 32.0 * kMmaKSteps * (double)iters * blocks;
  *ms = t;
  *flops_per_s = flops / (t * 1e-3);
  return KZ_OK;
}

extern "C" kz_status kz_probe_int_throughput(int32_t kind, double *ops_per_s, double *ms, void *stream) {
  if (!ops_per_s || !ms || kind < 0 || kind > 4) return KZ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KZ_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t *out = nullptr;
  if (cudaMallocAsync(&out, 16, s) != cudaSuccess) return KZ_ERR_CUDA;
  const int threads = 256, blocks = sms * 8;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  void (*const fns[5])(uint32_t, uint32_t *) = {int_probe_kernel<0>, int_probe_kernel<1>, int_probe_kernel<2>,
                                                 int_probe_kernel<3>, int_probe_kernel<4>};
  void (*fn)(uint32_t, uint32_t *) = fns[kind];
  fn<<<blocks, threads, 0, s>>>(12345u, out);  // warm-up
  cudaEventRecord(e0, s);
  fn<<<blocks, threads, 0, s>>>(54321u, out);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return KZ_ERR_CUDA;
  const double per_chain_step = kind == 3 ? 2.0 : (kind == 4 ? 3.0 : 1.0);
  const double ops = (double)blocks * threads * kIters * kChains * per_chain_step;
  *ms = t;
  *ops_per_s = ops / (t * 1e-3);
  return KZ_OK;
}
