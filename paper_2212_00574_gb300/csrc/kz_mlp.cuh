// kz_mlp.cuh -- the edge-scoring network of the learned schedule on the
// tensor cores: warp-level bf16 MMAs (mma.sync m16n8k16, fp32 accumulation)
// for the 16 -> 64 -> 64 -> 1 network of include/kz_learned.h.
//
// Rounding points (the CPU oracle of the network rounds at the same places):
//   every parameter is used as its bf16 value; the features x are rounded to
//   bf16; z1 = x W1^T + b1 is accumulated in fp32 and h1 = relu(z1) rounded to
//   bf16; z2 = h1 W2^T + b2 in fp32, h2 = relu(z2) kept in fp32; the output
//   logit = h2 . w3 + b3 in fp32.
//
// Fragment layouts of mma.m16n8k16 (PTX ISA, "Matrix fragments for
// mma.m16n8k16"): with g = lane / 4 and t = lane % 4,
//   A (16 x 16, row-major), four registers of two bf16 each:
//     a0: (row g,     cols 2t, 2t+1)     a1: (row g + 8, cols 2t, 2t+1)
//     a2: (row g,     cols 2t+8, 2t+9)   a3: (row g + 8, cols 2t+8, 2t+9)
//   B (16 x 8, K x N), two registers:
//     b0: (rows 2t, 2t+1, col g)         b1: (rows 2t+8, 2t+9, col g)
//   C/D (16 x 8, fp32), four registers:
//     c0, c1: (row g, cols 2t, 2t+1)     c2, c3: (row g + 8, cols 2t, 2t+1)
// The lower half of a packed register holds the element of smaller index.
// An accumulator pair of n-tiles (2s, 2s+1) of one layer is therefore, after
// the activation and a repack, exactly the A fragment of k-step s of the next
// layer: hidden activations never leave the registers.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/kz_learned.h"

namespace kz {
namespace mlp {

constexpr int F = KZ_MLP_FEATURES;
constexpr int H = KZ_MLP_HIDDEN;
constexpr int P = KZ_MLP_PARAMS;
// offsets of the weight blocks in the flat array
constexpr int oW1 = 0, ob1 = oW1 + H * F, oW2 = ob1 + H, ob2 = oW2 + H * H, ow3 = ob2 + H, ob3 = ow3 + H;
static_assert(ob3 + 1 == P, "weight layout");

// Row strides (in bf16 elements) of the shared-memory tiles: 8 elements of
// padding so that the eight row groups of a fragment load hit distinct banks.
constexpr int kXLd = F + 8;   // feature tile [rows][16]
constexpr int kWLd = H + 8;   // [64][64] weight tile
constexpr int kTileRows = 32; // edges per warp step (two m-tiles)

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16 *p) {
  return *reinterpret_cast<const uint32_t *>(p);
}

// The network's parameters as one CTA holds them: W2 in shared memory in its
// [j][i] layout (padded rows), the small vectors widened to fp32.
struct SmemNet {
  __nv_bfloat16 W2[H * kWLd];
  float b1[H], b2[H], w3[H];
  float b3;
};

// Cooperative load of the bf16 parameters into shared memory (whole block).
__device__ __forceinline__ void load_net(SmemNet &s, const __nv_bfloat16 *__restrict__ w16) {
  for (int e = threadIdx.x; e < H * H; e += blockDim.x) s.W2[(e / H) * kWLd + e % H] = w16[oW2 + e];
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    s.b1[j] = __bfloat162float(w16[ob1 + j]);
    s.b2[j] = __bfloat162float(w16[ob2 + j]);
    s.w3[j] = __bfloat162float(w16[ow3 + j]);
  }
  if (threadIdx.x == 0) s.b3 = __bfloat162float(w16[ob3]);
}

// B fragments of W1 (K = 16 features, N = 64 hidden: eight n-tiles), held in
// registers by each warp for its whole life.
__device__ __forceinline__ void load_w1_frags(uint32_t (&w1f)[8][2], const __nv_bfloat16 *__restrict__ w16) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    const __nv_bfloat16 *row = w16 + oW1 + (8 * nt + g) * F;
    w1f[nt][0] = ld_u32(row + 2 * t);
    w1f[nt][1] = ld_u32(row + 2 * t + 8);
  }
}

// Logits of the 32 rows of a warp's feature tile sx[32][kXLd] (bf16, written
// by the warp beforehand and synchronised with __syncwarp).  Returns the
// logit of row `lane`.
__device__ __forceinline__ float tile_logits(const SmemNet &net, const uint32_t (&w1f)[8][2],
                                             const __nv_bfloat16 *sx) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t a2[2][4][4];  // layer-2 A fragments: [m-tile][k-step][reg]
#pragma unroll
  for (int mt = 0; mt < 2; mt++) {
    uint32_t a[4];
    const __nv_bfloat16 *r0 = sx + (16 * mt + g) * kXLd, *r1 = r0 + 8 * kXLd;
    a[0] = ld_u32(r0 + 2 * t);
    a[1] = ld_u32(r1 + 2 * t);
    a[2] = ld_u32(r0 + 2 * t + 8);
    a[3] = ld_u32(r1 + 2 * t + 8);
#pragma unroll
    for (int s = 0; s < 4; s++) {
      float c[2][4];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int col = 8 * (2 * s + h) + 2 * t;
        c[h][0] = c[h][2] = net.b1[col];
        c[h][1] = c[h][3] = net.b1[col + 1];
        mma_bf16_16816(c[h], a, w1f[2 * s + h][0], w1f[2 * s + h][1]);
      }
      a2[mt][s][0] = pack_bf16x2(fmaxf(c[0][0], 0.f), fmaxf(c[0][1], 0.f));
      a2[mt][s][1] = pack_bf16x2(fmaxf(c[0][2], 0.f), fmaxf(c[0][3], 0.f));
      a2[mt][s][2] = pack_bf16x2(fmaxf(c[1][0], 0.f), fmaxf(c[1][1], 0.f));
      a2[mt][s][3] = pack_bf16x2(fmaxf(c[1][2], 0.f), fmaxf(c[1][3], 0.f));
    }
  }
  float out[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    const int col = 8 * nt + 2 * t;
    const float b2lo = net.b2[col], b2hi = net.b2[col + 1], w3lo = net.w3[col], w3hi = net.w3[col + 1];
    float c[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
      c[mt][0] = c[mt][2] = b2lo;
      c[mt][1] = c[mt][3] = b2hi;
    }
    const __nv_bfloat16 *wr = net.W2 + (8 * nt + g) * kWLd;
#pragma unroll
    for (int s = 0; s < 4; s++) {
      const uint32_t b0 = ld_u32(wr + 16 * s + 2 * t), b1 = ld_u32(wr + 16 * s + 2 * t + 8);
#pragma unroll
      for (int mt = 0; mt < 2; mt++) mma_bf16_16816(c[mt], a2[mt][s], b0, b1);
    }
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
      out[mt][0] = fmaf(w3lo, fmaxf(c[mt][0], 0.f), fmaf(w3hi, fmaxf(c[mt][1], 0.f), out[mt][0]));
      out[mt][1] = fmaf(w3lo, fmaxf(c[mt][2], 0.f), fmaf(w3hi, fmaxf(c[mt][3], 0.f), out[mt][1]));
    }
  }
  // sum over the four threads of a quad (they hold different columns)
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int h = 0; h < 2; h++) {
      out[mt][h] += __shfl_xor_sync(0xffffffffu, out[mt][h], 1);
      out[mt][h] += __shfl_xor_sync(0xffffffffu, out[mt][h], 2);
    }
  // row r = 16 mt + 8 h + g is held by lanes 4g..4g+3
  const int src = (lane & 7) << 2;
  const float v00 = __shfl_sync(0xffffffffu, out[0][0], src), v01 = __shfl_sync(0xffffffffu, out[0][1], src);
  const float v10 = __shfl_sync(0xffffffffu, out[1][0], src), v11 = __shfl_sync(0xffffffffu, out[1][1], src);
  const int mt = lane >> 4, h = (lane >> 3) & 1;
  const float v = mt ? (h ? v11 : v10) : (h ? v01 : v00);
  return v + net.b3;
}

// One row of the feature tile from fp32 features (rounded to bf16).
__device__ __forceinline__ void store_row(__nv_bfloat16 *row, const float *f) {
#pragma unroll
  for (int i = 0; i < F; i += 2) *reinterpret_cast<uint32_t *>(row + i) = pack_bf16x2(f[i], f[i + 1]);
}

}  // namespace mlp
}  // namespace kz
