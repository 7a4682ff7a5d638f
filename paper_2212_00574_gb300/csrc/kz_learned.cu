// kz_learned.cu -- the learned schedule (include/kz_learned.h): an edge-
// scoring MLP with hand-written forward / backward / Adam kernels, a trace
// collector for its training data, and the worklist schedule that uses it;
// and, sharing its row views and buffers, the support schedule's re-check
// sweeps on the bitset rows (recheck_kernelize).
//
// The schedule never changes the kernel (thesis Section 4.2 rules): every
// deletion it makes is of an element that fails its rule on the current
// graph, and it stops only after a full plain sweep deletes nothing, so the
// result is the unique greatest fixpoint.
//
// Round structure of a learned kernelization (bitset rows):
//   1. full passes (the multi-CTA sweep or the tensor form) while the
//      cascade is heavy: as long as the last pass deleted so many edges that
//      the frontier they leave would cost more to test than a full pass;
//   2. learned rounds: per-vertex statistics of the live graph (degree,
//      colour cover, per-class counts; the vertex rule falls out of them);
//      the frontier = the edges that may have started to fail.  After edge
//      deletions alone that is the dirty set: an edge fails only by losing a
//      common neighbour, so deleting {a, b} can only make {a, w} and {b, w}
//      fail, w a common neighbour of a and b; after vertex deletions it is
//      every live edge at a vertex whose live degree changed.  The MLP scores
//      the frontier on the tensor cores and only edges above the threshold
//      are tested (warp per edge, exact, stopping once every needed class is
//      covered); the others wait in a pending set.  Failing vertices and
//      edges are removed in place;
//   3. when a learned round finds nothing, the pending edges are tested if
//      they are few (the score kernel keeps their count, so a large set
//      costs no flush), else a full pass certifies; if it deletes something,
//      learned rounds resume.
// A list that would cost more to test than a full pass (both timed during
// the run) gives way to the full pass.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/kz_learned.h"
#include "kz_internal.cuh"
#include "kz_mlp.cuh"
#include "kz_rules.cuh"

struct kz_model_s {
  float *w32 = nullptr;          // fp32 master weights
  __nv_bfloat16 *w16 = nullptr;  // bf16 inference copy
  float *m = nullptr, *v = nullptr;
  int64_t t = 0;
  int device = 0;
};

namespace kz {
namespace learned {

using namespace kz::mlp;

// ---------------------------------------------------------------------------
// MLP kernels (tensor cores: warp-level bf16 MMAs, see kz_mlp.cuh)
// ---------------------------------------------------------------------------

constexpr int kFwdWarps = 8;

// Logits of B feature rows X (fp32 [B][16]), 32 rows per warp step.
__global__ void __launch_bounds__(32 * kFwdWarps) mlp_forward_kernel(const __nv_bfloat16 *__restrict__ w16,
                                                                      const float *__restrict__ X, int64_t B,
                                                                      float *__restrict__ logits) {
  __shared__ SmemNet net;
  __shared__ __align__(16) __nv_bfloat16 sx[kFwdWarps][kTileRows * kXLd];
  load_net(net, w16);
  uint32_t w1f[8][2];
  load_w1_frags(w1f, w16);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * kFwdWarps * kTileRows;
  for (int64_t base = ((int64_t)blockIdx.x * kFwdWarps + warp) * kTileRows; base < B; base += stride) {
    const int64_t q = base + lane;
    float f[F];
#pragma unroll
    for (int i = 0; i < F; i++) f[i] = q < B ? X[q * F + i] : 0.f;
    store_row(sx[warp] + lane * kXLd, f);
    __syncwarp();
    const float l = tile_logits(net, w1f, sx[warp]);
    if (q < B) logits[q] = l;
    __syncwarp();
  }
}

// Mean BCE and its gradient, four warps per CTA, 64 samples per chunk (16 per
// warp).  Each warp runs the forward pass and the per-sample backward pass of
// its 16 samples in registers (the layer outputs turn into the next product's
// A fragments), and leaves the product operands the weight gradients need in
// shared memory, transposed to [feature or hidden unit][sample]; then every
// warp forms 16 rows of dW2 = dz2^T h1 and dW1 = dz1^T x over the chunk's
// samples (K = samples), accumulated in registers across the CTA's chunks.
constexpr int kGradWarps = 4;
constexpr int kChunk = 16 * kGradWarps;
constexpr int kSLd = kChunk + 8;  // row stride of the [unit][sample] tiles

struct GradSmem {
  SmemNet net;
  __nv_bfloat16 W2T[H * kWLd];  // W2 transposed: [i][j]
  __nv_bfloat16 x[kGradWarps][16 * kXLd];
  __nv_bfloat16 xT[F * kSLd];
  __nv_bfloat16 h1T[H * kSLd];
  __nv_bfloat16 dz2T[H * kSLd];
  __nv_bfloat16 dz1T[H * kSLd];
  float gb1[H], gb2[H], gw3[H];
  float gb3, loss;
};

__device__ __forceinline__ float quad_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v + __shfl_xor_sync(0xffffffffu, v, 2);
}

// sum over the eight row groups (lanes with the same t)
__device__ __forceinline__ float column_sum(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  return v + __shfl_xor_sync(0xffffffffu, v, 16);
}

__global__ void __launch_bounds__(32 * kGradWarps) mlp_grad_kernel(const __nv_bfloat16 *__restrict__ w16,
                                                                    const float *__restrict__ X,
                                                                    const float *__restrict__ y, int64_t B,
                                                                    float *__restrict__ grad,
                                                                    float *__restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smraw[];
  GradSmem &S = *reinterpret_cast<GradSmem *>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  load_net(S.net, w16);
  for (int e = tid; e < H * H; e += blockDim.x) S.W2T[(e % H) * kWLd + e / H] = w16[oW2 + e];
  for (int j = tid; j < H; j += blockDim.x) S.gb1[j] = S.gb2[j] = S.gw3[j] = 0.f;
  if (tid == 0) S.gb3 = S.loss = 0.f;
  uint32_t w1f[8][2];
  load_w1_frags(w1f, w16);
  __syncthreads();
  const SmemNet &net = S.net;
  const float invB = 1.f / (float)B;
  float accW2[8][4], accW1[2][4];
#pragma unroll
  for (int i = 0; i < 8; i++) accW2[i][0] = accW2[i][1] = accW2[i][2] = accW2[i][3] = 0.f;
#pragma unroll
  for (int i = 0; i < 2; i++) accW1[i][0] = accW1[i][1] = accW1[i][2] = accW1[i][3] = 0.f;
  const int scol = 16 * warp;  // this warp's sample columns in the transposed tiles

  for (int64_t c0 = (int64_t)blockIdx.x * kChunk; c0 < B; c0 += (int64_t)gridDim.x * kChunk) {
    const int64_t sbase = c0 + scol;
    __nv_bfloat16 *sx = S.x[warp];
    if (lane < 16) {
      const int64_t q = sbase + lane;
      float f[F];
#pragma unroll
      for (int i = 0; i < F; i++) f[i] = q < B ? X[q * F + i] : 0.f;
      store_row(sx + lane * kXLd, f);
#pragma unroll
      for (int i = 0; i < F; i++) S.xT[i * kSLd + scol + lane] = sx[lane * kXLd + i];
    }
    __syncwarp();
    // forward, layer 1: rows g and g + 8 of this warp's 16 samples
    uint32_t a[4];
    a[0] = ld_u32(sx + g * kXLd + 2 * t);
    a[1] = ld_u32(sx + (g + 8) * kXLd + 2 * t);
    a[2] = ld_u32(sx + g * kXLd + 2 * t + 8);
    a[3] = ld_u32(sx + (g + 8) * kXLd + 2 * t + 8);
    uint32_t a2[4][4];
    uint32_t z1pos = 0;  // bit 4 nt + e: element e of n-tile nt has z1 > 0
#pragma unroll
    for (int s = 0; s < 4; s++) {
      float c[2][4];
#pragma unroll
      for (int hh = 0; hh < 2; hh++) {
        const int nt = 2 * s + hh, col = 8 * nt + 2 * t;
        c[hh][0] = c[hh][2] = net.b1[col];
        c[hh][1] = c[hh][3] = net.b1[col + 1];
        mma_bf16_16816(c[hh], a, w1f[nt][0], w1f[nt][1]);
#pragma unroll
        for (int e = 0; e < 4; e++) {
          if (c[hh][e] > 0.f) z1pos |= 1u << (4 * nt + e);
          const __nv_bfloat16 hv = __float2bfloat16_rn(fmaxf(c[hh][e], 0.f));
          S.h1T[(col + (e & 1)) * kSLd + scol + g + 8 * (e >> 1)] = hv;
        }
      }
      a2[s][0] = pack_bf16x2(fmaxf(c[0][0], 0.f), fmaxf(c[0][1], 0.f));
      a2[s][1] = pack_bf16x2(fmaxf(c[0][2], 0.f), fmaxf(c[0][3], 0.f));
      a2[s][2] = pack_bf16x2(fmaxf(c[1][0], 0.f), fmaxf(c[1][1], 0.f));
      a2[s][3] = pack_bf16x2(fmaxf(c[1][2], 0.f), fmaxf(c[1][3], 0.f));
    }
    // forward, layer 2
    float z2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      const int col = 8 * nt + 2 * t;
      z2[nt][0] = z2[nt][2] = net.b2[col];
      z2[nt][1] = z2[nt][3] = net.b2[col + 1];
      const __nv_bfloat16 *wr = net.W2 + (8 * nt + g) * kWLd;
#pragma unroll
      for (int s = 0; s < 4; s++) mma_bf16_16816(z2[nt], a2[s], ld_u32(wr + 16 * s + 2 * t), ld_u32(wr + 16 * s + 2 * t + 8));
    }
    // output and loss of rows g (index 0) and g + 8 (index 1)
    float o[2] = {0.f, 0.f};
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      const int col = 8 * nt + 2 * t;
      o[0] = fmaf(net.w3[col], fmaxf(z2[nt][0], 0.f), fmaf(net.w3[col + 1], fmaxf(z2[nt][1], 0.f), o[0]));
      o[1] = fmaf(net.w3[col], fmaxf(z2[nt][2], 0.f), fmaf(net.w3[col + 1], fmaxf(z2[nt][3], 0.f), o[1]));
    }
    float dl[2], lterm = 0.f, dsum = 0.f;
#pragma unroll
    for (int r = 0; r < 2; r++) {
      const float logit = quad_sum(o[r]) + net.b3;
      const int64_t q = sbase + g + 8 * r;
      const bool valid = q < B;
      const float yy = valid ? y[q] : 0.f;
      const float sig = 1.f / (1.f + expf(-logit));
      dl[r] = valid ? (sig - yy) * invB : 0.f;
      if (valid && t == 0) {
        lterm += (fmaxf(logit, 0.f) - logit * yy + log1pf(expf(-fabsf(logit)))) * invB;
        dsum += dl[r];
      }
    }
    // per-sample backward of layer 3 and 2: dz2 = bf16(dl w3 [z2 > 0])
    uint32_t adz[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      const int col = 8 * nt + 2 * t;
      float dz[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int r = e >> 1, cc = col + (e & 1);
        dz[e] = __bfloat162float(__float2bfloat16_rn(z2[nt][e] > 0.f ? dl[r] * net.w3[cc] : 0.f));
        S.dz2T[cc * kSLd + scol + g + 8 * r] = __float2bfloat16_rn(dz[e]);
      }
      const float gw_lo = column_sum(dl[0] * fmaxf(z2[nt][0], 0.f) + dl[1] * fmaxf(z2[nt][2], 0.f));
      const float gw_hi = column_sum(dl[0] * fmaxf(z2[nt][1], 0.f) + dl[1] * fmaxf(z2[nt][3], 0.f));
      const float gb_lo = column_sum(dz[0] + dz[2]), gb_hi = column_sum(dz[1] + dz[3]);
      if (g == 0) {
        atomicAdd(&S.gw3[col], gw_lo);
        atomicAdd(&S.gw3[col + 1], gw_hi);
        atomicAdd(&S.gb2[col], gb_lo);
        atomicAdd(&S.gb2[col + 1], gb_hi);
      }
      const int s = nt >> 1, base = (nt & 1) * 2;
      adz[s][base] = pack_bf16x2(dz[0], dz[1]);
      adz[s][base + 1] = pack_bf16x2(dz[2], dz[3]);
    }
    // dh1 = dz2 W2 (K = hidden units j), then dz1 = bf16(dh1 [z1 > 0])
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      const __nv_bfloat16 *wr = S.W2T + (8 * nt + g) * kWLd;
#pragma unroll
      for (int s = 0; s < 4; s++) mma_bf16_16816(c, adz[s], ld_u32(wr + 16 * s + 2 * t), ld_u32(wr + 16 * s + 2 * t + 8));
      const int col = 8 * nt + 2 * t;
      float dz[4];
#pragma unroll
      for (int e = 0; e < 4; e++) {
        dz[e] = __bfloat162float(__float2bfloat16_rn(((z1pos >> (4 * nt + e)) & 1u) ? c[e] : 0.f));
        S.dz1T[(col + (e & 1)) * kSLd + scol + g + 8 * (e >> 1)] = __float2bfloat16_rn(dz[e]);
      }
      const float gb_lo = column_sum(dz[0] + dz[2]), gb_hi = column_sum(dz[1] + dz[3]);
      if (g == 0) {
        atomicAdd(&S.gb1[col], gb_lo);
        atomicAdd(&S.gb1[col + 1], gb_hi);
      }
    }
    // warp sums of the loss terms and of dl (one thread per row holds them)
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      lterm += __shfl_xor_sync(0xffffffffu, lterm, o2);
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o2);
    }
    if (lane == 0) {
      atomicAdd(&S.loss, lterm);
      atomicAdd(&S.gb3, dsum);
    }
    __syncthreads();
    // weight gradients over the chunk: warp w forms rows j in [16 w, 16 w + 16)
#pragma unroll
    for (int ks = 0; ks < kChunk / 16; ks++) {
      uint32_t ad2[4], ad1[4];
      const int r0 = 16 * warp + g, k0 = 16 * ks + 2 * t;
      ad2[0] = ld_u32(S.dz2T + r0 * kSLd + k0);
      ad2[1] = ld_u32(S.dz2T + (r0 + 8) * kSLd + k0);
      ad2[2] = ld_u32(S.dz2T + r0 * kSLd + k0 + 8);
      ad2[3] = ld_u32(S.dz2T + (r0 + 8) * kSLd + k0 + 8);
      ad1[0] = ld_u32(S.dz1T + r0 * kSLd + k0);
      ad1[1] = ld_u32(S.dz1T + (r0 + 8) * kSLd + k0);
      ad1[2] = ld_u32(S.dz1T + r0 * kSLd + k0 + 8);
      ad1[3] = ld_u32(S.dz1T + (r0 + 8) * kSLd + k0 + 8);
#pragma unroll
      for (int nt = 0; nt < 8; nt++) {
        const __nv_bfloat16 *hr = S.h1T + (8 * nt + g) * kSLd + k0;
        mma_bf16_16816(accW2[nt], ad2, ld_u32(hr), ld_u32(hr + 8));
      }
#pragma unroll
      for (int nt = 0; nt < 2; nt++) {
        const __nv_bfloat16 *xr = S.xT + (8 * nt + g) * kSLd + k0;
        mma_bf16_16816(accW1[nt], ad1, ld_u32(xr), ld_u32(xr + 8));
      }
    }
    __syncthreads();
  }
  // this CTA's sums into the global gradient
  {
    const int j0 = 16 * warp + g;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      const int i = 8 * nt + 2 * t;
      atomicAdd(&grad[oW2 + j0 * H + i], accW2[nt][0]);
      atomicAdd(&grad[oW2 + j0 * H + i + 1], accW2[nt][1]);
      atomicAdd(&grad[oW2 + (j0 + 8) * H + i], accW2[nt][2]);
      atomicAdd(&grad[oW2 + (j0 + 8) * H + i + 1], accW2[nt][3]);
    }
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
      const int i = 8 * nt + 2 * t;
      atomicAdd(&grad[oW1 + j0 * F + i], accW1[nt][0]);
      atomicAdd(&grad[oW1 + j0 * F + i + 1], accW1[nt][1]);
      atomicAdd(&grad[oW1 + (j0 + 8) * F + i], accW1[nt][2]);
      atomicAdd(&grad[oW1 + (j0 + 8) * F + i + 1], accW1[nt][3]);
    }
  }
  __syncthreads();
  for (int j = tid; j < H; j += blockDim.x) {
    atomicAdd(&grad[ob1 + j], S.gb1[j]);
    atomicAdd(&grad[ob2 + j], S.gb2[j]);
    atomicAdd(&grad[ow3 + j], S.gw3[j]);
  }
  if (tid == 0) {
    atomicAdd(&grad[ob3], S.gb3);
    atomicAdd(loss, S.loss);
  }
}

__global__ void adam_kernel(float *__restrict__ w32, __nv_bfloat16 *__restrict__ w16, float *__restrict__ m,
                            float *__restrict__ v, const float *__restrict__ g, float lr, float bc1, float bc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w32[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    w32[i] = wi;
    w16[i] = __float2bfloat16(wi);
  }
}

__global__ void to_bf16_kernel(const float *__restrict__ w32, __nv_bfloat16 *__restrict__ w16) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x)
    w16[i] = __float2bfloat16(w32[i]);
}

// ---------------------------------------------------------------------------
// per-vertex statistics of the live graph (bitset rows)
// ---------------------------------------------------------------------------

struct Stats {
  int32_t *deg;       // live degree
  int32_t *prevdeg;   // live degree at the previous round
  int32_t *cover;     // classes other than own with a live neighbour
  int32_t *minc;      // smallest neighbour count over the other classes
  uint8_t *vfail;     // vertex rule fails on this snapshot
  uint8_t *changed;   // live degree changed since the previous round
  int32_t *ccnt;      // n x k: live neighbours of each class
};

struct RowView {
  uint32_t *A;        // current rows (updated in place by learned rounds)
  uint32_t *V;        // current live words
  int32_t n, k, ldw, R;
  const int32_t *col;   // relabelled colour
  const int32_t *coff;  // k + 1
};

__device__ __forceinline__ bool vertex_live(const RowView &r, int x) {
  const int c = r.col[x], i = x - r.coff[c];
  return (r.V[(i >> 5) * r.k + c] >> (i & 31)) & 1u;
}

// One warp per vertex; per-class neighbour counts in shared memory.
__global__ void stats_kernel(RowView r, Stats s, int first_round, unsigned long long *dv_out) {
  __shared__ int cls[8][64];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long dv = 0;
  for (int64_t x = warp0; x < r.n; x += warps) {
    for (int c = lane; c < 64; c += 32) cls[wib][c] = 0;
    __syncwarp();
    const uint32_t *row = r.A + x * r.ldw;
    const int rk = r.R * r.k;
    for (int w = lane; w < rk; w += 32) {
      const uint32_t word = row[w];
      if (word) atomicAdd(&cls[wib][w % r.k], __popc(word));
    }
    __syncwarp();
    for (int c = lane; c < r.k; c += 32) s.ccnt[x * r.k + c] = cls[wib][c];
    if (lane == 0) {
      const int own = r.col[x];
      int deg = 0, cover = 0, minc = 0x7fffffff;
      for (int c = 0; c < r.k; c++) {
        deg += cls[wib][c];
        if (c == own) continue;
        cover += cls[wib][c] > 0;
        minc = min(minc, cls[wib][c]);
      }
      if (r.k == 1) minc = 0;
      const bool live = vertex_live(r, (int)x);
      const bool fail = live && cover < r.k - 1;
      s.vfail[x] = fail ? 1 : 0;
      dv += fail;
      s.changed[x] = first_round ? 1 : (uint8_t)(deg != s.deg[x]);
      s.prevdeg[x] = first_round ? deg : s.deg[x];
      s.deg[x] = deg;
      s.cover[x] = cover;
      s.minc[x] = minc;
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) dv += __shfl_down_sync(0xffffffffu, dv, o);
  if (lane == 0 && dv) atomicAdd(dv_out, dv);
}

// Frontier: live edges {x, y} with a changed endpoint, each emitted once.
__global__ void frontier_kernel(RowView r, Stats s, int2 *__restrict__ out, unsigned long long *count,
                                int64_t cap) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = warp0; x < r.n; x += warps) {
    if (!s.changed[x]) continue;
    const uint32_t *row = r.A + x * r.ldw;
    const int rk = r.R * r.k;
    for (int w0 = 0; w0 < rk; w0 += 32) {
      const int w = w0 + lane;
      uint32_t word = w < rk ? row[w] : 0u;
      const int c = w % r.k, rr = w / r.k;
      // keep y when y is unchanged or x < y (each edge once)
      uint32_t keep = 0;
      while (word) {
        const int b = __ffs(word) - 1;
        word &= word - 1;
        const int y = r.coff[c] + 32 * rr + b;
        if (!s.changed[y] || x < y) keep |= 1u << b;
      }
      const int cnt = __popc(keep);
      int incl = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      unsigned long long base = 0;
      if (lane == 31 && total) base = atomicAdd(count, (unsigned long long)total);
      base = __shfl_sync(0xffffffffu, base, 31);
      unsigned long long pos = base + (incl - cnt);
      while (keep) {
        const int b = __ffs(keep) - 1;
        keep &= keep - 1;
        if ((int64_t)pos < cap) out[pos] = make_int2((int)x, r.coff[c] + 32 * rr + b);
        pos++;
      }
    }
  }
}

__device__ __forceinline__ void edge_features(const RowView &r, const Stats &s, int x, int y, int round,
                                              float density, float live_frac, float *f) {
  const float n = (float)max(r.n, 1);
  const float k = (float)r.k;
  const float du = (float)s.deg[x], dvv = (float)s.deg[y];
  f[0] = du / n;
  f[1] = dvv / n;
  f[2] = ((float)s.cover[x] - (k - 1.f)) / k;
  f[3] = ((float)s.cover[y] - (k - 1.f)) / k;
  f[4] = (float)s.minc[x] / fmaxf(n / k, 1.f);
  f[5] = (float)s.minc[y] / fmaxf(n / k, 1.f);
  f[6] = (du - (float)s.prevdeg[x]) / fmaxf((float)s.prevdeg[x], 1.f);
  f[7] = (dvv - (float)s.prevdeg[y]) / fmaxf((float)s.prevdeg[y], 1.f);
  f[8] = k / 64.f;
  f[9] = (float)round / 32.f;
  f[10] = density;
  f[11] = fminf(du, dvv) / fmaxf(fmaxf(du, dvv), 1.f);
  f[12] = (du + dvv) / (2.f * n);
  f[13] = log2f(n) / 16.f;
  f[14] = live_frac;
  // the chance that some needed class holds no common neighbour if each
  // endpoint's neighbours in a class were drawn at random from it: with
  // lambda = sum over needed classes c of exp(-cnt_x[c] cnt_y[c] / |C_c|)
  // (the expected number of uncovered classes), 1 - exp(-lambda)
  const int cx = r.col[x], cy = r.col[y];
  const int32_t *ax = s.ccnt + (int64_t)x * r.k, *ay = s.ccnt + (int64_t)y * r.k;
  float lam = 0.f;
  for (int c = 0; c < r.k; c++) {
    if (c == cx || c == cy) continue;
    const float size = (float)max(r.coff[c + 1] - r.coff[c], 1);
    lam += __expf(-(float)ax[c] * (float)ay[c] / size);
  }
  f[15] = 1.f - __expf(-lam);
}

// Pending-set bit of the (unordered) pair {x, y}: kept in the row of the
// smaller id, at the word and bit of the larger one.
__device__ __forceinline__ void pend_bit(const RowView &r, int x, int y, int64_t &word, uint32_t &bit) {
  const int a = min(x, y), b = max(x, y);
  const int cb = r.col[b], ib = b - r.coff[cb];
  word = (int64_t)a * r.ldw + (ib >> 5) * r.k + cb;
  bit = 1u << (ib & 31);
}

// Scores the frontier on the tensor cores: each warp takes 32 frontier edges
// at a time, computes their features (one edge per lane) into a bf16 tile in
// shared memory and runs the network on it (kz_mlp.cuh).  Edges above the
// threshold are listed for an exact test this round (and leave the pending
// set); the others join the pending set, to be tested later unless they die
// first; n_pend keeps the size of the pending set (an upper bound on its
// live part: pending edges that lost an endpoint stay counted).  The live
// counts for the density features come from the device (cnt[4] = twice the
// live edges, cnt[5] = live vertices).
constexpr int kScoreWarps = 8;

__global__ void __launch_bounds__(32 * kScoreWarps) score_kernel(RowView r, Stats s,
                                                                  const __nv_bfloat16 *__restrict__ w16,
                                                                  const int2 *__restrict__ fr,
                                                                  const unsigned long long *__restrict__ cnt,
                                                                  float logit_threshold, int round,
                                                                  int2 *__restrict__ work,
                                                                  unsigned long long *n_work,
                                                                  uint32_t *__restrict__ pend,
                                                                  unsigned long long *n_pend) {
  __shared__ SmemNet net;
  __shared__ __align__(16) __nv_bfloat16 sx[kScoreWarps][kTileRows * kXLd];
  const bool all = !(logit_threshold > -INFINITY);
  if (!all) load_net(net, w16);
  uint32_t w1f[8][2];
  if (!all) load_w1_frags(w1f, w16);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t total = (int64_t)cnt[0];
  const double nn = (double)max(r.n, 1);
  const float density = (float)((double)cnt[4] / (nn * fmax(nn - 1.0, 1.0)));
  const float live_frac = (float)((double)cnt[5] / nn);
  const int64_t stride = (int64_t)gridDim.x * kScoreWarps * kTileRows;
  for (int64_t base = ((int64_t)blockIdx.x * kScoreWarps + warp) * kTileRows; base < total; base += stride) {
    const int64_t q = base + lane;
    const bool valid = q < total;
    const int2 e = valid ? fr[q] : make_int2(0, 0);
    bool take = valid;
    if (!all) {
      float f[F];
      if (valid) {
        edge_features(r, s, e.x, e.y, round, density, live_frac, f);
      } else {
#pragma unroll
        for (int i = 0; i < F; i++) f[i] = 0.f;
      }
      store_row(sx[warp] + lane * kXLd, f);
      __syncwarp();
      const float logit = tile_logits(net, w1f, sx[warp]);
      take = valid && logit > logit_threshold;
      __syncwarp();
    }
    int delta = 0;  // change of the pending count by this lane's edge
    if (valid) {
      int64_t pw;
      uint32_t pb;
      pend_bit(r, e.x, e.y, pw, pb);
      if (take) delta = (atomicAnd(&pend[pw], ~pb) & pb) ? -1 : 0;
      else delta = (atomicOr(&pend[pw], pb) & pb) ? 0 : 1;
    }
    delta = __reduce_add_sync(0xffffffffu, delta);
    if (lane == 0 && delta) atomicAdd(n_pend, (unsigned long long)(long long)delta);
    const uint32_t m = __ballot_sync(0xffffffffu, take);
    unsigned long long at = 0;
    if (lane == 0 && m) at = atomicAdd(n_work, (unsigned long long)__popc(m));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (take) work[at + __popc(m & ((1u << lane) - 1u))] = e;
  }
}

// Flush: every pending edge that is still live, listed once; the pending
// set is cleared.
__global__ void flush_pending_kernel(RowView r, uint32_t *__restrict__ pend, int2 *__restrict__ out,
                                     unsigned long long *count, int64_t cap) {
  const int rk = r.R * r.k;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = tid; t < (int64_t)r.n * rk; t += stride) {
    const int64_t x = t / rk;
    const int w = (int)(t - x * rk);
    const int64_t idx = x * r.ldw + w;
    uint32_t bits = pend[idx] & r.A[idx];
    if (!pend[idx]) continue;
    pend[idx] = 0u;
    const int c = w % r.k, rr = w / r.k;
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      const unsigned long long pos = atomicAdd(count, 1ull);
      if ((int64_t)pos < cap) out[pos] = make_int2((int)x, r.coff[c] + 32 * rr + b);
    }
  }
}

// Edges deleted by the last full pass (set in the old rows, clear in the new
// ones), each listed once, from its smaller end.
__global__ void diff_dead_kernel(RowView rold, const uint32_t *__restrict__ Anew, int2 *__restrict__ out,
                                 unsigned long long *count, int64_t cap) {
  const int rk = rold.R * rold.k;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = tid; t < (int64_t)rold.n * rk; t += stride) {
    const int64_t x = t / rk;
    const int w = (int)(t - x * rk);
    const int64_t idx = x * rold.ldw + w;
    uint32_t bits = rold.A[idx] & ~Anew[idx];
    const int c = w % rold.k, rr = w / rold.k;
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      const int y = rold.coff[c] + 32 * rr + b;
      if (y <= (int)x) continue;
      const unsigned long long pos = atomicAdd(count, 1ull);
      if ((int64_t)pos < cap) out[pos] = make_int2((int)x, y);
    }
  }
}

// Dirty pairs of a round's edge deletions.  An edge can start failing only
// by losing a common neighbour, so when {a, b} goes, the edges that can
// start failing are {a, w} and {b, w} for the w in N(a) and N(b) both (rows
// as they were before the deletions, so that two deletions at the same w
// are seen too).  Every such pair joins the dirty set (pending-set layout);
// n_marks counts the pairs newly set.  One warp per deleted edge, the two
// rows read four words a lane at a time.
__global__ void mark_dirty_kernel(RowView rold, const int2 *__restrict__ dead,
                                  const unsigned long long *__restrict__ n_dead, int64_t cap,
                                  uint32_t *__restrict__ dirty, unsigned long long *n_marks) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = min((int64_t)*n_dead, cap);
  const int rk = rold.R * rold.k;
  for (int64_t q = warp0; q < total; q += warps) {
    const int2 e = dead[q];
    const uint32_t *ra = rold.A + (int64_t)e.x * rold.ldw, *rb = rold.A + (int64_t)e.y * rold.ldw;
    unsigned int added = 0;
    for (int w = 4 * lane; w < rk; w += 128) {
      const uint4 a = *reinterpret_cast<const uint4 *>(ra + w);
      const uint4 b = *reinterpret_cast<const uint4 *>(rb + w);
      const uint32_t both[4] = {a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        uint32_t m = both[j];
        if (!m) continue;  // also every zero padding word past rk
        const int c = (w + j) % rold.k, rr = (w + j) / rold.k;
        while (m) {
          const int bit = __ffs(m) - 1;
          m &= m - 1;
          const int y = rold.coff[c] + 32 * rr + bit;
          int64_t pw;
          uint32_t pb;
          pend_bit(rold, e.x, y, pw, pb);
          added += (atomicOr(&dirty[pw], pb) & pb) ? 0u : 1u;
          pend_bit(rold, e.y, y, pw, pb);
          added += (atomicOr(&dirty[pw], pb) & pb) ? 0u : 1u;
        }
      }
    }
    added = __reduce_add_sync(0xffffffffu, added);
    if (lane == 0 && added) atomicAdd(n_marks, (unsigned long long)added);
  }
}

// Up to `cap` live edges {x, y}, x < y, from every `step`-th row (a sample
// spread over the classes, for timing the exact test).  The count may pass
// cap; clamp_kernel brings it back.
__global__ void sample_edges_kernel(RowView r, int2 *__restrict__ out, unsigned long long *count, int64_t cap,
                                    int32_t step) {
  const int rk = r.R * r.k;
  const int64_t rows = ((int64_t)r.n + step - 1) / step;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = tid; t < rows * rk; t += stride) {
    if (*(volatile unsigned long long *)count >= (unsigned long long)cap) return;
    const int64_t j = t / rk;
    const int w = (int)(t - j * rk);
    const int64_t x = j * step;
    uint32_t bits = r.A[x * r.ldw + w];
    const int c = w % r.k, rr = w / r.k;
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      const int y = r.coff[c] + 32 * rr + b;
      if (y <= (int)x) continue;
      const unsigned long long pos = atomicAdd(count, 1ull);
      if ((int64_t)pos >= cap) return;
      out[pos] = make_int2((int)x, y);
    }
  }
}

__global__ void clamp_kernel(unsigned long long *count, unsigned long long cap) {
  if (*count > cap) *count = cap;
}

// Vertex and edge deletions of the last productive full pass, from the
// device state's per-sweep record (all ones when the record is not kept).
__global__ void last_pass_kernel(const DevState *st, unsigned long long *out) {
  const int64_t i = st->sweeps - 1;
  const bool kept = i >= 0 && i < kTraceCap;
  out[0] = kept ? (unsigned long long)st->trace_dv[i] : ~0ull;
  out[1] = kept ? (unsigned long long)st->trace_de[i] : ~0ull;
}

// Exact edge rule for listed edges, one warp per edge.  The lanes read the
// two rows four words at a time (a row is 16-byte aligned and zero-padded to
// a multiple of four words) and stop as soon as every class the edge needs
// has a common neighbour: on a dense graph the first plane settles it.
__global__ void test_edges_kernel(RowView r, const int2 *__restrict__ work, const unsigned long long *__restrict__ n_work,
                                  int2 *__restrict__ dead, unsigned long long *n_dead) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = (int64_t)*n_work;
  const int rk = r.R * r.k;
  const uint64_t every = r.k >= 64 ? ~0ull : ((1ull << r.k) - 1ull);
  for (int64_t q = warp0; q < total; q += warps) {
    const int2 e = work[q];
    const uint32_t *ru = r.A + (int64_t)e.x * r.ldw, *rv = r.A + (int64_t)e.y * r.ldw;
    const uint64_t need = every & ~((1ull << r.col[e.x]) | (1ull << r.col[e.y]));
    uint64_t all = 0;
    for (int w0 = 0; w0 < rk; w0 += 128) {
      const int w = w0 + 4 * lane;
      uint64_t cov = 0;
      if (w < rk) {
        const uint4 a = *reinterpret_cast<const uint4 *>(ru + w);
        const uint4 b = *reinterpret_cast<const uint4 *>(rv + w);
        const int c = w % r.k;
        if (a.x & b.x) cov |= 1ull << c;
        if (a.y & b.y) cov |= 1ull << ((c + 1) % r.k);
        if (a.z & b.z) cov |= 1ull << ((c + 2) % r.k);
        if (a.w & b.w) cov |= 1ull << ((c + 3) % r.k);
      }
      const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)cov);
      const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(cov >> 32));
      all |= ((uint64_t)hi << 32) | lo;
      if ((all & need) == need) break;
    }
    if (lane == 0 && __popcll(all & need) < r.k - 2) dead[atomicAdd(n_dead, 1ull)] = e;
  }
}

// Removes the failing edges and the failing vertices (with all their edges)
// in place, recording each failing vertex's sweep.
__global__ void apply_kernel(RowView r, const uint8_t *__restrict__ vfail, const int2 *__restrict__ dead,
                             const unsigned long long *__restrict__ n_dead, int32_t *__restrict__ v_sweep,
                             const DevState *st) {
  const int lane = threadIdx.x & 31;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nd = (int64_t)*n_dead;
  for (int64_t q = tid; q < nd; q += stride) {
    const int x = dead[q].x, y = dead[q].y;
    const int cx = r.col[x], cy = r.col[y], ix = x - r.coff[cx], iy = y - r.coff[cy];
    atomicAnd(&r.A[(int64_t)x * r.ldw + (iy >> 5) * r.k + cy], ~(1u << (iy & 31)));
    atomicAnd(&r.A[(int64_t)y * r.ldw + (ix >> 5) * r.k + cx], ~(1u << (ix & 31)));
  }
  const int64_t warp0 = tid >> 5, warps = stride >> 5;
  const int rk = r.R * r.k;
  for (int64_t x = warp0; x < r.n; x += warps) {
    if (!vfail[x]) continue;
    const int cx = r.col[x], ix = (int)x - r.coff[cx];
    uint32_t *row = r.A + x * r.ldw;
    for (int w = lane; w < rk; w += 32) {
      uint32_t word = row[w];
      const int c = w % r.k, rr = w / r.k;
      while (word) {
        const int b = __ffs(word) - 1;
        word &= word - 1;
        const int y = r.coff[c] + 32 * rr + b;
        atomicAnd(&r.A[(int64_t)y * r.ldw + (ix >> 5) * r.k + cx], ~(1u << (ix & 31)));
      }
      row[w] = 0u;
    }
    if (lane == 0) {
      atomicAnd(&r.V[(ix >> 5) * r.k + cx], ~(1u << (ix & 31)));
      if (v_sweep) v_sweep[x] = (int32_t)(st->sweeps + 1);  // the productive sweep this round becomes
    }
  }
}

// ---------------------------------------------------------------------------
// dense support rounds (schedule SUPPORT on the bitset rows)
// ---------------------------------------------------------------------------

// Class-major copy of the rows: row x's words of class c (planes 0 .. R - 1,
// zero-padded to Rp, a multiple of four) at x * k * Rp + c * Rp, so that a
// class's words are contiguous for the re-checks.
__global__ void class_major_kernel(const uint32_t *__restrict__ A, int32_t n, int32_t k, int32_t R, int32_t ldw,
                                   int32_t Rp, uint32_t *__restrict__ cm) {
  const int64_t row = (int64_t)k * Rp;
  const int64_t total = (int64_t)n * row;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = t / row;
    const int q = (int)(t - x * row), c = q / Rp, rr = q - c * Rp;
    cm[t] = rr < R ? A[x * ldw + (int64_t)rr * k + c] : 0u;
  }
}

// Re-check of one live pair {x, y} in class c on the current rows: does it
// keep a common neighbour in c (class c's words of both rows from the
// class-major copy, eight at a time in 16-byte loads, stopping at the first
// step with one)?  A pair with none fails and is listed once
// (failed bitset, pending-set layout).  Returns 1 when the pair is
// re-checked for the first time this round (checked bitset).
__device__ __forceinline__ unsigned int recheck_pair(const RowView &r, const uint32_t *__restrict__ cm, int Rp,
                                                     int x, int y, int c, uint32_t *__restrict__ failed,
                                                     int2 *__restrict__ out, unsigned long long *n_out, int64_t cap,
                                                     uint32_t *__restrict__ checked) {
  int64_t pw;
  uint32_t pb;
  pend_bit(r, x, y, pw, pb);
  const unsigned int first = (atomicOr(&checked[pw], pb) & pb) ? 0u : 1u;
  const int64_t cmw = (int64_t)r.k * Rp;
  const uint4 *px = reinterpret_cast<const uint4 *>(cm + x * cmw + (int64_t)c * Rp);
  const uint4 *py = reinterpret_cast<const uint4 *>(cm + y * cmw + (int64_t)c * Rp);
  const int quads = Rp >> 2;
  for (int q = 0; q < quads; q += 2) {
    const uint4 a0 = px[q], b0 = py[q];
    uint32_t any = (a0.x & b0.x) | (a0.y & b0.y) | (a0.z & b0.z) | (a0.w & b0.w);
    if (q + 1 < quads) {
      const uint4 a1 = px[q + 1], b1 = py[q + 1];
      any |= (a1.x & b1.x) | (a1.y & b1.y) | (a1.z & b1.z) | (a1.w & b1.w);
    }
    if (any) return first;
  }
  if (!(atomicOr(&failed[pw], pb) & pb)) {
    const unsigned long long pos = atomicAdd(n_out, 1ull);
    if ((int64_t)pos < cap) out[pos] = make_int2(min(x, y), max(x, y));
  }
  return first;
}

// Resident CTAs of the re-check kernel per SM: it waits on scattered loads,
// so it is capped at 40 registers for six CTAs (48 warps) an SM, and its
// grid-strided launch is exactly that many CTAs.  (Measured on the C5-size
// cascade: 71 ms to the fixpoint at three CTAs an SM, 60 ms at six, 70 ms at
// eight, where 32 registers spill.)
constexpr int kRecheckCtasPerSm = 6;

// One sweep of the dense support schedule (over the deleted edges q0 .. q1 -
// 1 of the list).  The edges the previous sweep deleted are the only cause
// of new failures: deleting {a, b} takes the
// common neighbour b (class col b) from every pair {a, w} and a (class col a)
// from every {b, w}, w in N(a) and N(b) in the rows before that sweep
// (rold).  One warp per deleted edge walks those w (four row words a lane)
// and re-checks each (pair, class) on the current rows (rnew, and their
// class-major copy cm); every edge
// that fails the edge rule on the current graph is found this way, since it
// passed before the previous sweep.  A failing vertex's edges all fail the
// edge rule too (no common neighbour can have the colour it lost), so the
// listed edges are the sweep's whole edge deletion.
__global__ void __launch_bounds__(256, kRecheckCtasPerSm) recheck_kernel(RowView rold, RowView rnew, const uint32_t *__restrict__ cm, int32_t Rp,
                               const int2 *__restrict__ dead,
                               const unsigned long long *__restrict__ n_dead, int64_t q0, int64_t q1, int64_t cap,
                               uint32_t *__restrict__ failed, int2 *__restrict__ out, unsigned long long *n_out,
                               uint32_t *__restrict__ checked, unsigned long long *n_checked) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = min(min((int64_t)*n_dead, cap), q1);
  const int rk = rold.R * rold.k;
  unsigned int first = 0;
  for (int64_t q = q0 + warp0; q < total; q += warps) {
    const int2 e = dead[q];
    const int ca = rold.col[e.x], cb = rold.col[e.y];
    const uint32_t *ra = rold.A + (int64_t)e.x * rold.ldw, *rb = rold.A + (int64_t)e.y * rold.ldw;
    const uint32_t *na = rnew.A + (int64_t)e.x * rnew.ldw, *nb = rnew.A + (int64_t)e.y * rnew.ldw;
    for (int w = 4 * lane; w < rk; w += 128) {
      const uint4 a = *reinterpret_cast<const uint4 *>(ra + w);
      const uint4 b = *reinterpret_cast<const uint4 *>(rb + w);
      const uint32_t both[4] = {a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w};
      if (!(both[0] | both[1] | both[2] | both[3])) continue;
      // the same words of the current rows: which pairs {a, w}, {b, w} are live
      const uint4 a2 = *reinterpret_cast<const uint4 *>(na + w);
      const uint4 b2 = *reinterpret_cast<const uint4 *>(nb + w);
      const uint32_t live_a[4] = {a2.x, a2.y, a2.z, a2.w}, live_b[4] = {b2.x, b2.y, b2.z, b2.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        uint32_t m = both[j];
        if (!m) continue;  // also every zero padding word past rk
        const int c = (w + j) % rold.k, rr = (w + j) / rold.k;
        while (m) {
          const int bit = __ffs(m) - 1;
          m &= m - 1;
          const int y = rold.coff[c] + 32 * rr + bit;
          if ((live_a[j] >> bit) & 1u) first += recheck_pair(rnew, cm, Rp, e.x, y, cb, failed, out, n_out, cap, checked);
          if ((live_b[j] >> bit) & 1u) first += recheck_pair(rnew, cm, Rp, e.y, y, ca, failed, out, n_out, cap, checked);
        }
      }
    }
  }
  first = __reduce_add_sync(0xffffffffu, first);
  if (lane == 0 && first) atomicAdd(n_checked, (unsigned long long)first);
}

// Closes a dense support sweep: the counts, the trace, and the flip to the
// buffer that now holds the state.  Nothing deleted: one unproductive pass.
__global__ void recheck_finish_kernel(DevState *st, const unsigned long long *dv, const unsigned long long *de,
                                      const unsigned long long *tests) {
  st->passes += 1;
  st->tests += (int64_t)*tests;
  if (*dv + *de > 0) {
    if (st->sweeps < kTraceCap) {
      st->trace_dv[st->sweeps] = (int64_t)*dv;
      st->trace_de[st->sweeps] = (int64_t)*de;
    }
    st->sweeps += 1;
    st->cur ^= 1;
  }
}

// Records a learned round (no buffer flip: learned rounds work in place).
__global__ void learned_finish_kernel(DevState *st, const unsigned long long *dv, const unsigned long long *de,
                                      const unsigned long long *tests, int32_t *v_sweep_unused) {
  (void)v_sweep_unused;
  st->passes += 1;
  st->tests += (int64_t)*tests;
  if (*dv + *de > 0) {
    if (st->sweeps < kTraceCap) {
      st->trace_dv[st->sweeps] = (int64_t)*dv;
      st->trace_de[st->sweeps] = (int64_t)*de;
    }
    st->sweeps += 1;
  }
}

// Live edges counted from the rows (for the density feature and the check).
__global__ void count_live_kernel(RowView r, unsigned long long *edges2, unsigned long long *verts) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long e = 0, v = 0;
  const int rk = r.R * r.k;
  for (int64_t t = tid; t < (int64_t)r.n * rk; t += stride) e += __popc(r.A[(t / rk) * r.ldw + t % rk]);
  for (int64_t x = tid; x < r.n; x += stride) v += vertex_live(r, (int)x);
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_down_sync(0xffffffffu, e, o);
    v += __shfl_down_sync(0xffffffffu, v, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (e) atomicAdd(edges2, e);
    if (v) atomicAdd(verts, v);
  }
}

// Trace records: features of a hashed subsample of the live edges of this
// sweep with the label "fails the edge rule on this snapshot".
__global__ void trace_kernel(RowView r, Stats s, int round, float density, float live_frac, uint64_t seed,
                             uint32_t keep_below, float *__restrict__ X, uint8_t *__restrict__ y,
                             unsigned long long *count, int64_t cap) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int rk = r.R * r.k;
  for (int64_t x = warp0; x < r.n; x += warps) {
    const uint32_t *ru = r.A + x * r.ldw;
    for (int w0 = 0; w0 < rk; w0 += 32) {
      const int w = w0 + lane;
      uint32_t word = w < rk ? ru[w] : 0u;
      const int c = w % r.k, rr = w / r.k;
      while (word) {
        const int b = __ffs(word) - 1;
        word &= word - 1;
        const int yv = r.coff[c] + 32 * rr + b;
        if (yv <= x) continue;
        uint64_t h = seed ^ ((uint64_t)x << 32 | (uint32_t)yv) ^ ((uint64_t)round * 0x9e3779b97f4a7c15ull);
        h ^= h >> 33;
        h *= 0xff51afd7ed558ccdull;
        h ^= h >> 33;
        if ((uint32_t)(h >> 32) >= keep_below) continue;
        // label: exact edge rule on this snapshot (serial over the rows)
        const uint32_t *rv = r.A + (int64_t)yv * r.ldw;
        uint64_t cov = 0;
        for (int q = 0; q < rk; q++)
          if (ru[q] & rv[q]) cov |= 1ull << (q % r.k);
        const uint64_t own = (1ull << r.col[x]) | (1ull << r.col[yv]);
        const bool fails = __popcll(cov & ~own) < r.k - 2;
        const unsigned long long pos = atomicAdd(count, 1ull);
        if ((int64_t)pos < cap) {
          float f[F];
          edge_features(r, s, (int)x, yv, round, density, live_frac, f);
#pragma unroll
          for (int i = 0; i < F; i++) X[pos * F + i] = f[i];
          y[pos] = fails ? 1 : 0;
        }
      }
    }
  }
}

}  // namespace learned
}  // namespace kz

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

using namespace kz;
using namespace kz::learned;

namespace {

int sms_now() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}

constexpr int kCounters = 10;

// Per-graph scratch of the learned schedule (allocated on first use).
struct LearnedBufs {
  Stats s;
  int2 *fr = nullptr, *work = nullptr, *dead = nullptr;
  uint32_t *pend = nullptr;   // pending edges (bitset rows, pair kept in the smaller id's row)
  uint32_t *dirty = nullptr;  // dirty edges: may have started failing (same layout)
  uint32_t *cm = nullptr;     // class-major copy of the current rows (support re-checks), on first use
  // [0] frontier [1] work [2] dead [3] dv [4] edges2 [5] verts [6] pending
  // [7] dirty [8] last full pass's dv [9] its de
  unsigned long long *cnt = nullptr;
  int32_t *col = nullptr;
};

kz_status ensure_bufs(kz_graph g, LearnedBufs &b, cudaStream_t s) {
  const size_t n = (size_t)std::max(g->n, 1), m = (size_t)std::max<int64_t>(g->m, 1);
  KZ_TRY(graph_alloc(g, &b.s.deg, n, s));
  KZ_TRY(graph_alloc(g, &b.s.prevdeg, n, s));
  KZ_TRY(graph_alloc(g, &b.s.cover, n, s));
  KZ_TRY(graph_alloc(g, &b.s.minc, n, s));
  KZ_TRY(graph_alloc(g, &b.s.vfail, n, s));
  KZ_TRY(graph_alloc(g, &b.s.changed, n, s));
  KZ_TRY(graph_alloc(g, &b.s.ccnt, n * (size_t)g->k, s));
  KZ_TRY(graph_alloc(g, &b.fr, m, s));
  KZ_TRY(graph_alloc(g, &b.work, m, s));
  KZ_TRY(graph_alloc(g, &b.dead, m, s));
  KZ_TRY(graph_alloc(g, &b.cnt, kCounters, s));
  KZ_TRY(graph_alloc(g, &b.pend, (size_t)std::max(g->n, 1) * g->ldw, s));
  KZ_TRY(graph_alloc(g, &b.dirty, (size_t)std::max(g->n, 1) * g->ldw, s));
  KZ_CUDA_TRY(cudaMemsetAsync(b.pend, 0, (size_t)std::max(g->n, 1) * g->ldw * 4, s));
  KZ_CUDA_TRY(cudaMemsetAsync(b.dirty, 0, (size_t)std::max(g->n, 1) * g->ldw * 4, s));
  std::vector<int32_t> col_new((size_t)g->n);
  for (int c = 0; c < g->k; c++)
    for (int x = g->coff[c]; x < g->coff[c + 1]; x++) col_new[x] = c;
  KZ_TRY(graph_alloc(g, &b.col, n, s));
  if (g->n) KZ_CUDA_TRY(cudaMemcpyAsync(b.col, col_new.data(), 4 * (size_t)g->n, cudaMemcpyHostToDevice, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  return KZ_OK;
}

RowView view_of(kz_graph g, const LearnedBufs &b, int cur) {
  RowView r;
  r.A = g->A[cur & 1];
  r.V = g->V[cur & 1];
  r.n = g->n;
  r.k = g->k;
  r.ldw = g->ldw;
  r.R = g->R;
  r.col = b.col;
  r.coff = g->d_coff;
  return r;
}

kz_status read_u64(const unsigned long long *d, unsigned long long *h, int count, cudaStream_t s) {
  KZ_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, s));
  KZ_CUDA_TRY(cudaStreamSynchronize(s));
  return KZ_OK;
}

int32_t read_cur(kz_graph g, cudaStream_t s) {
  int32_t cur = 0;
  cudaMemcpyAsync(&cur, &g->st->cur, 4, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return cur;
}

}  // namespace

namespace kz {

// Whether testing a list of edges one by one beats a full pass.  Both costs
// are measured during the run (CUDA events around the full passes and the
// list tests): a list is worth it while its estimated time stays under
// kListGain of the last full pass's (the rest pays for the round's
// statistics, scoring and marking).  Until a list test of at least
// kMinTimedList edges has been timed, a list may hold an eighth of the live
// edges.
constexpr unsigned long long kListShareInv = 8;
constexpr double kListGain = 0.7;
constexpr unsigned long long kMinTimedList = 1 << 16;
constexpr int64_t kCalibrationEdges = 1 << 20;  // the sample that times the exact test

struct ListBudget {
  double full_ms = -1.0;      // last full pass
  double per_edge_ms = -1.0;  // list test time per listed edge
  bool fits(double list, double live_edges) const {
    if (per_edge_ms < 0.0 || full_ms < 0.0) return list * (double)kListShareInv <= live_edges;
    return list * per_edge_ms <= kListGain * full_ms;
  }
};

// The dirty set that de edge deletions leave: about 2 de times the mean
// common-neighbour count of a live edge (a random-graph estimate from the
// live density) marks, landing on the live edges at random.
static double dirty_estimate(kz_graph g, unsigned long long de, double live_edges) {
  const double n = std::max(g->n, 2), k = std::max(g->k, 3);
  const double pairs = n * n * (k - 1.0) / (2.0 * k);  // vertex pairs in different classes
  const double dens = live_edges / pairs;
  const double common = n * (k - 2.0) / k * dens * dens;
  const double marks = 2.0 * (double)de * common;
  return live_edges > 0.0 ? live_edges * -std::expm1(-marks / live_edges) : 0.0;
}

// Timing events of one run (destroyed with it).
struct RunEvents {
  cudaEvent_t a = nullptr, b = nullptr;
  ~RunEvents() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  double ms() const {
    float v = 0.f;
    return cudaEventElapsedTime(&v, a, b) == cudaSuccess ? (double)v : -1.0;
  }
};

// Learned schedule (see the file comment).  full_path is the path of the
// full passes: KZ_PATH_BITSET (the multi-CTA sweep) or KZ_PATH_TENSOR.
kz_status learned_kernelize(kz_graph g, const kz_options &opt, int full_path, cudaStream_t s) {
  if (!g->model) return KZ_ERR_UNSUPPORTED;
  if (!g->learned_bufs) {
    LearnedBufs *b = new LearnedBufs();
    kz_status st = ensure_bufs(g, *b, s);
    if (st != KZ_OK) {
      delete b;
      return st;
    }
    g->learned_bufs = b;
  }
  LearnedBufs &b = *static_cast<LearnedBufs *>(g->learned_bufs);
  const int64_t max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : (int64_t)g->n + g->m + 1;
  const float p = std::min(std::max(g->learned_threshold, 0.f), 0.999999f);
  const float logit_thr = p <= 0.f ? -INFINITY : std::log(p / (1.f - p));
  const int sms = sms_now();
  const int grid = 8 * sms;
  KZ_TRY(bitset_begin_run(g, max_sweeps, s));
  if (g->n == 0) return KZ_OK;
  const int64_t cap = std::max<int64_t>(g->m, 1);
  const size_t set_bytes = (size_t)g->n * g->ldw * 4;
  RunEvents ev;
  KZ_CUDA_TRY(cudaEventCreate(&ev.a));
  KZ_CUDA_TRY(cudaEventCreate(&ev.b));
  ListBudget budget;
  bool calibrated = false;
  auto full_pass = [&](int *cont) -> kz_status {
    KZ_CUDA_TRY(cudaEventRecord(ev.a, s));
    const kz_status st = full_path == KZ_PATH_TENSOR ? tensor_one_pass(g, opt, s, cont) : bitset_one_pass(g, s, cont);
    KZ_CUDA_TRY(cudaEventRecord(ev.b, s));
    KZ_CUDA_TRY(cudaEventSynchronize(ev.b));
    const double ms = ev.ms();
    if (ms > 0.0) budget.full_ms = ms;
    return st;
  };
  // an exact test of a list, timed for the budget when the list is long
  auto test_list = [&](const RowView &rv, const int2 *list, unsigned long long *n_list) -> kz_status {
    KZ_CUDA_TRY(cudaEventRecord(ev.a, s));
    test_edges_kernel<<<grid, 256, 0, s>>>(rv, list, n_list, b.dead, b.cnt + 2);
    KZ_CUDA_TRY(cudaGetLastError());
    KZ_CUDA_TRY(cudaEventRecord(ev.b, s));
    return KZ_OK;
  };
  // after the counts of a timed list test are read back
  auto time_list = [&](unsigned long long listed) {
    if (listed < kMinTimedList) return;
    const double ms = ev.ms();
    if (ms > 0.0) budget.per_edge_ms = ms / (double)listed;
  };
  // counters and the run's productive sweeps, read back in one wait
  unsigned long long h[kCounters];
  int64_t sweeps = 0;
  auto read_counts = [&]() -> kz_status {
    KZ_CUDA_TRY(cudaMemcpyAsync(h, b.cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaMemcpyAsync(&sweeps, &g->st->sweeps, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaStreamSynchronize(s));
    return KZ_OK;
  };
  // the pending and dirty sets emptied: a full pass tests every edge
  bool dirty_valid = false;
  auto clear_sets = [&]() -> kz_status {
    KZ_CUDA_TRY(cudaMemsetAsync(b.pend, 0, set_bytes, s));
    KZ_CUDA_TRY(cudaMemsetAsync(b.dirty, 0, set_bytes, s));
    KZ_CUDA_TRY(cudaMemsetAsync(b.cnt + 6, 0, sizeof(unsigned long long) * 2, s));
    dirty_valid = false;
    return KZ_OK;
  };
  // degrees before the first pass, so that a degree frontier after it is
  // what that pass changed
  {
    RowView r0 = view_of(g, b, read_cur(g, s));
    KZ_CUDA_TRY(cudaMemsetAsync(b.cnt, 0, sizeof(unsigned long long) * kCounters, s));
    stats_kernel<<<grid, 256, 0, s>>>(r0, b.s, 1, b.cnt + 3);
    KZ_CUDA_TRY(cudaGetLastError());
  }
  KZ_TRY(clear_sets());
  int round = 1;
  bool need_full = true;
  RowView r;
  for (;;) {
    if (need_full) {
      // a full pass: the first one, those of the cascade's heavy sweeps, and
      // the certifying ones
      int cont = 0;
      KZ_TRY(full_pass(&cont));
      if (!cont) return KZ_OK;  // nothing deleted (or the sweep limit): certified / stopped
      need_full = false;
      const int cur = read_cur(g, s);
      r = view_of(g, b, cur);
      KZ_CUDA_TRY(cudaMemsetAsync(b.cnt, 0, sizeof(unsigned long long) * 6, s));
      count_live_kernel<<<grid, 256, 0, s>>>(r, b.cnt + 4, b.cnt + 5);
      last_pass_kernel<<<1, 1, 0, s>>>(g->st, b.cnt + 8);
      KZ_CUDA_TRY(cudaGetLastError());
      KZ_TRY(read_counts());
      round = (int)std::min<int64_t>(sweeps, 1 << 20);
      if (!calibrated) {
        // time the exact test once, on a sample of live edges (results dropped)
        calibrated = true;
        KZ_CUDA_TRY(cudaMemsetAsync(b.cnt + 1, 0, sizeof(unsigned long long) * 2, s));
        sample_edges_kernel<<<grid, 256, 0, s>>>(r, b.work, b.cnt + 1, std::min<int64_t>(kCalibrationEdges, cap),
                                                 std::max(1, g->n / 1024));
        clamp_kernel<<<1, 1, 0, s>>>(b.cnt + 1, (unsigned long long)std::min<int64_t>(kCalibrationEdges, cap));
        KZ_TRY(test_list(r, b.work, b.cnt + 1));
        KZ_TRY(read_counts());
        time_list(h[1]);
        KZ_CUDA_TRY(cudaMemsetAsync(b.cnt + 1, 0, sizeof(unsigned long long) * 2, s));
      }
      if (h[8] == 0) {
        const double live = (double)(h[4] / 2);
        if (!budget.fits(dirty_estimate(g, h[9], live), live)) {
          // still in the cascade's heavy sweeps: the next one is a full pass
          need_full = true;
          continue;
        }
        // few edge deletions: the next frontier is their dirty set, marked
        // from the pass's old rows (the other ping-pong buffer)
        const RowView rold = view_of(g, b, cur ^ 1);
        diff_dead_kernel<<<grid, 256, 0, s>>>(rold, r.A, b.dead, b.cnt + 2, cap);
        mark_dirty_kernel<<<grid, 256, 0, s>>>(rold, b.dead, b.cnt + 2, cap, b.dirty, b.cnt + 7);
        KZ_CUDA_TRY(cudaGetLastError());
        dirty_valid = true;
      }
      // (a pass that deleted vertices leaves the degree frontier)
    }
    KZ_CUDA_TRY(cudaMemsetAsync(b.cnt, 0, sizeof(unsigned long long) * 6, s));
    count_live_kernel<<<grid, 256, 0, s>>>(r, b.cnt + 4, b.cnt + 5);
    stats_kernel<<<grid, 256, 0, s>>>(r, b.s, 0, b.cnt + 3);
    if (dirty_valid) {
      // the dirty pairs still live, listed once; the dirty set empties
      flush_pending_kernel<<<grid, 256, 0, s>>>(r, b.dirty, b.fr, b.cnt + 0, cap);
      KZ_CUDA_TRY(cudaMemsetAsync(b.cnt + 7, 0, sizeof(unsigned long long), s));
    } else {
      frontier_kernel<<<grid, 256, 0, s>>>(r, b.s, b.fr, b.cnt + 0, cap);
    }
    score_kernel<<<2 * sms, 32 * kScoreWarps, 0, s>>>(r, b.s, g->model->w16, b.fr, b.cnt, logit_thr, round, b.work,
                                                      b.cnt + 1, b.pend, b.cnt + 6);
    KZ_CUDA_TRY(cudaGetLastError());
    KZ_TRY(read_counts());
    const unsigned long long live_edges = h[4] / 2;
    if (!budget.fits((double)h[1], (double)live_edges)) {
      // so many edges listed that testing them one by one costs more than a
      // full pass, which tests every edge anyway
      KZ_TRY(clear_sets());
      need_full = true;
      continue;
    }
    KZ_TRY(test_list(r, b.work, b.cnt + 1));
    KZ_TRY(read_counts());
    time_list(h[1]);
    unsigned long long dv = h[3], de = h[2];
    if (dv + de == 0) {
      // the scored edges found nothing: the pending ones next, when they are
      // few; otherwise (or when they hold no failure either) a full pass
      learned_finish_kernel<<<1, 1, 0, s>>>(g->st, b.cnt + 3, b.cnt + 2, b.cnt + 1, nullptr);
      if (!budget.fits((double)h[6], (double)live_edges)) {
        // the pending set's count already rules the list out: no flush
        KZ_TRY(clear_sets());
        need_full = true;
        continue;
      }
      KZ_CUDA_TRY(cudaMemsetAsync(b.cnt + 1, 0, sizeof(unsigned long long) * 2, s));
      flush_pending_kernel<<<grid, 256, 0, s>>>(r, b.pend, b.work, b.cnt + 1, cap);
      KZ_CUDA_TRY(cudaMemsetAsync(b.cnt + 6, 0, sizeof(unsigned long long), s));  // flushed
      KZ_TRY(read_counts());
      const unsigned long long pending = h[1];
      if (pending == 0 || !budget.fits((double)pending, (double)live_edges)) {
        KZ_TRY(clear_sets());
        need_full = true;
        continue;
      }
      KZ_TRY(test_list(r, b.work, b.cnt + 1));
      KZ_TRY(read_counts());
      time_list(h[1]);
      dv = 0;
      de = h[2];
      if (de == 0) {
        learned_finish_kernel<<<1, 1, 0, s>>>(g->st, b.cnt + 3, b.cnt + 2, b.cnt + 1, nullptr);
        KZ_TRY(clear_sets());
        need_full = true;
        continue;
      }
      KZ_CUDA_TRY(cudaMemsetAsync(b.s.vfail, 0, (size_t)g->n, s));
      KZ_CUDA_TRY(cudaMemsetAsync(b.cnt + 3, 0, sizeof(unsigned long long), s));
    }
    if (sweeps >= max_sweeps) {
      int32_t lim = KZ_ERR_LIMIT;
      KZ_CUDA_TRY(cudaMemcpyAsync(&g->st->status, &lim, 4, cudaMemcpyHostToDevice, s));
      KZ_CUDA_TRY(cudaStreamSynchronize(s));
      return KZ_OK;
    }
    if (dv == 0) {
      // the next frontier: the dirty pairs of this round's deletions, marked
      // while the rows still hold them
      mark_dirty_kernel<<<grid, 256, 0, s>>>(r, b.dead, b.cnt + 2, cap, b.dirty, b.cnt + 7);
      dirty_valid = true;
    } else if (dirty_valid) {
      // vertex deletions: the degree frontier covers them and the dirty pairs
      KZ_CUDA_TRY(cudaMemsetAsync(b.dirty, 0, set_bytes, s));
      KZ_CUDA_TRY(cudaMemsetAsync(b.cnt + 7, 0, sizeof(unsigned long long), s));
      dirty_valid = false;
    }
    apply_kernel<<<grid, 256, 0, s>>>(r, b.s.vfail, b.dead, b.cnt + 2, g->v_sweep, g->st);
    learned_finish_kernel<<<1, 1, 0, s>>>(g->st, b.cnt + 3, b.cnt + 2, b.cnt + 1, nullptr);
    KZ_CUDA_TRY(cudaGetLastError());
    round++;
    if (dirty_valid) {
      KZ_TRY(read_counts());
      if (!budget.fits((double)h[7], (double)(h[4] / 2))) {
        // a dirty set beyond the list budget: a full pass next
        KZ_TRY(clear_sets());
        need_full = true;
      }
    }
  }
}

// Dense support schedule: the first sweep is a full pass (the bitset sweep
// or the tensor form); every later sweep either re-checks only the (pair,
// class) combinations the previous sweep's deletions touched
// (recheck_kernel, with the vertex rule on the current rows) or, when that
// would cost more, is a full pass.  Both compute the same Jacobi sweep, so
// the sweeps and their deletions are the plain method's; a re-check sweep
// that finds nothing proves the fixpoint.  The choice compares the measured
// time of a full pass with the measured re-check time per deleted edge
// (timed first on a sample of kRecheckSample deleted edges, whose work is
// kept when the rest follows).  The two ping-pong buffers hold the rows
// before and after a sweep.
constexpr int64_t kRecheckSample = 1 << 15;
constexpr double kRecheckGain = 0.8;

kz_status recheck_kernelize(kz_graph g, const kz_options &opt, int full_path, cudaStream_t s) {
  if (!g->learned_bufs) {
    LearnedBufs *b = new LearnedBufs();
    kz_status st = ensure_bufs(g, *b, s);
    if (st != KZ_OK) {
      delete b;
      return st;
    }
    g->learned_bufs = b;
  }
  LearnedBufs &b = *static_cast<LearnedBufs *>(g->learned_bufs);
  const int64_t max_sweeps = opt.max_sweeps > 0 ? opt.max_sweeps : (int64_t)g->n + g->m + 1;
  const int grid = 8 * sms_now();
  KZ_TRY(bitset_begin_run(g, max_sweeps, s));
  if (g->n == 0) return KZ_OK;
  const int64_t cap = std::max<int64_t>(g->m, 1);
  const size_t set_bytes = (size_t)g->n * g->ldw * 4;
  const size_t row_bytes = (size_t)g->n * g->ldw * 4, v_bytes = (size_t)g->ldw * 4;
  unsigned long long h[kCounters];
  int64_t sweeps = 0;
  auto read_counts = [&]() -> kz_status {
    KZ_CUDA_TRY(cudaMemcpyAsync(h, b.cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaMemcpyAsync(&sweeps, &g->st->sweeps, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    KZ_CUDA_TRY(cudaStreamSynchronize(s));
    return KZ_OK;
  };
  const int32_t Rp = (g->R + 3) / 4 * 4;
  if (!b.cm) KZ_TRY(graph_alloc(g, &b.cm, (size_t)std::max(g->n, 1) * g->k * Rp, s));
  RunEvents ev;
  KZ_CUDA_TRY(cudaEventCreate(&ev.a));
  KZ_CUDA_TRY(cudaEventCreate(&ev.b));
  double full_ms = -1.0, per_dead_ms = -1.0;
  int cur = 0;
  int2 *dead = b.dead, *fresh = b.work;
  // a full pass, timed; then its deletions listed from the two buffers
  auto full_sweep = [&](int *cont) -> kz_status {
    KZ_CUDA_TRY(cudaEventRecord(ev.a, s));
    KZ_TRY(full_path == KZ_PATH_TENSOR ? tensor_one_pass(g, opt, s, cont) : bitset_one_pass(g, s, cont));
    KZ_CUDA_TRY(cudaEventRecord(ev.b, s));
    KZ_CUDA_TRY(cudaEventSynchronize(ev.b));
    const double ms = ev.ms();
    if (ms > 0.0) full_ms = ms;
    if (!*cont) return KZ_OK;
    cur = read_cur(g, s);
    KZ_CUDA_TRY(cudaMemsetAsync(b.cnt + 2, 0, sizeof(unsigned long long), s));
    diff_dead_kernel<<<grid, 256, 0, s>>>(view_of(g, b, cur ^ 1), g->A[cur & 1], dead, b.cnt + 2, cap);
    KZ_CUDA_TRY(cudaGetLastError());
    return KZ_OK;
  };
  int cont = 0;
  KZ_TRY(full_sweep(&cont));
  if (!cont) return KZ_OK;  // nothing deleted (or the sweep limit)
  for (;;) {
    // [0] failures found [1] pairs re-checked [2] deleted by the last sweep [3] failing vertices
    KZ_TRY(read_counts());
    const int64_t n_dead = (int64_t)std::min<unsigned long long>(h[2], (unsigned long long)cap);
    const RowView rnew = view_of(g, b, cur), rold = view_of(g, b, cur ^ 1);
    bool cm_built = false;
    auto recheck = [&](int64_t q0, int64_t q1) -> kz_status {
      KZ_CUDA_TRY(cudaEventRecord(ev.a, s));
      if (!cm_built) {
        class_major_kernel<<<grid, 256, 0, s>>>(rnew.A, g->n, g->k, g->R, g->ldw, Rp, b.cm);
        cm_built = true;
      }
      recheck_kernel<<<kRecheckCtasPerSm * sms_now(), 256, 0, s>>>(rold, rnew, b.cm, Rp, dead, b.cnt + 2, q0, q1,
                                                                    cap, b.pend, fresh, b.cnt + 0, b.dirty,
                                                                    b.cnt + 1);
      KZ_CUDA_TRY(cudaGetLastError());
      KZ_CUDA_TRY(cudaEventRecord(ev.b, s));
      KZ_CUDA_TRY(cudaEventSynchronize(ev.b));
      const double ms = ev.ms();
      if (ms > 0.0 && q1 - q0 >= 4096) per_dead_ms = ms / (double)(q1 - q0);
      return KZ_OK;
    };
    KZ_CUDA_TRY(cudaMemsetAsync(b.pend, 0, set_bytes, s));
    KZ_CUDA_TRY(cudaMemsetAsync(b.dirty, 0, set_bytes, s));
    KZ_CUDA_TRY(cudaMemsetAsync(b.cnt, 0, sizeof(unsigned long long) * 2, s));
    KZ_CUDA_TRY(cudaMemsetAsync(b.cnt + 3, 0, sizeof(unsigned long long), s));
    bool by_recheck = true;
    int64_t done = 0;
    if (full_ms > 0.0) {
      if (per_dead_ms < 0.0 && n_dead > kRecheckSample) {
        KZ_TRY(recheck(0, kRecheckSample));
        done = kRecheckSample;
      }
      if (per_dead_ms > 0.0 && (double)(n_dead - done) * per_dead_ms > kRecheckGain * full_ms) by_recheck = false;
    }
    if (!by_recheck) {
      // this sweep as a full pass (what a sample re-checked is dropped); the
      // pass applies the sweep limit itself
      KZ_TRY(full_sweep(&cont));
      if (!cont) return KZ_OK;
      continue;
    }
    if (done < n_dead) KZ_TRY(recheck(done, n_dead));
    stats_kernel<<<grid, 256, 0, s>>>(rnew, b.s, 0, b.cnt + 3);
    KZ_CUDA_TRY(cudaGetLastError());
    KZ_TRY(read_counts());
    const unsigned long long de = std::min<unsigned long long>(h[0], (unsigned long long)cap), dv = h[3];
    if (de + dv > 0 && sweeps >= max_sweeps) {
      int32_t lim = KZ_ERR_LIMIT;
      KZ_CUDA_TRY(cudaMemcpyAsync(&g->st->status, &lim, 4, cudaMemcpyHostToDevice, s));
      KZ_CUDA_TRY(cudaStreamSynchronize(s));
      return KZ_OK;
    }
    if (de + dv > 0) {
      // the next state in the other buffer: a copy of the current rows with
      // this sweep's deletions applied
      KZ_CUDA_TRY(cudaMemcpyAsync(g->A[(cur & 1) ^ 1], g->A[cur & 1], row_bytes, cudaMemcpyDeviceToDevice, s));
      KZ_CUDA_TRY(cudaMemcpyAsync(g->V[(cur & 1) ^ 1], g->V[cur & 1], v_bytes, cudaMemcpyDeviceToDevice, s));
      apply_kernel<<<grid, 256, 0, s>>>(view_of(g, b, cur ^ 1), b.s.vfail, fresh, b.cnt + 0, g->v_sweep, g->st);
      KZ_CUDA_TRY(cudaGetLastError());
    }
    recheck_finish_kernel<<<1, 1, 0, s>>>(g->st, b.cnt + 3, b.cnt + 0, b.cnt + 1);
    KZ_CUDA_TRY(cudaGetLastError());
    if (de + dv == 0) return KZ_OK;  // the fixpoint: the last sweep broke nothing
    cur ^= 1;
    std::swap(dead, fresh);
    KZ_CUDA_TRY(cudaMemcpyAsync(b.cnt + 2, b.cnt + 0, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s));
  }
}

kz_status learned_collect(kz_graph g, int64_t per_sweep_cap, uint64_t seed, float *X, uint8_t *y, int64_t cap,
                          int64_t *count) {
  cudaStream_t s = g->stream;
  if (!g->learned_bufs) {
    LearnedBufs *b = new LearnedBufs();
    kz_status st = ensure_bufs(g, *b, s);
    if (st != KZ_OK) {
      delete b;
      return st;
    }
    g->learned_bufs = b;
  }
  LearnedBufs &b = *static_cast<LearnedBufs *>(g->learned_bufs);
  float *dX = nullptr;
  uint8_t *dy = nullptr;
  unsigned long long *dcnt = nullptr;
  const size_t capz = (size_t)std::max<int64_t>(cap, 1);
  dX = (float *)dev_alloc(capz * F * 4, s);
  dy = (uint8_t *)dev_alloc(capz, s);
  dcnt = (unsigned long long *)dev_alloc(64, s);
  kz_status st = (dX && dy && dcnt) ? KZ_OK : KZ_ERR_OOM;
  if (st == KZ_OK) st = cuda_status(cudaMemsetAsync(dcnt, 0, 64, s));
  if (st == KZ_OK) st = bitset_begin_run(g, (int64_t)g->n + g->m + 1, s);
  const int grid = 8 * sms_now();
  int round = 0;
  while (st == KZ_OK) {
    const int cur = read_cur(g, s);
    RowView r = view_of(g, b, cur);
    st = cuda_status(cudaMemsetAsync(b.cnt, 0, sizeof(unsigned long long) * 8, s));
    count_live_kernel<<<grid, 256, 0, s>>>(r, b.cnt + 4, b.cnt + 5);
    stats_kernel<<<grid, 256, 0, s>>>(r, b.s, round == 0 ? 1 : 0, b.cnt + 3);
    unsigned long long h[8];
    if (st == KZ_OK) st = read_u64(b.cnt, h, 8, s);
    if (st != KZ_OK) break;
    const double n = std::max(g->n, 1);
    const double live_edges = (double)h[4] / 2.0;
    const float density = (float)((double)h[4] / (n * std::max(n - 1.0, 1.0)));
    const float live_frac = (float)(h[5] / n);
    // keep about per_sweep_cap of this sweep's live edges
    const double frac = live_edges > 0 ? std::min(1.0, (double)per_sweep_cap / live_edges) : 1.0;
    const uint32_t keep_below = frac >= 1.0 ? 0xffffffffu : (uint32_t)(frac * 4294967295.0);
    trace_kernel<<<grid, 256, 0, s>>>(r, b.s, round, density, live_frac, seed, keep_below, dX, dy, dcnt, cap);
    int cont = 0;
    st = bitset_one_pass(g, s, &cont);
    if (st != KZ_OK || !cont) break;
    round++;
  }
  unsigned long long total = 0;
  if (st == KZ_OK) st = read_u64(dcnt, &total, 1, s);
  const int64_t got = std::min<int64_t>((int64_t)total, cap);
  if (st == KZ_OK && got > 0) {
    st = cuda_status(cudaMemcpy(X, dX, (size_t)got * F * 4, cudaMemcpyDeviceToHost));
    if (st == KZ_OK) st = cuda_status(cudaMemcpy(y, dy, (size_t)got, cudaMemcpyDeviceToHost));
  }
  if (count) *count = got;
  if (dX) dev_free(dX, capz * F * 4, s);
  if (dy) dev_free(dy, capz, s);
  if (dcnt) dev_free(dcnt, 64, s);
  if (st == KZ_OK) st = cuda_status(cudaStreamSynchronize(s));
  return st;
}

void learned_release(kz_graph g) {
  delete static_cast<LearnedBufs *>(g->learned_bufs);
  g->learned_bufs = nullptr;
}

}  // namespace kz

// ---------------------------------------------------------------------------
// C ABI of the model
// ---------------------------------------------------------------------------

extern "C" {

kz_status kz_model_create(const float *weights, kz_model *out) {
  if (!out) return KZ_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return KZ_ERR_CUDA;
  }
  kz_model m = new (std::nothrow) kz_model_s();
  if (!m) return KZ_ERR_OOM;
  cudaGetDevice(&m->device);
  cudaError_t e = cudaMalloc(&m->w32, P * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->w16, P * 2);
  if (e == cudaSuccess) e = cudaMalloc(&m->m, P * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->v, P * 4);
  if (e == cudaSuccess) e = cudaMemset(m->m, 0, P * 4);
  if (e == cudaSuccess) e = cudaMemset(m->v, 0, P * 4);
  if (e == cudaSuccess)
    e = weights ? cudaMemcpy(m->w32, weights, P * 4, cudaMemcpyHostToDevice) : cudaMemset(m->w32, 0, P * 4);
  if (e == cudaSuccess) {
    to_bf16_kernel<<<8, 256>>>(m->w32, m->w16);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    kz_model_free(m);
    return cuda_status(e);
  }
  *out = m;
  return KZ_OK;
}

kz_status kz_model_get(kz_model m, float *weights) {
  if (!m || !weights) return KZ_ERR_ARG;
  KZ_CUDA_TRY(cudaDeviceSynchronize());
  KZ_CUDA_TRY(cudaMemcpy(weights, m->w32, P * 4, cudaMemcpyDeviceToHost));
  return KZ_OK;
}

void kz_model_free(kz_model m) {
  if (!m) return;
  cudaDeviceSynchronize();
  cudaFree(m->w32);
  cudaFree(m->w16);
  cudaFree(m->m);
  cudaFree(m->v);
  delete m;
}

kz_status kz_mlp_forward(kz_model m, const float *X, int64_t B, float *logits, void *stream) {
  if (!m || B < 0 || (B > 0 && (!X || !logits))) return KZ_ERR_ARG;
  if (B == 0) return KZ_OK;
  const int64_t per_block = (int64_t)kFwdWarps * kTileRows;
  const int grid = (int)std::min<int64_t>((B + per_block - 1) / per_block, 2 * sms_now());
  mlp_forward_kernel<<<grid, 32 * kFwdWarps, 0, (cudaStream_t)stream>>>(m->w16, X, B, logits);
  return cuda_status(cudaGetLastError());
}

kz_status kz_mlp_grad(kz_model m, const float *X, const float *y, int64_t B, float *grad, float *loss,
                      void *stream) {
  if (!m || B <= 0 || !X || !y || !grad || !loss) return KZ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t smem = sizeof(GradSmem);
  {
    static std::mutex mu;
    static bool configured[64] = {};
    int dev = 0;
    KZ_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && !configured[dev]) {
      KZ_CUDA_TRY(cudaFuncSetAttribute((const void *)mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
      configured[dev] = true;
    }
  }
  KZ_CUDA_TRY(cudaMemsetAsync(grad, 0, P * 4, s));
  KZ_CUDA_TRY(cudaMemsetAsync(loss, 0, 4, s));
  const int64_t blocks = std::min<int64_t>((B + kChunk - 1) / kChunk, 2 * sms_now());
  mlp_grad_kernel<<<(unsigned)blocks, 32 * kGradWarps, smem, s>>>(m->w16, X, y, B, grad, loss);
  return cuda_status(cudaGetLastError());
}

kz_status kz_mlp_adam(kz_model m, const float *grad, float lr, void *stream) {
  if (!m || !grad) return KZ_ERR_ARG;
  m->t += 1;
  const float bc1 = 1.f - std::pow(0.9f, (float)m->t);
  const float bc2 = 1.f - std::pow(0.999f, (float)m->t);
  adam_kernel<<<8, 256, 0, (cudaStream_t)stream>>>(m->w32, m->w16, m->m, m->v, grad, lr, bc1, bc2);
  return cuda_status(cudaGetLastError());
}

kz_status kz_collect_trace(kz_graph g, int64_t per_sweep_cap, uint64_t seed, float *X, uint8_t *y, int64_t cap,
                           int64_t *count) {
  if (!g || per_sweep_cap < 0 || cap < 0 || (cap > 0 && (!X || !y)) || !count) return KZ_ERR_ARG;
  if (!g->has_bitset) return KZ_ERR_UNSUPPORTED;
  g->slack = 0;  // traces follow the thesis's rules (q = k)
  KZ_TRY(state_to_bitset(g, g->stream));
  g->ab_synced = false;
  KZ_TRY(learned_collect(g, per_sweep_cap, seed, X, y, cap, count));
  g->kernelized = true;
  g->path_ran = KZ_PATH_BITSET;
  return KZ_OK;
}

kz_status kz_attach_model(kz_graph g, kz_model m, float threshold) {
  if (!g) return KZ_ERR_ARG;
  g->model = m;
  g->learned_threshold = threshold;
  return KZ_OK;
}

}  // extern "C"
