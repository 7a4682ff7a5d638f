// kz_pack.cu -- loading and fetching the bitset rows of the colour-index
// kernelization: the caller's graph (an edge list or a dense 0/1 bit matrix,
// caller vertex ids) packed into the block-plane rows of the sweep kernels
// (vertices relabelled class by class, word r k + c of a row holding members
// 32 r .. 32 r + 31 of class c), and the rows unpacked back to caller ids.
// The kernels move bits; the rules of thesis Section 4.2 run elsewhere.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "kz_internal.cuh"
#include "kz_rules.cuh"

namespace kz {

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

// The library's copy stream on the current device (created on first use,
// never destroyed): host copies of the dense load and fetch run on it, in
// row chunks, while the packing kernels work on the chunks already moved.
static cudaStream_t copy_stream() {
  static std::mutex mu;
  static std::map<int, cudaStream_t> streams;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = streams.find(dev);
  if (it != streams.end()) return it->second;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  streams[dev] = cs;
  return cs;
}

// Row chunks of a dense copy: one below 16 MiB (nothing to overlap), else
// eight.
static int copy_chunks(size_t bytes) { return bytes < (size_t(16) << 20) ? 1 : 8; }

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

// Row form of the dense packer, first half, over caller rows [r0, r1).  A CTA
// stages kPackRows caller rows (4, or fewer when the rows are long) at a time in shared memory and writes the relabelled rows inv[i].
// Word w = rr k + c of a relabelled row holds the relabelled vertices
// y = coff[c] + 32 rr + b, b = 0..31: lane b looks up y's caller column
// perm[y] once for all the staged rows, tests it in each of them, and one
// ballot per row assembles the word.  A warp builds 32 consecutive words
// this way, lane t keeping word t of every staged row, and stores each row's
// 32 words in one coalesced transaction.  Only columns j > i are taken (the
// upper triangle): every edge lands in the row of its endpoint with the
// smaller caller id, and symmetrize_kernel adds the other half.  A bit in an
// own-class word is an edge inside one class: an illegal colouring.
constexpr int kPackThreads = 256;
constexpr size_t kRowSmemBytes = 200 * 1024;  // shared memory the staged rows may take

template <int kPackRows>
__global__ void __launch_bounds__(kPackThreads) pack_dense_rows_kernel(PackArgs a, const uint64_t *__restrict__ bits,
                                                                     int64_t row_words, int32_t n, int32_t R,
                                                                     const int32_t *__restrict__ perm, int64_t r0,
                                                                     int64_t r1) {
  extern __shared__ __align__(16) uint32_t psm[];
  const int32_t nw = (n + 31) >> 5;
  uint32_t *srow = psm;  // kPackRows rows of nw 32-bit words
  int32_t *scoff = reinterpret_cast<int32_t *>(psm + (size_t)kPackRows * nw);  // k + 1
  const int k = a.k, rk = R * k;
  for (int c = threadIdx.x; c <= k; c += blockDim.x) scoff[c] = a.coff[c];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned long long mine = 0;
  for (int64_t i0 = r0 + (int64_t)blockIdx.x * kPackRows; i0 < r1; i0 += (int64_t)gridDim.x * kPackRows) {
    __syncthreads();  // the previous rows are consumed (and scoff is written)
    const int rows = r1 - i0 < kPackRows ? (int)(r1 - i0) : kPackRows;
    // (a 64-bit caller word w holds 32-bit words 2w and 2w + 1, low half first)
    const uint32_t *bits32 = reinterpret_cast<const uint32_t *>(bits);
    for (int32_t q = threadIdx.x; q < kPackRows * nw; q += blockDim.x) {
      const int r = q / nw, w = q - r * nw;
      srow[q] = r < rows ? bits32[(i0 + r) * 2 * row_words + w] : 0u;
    }
    __syncthreads();
    int32_t xr[kPackRows], own[kPackRows];
#pragma unroll
    for (int r = 0; r < kPackRows; r++) {
      xr[r] = r < rows ? a.inv[i0 + r] : 0;
      own[r] = r < rows ? a.col[xr[r]] : -1;
    }
    for (int w0 = warp * 32; w0 < a.ldw; w0 += nwarps * 32) {
      uint32_t keep[kPackRows];
#pragma unroll
      for (int r = 0; r < kPackRows; r++) keep[r] = 0u;
      int c = w0 % k, rr = w0 / k;  // class and round of word w0 + t
      for (int t = 0; t < 32; t++) {
        int32_t j = -1;  // caller column of this lane's bit
        if (w0 + t < rk) {
          const int32_t y = scoff[c] + 32 * rr + lane;
          if (y < scoff[c + 1]) j = perm[y];
        }
#pragma unroll
        for (int r = 0; r < kPackRows; r++) {
          const bool bit = j > i0 + r && ((srow[r * nw + (j >> 5)] >> (j & 31)) & 1u);
          const uint32_t word = __ballot_sync(0xffffffffu, bit);
          if (lane == t) keep[r] = word;
        }
        if (++c == k) {
          c = 0;
          ++rr;
        }
      }
      const int w = w0 + lane;
      if (w < a.ldw) {
#pragma unroll
        for (int r = 0; r < kPackRows; r++) {
          if (r >= rows) break;
          uint32_t out = keep[r];
          if (out && w < rk && w % k == own[r]) {
            atomicCAS(a.error, 0, (int32_t)KZ_ERR_ILLEGAL_COLOURING);
            out = 0u;
          }
          a.A[(int64_t)xr[r] * a.ldw + w] = out;
          mine += __popc(out);
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(a.edge_count, mine);
}

// Tile form of the dense packer, first half, over caller rows [r0, r1): the
// relabelling moves columns, so a CTA takes 32 caller rows i0 .. i0 + 31 at
// a time and turns the bit permutation into a word gather between two warp
// transposes.  (1) Column words: lane r reads 32 bytes of row i0 + r (every
// sector used), and per 32 columns a transpose gives lane b the word of
// column 32 q + b over the 32 rows, kept in shared memory (colw, one word
// per caller column).  (2) Output: for word w = rr k + c of the relabelled
// rows, lane b fetches the column word of caller column perm[y], y = coff[c]
// + 32 rr + b, keeps only the rows r with i0 + r < perm[y] (the upper
// triangle; symmetrize_kernel adds the other half), and a transpose gives
// lane r word w of row inv[i0 + r].  Lane r collects kTileWords consecutive
// words before one 32-byte store.  A set bit in an own-class word is an edge
// inside one class: an illegal colouring.  colw takes 4 bytes per caller
// column, so this form serves graphs up to kTileMaxN vertices; larger ones
// take the row form.
constexpr int kTileThreads = 512;
constexpr int kTileWords = 8;
constexpr int kTileMaxN = 48 * 1024;
constexpr size_t kTileSmemBytes = 216 * 1024;

__global__ void __launch_bounds__(kTileThreads) pack_dense_tiles_kernel(PackArgs a, const uint64_t *__restrict__ bits,
                                                                       int64_t row_words, int32_t n, int32_t R,
                                                                       const int32_t *__restrict__ perm, int64_t r0,
                                                                       int64_t r1) {
  extern __shared__ __align__(16) uint32_t colw[];  // 32 * ceil(n / 32) column words
  const int nq = (n + 31) >> 5;
  int32_t *scoff = reinterpret_cast<int32_t *>(colw + 32 * nq);  // k + 1
  const int k = a.k, rk = R * k;
  for (int c = threadIdx.x; c <= k; c += blockDim.x) scoff[c] = a.coff[c];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned long long mine = 0;
  for (int64_t i0 = r0 + (int64_t)blockIdx.x * 32; i0 < r1; i0 += (int64_t)gridDim.x * 32) {
    const int rows = r1 - i0 < 32 ? (int)(r1 - i0) : 32;
    __syncthreads();  // the previous rows' column words are consumed (and scoff is written)
    // (1) column words, kTileWords 32-bit words (256 columns) of a row per lane
    const uint64_t *row = bits + (i0 + lane) * row_words;
    for (int q0 = warp * kTileWords; q0 < nq; q0 += nwarps * kTileWords) {
      uint32_t v[kTileWords];
#pragma unroll
      for (int u = 0; u < kTileWords; u += 2) {
        const int64_t w64 = (q0 + u) >> 1;
        const uint64_t x = (lane < rows && w64 < row_words) ? row[w64] : 0ull;
        v[u] = (uint32_t)x;
        v[u + 1] = (uint32_t)(x >> 32);
      }
#pragma unroll
      for (int u = 0; u < kTileWords; u++) {
        const uint32_t col = transpose32(v[u]);
        if (q0 + u < nq) colw[32 * (q0 + u) + lane] = col;
      }
    }
    __syncthreads();
    const int64_t i = i0 + lane;  // this lane's row after the second transpose
    const int32_t x = lane < rows ? a.inv[i] : 0;
    const int own = lane < rows ? a.col[x] : -1;
    // (2) the relabelled words, kTileWords per lane before a store
    for (int w0 = warp * kTileWords; w0 < a.ldw; w0 += nwarps * kTileWords) {
      uint32_t out[kTileWords];
      int c = w0 % k, rr = w0 / k;  // class and round of word w0 + u
#pragma unroll
      for (int u = 0; u < kTileWords; u++) {
        uint32_t col = 0u;
        if (w0 + u < rk) {
          const int32_t y = scoff[c] + 32 * rr + lane;
          if (y < scoff[c + 1]) {
            const int32_t j = perm[y];
            const int64_t above = (int64_t)j - i0;  // rows r < above lie above the diagonal
            const uint32_t keep = above >= 32 ? 0xffffffffu : above <= 0 ? 0u : ((1u << above) - 1u);
            col = colw[j] & keep;
          }
        }
        out[u] = transpose32(col);
        if (out[u] && w0 + u < rk && c == own) {
          atomicCAS(a.error, 0, (int32_t)KZ_ERR_ILLEGAL_COLOURING);
          out[u] = 0u;
        }
        if (++c == k) {
          c = 0;
          ++rr;
        }
      }
      if (lane < rows) {
        uint32_t *dst = a.A + (int64_t)x * a.ldw + w0;
        *reinterpret_cast<uint4 *>(dst) = make_uint4(out[0], out[1], out[2], out[3]);
        if (w0 + kTileWords <= a.ldw) *reinterpret_cast<uint4 *>(dst + 4) = make_uint4(out[4], out[5], out[6], out[7]);
        mine += __popc(out[0]) + __popc(out[1]) + __popc(out[2]) + __popc(out[3]);
        if (w0 + kTileWords <= a.ldw) mine += __popc(out[4]) + __popc(out[5]) + __popc(out[6]) + __popc(out[7]);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(a.edge_count, mine);
}

// Second half: every 32 x 32 tile of rows of block X (word position p of
// the layout, p = r k + c: members 32 r .. 32 r + 31 of class c) at the word
// of block Y becomes the OR of itself and the transpose of the tile of Y's
// rows at X's word, and that tile the transpose of the result.  The word
// positions fall into groups of kSymGroup; a CTA takes one pair of groups
// (g1 <= g2) at a time: warp i stages the rows of block g1 kSymGroup + i at
// the words of group g2, and the rows of block g2 kSymGroup + i at the words
// of group g1, each lane reading its row's kSymGroup words in two 16-byte
// loads (every sector fully used), updates the tiles of its block against
// the other group's blocks in shared memory, and writes its rows back.  Each
// word of the matrix belongs to exactly one pair of groups; a block that
// does not exist (a class with fewer rounds) has no rows, and a tile of two
// blocks of one class is zero.
constexpr int kSymGroup = 8;

__device__ __forceinline__ void sym_block(const int32_t *__restrict__ coff, int k, int rk, int p, int &base,
                                          int &size) {
  base = 0;
  size = 0;
  if (p >= rk) return;
  const int c = p % k, r = p / k;
  const int rem = coff[c + 1] - coff[c] - 32 * r;
  if (rem <= 0) return;
  base = coff[c] + 32 * r;
  size = rem < 32 ? rem : 32;
}

__device__ __forceinline__ void sym_load(const uint32_t *__restrict__ A, int ldw, int base, int size, int word0,
                                         uint32_t (*s)[kSymGroup + 1]) {
  const int lane = threadIdx.x & 31;
  uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
  if (lane < size) {
    const uint32_t *row = A + (int64_t)(base + lane) * ldw + word0;
    lo = *reinterpret_cast<const uint4 *>(row);
    if (word0 + kSymGroup <= ldw) hi = *reinterpret_cast<const uint4 *>(row + 4);
  }
  s[lane][0] = lo.x, s[lane][1] = lo.y, s[lane][2] = lo.z, s[lane][3] = lo.w;
  s[lane][4] = hi.x, s[lane][5] = hi.y, s[lane][6] = hi.z, s[lane][7] = hi.w;
}

__device__ __forceinline__ void sym_store(uint32_t *__restrict__ A, int ldw, int base, int size, int word0,
                                          const uint32_t (*s)[kSymGroup + 1]) {
  const int lane = threadIdx.x & 31;
  if (lane >= size) return;
  uint32_t *row = A + (int64_t)(base + lane) * ldw + word0;
  *reinterpret_cast<uint4 *>(row) = make_uint4(s[lane][0], s[lane][1], s[lane][2], s[lane][3]);
  if (word0 + kSymGroup <= ldw) *reinterpret_cast<uint4 *>(row + 4) = make_uint4(s[lane][4], s[lane][5], s[lane][6], s[lane][7]);
}

__global__ void __launch_bounds__(32 * kSymGroup) symmetrize_kernel(uint32_t *__restrict__ A,
                                                                    const int32_t *__restrict__ coff, int32_t k,
                                                                    int32_t R, int32_t ldw) {
  __shared__ uint32_t sx[kSymGroup][32][kSymGroup + 1];  // rows of group g1's blocks, words of g2
  __shared__ uint32_t sy[kSymGroup][32][kSymGroup + 1];  // rows of group g2's blocks, words of g1
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rk = R * k;
  const int64_t ng = (rk + kSymGroup - 1) / kSymGroup;
  const int64_t total = ng * (ng + 1) / 2;
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    // pair t: g1 is the last group whose row of pairs starts at or before t
    int64_t lo = 0, hi = ng;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (mid * ng - mid * (mid - 1) / 2 <= t) lo = mid;
      else hi = mid;
    }
    const int g1 = (int)lo, g2 = (int)(lo + t - (lo * ng - lo * (lo - 1) / 2));
    const bool diag = g1 == g2;
    int xb, xs, yb, ys;
    sym_block(coff, k, rk, g1 * kSymGroup + warp, xb, xs);
    sym_block(coff, k, rk, g2 * kSymGroup + warp, yb, ys);
    __syncthreads();  // the previous pair's stores have read the tiles
    sym_load(A, ldw, xb, xs, g2 * kSymGroup, sx[warp]);
    if (!diag) sym_load(A, ldw, yb, ys, g1 * kSymGroup, sy[warp]);
    __syncthreads();
    if (diag) {
      // tiles (i, j) and (j, i) of one group: warp min(i, j) owns both
      for (int j = warp + 1; j < kSymGroup; j++) {
        const uint32_t nw = sx[warp][lane][j] | transpose32(sx[j][lane][warp]);
        sx[warp][lane][j] = nw;
        sx[j][lane][warp] = transpose32(nw);
      }
    } else {
      for (int j = 0; j < kSymGroup; j++) {
        const uint32_t nw = sx[warp][lane][j] | transpose32(sy[j][lane][warp]);
        sx[warp][lane][j] = nw;
        sy[j][lane][warp] = transpose32(nw);
      }
    }
    __syncthreads();
    sym_store(A, ldw, xb, xs, g2 * kSymGroup, sx[warp]);
    if (!diag) sym_store(A, ldw, yb, ys, g1 * kSymGroup, sy[warp]);
  }
}


// ---------------------------------------------------------------------------
// unpacking to caller ids
// ---------------------------------------------------------------------------

// Row form of the unpacker, over caller rows [r0, r1): a CTA stages the
// relabelled rows inv[ox] of kPackRows caller rows ox at a time in shared
// memory.  Each warp builds 32
// caller words (2048 columns) of every staged row in 64 rounds: in a round
// the lanes take 32 consecutive columns, look up their positions in the
// block-plane row once (cpos, consecutive and so coalesced), test them in
// each staged row, and a ballot per row gives half of one word, kept by the
// lane that writes it.  The CTA also writes the rows' vertex flags.
template <int kPackRows>
__global__ void __launch_bounds__(kPackThreads) unpack_rows_kernel(
    const uint32_t *__restrict__ A0, const uint32_t *__restrict__ A1, const uint32_t *__restrict__ V0,
    const uint32_t *__restrict__ V1, const int32_t *__restrict__ cur, int32_t n, int32_t ldw,
    const int32_t *__restrict__ inv, const int32_t *__restrict__ cpos, uint64_t *__restrict__ out,
    int64_t row_words, uint8_t *__restrict__ alive, unsigned long long *__restrict__ edge_count, int64_t r0,
    int64_t r1) {
  extern __shared__ __align__(16) uint32_t usm[];  // kPackRows rows of ldw words
  const bool one = (*cur & 1) != 0;
  const uint32_t *A = one ? A1 : A0;
  const uint32_t *V = one ? V1 : V0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned long long mine = 0;
  for (int64_t o0 = r0 + (int64_t)blockIdx.x * kPackRows; o0 < r1; o0 += (int64_t)gridDim.x * kPackRows) {
    __syncthreads();  // the previous rows are consumed
    const int rows = r1 - o0 < kPackRows ? (int)(r1 - o0) : kPackRows;
    for (int32_t q = threadIdx.x; q < kPackRows * ldw; q += blockDim.x) {
      const int r = q / ldw, w = q - r * ldw;
      usm[q] = r < rows ? A[(int64_t)inv[o0 + r] * ldw + w] : 0u;
    }
    __syncthreads();
    for (int64_t w0 = (int64_t)warp * 32; w0 < row_words; w0 += (int64_t)nwarps * 32) {
      uint64_t word[kPackRows];
#pragma unroll
      for (int r = 0; r < kPackRows; r++) word[r] = 0ull;
      for (int h = 0; h < 64; h++) {
        const int64_t col = w0 * 64 + 32 * h + lane;
        const int32_t p = col < n ? cpos[col] : -1;
#pragma unroll
        for (int r = 0; r < kPackRows; r++) {
          const bool bit = p >= 0 && ((usm[r * ldw + (p >> 5)] >> (p & 31)) & 1u);
          const uint32_t half = __ballot_sync(0xffffffffu, bit);
          if (lane == (h >> 1)) word[r] |= (uint64_t)half << ((h & 1) * 32);
        }
      }
      if (w0 + lane < row_words) {
#pragma unroll
        for (int r = 0; r < kPackRows; r++) {
          if (r >= rows) break;
          out[(o0 + r) * row_words + w0 + lane] = word[r];
          mine += __popcll(word[r]);
        }
      }
    }
    if (threadIdx.x < rows) {
      const int32_t p = cpos[o0 + threadIdx.x];
      alive[o0 + threadIdx.x] = (uint8_t)((V[p >> 5] >> (p & 31)) & 1u);
    }
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(edge_count, mine);
}

// Tile form of the unpacker, over caller rows [r0, r1): 32 caller rows o0 ..
// o0 + 31 at a time, their relabelled rows x_r = inv[o0 + r].  (1) Position
// words: lane r reads kTileWords consecutive words of row x_r (32 bytes),
// and per word w a transpose gives lane b the word of position 32 w + b (bit
// b of word w) over the 32 rows, kept in shared memory.  (2) Output: for
// caller columns 32 h .. 32 h + 31, lane b fetches the position word of
// column 32 h + b (cpos), and a transpose gives lane r those 32 bits of
// caller row o0 + r; lane r collects kTileWords of them (four 64-bit words)
// before storing.  Graphs whose rows exceed kTileMaxN positions take the
// row form.
__global__ void __launch_bounds__(kTileThreads) unpack_tiles_kernel(
    const uint32_t *__restrict__ A0, const uint32_t *__restrict__ A1, const uint32_t *__restrict__ V0,
    const uint32_t *__restrict__ V1, const int32_t *__restrict__ cur, int32_t n, int32_t ldw,
    const int32_t *__restrict__ inv, const int32_t *__restrict__ cpos, uint64_t *__restrict__ out,
    int64_t row_words, uint8_t *__restrict__ alive, unsigned long long *__restrict__ edge_count, int64_t r0,
    int64_t r1) {
  extern __shared__ __align__(16) uint32_t posw[];  // 32 * ldw position words
  const bool one = (*cur & 1) != 0;
  const uint32_t *A = one ? A1 : A0;
  const uint32_t *V = one ? V1 : V0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nh = (n + 31) >> 5;  // 32-bit halves of an output row that hold columns
  unsigned long long mine = 0;
  for (int64_t o0 = r0 + (int64_t)blockIdx.x * 32; o0 < r1; o0 += (int64_t)gridDim.x * 32) {
    const int rows = r1 - o0 < 32 ? (int)(r1 - o0) : 32;
    __syncthreads();  // the previous rows' position words are consumed
    const uint32_t *row = A + (int64_t)(lane < rows ? inv[o0 + lane] : 0) * ldw;
    for (int w0 = warp * kTileWords; w0 < ldw; w0 += nwarps * kTileWords) {
      uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
      if (lane < rows) {
        lo = *reinterpret_cast<const uint4 *>(row + w0);
        if (w0 + kTileWords <= ldw) hi = *reinterpret_cast<const uint4 *>(row + w0 + 4);
      }
      const uint32_t v[kTileWords] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
      for (int u = 0; u < kTileWords; u++) {
        const uint32_t pw = transpose32(v[u]);
        if (w0 + u < ldw) posw[32 * (w0 + u) + lane] = pw;
      }
    }
    __syncthreads();
    uint64_t *orow = out + (o0 + lane) * row_words;
    for (int h0 = warp * kTileWords; h0 < 2 * row_words; h0 += nwarps * kTileWords) {
      uint32_t half[kTileWords];
#pragma unroll
      for (int u = 0; u < kTileWords; u++) {
        uint32_t pw = 0u;
        if (h0 + u < nh) {
          const int64_t col = 32 * (int64_t)(h0 + u) + lane;
          if (col < n) pw = posw[cpos[col]];
        }
        half[u] = transpose32(pw);
      }
      if (lane < rows) {
#pragma unroll
        for (int u = 0; u < kTileWords; u += 2) {
          const int64_t w64 = (h0 + u) >> 1;
          if (w64 < row_words) {
            const uint64_t word = (uint64_t)half[u] | ((uint64_t)half[u + 1] << 32);
            orow[w64] = word;
            mine += __popcll(word);
          }
        }
      }
    }
    if (threadIdx.x < rows) {
      const int32_t p = cpos[o0 + threadIdx.x];
      alive[o0 + threadIdx.x] = (uint8_t)((V[p >> 5] >> (p & 31)) & 1u);
    }
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(edge_count, mine);
}

kz_status bitset_fetch_dense(kz_graph g, uint64_t *h_out, int64_t row_words, uint8_t *d_alive,
                             unsigned long long *d_edge_count, cudaStream_t s) {
  KZ_CUDA_TRY(cudaMemsetAsync(d_edge_count, 0, sizeof(unsigned long long), s));
  if (g->n == 0) return KZ_OK;
  const size_t row = (size_t)g->ldw * 4;
  if (row > kRowSmemBytes) return KZ_ERR_UNSUPPORTED;  // beyond the bitset budget's reach
  // the tile form while 32 rows of position words fit in shared memory
  const bool tiles = 32 * row <= kTileSmemBytes;
  const int rows = tiles ? 32 : 4 * row <= kRowSmemBytes ? 4 : 2 * row <= kRowSmemBytes ? 2 : 1;
  const int threads = tiles ? kTileThreads : kPackThreads;
  const size_t smem = rows * row;
  auto fn = tiles ? unpack_tiles_kernel
                  : rows == 4 ? unpack_rows_kernel<4> : rows == 2 ? unpack_rows_kernel<2> : unpack_rows_kernel<1>;
  int per_sm = 0;
  KZ_CUDA_TRY(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  KZ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
  const size_t bytes = (size_t)g->n * row_words * 8;
  // row chunks: the unpacking kernel of chunk c + 1 runs while chunk c
  // travels to the host on the copy stream (a copy into pageable memory
  // returns only when done, so the next kernel is enqueued first)
  const int chunks = copy_chunks(bytes);
  cudaStream_t cs = chunks > 1 ? copy_stream() : s;
  if (chunks > 1 && !cs) return KZ_ERR_CUDA;
  uint64_t *d_out = (uint64_t *)dev_alloc(bytes, s);
  if (!d_out) return KZ_ERR_OOM;
  const int64_t per = ((int64_t)g->n + chunks - 1) / chunks;
  std::vector<cudaEvent_t> ev((size_t)chunks, nullptr);
  kz_status st = KZ_OK;
  for (int c = 0; c < chunks && st == KZ_OK; c++)
    if (cs != s) st = cuda_status(cudaEventCreateWithFlags(&ev[c], cudaEventDisableTiming));
  auto launch = [&](int c) -> kz_status {
    const int64_t r0 = std::min<int64_t>(c * per, g->n), r1 = std::min<int64_t>(r0 + per, g->n);
    if (r1 <= r0) return KZ_OK;
    const int64_t groups = (r1 - r0 + rows - 1) / rows;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)std::max(per_sm, 1) * sm_count()));
    fn<<<grid, threads, smem, s>>>(g->A[0], g->A[1], g->V[0], g->V[1], &g->st->cur, g->n, g->ldw, g->d_inv,
                                   g->d_cpos, d_out, row_words, d_alive, d_edge_count, r0, r1);
    KZ_CUDA_TRY(cudaGetLastError());
    if (cs != s) KZ_CUDA_TRY(cudaEventRecord(ev[c], s));
    return KZ_OK;
  };
  if (st == KZ_OK) st = launch(0);
  for (int c = 0; c < chunks && st == KZ_OK; c++) {
    if (c + 1 < chunks) st = launch(c + 1);
    const int64_t r0 = std::min<int64_t>(c * per, g->n), r1 = std::min<int64_t>(r0 + per, g->n);
    if (st != KZ_OK || r1 <= r0) continue;
    if (cs != s) st = cuda_status(cudaStreamWaitEvent(cs, ev[c], 0));
    if (st == KZ_OK)
      st = cuda_status(cudaMemcpyAsync(h_out + r0 * row_words, d_out + r0 * row_words,
                                       (size_t)(r1 - r0) * row_words * 8, cudaMemcpyDeviceToHost, cs));
  }
  if (cs != s) {
    // the caller's stream covers the copies (and so the buffer's release)
    cudaEvent_t done = nullptr;
    kz_status st2 = cuda_status(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    if (st2 == KZ_OK) st2 = cuda_status(cudaEventRecord(done, cs));
    if (st2 == KZ_OK) st2 = cuda_status(cudaStreamWaitEvent(s, done, 0));
    if (done) cudaEventDestroy(done);
    if (st2 != KZ_OK && st == KZ_OK) st = st2;
    // after a failure the caller does not wait: no copy may outlive the call
    if (st != KZ_OK) cudaStreamSynchronize(cs);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
  dev_free(d_out, bytes, s);
  return st;
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
  // small tables of the packers: carved from the graph's chunks (one
  // allocator call at most), released with the graph
  int32_t *d_inv = nullptr, *d_col = nullptr, *d_coff = nullptr, *d_err = nullptr;
  unsigned long long *d_cnt = nullptr;
  const size_t nn = (size_t)std::max(g->n, 1);
  KZ_TRY(graph_alloc(g, &d_inv, nn, s));
  KZ_TRY(graph_alloc(g, &d_col, nn, s));
  KZ_TRY(graph_alloc(g, &d_coff, (size_t)g->k + 1, s));
  KZ_TRY(graph_alloc(g, &d_err, 4, s));
  KZ_TRY(graph_alloc(g, &d_cnt, 2, s));
  tmp.clear();
  if (g->n) {
    KZ_TRY(h2d(d_inv, g->inv.data(), (size_t)g->n * 4, s));
    KZ_TRY(h2d(d_col, col_new.data(), (size_t)g->n * 4, s));
  }
  KZ_TRY(h2d(d_coff, g->coff.data(), ((size_t)g->k + 1) * 4, s));
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
  kz_status st2 = st == KZ_OK ? pack_finish(g, s, a, tmp) : KZ_OK;
  return st != KZ_OK ? st : st2;
}

kz_status bitset_pack_dense(kz_graph g, const uint64_t *h_bits, int64_t row_words, cudaStream_t s) {
  PackArgs a;
  std::vector<void *> tmp;
  kz_status st = pack_setup(g, s, a, tmp);
  const int64_t words = (int64_t)g->n * g->ldw;
  if (st == KZ_OK && words > 0) {
    // the upper triangle row by row, then the transposed half tile by tile
    const size_t row = (size_t)((g->n + 31) / 32) * 4, coff = (size_t)(g->k + 1) * 4;
    if (row + coff > kRowSmemBytes) st = KZ_ERR_UNSUPPORTED;  // beyond the bitset budget's reach
    // the tile form while one column word per caller column fits in shared
    // memory (32 rows x n bits)
    const bool tiles = g->n <= kTileMaxN && 32 * row + coff <= kTileSmemBytes;
    const int rows = tiles ? 32 : 4 * row + coff <= kRowSmemBytes ? 4 : 2 * row + coff <= kRowSmemBytes ? 2 : 1;
    const int threads = tiles ? kTileThreads : kPackThreads;
    const size_t smem = rows * row + coff;
    auto fn = tiles ? pack_dense_tiles_kernel
                    : rows == 4 ? pack_dense_rows_kernel<4> : rows == 2 ? pack_dense_rows_kernel<2> : pack_dense_rows_kernel<1>;
    int per_sm = 0;
    if (st == KZ_OK)
      st = cuda_status(cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (st == KZ_OK) st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    const size_t bytes = (size_t)g->n * row_words * 8;
    uint64_t *d_bits = st == KZ_OK ? (uint64_t *)dev_alloc(bytes, s) : nullptr;
    if (st == KZ_OK && !d_bits) st = KZ_ERR_OOM;
    // row chunks: chunk c + 1 travels on the copy stream while the packing
    // kernel of chunk c runs; the copy stream first waits for the caller's
    // stream, which owns the fresh buffer
    const int chunks = copy_chunks(bytes);
    cudaStream_t cs = chunks > 1 ? copy_stream() : s;
    if (st == KZ_OK && chunks > 1 && !cs) st = KZ_ERR_CUDA;
    const int64_t per = ((int64_t)g->n + chunks - 1) / chunks;
    std::vector<cudaEvent_t> ev;
    if (st == KZ_OK && cs != s) {
      ev.assign((size_t)chunks + 1, nullptr);
      for (auto &e : ev)
        if (st == KZ_OK) st = cuda_status(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      if (st == KZ_OK) st = cuda_status(cudaEventRecord(ev[chunks], s));
      if (st == KZ_OK) st = cuda_status(cudaStreamWaitEvent(cs, ev[chunks], 0));
    }
    bool copied_any = false;
    for (int c = 0; c < chunks && st == KZ_OK; c++) {
      const int64_t r0 = std::min<int64_t>(c * per, g->n), r1 = std::min<int64_t>(r0 + per, g->n);
      if (r1 <= r0) continue;
      st = cuda_status(cudaMemcpyAsync(d_bits + r0 * row_words, h_bits + r0 * row_words,
                                       (size_t)(r1 - r0) * row_words * 8, cudaMemcpyHostToDevice, cs));
      copied_any = true;
      if (st == KZ_OK && cs != s) st = cuda_status(cudaEventRecord(ev[c], cs));
      if (st == KZ_OK && cs != s) st = cuda_status(cudaStreamWaitEvent(s, ev[c], 0));
      if (st != KZ_OK) break;
      const int64_t groups = (r1 - r0 + rows - 1) / rows;
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)std::max(per_sm, 1) * sm_count()));
      fn<<<grid, threads, smem, s>>>(a, d_bits, row_words, g->n, g->R, g->d_perm, r0, r1);
      st = cuda_status(cudaGetLastError());
    }
    if (st != KZ_OK && copied_any && cs != s) cudaStreamSynchronize(cs);  // no release under a running copy
    if (st == KZ_OK) {
      const int64_t ng = ((int64_t)g->R * g->k + kSymGroup - 1) / kSymGroup;
      const int64_t pairs = ng * (ng + 1) / 2;
      const int sgrid = (int)std::max<int64_t>(1, std::min<int64_t>(pairs, 8 * sm_count()));
      symmetrize_kernel<<<sgrid, 32 * kSymGroup, 0, s>>>(g->A0, a.coff, g->k, g->R, g->ldw);
      st = cuda_status(cudaGetLastError());
    }
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (d_bits) dev_free(d_bits, bytes, s);
  }
  kz_status st2 = st == KZ_OK ? pack_finish(g, s, a, tmp) : KZ_OK;
  return st != KZ_OK ? st : st2;
}

}  // namespace kz
