// kz_rules.cuh -- warp-level evaluation of the two Section 4.2 rules on the
// block-plane bitset layout (see kz_internal.cuh), shared by the multi-CTA
// sweep kernel and the whole-fixpoint-in-one-CTA kernel.
//
// Vertex rule: a live vertex u fails when the classes other than col(u) that
// hold a live neighbour number fewer than q-1.
// Edge rule: a live edge {u,v} fails when the classes other than col(u),
// col(v) that hold a live common neighbour number fewer than q-2.
// q is the clique size sought, at most the number of colours k; the thesis
// states the rules for q = k.  With slack = k - q the rules read "more than
// slack needed classes uncovered", so the all-covered tests below settle a
// pair for every q and only the recounts take slack.
//
// A warp works on a block X (lane = member u) against a block Y of a higher
// class.  Plane 0 of row u (the first 32 members of every class) sits in
// registers as Fu[c]; a per-pair mask P[c] is all ones for c = col(u),
// c = col(v) and padding classes c >= k, zero elsewhere.  The pair is covered
// in every needed class at once when
//     min_c ((Fu[c] & Fv[c]) | P[c]) != 0,
// one LOP3 and half a three-input min per class.  A live edge that fails this
// plane-0 test is recounted exactly over all planes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kz_internal.cuh"

namespace kz {

__device__ __forceinline__ uint32_t kz_min3(uint32_t a, uint32_t b, uint32_t c) {
  return __vimin3_u32(a, b, c);
}

// Exact count over all planes of the classes (other than cu) in which row u
// has a set bit.
static __device__ __noinline__ int exact_vertex_cover_row(const uint32_t *ru, int k,
                                                   const int32_t *__restrict__ rounds, int cu) {
  int cnt = 0;
  for (int c = 0; c < k; c++) {
    if (c == cu) continue;
    const int R = rounds[c];
    for (int r = 0; r < R; r++) {
      if (ru[r * k + c]) {
        cnt++;
        break;
      }
    }
  }
  return cnt;
}

// Plane 0 of a row into registers (zero when the lane has no vertex).
template <int KMAX>
__device__ __forceinline__ void load_plane0(uint32_t (&Fu)[KMAX], const uint32_t *row, int k,
                                            bool valid) {
#pragma unroll
  for (int q = 0; q < KMAX / 4; q++) {
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (valid && 4 * q < k) w = reinterpret_cast<const uint4 *>(row)[q];
    // words at or beyond k belong to the next plane: never counted
    if (4 * q + 0 >= k) w.x = 0u;
    if (4 * q + 1 >= k) w.y = 0u;
    if (4 * q + 2 >= k) w.z = 0u;
    if (4 * q + 3 >= k) w.w = 0u;
    Fu[4 * q + 0] = w.x;
    Fu[4 * q + 1] = w.y;
    Fu[4 * q + 2] = w.z;
    Fu[4 * q + 3] = w.w;
  }
}

template <int KMAX>
__device__ __forceinline__ void pair_mask(uint32_t (&P)[KMAX], int k, int cu, int cv) {
#pragma unroll
  for (int c = 0; c < KMAX; c++) P[c] = (c == cu || c == cv || c >= k) ? 0xffffffffu : 0u;
}

// True when plane 0 alone shows every needed class covered.  fv points at
// the first word of v's row (16-byte aligned); words at or beyond k are not
// read.
template <int KMAX>
__device__ __forceinline__ bool plane0_covered(const uint32_t (&Fu)[KMAX], const uint32_t (&P)[KMAX],
                                               const uint32_t *fv, int k) {
  uint32_t m0 = 0xffffffffu, m1 = 0xffffffffu;
#pragma unroll
  for (int q = 0; q < KMAX / 4; q++) {
    if (4 * q >= k) break;  // k is uniform: one kernel serves every k <= KMAX
    const uint4 w = reinterpret_cast<const uint4 *>(fv)[q];
    m0 = kz_min3(m0, (Fu[4 * q + 0] & w.x) | P[4 * q + 0], (Fu[4 * q + 1] & w.y) | P[4 * q + 1]);
    m1 = kz_min3(m1, (Fu[4 * q + 2] & w.z) | P[4 * q + 2], (Fu[4 * q + 3] & w.w) | P[4 * q + 3]);
  }
  return min(m0, m1) != 0u;
}

// Number of classes other than cu whose plane-0 word of row u is non-zero.
template <int KMAX>
__device__ __forceinline__ int plane0_vertex_cover(const uint32_t (&Fu)[KMAX], int k, int cu) {
  int cnt = 0;
#pragma unroll
  for (int c = 0; c < KMAX; c++) cnt += (c < k && c != cu && Fu[c] != 0u) ? 1 : 0;
  return cnt;
}

// Classes (bit c) other than cu whose plane-0 word of row u is zero.
template <int KMAX>
__device__ __forceinline__ uint64_t plane0_vertex_missing(const uint32_t (&Fu)[KMAX], int k, int cu) {
  uint64_t miss = 0;
#pragma unroll
  for (int c = 0; c < KMAX; c++)
    if (c < k && c != cu && Fu[c] == 0u) miss |= 1ull << c;
  return miss;
}

// Classes in miss0 (none of their first 32 members is a neighbour of u) that
// a later plane of row u covers.  Reads only the later planes of those
// classes; `rounds` (blocks per class) is best in shared memory.
static __device__ __noinline__ int vertex_cover_beyond_plane0(const uint32_t *ru, int k,
                                                             const int32_t *__restrict__ rounds, uint64_t miss0) {
  int cnt = 0;
  while (miss0) {
    const int c = __ffsll((long long)miss0) - 1;
    miss0 &= miss0 - 1;
    const int R = rounds[c];
    for (int r = 1; r < R; r++) {
      if (ru[r * k + c]) {
        cnt++;
        break;
      }
    }
  }
  return cnt;
}

// Classes (bit c) that plane 0 leaves uncovered for the pair: needed classes
// whose plane-0 word AND is zero.
template <int KMAX>
__device__ __forceinline__ uint64_t plane0_missing(const uint32_t (&Fu)[KMAX], const uint32_t (&P)[KMAX],
                                                   const uint32_t *fv, int k) {
  uint64_t miss = 0;
#pragma unroll
  for (int c = 0; c < KMAX; c++) {
    if (c >= k) break;
    if (((Fu[c] & fv[c]) | P[c]) == 0u) miss |= 1ull << c;
  }
  return miss;
}

// Exact edge rule for a pair that plane 0 did not settle: every class in
// `miss` must show a common neighbour in some later plane.  Returns true
// when the edge fails (some needed class has none in any plane).
__device__ __forceinline__ bool edge_fails_beyond_plane0(const uint32_t *ru, const uint32_t *rv, int k,
                                                         const int32_t *__restrict__ rounds, uint64_t miss,
                                                         int slack) {
  // the edge fails when more than `slack` needed classes hold no common
  // neighbour (slack = colours - clique size: 0 for the thesis's rule)
  if (__popcll(miss) <= slack) return false;
  int missing = 0;
  while (miss) {
    const int c = __ffsll((long long)miss) - 1;
    miss &= miss - 1;
    const int R = rounds[c];
    bool found = false;
    for (int r = 1; r < R; r++) {
      if (ru[r * k + c] & rv[r * k + c]) {
        found = true;
        break;
      }
    }
    if (!found && ++missing > slack) return true;
  }
  return false;
}

// Tests every live edge between the lane's vertex u (row ru, plane 0 in Fu)
// and the members of block Y.  adjw = row u's word for Y (bit b = edge to
// member b).  fv_row(b) returns plane 0 of member b's row; row_v(b) returns
// member b's full row.  Returns the lane's deletion mask over Y's members.
// Must be called by all 32 lanes.  A pair that plane 0 does not settle is
// recounted by its own lane over the later planes of the uncovered classes
// only; the lanes' recounts run side by side, so their loads overlap.
template <int KMAX, class FvRow, class FullRow>
__device__ __forceinline__ uint32_t edge_rule_block(const uint32_t (&Fu)[KMAX], const uint32_t (&P)[KMAX],
                                                    const uint32_t *ru, uint32_t adjw, int k, int slack,
                                                    const int32_t *__restrict__ rounds, int cu, int cv,
                                                    FvRow fv_row, FullRow row_v) {
  (void)cu;
  (void)cv;
  uint32_t bits = __reduce_or_sync(0xffffffffu, adjw);
  uint32_t del = 0;
  while (bits) {
    const int b = __ffs(bits) - 1;
    bits &= bits - 1;
    const uint32_t *fv = fv_row(b);
    const bool covered = plane0_covered<KMAX>(Fu, P, fv, k);
    if (((adjw >> b) & 1u) && !covered) {
      const uint64_t miss = plane0_missing<KMAX>(Fu, P, fv, k);
      if (edge_fails_beyond_plane0(ru, row_v(b), k, rounds, miss, slack)) del |= 1u << b;
    }
  }
  return del;
}

// Hot loop of the sweep kernels: the plane-0 test of every member of block Y
// (rows staged in shared memory, KMAX words apart) against every lane's u,
// two members at a time (four independent min chains).  Returns the lane's
// live edges that plane 0 does not settle; the recount is done afterwards
// by recount_unsettled, outside this loop.
template <int KMAX>
__device__ __forceinline__ uint32_t plane0_unsettled(const uint32_t (&Fu)[KMAX], const uint32_t (&P)[KMAX],
                                                     const uint32_t *sv, uint32_t adjw, int k) {
  uint32_t bits = __reduce_or_sync(0xffffffffu, adjw);
  uint32_t open = 0;
  while (bits) {
    const int b0 = __ffs(bits) - 1;
    bits &= bits - 1;
    const uint4 *f0 = reinterpret_cast<const uint4 *>(sv + b0 * KMAX);
    if (bits) {
      const int b1 = __ffs(bits) - 1;
      bits &= bits - 1;
      const uint4 *f1 = reinterpret_cast<const uint4 *>(sv + b1 * KMAX);
      uint32_t m0 = 0xffffffffu, m1 = 0xffffffffu, m2 = 0xffffffffu, m3 = 0xffffffffu;
#pragma unroll
      for (int q = 0; q < KMAX / 4; q++) {
        // words >= k are forced by P, but the bound check keeps the compiler
        // from rebuilding P inside the loop (measured: 1.6x the instructions)
        if (4 * q >= k) break;
        const uint4 w0 = f0[q], w1 = f1[q];
        m0 = kz_min3(m0, (Fu[4 * q + 0] & w0.x) | P[4 * q + 0], (Fu[4 * q + 1] & w0.y) | P[4 * q + 1]);
        m1 = kz_min3(m1, (Fu[4 * q + 2] & w0.z) | P[4 * q + 2], (Fu[4 * q + 3] & w0.w) | P[4 * q + 3]);
        m2 = kz_min3(m2, (Fu[4 * q + 0] & w1.x) | P[4 * q + 0], (Fu[4 * q + 1] & w1.y) | P[4 * q + 1]);
        m3 = kz_min3(m3, (Fu[4 * q + 2] & w1.z) | P[4 * q + 2], (Fu[4 * q + 3] & w1.w) | P[4 * q + 3]);
      }
      if (min(m0, m1) == 0u) open |= 1u << b0;
      if (min(m2, m3) == 0u) open |= 1u << b1;
    } else {
      uint32_t m0 = 0xffffffffu, m1 = 0xffffffffu;
#pragma unroll
      for (int q = 0; q < KMAX / 4; q++) {
        if (4 * q >= k) break;
        const uint4 w0 = f0[q];
        m0 = kz_min3(m0, (Fu[4 * q + 0] & w0.x) | P[4 * q + 0], (Fu[4 * q + 1] & w0.y) | P[4 * q + 1]);
        m1 = kz_min3(m1, (Fu[4 * q + 2] & w0.z) | P[4 * q + 2], (Fu[4 * q + 3] & w0.w) | P[4 * q + 3]);
      }
      if (min(m0, m1) == 0u) open |= 1u << b0;
    }
  }
  return open & adjw;
}

// ---------------------------------------------------------------------------
// Half-word form of plane 0, for dense graphs: word j holds the first 16
// members of class 2j (low half) and of class 2j+1 (high half), so one LOP3
// tests two classes and one three-input 16x2 min reduces four.  A pair is
// settled when every needed class has a common neighbour among the first 16
// members; anything else goes to the exact recount over the full rows.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t pack_halves(uint32_t lo, uint32_t hi) {
  return __byte_perm(lo, hi, 0x5410);  // low 16 bits of lo, then low 16 bits of hi
}

// Half-word plane 0 of a full-word plane 0 (KH = KMAX / 2 words).
template <int KMAX, int KH>
__device__ __forceinline__ void halve_plane0(uint32_t (&H)[KH], const uint32_t (&F)[KMAX]) {
#pragma unroll
  for (int j = 0; j < KH; j++) H[j] = pack_halves(F[2 * j], F[2 * j + 1]);
}

// Forced half-words: all ones for the classes of u and v and for classes >= k.
template <int KH>
__device__ __forceinline__ void half_mask(uint32_t (&P)[KH], int k, int cu, int cv) {
#pragma unroll
  for (int j = 0; j < KH; j++) {
    const int c0 = 2 * j, c1 = 2 * j + 1;
    const bool f0 = c0 == cu || c0 == cv || c0 >= k;
    const bool f1 = c1 == cu || c1 == cv || c1 >= k;
    P[j] = (f0 ? 0x0000ffffu : 0u) | (f1 ? 0xffff0000u : 0u);
  }
}

// Row stride (words) of the half-word staging buffer: KMAX / 2 rounded up to
// a multiple of 4, so that every row starts on 16 bytes.
template <int KMAX>
__host__ __device__ constexpr int half_stride() {
  return (KMAX / 2 + 3) / 4 * 4;
}

// Half-word form of staged plane-0 rows (KMAX words apart in src) into dst
// (half_stride<KMAX>() words apart): lane b converts row b.  Words of classes
// >= k come out as anything; the forced mask covers them.
template <int KMAX>
__device__ __forceinline__ void halve_staged_rows(const uint32_t *src, uint32_t *dst, int rows, int lane) {
  constexpr int KH = KMAX / 2;
  if (lane < rows) {
    const uint32_t *row = src + lane * KMAX;
    uint32_t *out = dst + lane * half_stride<KMAX>();
    uint32_t w[KMAX];
#pragma unroll
    for (int q = 0; q < KMAX / 4; q++) {
      const uint4 v = reinterpret_cast<const uint4 *>(row)[q];
      w[4 * q + 0] = v.x;
      w[4 * q + 1] = v.y;
      w[4 * q + 2] = v.z;
      w[4 * q + 3] = v.w;
    }
    uint32_t h[KH];
    halve_plane0<KMAX, KH>(h, w);
#pragma unroll
    for (int q = 0; q < KH / 4; q++)
      reinterpret_cast<uint4 *>(out)[q] = make_uint4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
    if constexpr (KH % 4 == 2)
      reinterpret_cast<uint2 *>(out)[KH / 2 - 1] = make_uint2(h[KH - 2], h[KH - 1]);
  }
}

__device__ __forceinline__ bool has_zero_half(uint32_t m) { return (m & 0xffffu) == 0u || m < 0x10000u; }

// Folds the forced half-word ANDs of one staged member row f into a0, a1.
template <int KH>
__device__ __forceinline__ void half_fold(const uint32_t (&F)[KH], const uint32_t (&P)[KH], const uint32_t *f,
                                          uint32_t &a0, uint32_t &a1) {
#pragma unroll
  for (int q = 0; q < KH / 4; q++) {
    const uint4 w = reinterpret_cast<const uint4 *>(f)[q];
    a0 = __vimin3_u16x2(a0, (F[4 * q + 0] & w.x) | P[4 * q + 0], (F[4 * q + 1] & w.y) | P[4 * q + 1]);
    a1 = __vimin3_u16x2(a1, (F[4 * q + 2] & w.z) | P[4 * q + 2], (F[4 * q + 3] & w.w) | P[4 * q + 3]);
  }
  if constexpr (KH % 4 == 2) {
    const uint2 w = reinterpret_cast<const uint2 *>(f)[KH / 2 - 1];
    a0 = __vimin3_u16x2(a0, (F[KH - 2] & w.x) | P[KH - 2], (F[KH - 1] & w.y) | P[KH - 1]);
  }
}

// Hot loop of the half-word form (see plane0_unsettled) over half-word rows
// sv (half_stride<KMAX>() words apart): returns the lane's live edges that
// the first 16 members of each class do not settle.  When
// `try_fast` is set and all 32 members of Y are in play, one pass folds every
// pair of the block into the lanes' running minima; only a block in which
// some pair (edge or not) shows an uncovered class is redone member by
// member.  Lanes without a vertex must hold all-ones in F.
template <int KMAX, int KH>
__device__ __forceinline__ uint32_t half_unsettled(const uint32_t (&F)[KH], const uint32_t (&P)[KH],
                                                   const uint32_t *sv, uint32_t adjw, bool try_fast) {
  uint32_t bits = __reduce_or_sync(0xffffffffu, adjw);
  if (try_fast && bits == 0xffffffffu) {
    uint32_t a0 = 0xffffffffu, a1 = 0xffffffffu, a2 = 0xffffffffu, a3 = 0xffffffffu;
#pragma unroll 2
    for (int b = 0; b < 32; b += 2) {
      half_fold<KH>(F, P, sv + b * half_stride<KMAX>(), a0, a1);
      half_fold<KH>(F, P, sv + (b + 1) * half_stride<KMAX>(), a2, a3);
    }
    const uint32_t a = __vimin3_u16x2(__vimin3_u16x2(a0, a1, a2), a3, 0xffffffffu);
    if (!__any_sync(0xffffffffu, has_zero_half(a))) return 0u;
  }
  uint32_t open = 0;
  while (bits) {
    const int b0 = __ffs(bits) - 1;
    bits &= bits - 1;
    uint32_t m0 = 0xffffffffu, m1 = 0xffffffffu;
    half_fold<KH>(F, P, sv + b0 * half_stride<KMAX>(), m0, m1);
    if (bits) {
      const int b1 = __ffs(bits) - 1;
      bits &= bits - 1;
      uint32_t m2 = 0xffffffffu, m3 = 0xffffffffu;
      half_fold<KH>(F, P, sv + b1 * half_stride<KMAX>(), m2, m3);
      if (has_zero_half(__vimin3_u16x2(m2, m3, 0xffffffffu))) open |= 1u << b1;
    }
    if (has_zero_half(__vimin3_u16x2(m0, m1, 0xffffffffu))) open |= 1u << b0;
  }
  return open & adjw;
}

// ---------------------------------------------------------------------------
// Two-plane form, for sparser graphs: the first test looks at the first 64
// members of each class (planes 0 and 1), so far fewer pairs go to the
// recount.  A staged row holds plane 0 in words [0, KMAX) and plane 1 in
// words [KMAX, 2 KMAX).
// ---------------------------------------------------------------------------

// Plane 1 of a row into registers (k words from row + k; zero when the lane
// has no vertex).  Plane 1 need not start on 16 bytes: scalar loads.
template <int KMAX>
__device__ __forceinline__ void load_plane1(uint32_t (&F1)[KMAX], const uint32_t *row, int k, bool valid) {
#pragma unroll
  for (int c = 0; c < KMAX; c++) F1[c] = (valid && c < k) ? row[k + c] : 0u;
}

// Staged rows hold the first round_up(2k, 4) words of each row at their own
// offsets; lane b moves plane 1 of row b from word k to word KMAX.
template <int KMAX>
__device__ __forceinline__ void spread_plane1(uint32_t *buf, int rows, int k, int lane) {
  if (k == KMAX || lane >= rows) return;
  uint32_t *row = buf + lane * 2 * KMAX;
  uint32_t t[KMAX];
#pragma unroll
  for (int c = 0; c < KMAX; c++) t[c] = c < k ? row[k + c] : 0u;
#pragma unroll
  for (int q = 0; q < KMAX / 4; q++)
    reinterpret_cast<uint4 *>(row + KMAX)[q] = make_uint4(t[4 * q], t[4 * q + 1], t[4 * q + 2], t[4 * q + 3]);
}

// Hot loop of the two-plane form (see plane0_unsettled): per class
// (F0 & w0) | (F1 & w1) | P, two LOP3s.  Returns the lane's live edges that
// the first 64 members of each class do not settle.
template <int KMAX>
__device__ __forceinline__ uint32_t two_unsettled(const uint32_t (&F0)[KMAX], const uint32_t (&F1)[KMAX],
                                                  const uint32_t (&P)[KMAX], const uint32_t *sv, uint32_t adjw,
                                                  int k) {
  uint32_t bits = __reduce_or_sync(0xffffffffu, adjw);
  uint32_t open = 0;
  while (bits) {
    const int b0 = __ffs(bits) - 1;
    bits &= bits - 1;
    const uint4 *f0 = reinterpret_cast<const uint4 *>(sv + b0 * 2 * KMAX);
    uint32_t m0 = 0xffffffffu, m1 = 0xffffffffu;
#pragma unroll
    for (int q = 0; q < KMAX / 4; q++) {
      if (4 * q >= k) break;  // see plane0_unsettled
      const uint4 a = f0[q], b = f0[KMAX / 4 + q];
      m0 = kz_min3(m0, (F0[4 * q + 0] & a.x) | (F1[4 * q + 0] & b.x) | P[4 * q + 0],
                   (F0[4 * q + 1] & a.y) | (F1[4 * q + 1] & b.y) | P[4 * q + 1]);
      m1 = kz_min3(m1, (F0[4 * q + 2] & a.z) | (F1[4 * q + 2] & b.z) | P[4 * q + 2],
                   (F0[4 * q + 3] & a.w) | (F1[4 * q + 3] & b.w) | P[4 * q + 3]);
    }
    if (min(m0, m1) == 0u) open |= 1u << b0;
  }
  return open & adjw;
}

// Recount, lane by lane, the edges plane 0 left open: the classes plane 0
// leaves uncovered (from the row of u and the staged row of v) are searched
// in their later planes.  Returns the lane's deletion mask.  Takes pointers
// only, so the hot loop's register arrays stay in registers.
static __device__ __noinline__ uint32_t recount_unsettled(const uint32_t *ru, const uint32_t *sv, int kmax_stride,
                                                         const uint32_t *ybase, int ldw, uint32_t open, int k,
                                                         int cu, int cv, const int32_t *__restrict__ rounds,
                                                         int slack) {
  uint32_t del = 0;
  while (open) {
    const int b = __ffs(open) - 1;
    open &= open - 1;
    const uint32_t *fv = sv + b * kmax_stride;
    uint64_t miss = 0;
    for (int c = 0; c < k; c++)
      if (c != cu && c != cv && (ru[c] & fv[c]) == 0u) miss |= 1ull << c;
    if (edge_fails_beyond_plane0(ru, ybase + (int64_t)b * ldw, k, rounds, miss, slack)) del |= 1u << b;
  }
  return del;
}

// Column view of the lanes' deletion masks: lane b receives the mask of the
// lanes (members of X) whose edge to member b of Y was deleted.
__device__ __forceinline__ uint32_t transpose_deletions(uint32_t del) {
  uint32_t delT = 0;
  uint32_t any = __reduce_or_sync(0xffffffffu, del);
  const int lane = threadIdx.x & 31;
  while (any) {
    const int b = __ffs(any) - 1;
    any &= any - 1;
    const uint32_t col = __ballot_sync(0xffffffffu, (del >> b) & 1u);
    if (lane == b) delT = col;
  }
  return delT;
}

// 32 x 32 bit-matrix transpose across the warp: lane i holds row i (bit j =
// entry (i, j)); lane j receives column j (bit i = entry (i, j)).  Five
// butterfly stages swap the off-diagonal half-blocks of 16, 8, 4, 2 and 1.
__device__ __forceinline__ uint32_t transpose32(uint32_t w) {
  const int lane = threadIdx.x & 31;
  const uint32_t masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int i = 0; i < 5; i++) {
    const int sft = 16 >> i;
    const uint32_t m = masks[i];
    const uint32_t q = __shfl_xor_sync(0xffffffffu, w, sft);
    w = (lane & sft) ? ((w & ~m) | ((q >> sft) & m)) : ((w & m) | ((q << sft) & ~m));
  }
  return w;
}

// Records a finished pass in the device state and decides whether another
// pass follows: a pass that deleted something is applied (sweeps + 1, the
// ping-pong buffers flip) unless the sweep limit is reached, in which case it
// is dropped and KZ_ERR_LIMIT recorded.  Returns 1 to continue.
__device__ __forceinline__ int finish_pass(DevState *st, unsigned long long dv, unsigned long long de,
                                           unsigned long long tests) {
  // every field is read before any is written, so the reads travel together
  // (one memory round trip instead of a chain of read-modify-writes)
  const int64_t passes = st->passes, total = st->tests, sweeps = st->sweeps, max_sweeps = st->max_sweeps;
  const int32_t cur = st->cur;
  const bool productive = dv + de > 0;
  const bool limited = productive && sweeps >= max_sweeps;
  const int cont = productive && !limited ? 1 : 0;
  st->passes = passes + 1;
  st->tests = total + (int64_t)tests;
  st->full_write = 0;
  if (limited) st->status = KZ_ERR_LIMIT;
  if (cont) {
    if (sweeps < kTraceCap) {
      st->trace_dv[sweeps] = (int64_t)dv;
      st->trace_de[sweeps] = (int64_t)de;
    }
    st->sweeps = sweeps + 1;
    st->cur = cur ^ 1;
  }
  st->cont = cont;
  return cont;
}

}  // namespace kz
