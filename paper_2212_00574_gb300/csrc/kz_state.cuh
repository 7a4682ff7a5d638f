// kz_state.cuh -- the data the library's kernels share: block descriptors,
// work items, the per-graph device state word block and the in-CTA graph
// descriptor.  The bitset layout these refer to is described in
// kz_internal.cuh.  Host-only declarations live there, so that changing them
// leaves every kernel's sources as they were.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kz {

constexpr int kWarp = 32;
constexpr int kTraceCap = 1 << 16;  // per-sweep trace entries kept on the device

// One block of up to 32 same-coloured vertices.
struct BlockDesc {
  int32_t c;     // colour class
  int32_t r;     // plane (round) within the class
  int32_t base;  // first vertex (relabelled id)
  int32_t size;  // members, 1..32
};

// Work item of the sweep kernel: block x against blocks [y0, y1) of higher
// classes; vflag marks the one item per x that also evaluates the vertex rule.
struct WorkItem {
  int32_t x;
  int32_t y0;
  int32_t y1;
  int32_t vflag;
};

// Device-resident loop state of one graph.  Written by the sweep kernels'
// last warp; read by the host only after a synchronisation.
struct DevState {
  int32_t cur;        // which ping-pong buffer holds the live state
  int32_t status;     // kz_status of the running / last kernelize
  int32_t cont;       // 1 while another pass is needed
  int32_t full_write; // next pass writes every word of the next buffer (cleared after a pass)
  int64_t sweeps;     // productive sweeps so far
  int64_t passes;     // passes so far
  int64_t tests;      // live edges tested, all passes
  int64_t max_sweeps;
  unsigned long long pass_dv;     // counters of the running pass
  unsigned long long pass_de;
  unsigned long long pass_tests;
  unsigned int ticket;            // warps finished in the running pass
  unsigned int pad1;
  unsigned int bar_count;         // grid barrier of the persistent sweep kernel
  unsigned int bar_gen;
  int32_t bar_abort;              // a bounded barrier wait ran out
  int32_t pad2;
  unsigned long long pass_word;   // persistent sweep kernel: barrier generation and next-pass state
  unsigned long long ppass[2][3]; // persistent sweep kernel: pass counters (tests, de, dv) by pass parity
  int64_t trace_dv[kTraceCap];
  int64_t trace_de[kTraceCap];
};

// The persistent sweep kernel's barrier word: the generation (20 bits), then
// whether another pass follows, the buffer it reads and its sweep number.
// The pass-closing CTA writes it once; waiting CTAs need no other read.
__host__ __device__ inline unsigned long long pass_word(uint32_t gen, int cont, int cur, int64_t sweeps) {
  return (unsigned long long)(gen & 0xfffffu) | ((unsigned long long)(cont & 1) << 20) |
         ((unsigned long long)(cur & 1) << 21) | ((unsigned long long)sweeps << 22);
}
__host__ __device__ inline uint32_t pass_word_gen(unsigned long long w) { return (uint32_t)(w & 0xfffffu); }
__host__ __device__ inline int pass_word_cont(unsigned long long w) { return (int)((w >> 20) & 1u); }
__host__ __device__ inline int pass_word_cur(unsigned long long w) { return (int)((w >> 21) & 1u); }
__host__ __device__ inline int64_t pass_word_sweeps(unsigned long long w) { return (int64_t)(w >> 22); }

// Per-graph descriptor of the whole-fixpoint-in-one-CTA kernel.
struct CtaGraph {
  uint32_t *A0, *A1;      // ping-pong adjacency rows
  uint32_t *V0, *V1;      // ping-pong vertex live words
  int32_t *v_sweep;
  DevState *st;
  const BlockDesc *blocks;
  const int32_t *rounds;
  const int32_t *pair_off;  // nb + 1 prefix of block pairs per x
  const int32_t *boff;      // k + 1 first block of each class
  int32_t n, k, ldw, nb;
  int32_t smem_words;       // words the shared mode needs (-1: too many)
  int32_t pad;
  int64_t m;                // edges (default sweep limit n + m + 1)
  int64_t cost;
};

}  // namespace kz
