// kz_internal.cuh -- layouts, handle and helpers shared by the library's
// translation units.  Nothing here is part of the C ABI (see include/kz.h).
//
// Bitset layout ("block-plane rows")
// ----------------------------------
// Vertices are relabelled so that colour class c occupies the contiguous id
// range [coff[c], coff[c] + csz[c]).  A class is cut into *blocks* of 32
// consecutive vertices: block (c, r) holds class members 32r .. 32r+31.  A
// vertex x of class c, member index i = x - coff[c], lives in block
// (c, i / 32) at bit i % 32.
//
// Every adjacency row is an array of 32-bit words, one word per block, laid
// out plane-major: the word of block (c, r) sits at index r * k + c.  Plane 0
// (the first k words of a row) therefore holds the first 32 members of every
// class, which is all a dense graph needs to show that an edge is covered.
// R = max_c ceil(csz[c] / 32) planes; rows are padded to ldw = round_up(R*k, 4)
// words so that every row starts on a 16-byte boundary.  Words of a vertex's
// own class and words of planes a class does not reach stay zero forever.
//
// The vertex live mask uses the same word indexing (one row of ldw words).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/kz.h"

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
  int32_t pad0;
  int64_t sweeps;     // productive sweeps so far
  int64_t passes;     // passes so far
  int64_t tests;      // live edges tested, all passes
  int64_t max_sweeps;
  unsigned long long pass_dv;     // counters of the running pass
  unsigned long long pass_de;
  unsigned long long pass_tests;
  unsigned int ticket;            // warps finished in the running pass
  unsigned int pad1;
  int64_t trace_dv[kTraceCap];
  int64_t trace_de[kTraceCap];
};

// Device allocation through the registered allocator.
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, size_t bytes, cudaStream_t s);

}  // namespace kz

// The handle behind kz_graph.
struct kz_graph_s {
  int32_t n = 0, k = 0;
  int64_t m = 0;          // edges after merging duplicates
  int device = 0;
  cudaStream_t stream = nullptr;  // stream of the last enqueued work
  bool kernelized = false;
  int32_t path_ran = KZ_PATH_BITSET;

  // relabelling (host)
  std::vector<int32_t> perm;  // new id -> caller id
  std::vector<int32_t> inv;   // caller id -> new id
  std::vector<int32_t> coff;  // k + 1 class offsets
  std::vector<int32_t> rounds;  // k: blocks per class
  std::vector<kz::BlockDesc> blocks;
  std::vector<int32_t> boff;  // k + 1: first block of each class

  // bitset layout
  int32_t R = 0, ldw = 0;
  size_t row_bytes = 0;

  // device buffers (owned)
  uint32_t *A0 = nullptr;     // pristine adjacency, n * ldw words
  uint32_t *A[2] = {nullptr, nullptr};
  uint32_t *V0 = nullptr;     // pristine live words, ldw
  uint32_t *V[2] = {nullptr, nullptr};
  int32_t *v_sweep = nullptr;  // n (relabelled ids)
  int32_t *d_rounds = nullptr; // k
  int32_t *d_coff = nullptr;   // k + 1
  int32_t *d_perm = nullptr;   // n
  kz::BlockDesc *d_blocks = nullptr;
  kz::WorkItem *d_items = nullptr;
  int32_t n_items = 0;
  kz::DevState *st = nullptr;

  // executable CUDA graph of the device-side sweep loop (built lazily)
  cudaGraphExec_t loop_exec = nullptr;
  int loop_grid = 0;

  // every device allocation, for kz_free_graph
  struct Alloc { void *p; size_t bytes; };
  std::vector<Alloc> allocs;
};

namespace kz {

// Kernels and host helpers of the bitset path (kz_bitset.cu).
kz_status bitset_build_layout(kz_graph g);
kz_status bitset_pack_edges(kz_graph g, const int32_t *d_edges, int64_t m, bool dedup,
                            cudaStream_t s);
kz_status bitset_pack_dense(kz_graph g, const uint64_t *d_bits, int64_t row_words,
                            const int32_t *d_colour_caller, cudaStream_t s);
kz_status bitset_finish_load(kz_graph g, cudaStream_t s);
kz_status bitset_reset(kz_graph g, cudaStream_t s);
kz_status bitset_kernelize(kz_graph g, const kz_options &opt, cudaStream_t s);
kz_status bitset_unpack_dense(kz_graph g, uint64_t *d_out, int64_t row_words,
                              unsigned long long *d_edge_count, cudaStream_t s);
kz_status bitset_vertex_alive(kz_graph g, uint8_t *host_alive, int64_t *n_live);

// Allocation bookkeeping on the handle.
template <class T>
kz_status graph_alloc(kz_graph g, T **out, size_t count, cudaStream_t s) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 16;
  void *p = dev_alloc(bytes, s);
  if (!p) {
    *out = nullptr;
    return KZ_ERR_OOM;
  }
  g->allocs.push_back({p, bytes});
  *out = static_cast<T *>(p);
  return KZ_OK;
}

inline kz_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return KZ_OK;
  if (e == cudaErrorMemoryAllocation) return KZ_ERR_OOM;
  return KZ_ERR_CUDA;
}

}  // namespace kz

#define KZ_CUDA_TRY(expr)                            \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) return kz::cuda_status(_e); \
  } while (0)

#define KZ_TRY(expr)                  \
  do {                                \
    kz_status _s = (expr);            \
    if (_s != KZ_OK) return _s;       \
  } while (0)
