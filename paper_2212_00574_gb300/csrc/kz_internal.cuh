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

#include "kz_state.cuh"

namespace kz {

// Device allocation through the registered allocator.
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, size_t bytes, cudaStream_t s);

// Host-to-device copy of a host table.  While a LoadStage is active on this
// thread the bytes are first copied into one pinned staging arena, so the
// copy is asynchronous (the host does not wait for the stream's earlier work)
// and the source may be released at once; otherwise an ordinary copy.
kz_status h2d(void *dst, const void *src, size_t bytes, cudaStream_t s);

// Scope of one graph load: holds the staging arena for this thread and waits
// for the stream at its end (so the arena is free for the next load).
struct LoadStage {
  explicit LoadStage(cudaStream_t s);
  ~LoadStage();
  LoadStage(const LoadStage &) = delete;
  LoadStage &operator=(const LoadStage &) = delete;
  cudaStream_t stream;
};

}  // namespace kz

namespace kz {
struct CtaGraph;
// Grid and work split of the multi-CTA sweep kernels for one plane-0 form
// (built when the form is first used).
struct SweepPlan {
  int32_t grid = 0;                 // CTAs, one per SM at most (0: not built)
  int32_t *d_cta_begin = nullptr;   // first unit of each CTA's range, grid + 1
};
}  // namespace kz
typedef kz::CtaGraph *CtaGraphPtr;

// The handle behind kz_graph.
struct kz_graph_s {
  int32_t n = 0, k = 0;
  int64_t m = 0;          // edges after merging duplicates
  uint64_t uid = 0;       // unique per loaded graph (batch plans are keyed by it)
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
  int32_t *d_boff = nullptr;   // k + 1
  int32_t *d_pair_off = nullptr;  // blocks + 1
  int64_t n_pairs = 0;
  CtaGraphPtr d_cta_desc = nullptr;  // this graph's in-CTA descriptor
  int32_t *d_zero = nullptr;         // a device 0 (queue order of a single graph)
  int32_t *d_perm = nullptr;   // n
  kz::BlockDesc *d_blocks = nullptr;
  kz::SweepPlan plan[3];              // work of the sweep kernels per form (full, half-word, two-plane)
  uint8_t *d_changed = nullptr;       // per unit: low byte of the sweep that last changed it
  int2 *d_units = nullptr;            // (x, y) of every unit, in pass order
  int64_t n_units = 0;
  // true when the two row buffers differ only in the words of units whose
  // change tag names the current sweep (false after any other path or a
  // conversion wrote the rows; the next bitset pass then writes every word)
  bool ab_synced = false;
  double density = 0;                // edges / pairs of vertices in different classes, at load
  int32_t slack = 0;                  // k minus the clique size of the current kz_kernelize (0: q = k)
  int32_t form = 0;                   // the sweep kernels' first test chosen by density
  bool fast_half = false;             // half-word form: fold whole blocks first (very dense graphs)
  kz::DevState *st = nullptr;

  // which representation holds the live state: KZ_PATH_BITSET (bitset rows,
  // also used by the in-CTA path) or KZ_PATH_SPARSE (CSR flags)
  bool has_bitset = false;
  bool has_csr = false;
  int32_t owner = KZ_PATH_BITSET;
  int32_t *d_inv = nullptr;    // caller id -> relabelled id (bitset layout)
  int32_t *d_cpos = nullptr;   // caller id -> (word << 5) | bit of its relabelled vertex inside any row

  // CSR path (caller ids)
  int64_t *sp_row0 = nullptr;  // n + 1, all edges
  int32_t *sp_adj0 = nullptr, *sp_eid0 = nullptr;
  int64_t *sp_row[2] = {nullptr, nullptr};  // compacted live rows (ping-pong)
  int32_t *sp_adj[2] = {nullptr, nullptr};
  int32_t *sp_eid[2] = {nullptr, nullptr};
  uint8_t *sp_elive[2] = {nullptr, nullptr};
  uint8_t *sp_vlive[2] = {nullptr, nullptr};
  int32_t sp_cur = 0;
  int64_t *sp_orow = nullptr;  // oriented live CSR
  int32_t *sp_oadj = nullptr, *sp_oeid = nullptr, *sp_osrc = nullptr;
  int32_t *sp_eu = nullptr, *sp_ev = nullptr;  // canonical sorted edges
  int32_t *sp_col = nullptr, *sp_rank = nullptr;
  unsigned long long *sp_mask = nullptr;
  int32_t *sp_cnt_live = nullptr, *sp_cnt_or = nullptr;
  int64_t *sp_sums = nullptr, *sp_totals = nullptr;
  int32_t *sp_v_sweep = nullptr;

  // learned schedule: attached model, threshold, per-graph scratch
  struct kz_model_s *model = nullptr;
  float learned_threshold = 0.5f;
  void *learned_bufs = nullptr;
  void *tensor_bufs = nullptr;  // tensor-core path scratch
  void *support_bufs = nullptr; // per-class support counts (CSR path, support schedule)
  void *dominance_bufs = nullptr;  // vertex dominance rounds
  int32_t dom_rounds = 0;          // dominance rounds of the last kz_kernelize that deleted something
  int64_t dom_removed = 0;         // vertices they deleted

  // executable CUDA graph of the device-side sweep loop (built lazily)
  cudaGraphExec_t loop_exec = nullptr;
  // executable CUDA graph of one persistent run: run-start kernel, then the
  // cooperative sweep kernel (built lazily; one launch per kz_kernelize)
  cudaGraphExec_t run_exec = nullptr;
  int64_t run_max_sweeps = 0;
  int32_t run_form = -1;
  int32_t run_slack = 0;
  int loop_grid = 0;
  int64_t loop_max_sweeps = 0;
  int32_t loop_form = 0;
  int32_t loop_slack = 0;

  // every device allocation, for kz_free_graph
  struct Alloc { void *p; size_t bytes; };
  std::vector<Alloc> allocs;
  // small allocations are carved from chunks (one allocator call per chunk)
  uint8_t *arena = nullptr;
  size_t arena_size = 0, arena_used = 0, arena_next = 256 << 10;
};

namespace kz {

// Kernels and host helpers of the bitset path (kz_bitset.cu; loading and
// fetching in kz_pack.cu).
kz_status bitset_build_layout(kz_graph g);
kz_status bitset_pack_edges(kz_graph g, const int32_t *d_edges, int64_t m, bool dedup,
                            cudaStream_t s);
// Packs a host dense bit matrix (row-major, row_words words a row), copied
// in row chunks that overlap the packing; synchronous.
kz_status bitset_pack_dense(kz_graph g, const uint64_t *h_bits, int64_t row_words, cudaStream_t s);
kz_status bitset_finish_load(kz_graph g, cudaStream_t s);
kz_status bitset_reset(kz_graph g, cudaStream_t s);
kz_status bitset_kernelize(kz_graph g, const kz_options &opt, cudaStream_t s);
// Caller-ordered dense rows of the current state into host memory (row
// chunks, each copied while the next is unpacked), vertex flags (bytes, on
// the device) and the count of set bits (twice the edges, on the device).
// Asynchronous on s: the caller's wait on s covers every copy.
kz_status bitset_fetch_dense(kz_graph g, uint64_t *h_out, int64_t row_words, uint8_t *d_alive,
                             unsigned long long *d_edge_count, cudaStream_t s);
kz_status bitset_vertex_alive(kz_graph g, uint8_t *host_alive, int64_t *n_live);

// One plain multi-CTA sweep pass (no loop graph); *cont = 1 when it deleted
// something and another pass should follow.
kz_status bitset_one_pass(kz_graph g, cudaStream_t s, int *cont);
// Failure-path probe of the persistent kernel's bounded grid barrier.
kz_status bitset_barrier_timeout_probe(kz_graph g, uint32_t spin_limit, cudaStream_t s);
// Run start (counters zero, sweep limit) without a pass.
kz_status bitset_begin_run(kz_graph g, int64_t max_sweeps, cudaStream_t s);

// Tensor-core edge rule (kz_tensor.cu).
kz_status tensor_kernelize(kz_graph g, const kz_options &opt, cudaStream_t s);
// One pass of the tensor form (the run started by bitset_begin_run); *cont = 1
// when it deleted something and the run may go on.
kz_status tensor_one_pass(kz_graph g, const kz_options &opt, cudaStream_t s, int *cont);
void tensor_release(kz_graph g);
// The driver's cuTensorMapEncodeTiled, found through the runtime's entry-point
// query (null when the driver does not provide it).
void *tensor_map_encoder();
// One round of vertex dominance (Definition 4.3.1) on the current bitset rows;
// synchronous, returns the vertices deleted.
kz_status dominance_round(kz_graph g, int64_t *removed, cudaStream_t s);
// One round of edge dominance (Definitions 4.3.2, 4.3.3) on the current rows;
// *removed = edges deleted.  Needs a colour-index fixpoint for q >= 3 first.
kz_status edge_dominance_round(kz_graph g, int64_t *removed, cudaStream_t s);
void dominance_release(kz_graph g);

// Learned schedule (kz_learned.cu).
kz_status learned_kernelize(kz_graph g, const kz_options &opt, int full_path, cudaStream_t s);
// Schedule SUPPORT on the bitset rows: a full first sweep, then sweeps that
// re-check only the (pair, class) combinations the last one touched.
kz_status recheck_kernelize(kz_graph g, const kz_options &opt, int full_path, cudaStream_t s);
void learned_release(kz_graph g);

// Whole-fixpoint-in-one-CTA kernel (kz_cta.cu).
kz_status cta_prepare(kz_graph g, cudaStream_t s);
kz_status cta_upload_descriptor(kz_graph g, cudaStream_t s);
bool cta_fits_shared(kz_graph g);
// force_mode: 1 = shared mode where it fits, 0 = global mode for every graph
kz_status cta_kernelize(kz_graph *gs, int count, const kz_options &opt, cudaStream_t s, int force_mode);
// One graph, one CTA, no allocation or copy per call.
kz_status cta_kernelize_one(kz_graph g, const kz_options &opt, cudaStream_t s);

// CSR path (kz_sparse.cu).
// Edges: device int32[2 m], caller ids (validated on the host).
kz_status sparse_load(kz_graph g, const int32_t *colour, int64_t m, const int32_t *d_edges, bool dedup,
                      cudaStream_t s);
// The sorted edge list, CSR and orientation rank on the device (kz_csr.cu).
kz_status sparse_build_csr(kz_graph g, const int32_t *d_edges, int64_t m, bool dedup, cudaStream_t s);
// out[0..n] = exclusive prefix of in[0..n-1], out[n] = total (kz_sparse.cu);
// sums holds n / 1024 + 1 partial sums.
kz_status scan_counts(const int32_t *in, int64_t n, int64_t *out, int64_t *sums, int64_t *total, cudaStream_t s);
kz_status sparse_reset(kz_graph g, cudaStream_t s);
kz_status sparse_kernelize(kz_graph g, const kz_options &opt, cudaStream_t s);
kz_status sparse_fetch(kz_graph g, uint8_t *vertex_alive, int32_t *edges_out, int64_t cap, int64_t *m_live);
kz_status sparse_vertex_alive(kz_graph g, uint8_t *host_alive, int64_t *n_live);
kz_status sparse_v_sweep(kz_graph g, int32_t *host);
// Oriented CSR of the live edges of the current CSR state.
kz_status sparse_orient_live(kz_graph g, cudaStream_t s);
// The CSR path with incremental per-class support counts (kz_support.cu).
kz_status sparse_kernelize_support(kz_graph g, const kz_options &opt, cudaStream_t s);
void support_release(kz_graph g);
// Move the live state between the two representations.
kz_status state_to_sparse(kz_graph g, cudaStream_t s);
kz_status state_to_bitset(kz_graph g, cudaStream_t s);

// Batched Jacobi loop over many graphs (kz_batch.cu); every k <= 32.
kz_status batch_kernelize(kz_graph *gs, int count, const kz_options &opt, cudaStream_t s);

// Allocation bookkeeping on the handle.
// Device memory owned by the graph (freed with it).  Requests below 1 MiB
// are carved, 256-byte aligned, from chunks of at least 256 KiB (each chunk
// twice the last), so loading a graph makes few allocator calls; larger ones
// get their own allocation.
template <class T>
kz_status graph_alloc(kz_graph g, T **out, size_t count, cudaStream_t s) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void *p = nullptr;
  if (bytes < ((size_t)1 << 20)) {
    if (!g->arena || g->arena_used + bytes > g->arena_size) {
      const size_t chunk = g->arena_next > bytes ? g->arena_next : bytes;
      void *c = dev_alloc(chunk, s);
      if (!c) {
        *out = nullptr;
        return KZ_ERR_OOM;
      }
      g->allocs.push_back({c, chunk});
      g->arena = static_cast<uint8_t *>(c);
      g->arena_size = chunk;
      g->arena_used = 0;
      g->arena_next = chunk * 2;
    }
    p = g->arena + g->arena_used;
    g->arena_used += bytes;
  } else {
    p = dev_alloc(bytes, s);
    if (!p) {
      *out = nullptr;
      return KZ_ERR_OOM;
    }
    g->allocs.push_back({p, bytes});
  }
  *out = static_cast<T *>(p);
  return KZ_OK;
}

inline kz_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return KZ_OK;
  if (e == cudaErrorMemoryAllocation) return KZ_ERR_OOM;
  return KZ_ERR_CUDA;
}

}  // namespace kz

// On failure the runtime's last-error state is consumed, so that a refused
// launch (a non-sticky error) does not resurface in a later, unrelated call.
#define KZ_CUDA_TRY(expr)                            \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) {                         \
      cudaGetLastError();                            \
      return kz::cuda_status(_e);                    \
    }                                                \
  } while (0)

#define KZ_TRY(expr)                  \
  do {                                \
    kz_status _s = (expr);            \
    if (_s != KZ_OK) return _s;       \
  } while (0)
