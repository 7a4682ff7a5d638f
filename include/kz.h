/*
 * kz.h -- C ABI of the GB300 colour-index kernelization library (libkz.so).
 *
 * The library computes the kernel of a legally k-coloured graph under the two
 * colour-index rules of the thesis "Kernelization of Discrete Optimization
 * Problems on Parallel Architectures" (arXiv 2212.00574), Section 4.2:
 *
 *   - Definition 4.2.1: the graph is legally coloured with k colours, the
 *     colour classes being c_1..c_k (0..k-1 here).
 *   - Vertex rule (colour index of a node, and the remark after it): a vertex
 *     whose neighbours cover fewer than k-1 colour classes lies in no k-clique
 *     and is deleted.
 *   - Edge rule (colour index of an edge, and the remark after it): an edge
 *     {u,v} whose common neighbours cover fewer than k-2 colour classes lies
 *     in no k-clique and is deleted; u and v are kept.
 *
 * The rules are applied to the live graph, sweep after sweep, until neither
 * fires.  Each sweep is a Jacobi sweep: both rules read the same snapshot and
 * their deletions are applied together.  The result is the unique greatest
 * subgraph closed under both rules, so no k-clique is ever lost.
 *
 * Conventions shared by every entry point:
 *   - Every call returns a kz_status and never aborts, traps or exits.
 *   - `void* stream` is a cudaStream_t on the current device (NULL = the
 *     legacy default stream).  Work is enqueued on it; the calls marked
 *     "synchronous" wait for it.
 *   - Host pointers stay owned by the caller and are not retained after the
 *     call returns.  A kz_graph owns all the device memory it uses; it is
 *     allocated at load through the registered allocator (kz_set_allocator)
 *     or cudaMallocAsync, and released by kz_free_graph.
 *   - Vertex ids at the boundary are the caller's ids 0..n-1.  Internally the
 *     library relabels vertices so that every colour class is contiguous.
 *   - There is no CPU fallback: without a usable CUDA device the calls that
 *     need one return KZ_ERR_CUDA.
 *   - Asynchronous failures (sweep limit, a bounds check in a kernel) are
 *     recorded on the device and reported by the next synchronous call on the
 *     same graph (kz_fetch_kernel, kz_fetch_kernel_dense, kz_fetch_stats).
 */
#ifndef KZ_H
#define KZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kz_graph_s *kz_graph; /* opaque handle */

typedef enum {
    KZ_OK = 0,
    KZ_ERR_ARG = 1,                /* null pointer, negative size, k outside [1, 64], bad option */
    KZ_ERR_COLOUR_RANGE = 2,       /* a colour outside [0, k) */
    KZ_ERR_ILLEGAL_COLOURING = 3,  /* an edge joins two vertices of one colour (Definition 4.2.1) */
    KZ_ERR_SELF_LOOP = 4,          /* an edge {v, v} */
    KZ_ERR_VERTEX_RANGE = 5,       /* an endpoint outside [0, n) */
    KZ_ERR_DUPLICATE_EDGE = 6,     /* an edge given twice (either orientation) without KZ_DEDUP */
    KZ_ERR_OOM = 7,                /* device allocation failed */
    KZ_ERR_CUDA = 8,               /* a CUDA runtime call failed (no device, launch failure, ...) */
    KZ_ERR_LIMIT = 9,              /* max_sweeps productive sweeps ran and a rule still fired */
    KZ_ERR_TIMEOUT = 10,           /* a bounded device wait gave up */
    KZ_ERR_NOT_READY = 11,         /* fetch before any kz_kernelize on this graph */
    KZ_ERR_BUFFER = 12,            /* output capacity too small (the needed size is still reported) */
    KZ_ERR_UNSUPPORTED = 13,       /* the requested path cannot hold this graph */
    KZ_ERR_INTERNAL = 14           /* a kernel's own consistency check failed */
} kz_status;

/* kz_load_graph / kz_load_graph_dense flags */
#define KZ_DEDUP 0x1u /* merge duplicate and reversed edge pairs instead of failing */

/* Which kernels evaluate the rules (kz_options.path). */
typedef enum {
    KZ_PATH_AUTO = 0,   /* SPARSE for a graph loaded as an edge list without bitset rows; SMALL up to 64
                           vertices; otherwise BITSET or TENSOR from a table of measured times to fixpoint
                           over n, k and edge density (TENSOR for larger, sparser graphs) */
    KZ_PATH_BITSET = 1, /* per-colour bitset rows in HBM, warp-per-block-pair sweep kernel */
    KZ_PATH_SMALL = 2,  /* whole fixpoint inside one CTA, graph held in shared memory */
    KZ_PATH_SPARSE = 3, /* CSR adjacency, per-edge colour masks from triangle enumeration */
    KZ_PATH_TENSOR = 4  /* per-colour common-neighbour counts on tcgen05 tensor cores */
} kz_path;

/* Order in which elements are tested (kz_options.schedule).  Neither changes
 * the result: the greatest fixpoint of monotone deletion rules is unique. */
typedef enum {
    KZ_SCHED_PLAIN = 0,   /* Jacobi sweeps over every live element */
    KZ_SCHED_LEARNED = 1, /* MLP-ranked worklist, then a full certifying sweep */
    KZ_SCHED_SUPPORT = 2  /* the same Jacobi sweeps, re-testing only what the last sweep's
                             deletions can have broken.  On the CSR state (graphs loaded from an
                             edge list; path AUTO or SPARSE): per-class common-neighbour counts
                             kept up to date as triangles break; needs about 4 m k bytes
                             (KZ_ERR_UNSUPPORTED above 6 GiB).  On the bitset rows (graphs
                             without a CSR, or path BITSET or TENSOR): a full first sweep on that
                             path, then each sweep re-checks, for every edge {a, b} the last one
                             deleted and every common neighbour w, the pairs {a, w} and {b, w} in
                             the class of the neighbour they lost.  Either way the sweeps and
                             per-sweep deletions equal PLAIN's; edge_tests counts the tests made
                             (distinct pairs re-checked per sweep) */
} kz_schedule;

/* First test of a pair in the BITSET path's sweep kernels (kz_options.plane0).
 * Both are exact: a pair the first test leaves open is recounted over all
 * planes.  Only the speed differs. */
typedef enum {
    KZ_PLANE0_AUTO = 0, /* by edge density: half words from 0.8, two planes below 0.42 */
    KZ_PLANE0_FULL = 1, /* the first 32 members of each class, one word per class */
    KZ_PLANE0_HALF = 2, /* the first 16 members of each class, two classes per word */
    KZ_PLANE0_TWO = 3   /* the first 64 members of each class (k <= 32 and classes of more than
                           32 members; otherwise FULL) */
} kz_plane0;

/* How kz_kernelize_batch runs its graphs (kz_options.batch).  All give the
 * same results; only the scheduling differs. */
typedef enum {
    KZ_BATCH_CONCURRENT = 0, /* each graph on its own path (kz_options.path; AUTO per graph), spread
                                over the library's internal streams longest first, joined back
                                into the caller's stream */
    KZ_BATCH_SEQUENTIAL = 1, /* each graph on its own path, one after another on the caller's stream */
    KZ_BATCH_FUSED = 2       /* one launch for all graphs: the in-CTA persistent kernel (path SMALL,
                                and graphs with k > 32), otherwise the batched multi-graph Jacobi
                                kernel; graphs without bitset rows run on the CSR path first */
} kz_batch_mode;

typedef struct {
    int32_t path;         /* kz_path */
    int32_t schedule;     /* kz_schedule */
    int64_t max_sweeps;   /* productive sweeps allowed; <= 0 means n + m + 1 (always enough) */
    int32_t use_graph;    /* device-side pass loop: 1 (default) one cooperative persistent launch,
                             2 a CUDA-graph while node (one launch per pass), 0 host-driven loop */
    int32_t plane0;       /* kz_plane0 (BITSET path only) */
    int32_t batch;        /* kz_batch_mode (kz_kernelize_batch only) */
    int32_t clique_k;     /* clique size q sought, 1 <= q <= k; 0 means q = k.  The rules delete a
                             vertex whose live neighbours cover fewer than q-1 classes and an edge whose
                             live common neighbours cover fewer than q-2 (thesis Section 4.2, Remarks:
                             a q-clique survives whenever the colouring is legal, whatever k >= q).
                             q < k runs on the BITSET, SMALL, SPARSE and TENSOR paths with the plain
                             schedule; the LEARNED and SUPPORT schedules and the FUSED batch return
                             KZ_ERR_UNSUPPORTED for it */
    int32_t dominance;    /* 1: after the colour-index fixpoint, rounds of vertex dominance (thesis
                             Section 4.3, Definition 4.3.1), each followed by the fixpoint again, until
                             a round deletes nothing.  2: the same with rounds of edge dominance
                             (Definitions 4.3.2 and 4.3.3: an edge {x, y} goes when another live edge
                             {u, v} has every common neighbour of x and y as a common neighbour; in one
                             round, of dominated edges whose records {x, y, u, v} share a vertex only
                             the one with the smallest caller-id key goes); needs a clique size of at
                             least 3.  0 (default): off.  Opt-in because dominance keeps the clique
                             number but may delete some maximum cliques.  Needs bitset rows (paths
                             BITSET, SMALL, TENSOR) and the plain schedule, else KZ_ERR_UNSUPPORTED;
                             kz_kernelize_batch refuses it.  The statistics and the trace then cover
                             the last colour-index run */
    int32_t tensor_precision;  /* TENSOR path operands: 0 (default) E4M3 0/1 through
                                  tcgen05.mma kind::f8f6f4; 1 BF16 0/1 through kind::f16 (twice
                                  the operand bytes and MMAs; the same exact counts) */
    int32_t reserved[4];  /* must be zero */
} kz_options;

/* Fill *opt with the defaults (AUTO path, PLAIN schedule, no sweep limit,
 * device-side pass loop in one persistent launch). */
void kz_default_options(kz_options *opt);

typedef struct {
    int64_t n, m;          /* input vertices and edges (after KZ_DEDUP merging) */
    int64_t n_live;        /* vertices in the kernel */
    int64_t m_live;        /* edges in the kernel */
    int64_t sweeps;        /* productive Jacobi sweeps of the last kz_kernelize */
    int64_t passes;        /* rule evaluations over the whole graph, the certifying one included */
    int64_t edge_tests;    /* live edges tested, summed over passes */
    int32_t path;          /* kz_path that ran */
    int32_t status;        /* kz_status recorded on the device by the last kz_kernelize */
    int32_t k;             /* colours */
    int32_t clique_k;      /* clique size q the last kz_kernelize used */
    int32_t dominance_rounds;  /* dominance rounds of the last kz_kernelize that deleted something */
    int32_t dominated;     /* vertices (vertex dominance) or edges (edge dominance) those rounds deleted */
    int32_t reserved[2];
} kz_stats;

/* Optional device allocator (for example a caching allocator owned by the
 * caller).  alloc returns NULL on failure; both are called on the host with
 * the stream the allocation is used on.  Passing NULL restores
 * cudaMallocAsync / cudaFreeAsync.  Applies to graphs loaded afterwards. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} kz_allocator;

kz_status kz_set_allocator(const kz_allocator *allocator);

/*
 * Load a graph given as an edge list (synchronous).
 *   n       vertices (ids 0..n-1), n >= 0
 *   k       colours, 1 <= k <= 64; the clique size searched for is also k
 *           (Definition 4.2.1 uses one k for both)
 *   colour  host int32[n], colour[v] in [0, k); must be a legal colouring
 *   m       number of edges, m >= 0
 *   edges   host int32[2*m]: pairs (u, v), any orientation
 *   flags   KZ_DEDUP or 0
 *   stream  stream for the copies and the packing kernels
 *   out     receives the handle (NULL on failure)
 * Input errors (KZ_ERR_COLOUR_RANGE, _VERTEX_RANGE, _SELF_LOOP,
 * _ILLEGAL_COLOURING, _ARG) are found on the host before any CUDA call;
 * duplicates are found on the device during packing.
 */
kz_status kz_load_graph(int32_t n, int32_t k, const int32_t *colour, int64_t m,
                        const int32_t *edges, uint32_t flags, void *stream, kz_graph *out);

/*
 * Load a graph given as a dense adjacency bit matrix (synchronous).
 *   adj_bits   host uint64[n * row_words], row-major; bit (j % 64) of word
 *              (j / 64) in row i is set iff {i, j} is an edge.  Only bits with
 *              j > i are read: the diagonal and the lower triangle are ignored,
 *              so the matrix need not be symmetric.  Bits j >= n are ignored.
 *   row_words  words per row, >= ceil(n / 64)
 * Other arguments as kz_load_graph.  An upper-triangle bit joining two
 * vertices of one colour gives KZ_ERR_ILLEGAL_COLOURING.
 */
kz_status kz_load_graph_dense(int32_t n, int32_t k, const int32_t *colour,
                              const uint64_t *adj_bits, int64_t row_words, uint32_t flags,
                              void *stream, kz_graph *out);

/*
 * Run the rules to their fixpoint, starting from the graph's current live
 * state (as loaded, as left by an earlier kz_kernelize, or as restored by
 * kz_reset).  Asynchronous: enqueued on `stream`.  opt may be NULL (defaults).
 * The per-run counters (sweeps, passes, edge_tests, status) restart at zero.
 */
kz_status kz_kernelize(kz_graph g, const kz_options *opt, void *stream);

/*
 * Kernelize `count` graphs (asynchronous).  Every graph ends exactly as
 * kz_kernelize would leave it.  opt as kz_kernelize; opt->path selects the
 * per-graph path (AUTO lets the measured table choose per graph), and
 * opt->batch how the graphs are scheduled (kz_batch_mode): by default each
 * graph runs on its own path over the library's internal streams (one or a
 * few launches per graph); KZ_BATCH_FUSED runs them all in one persistent
 * launch.  The caller's stream waits for every graph.
 */
kz_status kz_kernelize_batch(kz_graph *graphs, int32_t count, const kz_options *opt, void *stream);

/*
 * Tuning of the fused batch (kz_options.batch = KZ_BATCH_FUSED).  Its cost
 * model gives each graph a group of clamp(cost / unit, 1, max_group) CTAs of
 * the persistent launch, where a graph's cost is its block pairs times k and
 * unit is the batch's total cost over group_spread times the resident CTAs;
 * a graph's pass is split into about items_per_warp work items per warp of
 * its group.  A value <= 0 restores the default (the values the batch
 * autotuner measured best on the 1024-graph workload).  Applies to the next
 * fused batch (a changed setting rebuilds the batch's plan).  Process-wide.
 * Returns KZ_ERR_ARG for a NaN group_spread.
 */
kz_status kz_set_batch_tuning(double group_spread, int32_t items_per_warp, int32_t max_group);

/*
 * Copy the kernel back (synchronous: waits for the graph's last stream).
 *   vertex_alive  host uint8[n] (may be NULL): 1 if the vertex survives
 *   edges_out     host int32[2*cap] (may be NULL when cap == 0): surviving
 *                 edges as (u, v) with u < v in caller ids, sorted
 *                 lexicographically
 *   cap           capacity of edges_out in edges
 *   m_out         receives the number of surviving edges (always written,
 *                 also when KZ_ERR_BUFFER is returned)
 *   stats         may be NULL
 * Returns the device status of the last kz_kernelize if it is not KZ_OK
 * (for example KZ_ERR_LIMIT; the partial kernel is still copied).
 */
kz_status kz_fetch_kernel(kz_graph g, uint8_t *vertex_alive, int32_t *edges_out, int64_t cap,
                          int64_t *m_out, kz_stats *stats);

/*
 * Copy the kernel back as a symmetric dense bit matrix in caller ids
 * (synchronous).  adj_bits host uint64[n * row_words], fully overwritten;
 * row_words >= ceil(n / 64).  vertex_alive and stats as kz_fetch_kernel.
 */
kz_status kz_fetch_kernel_dense(kz_graph g, uint8_t *vertex_alive, uint64_t *adj_bits,
                                int64_t row_words, kz_stats *stats);

/* Statistics only (synchronous, copies no kernel). */
kz_status kz_fetch_stats(kz_graph g, kz_stats *stats);

/*
 * Per-sweep trace of the last kz_kernelize (synchronous).
 *   dv, de   host int64[cap]: vertices / edges that failed their rule in each
 *            productive sweep (entries beyond `sweeps` are not written)
 *   v_sweep  host int32[n] (may be NULL): productive sweep (1-based) in which
 *            each caller vertex was deleted, 0 if it survives
 */
kz_status kz_fetch_trace(kz_graph g, int64_t *dv, int64_t *de, int64_t cap, int32_t *v_sweep);

/* Restore the live state to the graph as loaded (asynchronous). */
kz_status kz_reset(kz_graph g, void *stream);

/*
 * Clique search on the current kernel (synchronous; host branch and bound).
 * Looks for a clique of q vertices (0 <= q <= k) in the kernel that the last
 * kz_kernelize left; the kernel for clique size q holds every q-clique of the
 * graph (thesis Section 4.2, Remarks), so the answer is the graph's.  The
 * search is exact: colour-ordered branch and bound (at most one vertex per
 * class under the legal colouring), branching on the class with the fewest
 * candidates, pruned when fewer classes with candidates remain than vertices
 * are still needed.
 *   node_limit  search nodes allowed; <= 0 means no limit
 *   clique_out  host int32[q]: the clique's caller ids in ascending order
 *               (written when one is found)
 *   found       1 when a q-clique was found, 0 when there is none
 * Returns KZ_ERR_NOT_READY before any kz_kernelize, KZ_ERR_LIMIT when the
 * node limit ran out before the search ended (found = 0, unknown), KZ_ERR_ARG
 * for q outside [0, k], KZ_ERR_UNSUPPORTED when the kernel's adjacency
 * bitsets would exceed 8 GB of host memory.
 */
kz_status kz_find_clique(kz_graph g, int32_t q, int64_t node_limit, int32_t *clique_out, int32_t *found);

/*
 * Maximum clique through kernelization (synchronous): for q = k, k-1, ..., 1
 * the graph is reset, kernelized for clique size q (opt with clique_k = q;
 * opt may be NULL for the defaults) and searched with kz_find_clique; the
 * first q with a clique is the clique number (the thesis, Section 4: the
 * k-clique test run for decreasing k answers the maximum clique problem; a
 * legal k-colouring bounds it by k).  On return the handle holds the kernel
 * for *q_out.
 *   q_out       the clique number (0 for an empty graph)
 *   clique_out  host int32[k]: one maximum clique, caller ids ascending
 *               (its first *q_out entries)
 * Returns KZ_ERR_LIMIT when a search ran out of nodes (*q_out is the size
 * being searched then), or the first error of kz_reset / kz_kernelize.
 */
kz_status kz_max_clique(kz_graph g, const kz_options *opt, int64_t node_limit, int32_t *q_out, int32_t *clique_out,
                        void *stream);

/* Release the handle and its device memory (waits for its stream).  NULL is
 * ignored. */
void kz_free_graph(kz_graph g);

/* Static, NUL-terminated description of a status. */
const char *kz_status_string(kz_status s);

/*
 * kz_kernelize_dense_noalloc -- kernelize one graph without allocating any
 * memory.  The thesis has no counterpart: this is an interface for callers
 * that cannot allocate device memory.  Examples: a process whose device
 * memory is wholly reserved by another allocator (a framework's memory pool
 * that owns the GPU), code that runs inside such an allocator's callbacks,
 * and latency-critical loops that must not call cudaMalloc because it can
 * synchronise the device.  kz_load_graph and friends allocate per graph;
 * this entry point uses one fixed scratch array instead.
 *
 * Every intermediate (relabelling, bitset rows, ping-pong buffers, loop
 * state) lives in a static device array of about 9 MiB that each GPU loading
 * the library holds until the process exits.  The first call on a device
 * does the set-up: it looks up that array's device address (once per
 * device).  Make that first call before any stream capture, and while about
 * 9 MiB of device memory is still free: with lazy module loading the CUDA
 * runtime materialises the array at that first call, so a caller whose pool
 * will reserve the whole GPU should make one warm-up call before the pool
 * does.  The call itself makes no cudaMalloc, cudaFree or other allocating
 * call, host or device.
 *
 * All calls share the one array, which keeps the last call's contents (every
 * call re-initialises what it reads).  Calls that overlap on the GPU (two
 * host threads, or two streams) race on it and give wrong results: serialise
 * them.
 *
 * Arguments (all buffers are DEVICE memory owned by the caller):
 *   n, k          vertices (0 <= n <= KZ_NOALLOC_MAX_N) and colours (1..32)
 *   colour        int32[n], legal colouring
 *   adj_bits      uint64[n * row_words], as kz_load_graph_dense (strict upper
 *                 triangle read)
 *   max_sweeps    as kz_options.max_sweeps
 *   vertex_alive  uint8[n] out: 1 if the vertex is in the kernel
 *   adj_out       uint64[n * row_words] out: the kernel's symmetric bit matrix
 *   counts        int64[4] out: sweeps, passes, edge tests, status
 *   stream        stream for every launch; the call waits for it at the end,
 *                 so no call can be captured into a CUDA graph
 * Returns the status (also in counts[3]).  n > KZ_NOALLOC_MAX_N, or colour
 * classes so uneven that the bitset rows exceed KZ_NOALLOC_MAX_WORDS words,
 * give KZ_ERR_UNSUPPORTED.  Statuses found on the host (KZ_ERR_ARG, and
 * KZ_ERR_UNSUPPORTED for n) leave the outputs untouched; statuses found on
 * the device (KZ_ERR_COLOUR_RANGE, KZ_ERR_ILLEGAL_COLOURING, KZ_ERR_UNSUPPORTED
 * for uneven classes) leave vertex_alive and adj_out all zero and counts[0..2]
 * zero.  KZ_ERR_LIMIT leaves the partial kernel, as kz_fetch_kernel does.
 */
#define KZ_NOALLOC_MAX_N 4096
#define KZ_NOALLOC_MAX_WORDS (1 << 20)
kz_status kz_kernelize_dense_noalloc(int32_t n, int32_t k, const int32_t *colour,
                                     const uint64_t *adj_bits, int64_t row_words, int64_t max_sweeps,
                                     uint8_t *vertex_alive, uint64_t *adj_out, int64_t *counts,
                                     void *stream);

/* Library version as major * 10000 + minor * 100 + patch. */
int32_t kz_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KZ_H */
