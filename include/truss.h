/*
 * truss.h -- C ABI of the GB300 (sm_103a) exact truss-decomposition library.
 *
 * Problem (Wang & Cheng, "Truss Decomposition in Massive Networks", Section 2,
 * problem definition): for an undirected simple graph G, compute for every edge
 * e its support sup(e) -- the number of triangles of G containing e
 * (Definition 1) -- and its truss number phi(e) = max{k : e in T_k}, where the
 * k-truss T_k is the largest subgraph in which every edge lies in at least k-2
 * triangles (Definition 2).  The k-class Phi_k (Definition 3) is the set of
 * edges with phi(e) = k, so the per-edge truss numbers are the whole
 * decomposition.  The method follows Algorithm 2 (Section 3.2): supports first
 * (step 2), then edges are removed in ascending order of support, decrementing
 * the support of the other two edges of each destroyed triangle (steps 4-12).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Input is an edge list of `rows` rows: src[r], dst[r] are int32 vertex ids
 *   in [0, n).  Rows are undirected pairs in either orientation; duplicate and
 *   reversed rows are allowed and receive the values of their edge; a self-loop
 *   row (src == dst) receives -1 in every per-row output.
 * - After removing self-loops and duplicates the number of distinct edges m
 *   must be < 2^31 (edge ids are int32).  n must be < 2^31.
 * - Every per-row output is indexed by input row and is int32.
 * - Pointers may be device memory or host memory (pageable or pinned); the
 *   library detects which with cudaPointerGetAttributes.  truss_support,
 *   truss_decompose and truss_decompose_batch read pinned host rows and
 *   write pinned host per-row outputs in place from their kernels (through
 *   the memory's device address); every other host buffer is staged
 *   through device memory the library owns.  The caller owns every input and
 *   output buffer; the library owns its workspace (a per-context arena that
 *   grows on demand and is released by truss_ctx_destroy).
 * - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).  Work
 *   is enqueued on it; the call reads two small counters back from the device
 *   (the number of distinct edges and the number of triangles, to size the
 *   workspace), so it returns only after the outputs are complete.
 * - Return value: TRUSS_OK (0) or a negative TRUSS_E* code; nothing throws
 *   across the ABI.  On error the outputs are unspecified.
 * - A truss_ctx is not thread-safe: use one context per host thread.  The
 *   truss_serve_* functions below are thread-safe.
 */
#ifndef TRUSS_H
#define TRUSS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- errors --- */
#define TRUSS_OK 0
#define TRUSS_EINVAL (-1)    /* bad argument, vertex id out of [0, n), m >= 2^31 */
#define TRUSS_ENOMEM (-2)    /* device or host allocation failed */
#define TRUSS_ECUDA (-3)     /* a CUDA runtime call failed */
#define TRUSS_ETIMEOUT (-4)  /* a bounded device-side wait gave up */
#define TRUSS_EAGAIN (-5)    /* serve: result not ready yet */
#define TRUSS_EBUSY (-6)     /* serve: admission refused (queue full / over budget) */
#define TRUSS_ESHUTDOWN (-7) /* serve: server stopped */
#define TRUSS_ECHECK (-8)    /* an internal consistency check failed */

/* Human-readable message for a TRUSS_* code (static storage). */
const char *truss_strerror(int code);

/* ------------------------------------------------------------ context --- */
typedef struct truss_ctx truss_ctx;

typedef struct truss_opts {
  /* Upper limit, in nanoseconds, of any device-side wait (the grid-wide
   * barrier of the persistent peel kernel).  A wait that exceeds it makes the
   * call return TRUSS_ETIMEOUT.  0 = default (4 s). */
  int64_t wait_limit_ns;
  /* Non-zero: record CUDA events around each stage (build, support, triangle
   * lists, peel, scatter) so truss_last_stats reports stage times. */
  int32_t profile;
  /* Non-zero: also compute the algorithmic byte counts of the support and
   * peel kernels (one extra host pass over small arrays). */
  int32_t count_bytes;
  /* The fields below choose schedules only: every value gives the same
   * outputs.  0 selects the built-in default for each. */
  /* Hub threshold of the support walk: out-lists of at most this many
   * entries are staged in shared memory, longer ones are read from global
   * memory (0 = the staging capacity, 512; larger values are clamped). */
  int32_t support_stage_max;
  /* Peel kernel variant: 0 or 2 = two 512-thread blocks per SM, one work item
   * per lane group; 1 = one block per SM, two items per lane group; 3 = one
   * block per SM, one item; 4 = the barrier-free peel (a destroyed bit per
   * triangle and a work queue per level instead of sub-rounds; it needs the
   * triangle records and fewer than 2^32 of them, else variant 0 runs). */
  int32_t peel_variant;
  /* Target walk cost (out-list entries) of one warp range of the support
   * walk (0 = 16384). */
  int32_t support_range_work;
  /* Fixed cost, in out-list entries, charged for every oriented edge when
   * the support walk is split into equal-cost ranges (0 = 64, negative =
   * none). */
  int32_t support_pair_cost;
  /* Non-zero: build the triangle lists by a second walk of the graph, the
   * path taken anyway when the support walk's triangle records do not fit
   * in free device memory (0 = records whenever they fit). */
  int32_t lists_by_walk;
  /* Non-zero: whenever the triangle records are used, leave each edge's own
   * triangles (those it closes as the walked edge) in the records instead of
   * copying them into its list; the list pass then writes a third less, and
   * the peel reads each list in two stretches.  0 = whole lists when they fit
   * in free device memory, own parts in place when only those fit.  Ignored
   * by peel variant 4, which needs whole lists. */
  int32_t lists_in_place;
  int32_t reserved[5];
} truss_opts;

/* Create a context bound to CUDA device `device` (ordinal).  opts may be NULL
 * (all defaults).  *out receives the context.  Errors: TRUSS_EINVAL (bad
 * device or NULL out), TRUSS_ECUDA, TRUSS_ENOMEM. */
int truss_ctx_create(truss_ctx **out, int device, const truss_opts *opts);

/* Replace the options of an existing context; they apply from its next call
 * (the workspace is kept).  The library has no counterpart in the paper: it
 * lets a schedule search time candidates on one warm context.  Errors:
 * TRUSS_EINVAL (NULL ctx or opts). */
int truss_ctx_set_opts(truss_ctx *ctx, const truss_opts *opts);

/* Release the context and its workspace.  NULL is accepted. */
int truss_ctx_destroy(truss_ctx *ctx);

/* ------------------------------------------------------- single graph --- */
/* Support of every edge (Definition 1; Algorithm 2 step 2).
 * n: vertex count; rows: number of rows of src/dst (0 allowed).
 * support_out[r] = sup(e) of row r's edge, -1 for self-loop rows.
 * Errors: TRUSS_EINVAL, TRUSS_ENOMEM, TRUSS_ECUDA. */
int truss_support(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src,
                  const int32_t *dst, int32_t *support_out, void *cuda_stream);

/* Full truss decomposition (Algorithm 2; Definitions 1-3).
 * support_out (nullable): sup(e) per row, as truss_support.
 * truss_out: phi(e) per row (>= 2), -1 for self-loop rows.
 * kmax_out (nullable, host or device int32[1]): k_max = max phi (0 if the
 * graph has no edge).
 * Errors: TRUSS_EINVAL, TRUSS_ENOMEM, TRUSS_ECUDA, TRUSS_ETIMEOUT. */
int truss_decompose(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src,
                    const int32_t *dst, int32_t *support_out, int32_t *truss_out,
                    int32_t *kmax_out, void *cuda_stream);

/* ------------------------------------------------------------- top-t ---- */
/* Upper bound of the truss number of every edge (Procedure 6, Section 6.2,
 * with the whole graph as the neighbourhood subgraph):
 *   psi(e) = min{sup(e), x_u, x_v} + 2, e = (u, v),
 * where x_w is the largest x such that w has x incident edges other than e
 * with support >= x.  phi(e) <= psi(e) (Lemma 2).
 * support_out (nullable): sup(e) per row; psi_out: psi(e) per row; both -1
 * for self-loop rows.  Errors: TRUSS_EINVAL, TRUSS_ENOMEM, TRUSS_ECUDA. */
int truss_upper_bound(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src,
                      const int32_t *dst, int32_t *support_out, int32_t *psi_out,
                      void *cuda_stream);

/* The top-t k-classes, Phi_k for k_max >= k > k_max - t (Algorithm 7,
 * Section 6.3).  truss_out[r] = phi(e) of row r's edge if phi(e) >= k_max -
 * t + 1, else 0; -1 for self-loop rows.  kmax_out (nullable, host or device
 * int32[1]) receives k_max (0 for a graph without edges).  t >= 1; a t of at
 * least k_max - 1 gives every class.  The library decomposes only the
 * candidate subgraph of edges whose psi is at least a threshold that it
 * lowers until it is <= k_max - t + 1 (truss_last_stats: candidates,
 * rounds).  Errors: TRUSS_EINVAL (also t < 1), TRUSS_ENOMEM, TRUSS_ECUDA,
 * TRUSS_ETIMEOUT. */
int truss_top(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
              int32_t t, int32_t *truss_out, int32_t *kmax_out, void *cuda_stream);

/* ------------------------------------------------ working-set budget --- */
/* Truss decomposition by the bottom-up method of Section 5 (Algorithm 3
 * LowerBounding, Algorithm 4, Procedure 5), for graphs whose decomposition
 * working set (which grows with the number of triangles) does not fit in
 * device memory.  The canonical edge list stays resident; the in-memory
 * decomposition only runs on neighbourhood subgraphs (Definition 4) of about
 * budget_edges edges.  Outputs as truss_decompose (identical values).
 * truss_last_stats: rounds = neighbourhood subgraphs decomposed, candidates =
 * the largest one's edges.  A subgraph larger than the budget (one vertex
 * of higher degree, or a large NS(U_k)) is decomposed whole, so the budget
 * bounds the working set only as far as the graph allows.
 * Errors: TRUSS_EINVAL (also budget_edges < 1), TRUSS_ENOMEM, TRUSS_ECUDA,
 * TRUSS_ETIMEOUT. */
int truss_decompose_budget(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src,
                           const int32_t *dst, int64_t budget_edges, int32_t *support_out,
                           int32_t *truss_out, int32_t *kmax_out, void *cuda_stream);

/* ------------------------------------------------------------- k-core --- */
/* Core number of every vertex: the largest k such that the vertex lies in
 * the k-core, the largest subgraph in which every vertex has degree >= k.
 * The paper sets the k-truss against the k-core: a k-truss lies in the
 * (k-1)-core (Section 1), and Section 7 (Table 6) compares the k_max-truss
 * with the c_max-core; its edge bins reuse the core decomposition's
 * bin-sorted degree array (Section 3.2).  This entry point computes the core
 * decomposition on the same CSR.
 * core_out: n entries, indexed by vertex id (0 for a vertex without edges);
 * kmax_out (nullable, host or device int32[1]): the largest core number.
 * Errors: TRUSS_EINVAL, TRUSS_ENOMEM, TRUSS_ECUDA, TRUSS_ETIMEOUT. */
int truss_core(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
               int32_t *core_out, int32_t *kmax_out, void *cuda_stream);

/* ------------------------------------------------------------- batched --- */
/* Decompose G independent graphs in one pass.  Graph g has n[g] vertices and
 * rows row_off[g] .. row_off[g+1]-1 of src/dst, with ids local to the graph
 * (in [0, n[g])).  row_off has G+1 entries, row_off[0] = 0, non-decreasing.
 * n and row_off are HOST arrays.  Per-row outputs are as truss_decompose over
 * the concatenated rows; kmax_out (nullable, host or device int32[G]) receives
 * each graph's k_max.  The result for each graph equals truss_decompose on
 * that graph alone: the truss numbers of a disjoint union are those of its
 * components (Definition 2).  Errors as truss_decompose. */
int truss_decompose_batch(truss_ctx *ctx, int32_t G, const int64_t *n, const int64_t *row_off,
                          const int32_t *src, const int32_t *dst, int32_t *support_out,
                          int32_t *truss_out, int32_t *kmax_out, void *cuda_stream);

/* --------------------------------------------------------------- stats --- */
typedef struct truss_run_stats {
  int64_t n, rows, m;        /* vertices, input rows, distinct edges */
  int64_t triangles;         /* |triangles of G| = sum sup / 3 */
  int32_t kmax;              /* max truss number */
  int32_t levels;            /* levels k with a non-empty scan */
  int32_t subrounds;         /* peel sub-rounds over all levels */
  int32_t graphs;            /* 1, or G for a batch */
  /* stage times in ms (profile != 0), else 0 */
  float ms_build, ms_support, ms_lists, ms_peel, ms_scatter, ms_total;
  /* Algorithmic bytes of the three largest stages (count_bytes != 0, else
   * 0).  bytes_support = 4 * sum over oriented edges (u, v) of
   * (d+(u) + d+(v)) + 44 m + 24 T: the out-list entries a forward merge of
   * each edge's two out-lists reads, its offsets, endpoints and support
   * write, and three 8-byte read-modify-writes per triangle.  bytes_peel =
   * sum over edges e = (u, v) of 12 min(L_u, L_v) + 12 (min(L_u, L_v) - 1)
   * + 8, plus 16 T and 8 per edge present at each level that removes one:
   * reading the alive neighbours of e's endpoint with fewer of them (id,
   * edge id, state), looking each one up from the other endpoint, two
   * read-modify-writes per destroyed triangle and the level scans; L_x is 1
   * + the number of x's edges removed in a later sub-round than e (the
   * fewest that any one-at-a-time removal order with the same sub-rounds
   * leaves).
   * bytes_lists = the list passes this library runs (8-byte records read
   * twice, three list entries written, two cursor read-modify-writes per
   * triangle, and the per-edge offsets and cursors). */
  double bytes_support, bytes_lists, bytes_peel;
  /* kernels this call launched (own kernels plus the CUB sort/scan passes) */
  int64_t launches;
  /* truss_top only: edges of the last candidate subgraph, and how many
   * candidate subgraphs were decomposed */
  int64_t candidates;
  int32_t rounds;
  /* how the triangle lists were built: 0 = none (support only), 1 = by a
   * second walk of the graph, 2 = whole, from the records, 3 = from the
   * records with each edge's own part left in place */
  int32_t lists_layout;
  /* peel work (decompositions): triangle-list entries read, residual
   * decrements, alive-list entries scanned */
  int64_t peel_entries, peel_decrements, peel_scanned;
  /* count_bytes != 0: the same two stages priced by the per-unit figures of
   * the kernels this library runs (the support walk from each edge's middle
   * vertex; the peel's list entries, partner states, decrements and alive-
   * list entries), beside the formula figures above */
  double design_bytes_support, design_bytes_peel;
  /* count_bytes != 0: sum over edges of min(L_u, L_v) as above; the same
   * with L_x counting every edge of x not removed before e's sub-round; sum
   * over the levels that remove an edge of the edges present when they
   * start; list entries the peel read whose triangle had already lost an
   * edge, and those whose triangle lost it in an earlier level */
  int64_t peel_sum_min_alive, peel_sum_min_alive_start, peel_alive_levels;
  int64_t peel_dead_entries, peel_dead_earlier;
  /* device workspace the context holds after the call, and the most of it
   * the call used at once (bytes) */
  int64_t workspace_bytes, workspace_peak;
} truss_run_stats;

/* Statistics of the last successful call on this context. */
int truss_last_stats(truss_ctx *ctx, truss_run_stats *out);

/* ------------------------------------------------ allocation-free support --- */
/* Largest graph truss_support_noalloc accepts. */
#define TRUSS_NOALLOC_MAX_ROWS 65536
#define TRUSS_NOALLOC_MAX_N 65536

/* Per-row edge support, as truss_support, for a small graph and without
 * allocating any memory.  The paper has no counterpart to this entry point.
 * It is for callers that cannot allocate at the moment they need the result
 * and so cannot use a truss_ctx, whose workspace is allocated on demand: code
 * running inside an allocator or memory-pool callback, or a process whose
 * device memory is entirely handed out by another allocator.
 *
 * All working memory is one fixed array of about 5 MB in the library's device
 * image: every GPU that loads the library holds it until the process exits.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  Every call
 * on a device uses the same array and clears what it reads, so calls whose
 * work can overlap on the GPU (other streams, other host threads) race on it
 * and must be serialised by the caller.
 *
 * n must be <= TRUSS_NOALLOC_MAX_N and rows <= TRUSS_NOALLOC_MAX_ROWS;
 * anything larger is rejected with TRUSS_EINVAL before any device work.
 * src, dst and support_out must be reachable by a kernel on the current
 * device as given: memory of the current device, managed memory, or pinned
 * host memory mapped at the same address.  Memory of another GPU and pageable
 * host memory are refused with TRUSS_EINVAL before any launch.
 * support_out[r] is the support of row r's edge, -1 for a self-loop row.  The
 * work runs on the current device on cuda_stream and the call waits for it
 * (it reads back one status word).  Errors: TRUSS_EINVAL (sizes, null
 * pointers, pointers the current device cannot use as given, a vertex id
 * outside [0, n)),
 * TRUSS_ECUDA. */
int truss_support_noalloc(int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
                          int32_t *support_out, void *cuda_stream);

/* ------------------------------------------------------------- serving --- */
/* A request loop that decomposes many graphs of mixed sizes concurrently
 * (each request is the problem of the Section 2 problem definition, solved
 * as by truss_decompose).  Worker threads, each with its own context and CUDA
 * stream, take requests in arrival order; waiting requests of at most
 * `batch_rows` rows are grouped into one batched launch (as
 * truss_decompose_batch), larger ones run alone, and requests arriving while
 * others run are admitted as workers and memory free up (continuous
 * batching).  A request is admitted only while the projected device
 * footprint of all admitted, unfinished requests stays within
 * `hbm_budget_bytes` (truss_serve_footprint gives the projection).  Results
 * are exact and identical to a truss_decompose of the request alone. */
typedef struct truss_server truss_server;

typedef struct truss_serve_opts {
  int64_t hbm_budget_bytes; /* 0 = a third of the device memory free at start */
  int32_t max_inflight;     /* admitted, unfinished requests (0 = 256) */
  int32_t streams;          /* worker threads / streams (0 = 4) */
  int64_t batch_rows;       /* requests with <= this many rows are batched (0 = 65536) */
  int32_t max_batch;        /* requests per batched launch (0 = 512) */
  int32_t max_queue;        /* waiting requests before submit returns TRUSS_EBUSY (0 = 1<<20) */
  int32_t reserved[6];
} truss_serve_opts;

typedef struct truss_req_stats {
  int64_t m;          /* distinct edges */
  int64_t triangles;  /* triangles */
  int32_t kmax;       /* max truss number */
  int32_t batched;    /* requests in the launch that served this one */
  double queue_ms;    /* submit -> start of its launch */
  double run_ms;      /* start -> results ready in host memory */
  double total_ms;    /* submit -> results ready */
} truss_req_stats;

typedef struct truss_serve_stats {
  int64_t submitted, admitted, rejected, completed, failed;
  int64_t edges;            /* distinct edges of completed requests */
  double p50_ms, p99_ms;    /* submit -> ready latency of completed requests */
  double mean_ms, max_ms;
  double wall_s;            /* first submit -> last completion */
  double edges_per_s;       /* edges / wall_s */
  int64_t launches;         /* single + batched decompositions run */
  int64_t retried;          /* requests run again alone after exceeding their run's cap */
} truss_serve_stats;

/* Projected device footprint (bytes) used for admission of a request of
 * `rows` rows over `n` vertices: 96 bytes per row for the edge keys, CSR,
 * supports and peel queues, 16 per vertex, and 8-byte triangle-list entries
 * for an assumed 3 x 32 triangle incidences per row (the exact figure is
 * known only after the support pass).  A run's workspace is capped at twice
 * the projection of its requests; a request that needs more (a graph much
 * denser in triangles than assumed) fails that run with TRUSS_ENOMEM, is
 * queued again once at the head of the queue with the whole budget as its
 * footprint, and then runs alone with the whole budget as its cap: it
 * completes, or fails alone with TRUSS_ENOMEM, and no other request loses
 * memory to it. */
int64_t truss_serve_footprint(int64_t n, int64_t rows);

/* Start a server on ctx's device with ctx's options (ctx itself is not used
 * afterwards and may be destroyed).  opts may be NULL.  Errors: TRUSS_EINVAL,
 * TRUSS_ECUDA, TRUSS_ENOMEM. */
int truss_serve_start(truss_ctx *ctx, const truss_serve_opts *opts, truss_server **out);

/* Queue a request.  src/dst (host or device memory, `rows` rows over [0, n))
 * are read when the request runs, so they must stay valid and unchanged
 * until the request completes (truss_serve_poll/wait returns TRUSS_OK or an
 * error for it).  *ticket identifies the request.  Errors: TRUSS_EINVAL (bad
 * sizes), TRUSS_EBUSY (projected footprint above the whole budget, or queue
 * full), TRUSS_ESHUTDOWN (server stopping).  Thread-safe. */
int truss_serve_submit(truss_server *srv, int64_t n, int64_t rows, const int32_t *src,
                       const int32_t *dst, uint64_t *ticket);

/* If request `ticket` is done, copy its per-row support and truss numbers
 * into the caller's buffers (host memory, `rows` entries each, either may be
 * NULL), fill *st (nullable), release the request and return TRUSS_OK (or the
 * request's own error).  TRUSS_EAGAIN if it is still queued or running;
 * TRUSS_EINVAL for an unknown ticket.  Thread-safe. */
int truss_serve_poll(truss_server *srv, uint64_t ticket, int32_t *support_out,
                     int32_t *truss_out, truss_req_stats *st);

/* As truss_serve_poll, blocking up to timeout_ns (< 0: no limit) for the
 * request to finish; TRUSS_EAGAIN on timeout.  Thread-safe. */
int truss_serve_wait(truss_server *srv, uint64_t ticket, int64_t timeout_ns,
                     int32_t *support_out, int32_t *truss_out, truss_req_stats *st);

/* Stop accepting requests, finish the admitted and queued ones, join the
 * workers, fill *st (nullable) and free the server (results not yet polled
 * are discarded).  NULL is accepted. */
int truss_serve_stop(truss_server *srv, truss_serve_stats *st);

#ifdef __cplusplus
}
#endif
#endif /* TRUSS_H */
