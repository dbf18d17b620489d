/*
 * rcm.h -- C ABI of the GB300 (sm_103a) Reverse Cuthill-McKee ordering library.
 *
 * Method: Azad, Jacquelin, Buluc, Ng, "The Reverse Cuthill-McKee Algorithm in Distributed-Memory"
 * (arXiv:1610.08128). The ordering is the one of Sec. II-A / Sec. III with fixed tie rules:
 *   - D[v] (Alg. 3/4 input) = number of off-diagonal entries in row v; diagonal entries are ignored;
 *   - components (Sec. III-B: "invoking Alg. 3 for each connected component") are processed in
 *     start-rule order: each starts at the lowest-id vertex of minimum degree not yet numbered;
 *   - pseudo-peripheral root (Alg. 2, George-Liu): breadth-first sweeps, each from the lowest-id
 *     minimum-degree vertex of the previous sweep's last level, while the eccentricity grows
 *     strictly; the root is the last vertex swept;
 *   - labelled breadth-first traversal (Alg. 3): each newly reached vertex takes the smallest label
 *     among its neighbours in the current frontier (SpMSpV over (select2nd, min), Fig. 2); the new
 *     level is ordered by (parent label, degree, vertex id) (SortPerm, Sec. IV-B) and numbered
 *     consecutively; labels continue across components;
 *   - the sequence is reversed once at the end (Alg. 1 last line; Alg. 3 return).
 *
 * Conventions shared by every entry point
 *   Pattern   symmetric sparsity pattern of A in CSR with int32 indices: rowptr[n+1] (rowptr[0] = 0,
 *             non-decreasing), colidx[rowptr[n]] with 0 <= colidx < n. Values are not passed
 *             (Sec. III-A: only where the nonzeros are matters). Diagonal entries are allowed and
 *             ignored. Column order inside a row is free. Duplicate entries are not allowed.
 *             Symmetry is a precondition and is not checked (rcm_validate checks it).
 *   Output    perm[k] = original vertex placed at new position k (new -> old), so that
 *             (P A P^T)_{ij} = A_{perm[i], perm[j]}.
 *   Memory    Pointers documented as "device" must be device-accessible memory of the current
 *             CUDA device; "host" pointers are ordinary host memory. Inputs stay owned by the
 *             caller. The library allocates its own workspace (stream-ordered, from the device's
 *             default memory pool) and frees it in stream order.
 *   Streams   Device entry points are asynchronous and stream-ordered on `stream` (NULL = legacy
 *             default stream). Argument errors are returned synchronously. Errors the device
 *             detects (malformed CSR, a barrier that timed out) are latched per stream and returned
 *             by rcm_stream_status(). perm is undefined after any error.
 *   Limits    n < 2^31, nnz = rowptr[n] < 2^31.
 *   Threads   Entry points may be called from several host threads; calls on different streams
 *             run independently.
 */
#ifndef RCM_GB300_RCM_H
#define RCM_GB300_RCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t). NULL selects the legacy default stream. */
typedef struct CUstream_st *rcm_stream_t;

typedef enum {
    RCM_OK = 0,
    RCM_ERR_INVALID_ARG = 1,    /* bad argument (NULL pointer, negative size, bad options)          */
    RCM_ERR_BAD_CSR = 2,        /* malformed pattern: rowptr not monotone, colidx out of range     */
    RCM_ERR_OOM = 3,            /* a device or host allocation failed                              */
    RCM_ERR_TOO_LARGE = 4,      /* size beyond a documented limit or an admission budget           */
    RCM_ERR_CUDA = 5,           /* a CUDA runtime call failed                                      */
    RCM_ERR_TIMEOUT = 6,        /* a bounded device-side wait ran out (grid barrier, queue)        */
    RCM_ERR_NOT_READY = 7,      /* rcm_poll: the request has not finished                          */
    RCM_ERR_UNKNOWN_TICKET = 8  /* rcm_poll: no such request                                       */
} rcm_status;

/* Human-readable name of a status code (static storage). */
const char *rcm_status_string(rcm_status s);

/* Tuning knobs. None of them changes the result, except row_order: every other setting yields the
   same permutation. Zero-initialise and set what you need; 0 means "library default" in every field. */
typedef struct {
    int32_t narrow_threshold;  /* frontier size below which a single CTA runs the levels; -1 = never;
                                  0 = the CTA width, or 128 on a graph with a vertex of more than
                                  512 neighbours when fused_sweeps is 0 too (decided on the device) */
    int32_t grid_blocks;       /* CTAs of the persistent grid (<= co-resident limit); 0 = one per SM */
    int32_t block_threads;     /* threads per CTA of the persistent grid: 32 .. 1024 (power of 2); 0 = 512 */
    int32_t fused_sweeps;      /* 1 = label during sweeps 2.. (fused); 2 = label during every sweep,
                                  the first included (its labels are discarded); -1 = levels-only
                                  sweeps, then a separate labelled pass; 0 = 2 on a persistent grid
                                  of at least 64 CTAs (1 with async_sweeps, or on a graph with a
                                  vertex of more than 512 neighbours when narrow_threshold is 0
                                  too), 1 on smaller grids, clusters and the shared-memory CTA.
                                  Same result                                                      */
    int64_t spin_limit_ns;     /* bound of every device-side wait; 0 = 20 s                        */
    int64_t nnz;               /* rowptr[n] when the caller knows it: skips the synchronised 4-byte
                                  read (the device still checks it; a mismatch is RCM_ERR_BAD_CSR);
                                  0 = read it from the device                                       */
    int32_t debug_stall_barrier; /* test hook: CTA 0 never arrives at the first grid barrier, so
                                    the others' bounded waits run out and report RCM_ERR_TIMEOUT  */
    int32_t profile_phases;    /* 1 = CTA 0 accumulates %globaltimer time per phase into
                                  rcm_stats.phase_ns (small overhead)                              */
    int32_t cluster;           /* 1 = launch the persistent engine as ONE thread-block cluster of
                                  grid_blocks CTAs (2..16 as the device allows; 0 = the largest),
                                  co-scheduled by the hardware, instead of a cooperative grid;
                                  block_threads must be 0 or 512. RCM_ERR_INVALID_ARG if the
                                  device cannot launch that cluster                                */
    int32_t executor;          /* 0 = automatic: graphs of at most 4,608 vertices, with the grid options
                                  above at their defaults, run on one CTA that keeps the graph's
                                  traversal state in shared memory; others on the persistent grid.
                                  1 = always the persistent grid. 2 = always the shared-memory CTA
                                  (RCM_ERR_TOO_LARGE above 4,608 vertices); with 2, block_threads
                                  (32..512, 0 = automatic) sets that CTA's width                     */
    int32_t async_sweeps;      /* levels-only sweeps of the persistent grid (Alg. 2 needs only their
                                  eccentricity and last level): 1 = through an asynchronous work queue
                                  with no grid barrier per level (same result; 8n more workspace
                                  bytes; block_threads must be 0 or 512, else RCM_ERR_INVALID_ARG);
                                  0 or -1 = level by level (the default: faster on every graph
                                  measured on GB300). The shared-memory CTA ignores it.             */
    int32_t debug_async_slots; /* test hook: slots of the asynchronous sweeps' work queue (0 = 2n).
                                  A queue that runs full makes the sweep, and every later one of
                                  the call, run level by level instead: same result, slower.        */
    int32_t row_order;         /* 0 = the ordering above: each level by (parent label, degree, id).
                                  1 = the sort-free variant the paper's conclusion names (no sort
                                  beyond the parent order): a vertex's children are numbered in the
                                  order its row stores them. CHANGES THE RESULT (usually a somewhat
                                  larger bandwidth and profile); saves the degree gather of the
                                  row sort.                                                         */
    int32_t expand_mode;       /* expansion of the persistent grid's whole-grid levels; the result is
                                  the same in every mode:
                                  1 = top-down only: the frontier's atomicMin on its neighbours;
                                  2 = bottom-up on every whole-grid level: each vertex not yet reached
                                      scans its own row;
                                  3 = chosen per level: bottom-up once the frontier is a large part
                                      of the graph, top-down otherwise;
                                  0 = automatic: 3 for patterns averaging at least 8 stored entries
                                      per row (low-diameter graphs, whose frontiers grow wide), 1
                                      otherwise.
                                  Modes 2 and 3 need 512-thread CTAs and level-by-level sweeps
                                  (else RCM_ERR_INVALID_ARG; 0 then means 1). Narrow levels and the
                                  CTA executors are always top-down.                                */
    int32_t bottom_up_divisor; /* switch threshold of expand_mode 3 (and 0 when it picks 3): a level
                                  runs bottom-up when its frontier holds at least n / divisor vertices
                                  and at least a quarter of those not yet reached; 0 = 16          */
    int32_t l2_persist;        /* 1 = the persistent grid's launch marks its claim and stamp arrays
                                  (12 bytes per vertex) as persisting in L2, through an access-policy
                                  window, so that rows streaming through L2 do not evict them. This
                                  raises the context's persisting-L2 limit to the window's size (at
                                  most the device maximum); a small kernel after the traversal turns
                                  the window's lines back into normal ones, and the call then
                                  SYNCHRONISES `stream` and puts the previous limit back (a raised
                                  limit slows later kernels of the context). Cooperative grid only
                                  (ignored on clusters and the shared-memory CTA). 0 or -1 = off    */
    int32_t debug_order_bits;  /* test hook: width of the in-level order field of the labelled
                                  traversal's 64-bit claim keys; 0 = 64 minus the bits of n + 2 (the
                                  rest holds the level). The persistent grid runs at most
                                  floor((2^width - 1) / n) CTAs, so that any CTA's share of a level
                                  fits the field (the largest graphs run on fewer CTAs; n < 2^31
                                  always fits on at least one). With a forced width that clamp is
                                  skipped, and a level share that does not fit ends the call with
                                  RCM_ERR_TOO_LARGE. 1..(the width from n), else RCM_ERR_INVALID_ARG */
    int32_t mid_cluster;       /* middle tier of the persistent grid: the grid is launched in thread-
                                  block clusters of this many CTAs (2, 4, 8 or 16, as the device
                                  allows; the grid shrinks to the CTAs that fit in whole clusters),
                                  and labelled levels of narrow_threshold to mid_threshold vertices
                                  run on cluster 0 alone, exchanging through distributed shared
                                  memory instead of the grid's L2 atomics. Same result. 0 or -1 =
                                  off; cooperative grid only (not with cluster, RCM_ERR_INVALID_ARG
                                  otherwise)                                                        */
    int32_t mid_threshold;     /* with mid_cluster: levels below this many vertices (and at least
                                  narrow_threshold) run on the middle tier; 0 = 128 x mid_cluster   */
    int32_t components_first;  /* persistent grid: 1 = find every component (union-find, Sec. III-B's
                                  component loop) before the first sweep, instead of sweeping from
                                  the first start vertex and building the table only when that
                                  sweep does not reach every vertex. Faster on graphs known to be
                                  disconnected into components of similar size (that probe sweep is
                                  serial); one union-find pass more on a connected graph. Same
                                  result. 0 or -1 = off                                             */
} rcm_options;

/* Statistics of one ordering (filled by rcm_order_ex when requested). */
typedef struct {
    int64_t components;      /* connected components                                               */
    int64_t sweeps;          /* level structures computed by the pseudo-peripheral search (Alg. 2);
                                isolated vertices are numbered directly and count none (Alg. 2 on
                                one vertex would be two one-level sweeps)                        */
    int64_t traversals;      /* breadth-first traversals executed (a fused labelled sweep counts once) */
    int64_t levels;          /* levels expanded over all traversals                                */
    int64_t max_ecc;         /* largest eccentricity of a root                                     */
    int64_t isolated;        /* vertices of degree zero                                            */
    int64_t narrow_levels;   /* levels run by a single CTA                                         */
    int64_t grid_levels;     /* levels run by the whole persistent grid                            */
    double prep_ms;          /* device time of the preprocessing kernels (CUDA events)             */
    double traverse_ms;      /* device time of the persistent traversal kernel (CUDA events)       */
    int64_t phase_ns[8];     /* with profile_phases, CTA 0's time in: [0] levels-only expansion,
                                [1] labelled claims (phase A), [2] labelled ownership + numbering
                                (phase B), [3] label writes, [4] grid exchanges, [5] redistribution
                                exchanges, [6] waiting while CTA 0 runs narrow levels alone,
                                [7] start-vertex search, isolated vertices and claim resets       */
} rcm_stats;

/*
 * rcm_order -- RCM permutation of one symmetric pattern (Alg. 2 + Alg. 3, Sec. III).
 *   n        vertices (rows); 0 is allowed (nothing to do).
 *   rowptr   device, int32[n+1]; colidx device, int32[rowptr[n]].
 *   perm_out device, int32[n]; receives perm (new -> old). Also used as the level queue while running.
 * Reads rowptr[n] from the device once (a 4-byte copy synchronised on `stream`) to size the
 * workspace, then enqueues all work on `stream` and returns. Device-detected errors: see
 * rcm_stream_status.
 */
rcm_status rcm_order(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *perm_out,
                     rcm_stream_t stream);

/*
 * rcm_order_ex -- rcm_order with options and statistics.
 *   opts   host, may be NULL (defaults).
 *   stats  host, may be NULL. When given, the call records CUDA events around its kernels,
 *          synchronises `stream`, fills *stats, and its return value includes device-detected
 *          errors (as rcm_stream_status would).
 */
rcm_status rcm_order_ex(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *perm_out,
                        const rcm_options *opts, rcm_stats *stats, rcm_stream_t stream);

/*
 * rcm_order_host -- end-to-end ordering from host memory: copies the pattern to the device,
 * orders it on `stream`, copies perm back, and synchronises. Returns the final status
 * (device-detected errors included). On the persistent grid it uses the L2 window of
 * rcm_options.l2_persist (the call synchronises anyway; same result).
 *   rowptr host int32[n+1], colidx host int32[rowptr[n]], perm_out host int32[n].
 * Pinned (page-locked) host buffers give the fastest copies; pageable ones work.
 */
rcm_status rcm_order_host(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *perm_out,
                          rcm_stream_t stream);

/*
 * rcm_order_batch -- G independent patterns in one call (batched ordering; no counterpart in the
 * paper, which orders one matrix at a time). The patterns are stacked block-diagonally.
 *   G        number of graphs (>= 0).
 *   n_total  total vertices = goff[G] (host value; checked against the device copy).
 *   goff     device, int64[G+1]: graph g owns global rows goff[g] .. goff[g+1]-1.
 *   rowptr   device, int32[n_total+1] (global); colidx device, global column ids; every entry of
 *            graph g's rows must lie inside graph g's block.
 *   perm_out device, int32[n_total]; segment g receives graph g's perm in LOCAL ids 0..n_g-1, equal
 *            to rcm_order on that block alone.
 * Asynchronous on `stream`; device-detected errors as for rcm_order.
 */
rcm_status rcm_order_batch(int32_t G, int64_t n_total, const int64_t *goff, const int32_t *rowptr,
                           const int32_t *colidx, int32_t *perm_out, rcm_stream_t stream);

/* Tuning of the batched path (apart from row_order, every value gives the same permutations;
   only speed differs). */
typedef struct {
    int32_t block_threads;   /* threads per CTA of the batched executor: 128, 256 or 512; 0 = 256   */
    int32_t row_sort_split;  /* rows with at most this many stored entries are sorted by one thread,
                                longer rows by a whole CTA: 4..32; 0 = 32                          */
    int32_t row_order;       /* as rcm_options.row_order: 1 = sort-free variant (changes the result) */
    int32_t reserved[5];
} rcm_batch_options;

/* rcm_order_batch with tuning options (opts may be NULL = defaults). RCM_ERR_INVALID_ARG for
   values outside the ranges above. */
rcm_status rcm_order_batch_ex(int32_t G, int64_t n_total, const int64_t *goff, const int32_t *rowptr,
                              const int32_t *colidx, int32_t *perm_out, const rcm_batch_options *opts,
                              rcm_stream_t stream);

/*
 * Batched replay plan: the launches of rcm_order_batch_ex for fixed device buffers, captured once
 * into a CUDA graph with a workspace of their own, then replayed with one launch. Each replay
 * orders whatever pattern the buffers hold at that time; it must keep G, n_total and
 * rowptr[n_total] == nnz (a different stored-entry count is reported as RCM_ERR_BAD_CSR).
 *   create   goff, rowptr, colidx, perm_out: device buffers as for rcm_order_batch, kept by the
 *            caller for the plan's lifetime. Allocates the workspace; synchronous.
 *   launch   enqueues one replay on `stream` (asynchronous).
 *   status   synchronises `stream` and returns the device-detected status of the last replay.
 *   destroy  frees the graph and the workspace (after synchronising the device).
 */
typedef struct rcm_batch_plan rcm_batch_plan;
rcm_status rcm_batch_plan_create(int32_t G, int64_t n_total, int64_t nnz, const int64_t *goff,
                                 const int32_t *rowptr, const int32_t *colidx, int32_t *perm_out,
                                 const rcm_batch_options *opts, rcm_batch_plan **out);
rcm_status rcm_batch_plan_launch(rcm_batch_plan *plan, rcm_stream_t stream);
rcm_status rcm_batch_plan_status(rcm_batch_plan *plan, rcm_stream_t stream);
rcm_status rcm_batch_plan_destroy(rcm_batch_plan *plan);

/*
 * rcm_order_noalloc -- rcm_order for callers that must not allocate device memory (the paper has
 * no counterpart). Typical callers: an application whose memory framework has already reserved
 * the device memory for its own caching allocator, or a solver loop with a memory budget fixed
 * at start-up, where an allocation could fail or stall the device. Same arguments and result as
 * rcm_order; the workspace is a fixed device array inside this library (about 8 MiB, kept by
 * every GPU that loads the library until the process exits).
 *   Limits   n <= 65,536 vertices and rowptr[n] <= 1,048,576 stored entries; larger patterns
 *            return RCM_ERR_TOO_LARGE before any work is enqueued.
 *   Set-up   the first call on a device does a one-time set-up with that device current: it looks
 *            up the array's device address and loads every kernel the call can launch (CUDA
 *            loads device code lazily, and loading takes device memory). So that first call may
 *            allocate; later calls allocate nothing. Make the first call on each device at
 *            start-up, before the memory budget is handed out, and before any stream capture.
 *   Sharing  every call uses the same array, which keeps the previous call's contents (the call
 *            clears what must start at zero). Calls whose work overlaps on the GPU (different
 *            streams, or host threads) race on it and must be serialised by the caller.
 *   Sync     synchronises `stream`; the return value includes device-detected errors.
 */
rcm_status rcm_order_noalloc(int32_t n, const int32_t *rowptr, const int32_t *colidx, int32_t *perm_out,
                             rcm_stream_t stream);

/*
 * Serving (continuous batching; no counterpart in the paper, which orders one matrix at a time).
 * A server owns a device arena of hbm_budget_bytes (allocated once at creation) and up to
 * max_inflight concurrent requests. Each request needs one arena region: its CSR when given in
 * host memory, its output when the caller's buffer is in host memory, and the ordering's
 * workspace (rcm_request_bytes gives the exact size). Requests are admitted in
 * arrival order as regions and slots free up; each admitted request runs on its own stream (its
 * validation and sorted-row kernels, then one CTA of the batched executor), so requests that
 * arrive while others are on the GPU run alongside them.
 * Results are bit-identical to rcm_order on the same pattern.
 * Concurrency: CUDA maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8 by default),
 * and streams sharing a queue wait behind each other. Processes that serve many requests should
 * set it to 32 in the environment before their CUDA context is created: on GB300, with 4,000
 * requests at 2,000/s, that raised throughput by 4% and cut p50 / p99 latency by a third / a
 * quarter. The library cannot set it itself, because the context exists before it runs.
 */
typedef struct rcm_server rcm_server;

typedef struct {
    int64_t submitted, completed, failed, cancelled;
    int64_t waiting;            /* submitted, not admitted yet                                      */
    int64_t running;            /* admitted, not finished                                           */
    int64_t max_running;        /* largest number of requests on the GPU at once                    */
    int64_t arena_bytes;        /* budget                                                           */
    int64_t arena_peak_bytes;   /* largest arena use                                                */
    double latency_p50_s;       /* completion minus submission time, over completed requests       */
    double latency_p99_s;
    double latency_max_s;
} rcm_server_stats;

/*
 * Arena bytes one request of n vertices and nnz stored entries takes: the staged CSR when
 * host_csr != 0 (rowptr/colidx in host memory), the staged result when host_out != 0, a status
 * block, and the ordering's workspace (about 124 bytes per vertex, 4 per stored entry and 34 KB).
 * A budget of at least this many bytes admits the request. Pure host arithmetic.
 */
size_t rcm_request_bytes(int32_t n, int64_t nnz, int32_t host_csr, int32_t host_out);

/* Creates a server on the current device. max_inflight in [1, 4096]. */
rcm_status rcm_server_create(size_t hbm_budget_bytes, int32_t max_inflight, rcm_server **out);

/* Execution policy of a server (rcm_server_create uses the defaults, all fields 0). */
typedef struct {
    int64_t cluster_min_vertices; /* requests of at least this many vertices run the persistent
                                     engine of rcm_order launched as one thread-block cluster;
                                     smaller ones run on one CTA. 0 = 524,288; -1 = never         */
    int32_t cluster_blocks;       /* CTAs of that cluster, 2..16 as the device allows; 0 = 4       */
    int32_t debug_fail_after;     /* test hook: once this many requests have completed, the server
                                     acts as if a running request's stream reported a CUDA error
                                     (its failure path without a device fault); 0 = off           */
    int32_t reserved[4];
} rcm_server_options;

/* rcm_server_create with an execution policy (opts may be NULL). RCM_ERR_INVALID_ARG for values
   outside the ranges above. */
rcm_status rcm_server_create_ex(size_t hbm_budget_bytes, int32_t max_inflight, const rcm_server_options *opts,
                                rcm_server **out);

/*
 * Submits one ordering request and returns its ticket. rowptr/colidx may be host or device
 * memory, perm_out host or device memory (pinned host memory gives the fastest copies; results
 * bound for pageable memory are copied by a helper thread of the server once the ordering is
 * done); all must stay valid and unmodified until rcm_poll/rcm_wait reports the request
 * finished. A request that can never fit the budget returns RCM_ERR_TOO_LARGE (no ticket).
 */
rcm_status rcm_submit(rcm_server *srv, int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                      int32_t *perm_out, uint64_t *ticket);

/* RCM_ERR_NOT_READY while the request runs or waits; otherwise its final status, after which
   the ticket is forgotten (a later poll returns RCM_ERR_UNKNOWN_TICKET). */
rcm_status rcm_poll(rcm_server *srv, uint64_t ticket);

/* Blocks until the request finishes; returns its final status and forgets the ticket. */
rcm_status rcm_wait(rcm_server *srv, uint64_t ticket);

/* Withdraws a request that has not been admitted yet (RCM_OK); a running request cannot be
   withdrawn (RCM_ERR_NOT_READY). */
rcm_status rcm_cancel(rcm_server *srv, uint64_t ticket);

/* Counters and latency percentiles of the requests seen so far. */
rcm_status rcm_server_info(rcm_server *srv, rcm_server_stats *out);

/* Drops requests not admitted yet, waits for running ones, and frees the server. */
rcm_status rcm_server_destroy(rcm_server *srv);

/* Synchronises `stream` and returns (and clears) the error latched by earlier calls on it.
   Each stream that rcm_order / rcm_order_ex / rcm_order_batch(_ex) ran on holds one of 4,096 latch
   words of this process until this call reads it; the word is then free for any stream. An
   ordering call on a further stream while all 4,096 are held returns RCM_ERR_TOO_LARGE before any
   work (read the status of streams you are done with). */
rcm_status rcm_stream_status(rcm_stream_t stream);

/* Workspace bytes rcm_order allocates for a pattern of n vertices and nnz stored entries. */
size_t rcm_workspace_bytes(int32_t n, int64_t nnz);

/* What rcm_validate found. Counts are of stored entries unless named otherwise. */
typedef struct {
    int64_t bad_rows;       /* rows v with rowptr[v] < 0, rowptr[v+1] < rowptr[v] or rowptr[v+1] > rowptr[n];
                               rowptr[0] != 0 counts as one more                                      */
    int64_t bad_columns;    /* entries with a column outside [0, n)                                   */
    int64_t duplicates;     /* entries equal to another entry of the same row (each extra copy once);
                               -1 = not checked (rows or columns malformed)                           */
    int64_t asymmetric;     /* off-diagonal entries (v, w) whose row w holds no v; -1 = not checked   */
    int64_t diagonal;       /* diagonal entries (allowed; the ordering ignores them)                  */
    int64_t max_row;        /* stored entries of the longest well-formed row                          */
    int64_t first_bad_row;  /* smallest row holding a fault counted above, -1 if none                 */
    int64_t reserved;
} rcm_validate_report;

/*
 * rcm_validate -- checks a pattern against the contract every ordering call assumes (file header):
 * CSR structure, columns in range, no duplicate entries, and symmetry (the graph of A is
 * undirected, Sec. II-A; the ordering calls take symmetry as a precondition and do not check it).
 * rowptr, colidx: device, as for rcm_order. report: host, filled on RCM_OK and on RCM_ERR_BAD_CSR.
 * Returns RCM_OK when the pattern meets the contract, RCM_ERR_BAD_CSR when it does not (report
 * says why), RCM_ERR_INVALID_ARG for n < 0 or null pointers. Synchronous: waits for `stream`.
 * A debugging aid, off the ordering path: it sorts a copy of every row (4 bytes per entry of
 * workspace) and binary-searches each entry's partner row.
 */
rcm_status rcm_validate(int32_t n, const int32_t *rowptr, const int32_t *colidx, rcm_validate_report *report,
                        rcm_stream_t stream);

/*
 * rcm_bandwidth_profile -- bandwidth and profile of P A P^T (Sec. II-A): with pos = perm^-1 and
 * f_i = min(i, min{pos[w] : w adjacent to perm[i]}), beta_i = i - f_i, bandwidth = max beta_i,
 * profile = |Env| = sum beta_i. All pointers device except bw/profile (host). Synchronous.
 * Returns RCM_ERR_INVALID_ARG if perm is not a permutation of 0..n-1.
 */
rcm_status rcm_bandwidth_profile(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                                 const int32_t *perm, int64_t *bw, int64_t *profile, rcm_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* RCM_GB300_RCM_H */
