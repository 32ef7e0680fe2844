/*
 * mpld.h -- C ABI of libmpld: exact-cover (EC) multiple patterning layout
 * decomposition on one GB300 (sm_103a).
 *
 * Paper: G. Chen, H. Yang, B. Yu, "GPU-Accelerated Matrix Cover Algorithm for
 * Multiple Patterning Layout Decomposition".
 *
 * Problem (Sec. 2.1, Eq. 1a-1d): a layout graph with conflict edges CE and
 * stitch edges SE and k masks in; a mask x_i in {0..k-1} per segment out,
 * minimising  cost_conflict * #{(i,j) in CE : x_i == x_j}
 *           + cost_stitch   * #{(i,j) in SE : x_i != x_j}.
 * The paper's weights are 1 and alpha = 0.1 (Sec. 2.1); the defaults 10 and
 * 1 are the same objective in integers.  (Eq. 1d prints the mask domain as
 * {0..k}; k masks are meant.)
 *
 * Flow (Sec. 2.2): simplify the graph, split it into sub-graphs, solve each
 * with the matrix-cover search (Sec. 2.3, Algorithm 1), recover the removed
 * nodes, count conflicts and stitches.
 *
 * Conventions for every call:
 *   - all pointers in structs and arguments are HOST pointers unless named
 *     otherwise; the library never keeps a caller pointer after a call
 *     returns;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); all device work of a call is ordered on it;
 *   - return value: MPLD_OK (0), MPLD_BUDGET (1: at least one search
 *     instance hit its node budget or time limit and returned its best
 *     assignment so far), or a negative MPLD_E_* error code; on an error no
 *     output is written and the handle is left as it was.
 *   - calls on different handles may run concurrently from different host
 *     threads; calls on one handle must not.
 */
#ifndef MPLD_H
#define MPLD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPLD_OK 0
#define MPLD_BUDGET 1
#define MPLD_TIMEOUT 2         /* per-instance status: time limit reached */
#define MPLD_E_INVALID (-1)    /* malformed input: id out of range, self-loop, k not in [2,8], ... */
#define MPLD_E_OOM (-2)        /* host or device allocation failed */
#define MPLD_E_CUDA (-3)       /* a CUDA runtime call failed */
#define MPLD_E_TIMEOUT (-4)    /* a device-side wait ran out (status word set by the kernel) */
#define MPLD_E_TOO_LARGE (-5)  /* a search instance exceeds the supported size */
#define MPLD_E_STATE (-6)      /* call out of order (e.g. fetch before any solve) */

/* mpld_params.flags */
#define MPLD_NO_SIMPLIFY 1u      /* skip the simplification step (Sec. 2.2) */
#define MPLD_SINGLE_INSTANCE 2u  /* search all remaining segments as ONE instance (no sub-graph split) */
#define MPLD_COLUMN_BFS 8u       /* search with the paper's column rule (Algorithm 1): the lowest-index
                                    uncovered column with a single row left, else the uncovered column
                                    first in breadth-first order of the sub-graph (conflict and stitch
                                    edges, roots and neighbours in ascending id).  Default: the column
                                    with the fewest rows, lowest index on ties.  Read by the search
                                    calls and by mpld_server_create; not available to
                                    mpld_search_instance_noalloc. */
#define MPLD_BICONNECTED 16u     /* search the biconnected blocks of each sub-graph instead of the
                                    whole sub-graph (conflict and stitch edges together), then join
                                    them at their cut segments: every edge lies in exactly one
                                    block and renaming masks inside a block keeps its cost, so the
                                    blocks' optima join into the sub-graph's optimum.  Blocks are
                                    taken breadth-first over the block-cut tree (from the
                                    lexicographically first block holding the sub-graph's lowest
                                    segment; a block's segments in ascending id; at each, the
                                    untaken blocks in lexicographic order of their ascending
                                    segment lists), and a block's masks are renamed by the one
                                    transposition that keeps its attach segment's mask.  With a
                                    node budget each block has its own.  Read by
                                    mpld_build_matrix; not with MPLD_SINGLE_INSTANCE
                                    (MPLD_E_INVALID).  Instances are then blocks: a cut segment
                                    belongs to several, and mpld_component_results reports the
                                    first. */
#define MPLD_CLIQUE_BOUND 32u    /* second bound mode: at build, each instance's (k+1)-cliques of
                                    conflict edges are listed in lexicographic order of their
                                    ascending member lists and taken greedily when they share no
                                    edge with one taken before; the search then prunes when
                                    path cost + cost_conflict * (uncovered columns with no active
                                    row + taken cliques with no member assigned) reaches the
                                    incumbent.  Admissible: an untouched clique must repeat a mask
                                    on an edge between unassigned segments.  The first minimum-cost
                                    leaf is unchanged; fewer nodes.  Read by mpld_build_matrix
                                    (and mpld_server_submit); MPLD_E_TOO_LARGE above 65,535
                                    cliques in one instance. */
#define MPLD_PARALLEL_EXACT 64u  /* exact search (node_budget must be 0, else MPLD_E_INVALID) with
                                    many warps splitting each instance of at least 16 segments
                                    that fits the register-resident form (at most 128 segments,
                                    64 at k = 8): the tree is cut at the first depth D with
                                    k^D >= 16 * warps, and the warps take its k^D subtrees in
                                    depth-first order from a shared counter, sharing the
                                    incumbent as (cost, subtree).  An instance searched alone
                                    (mpld_solve, a one-instance problem) is split by every warp
                                    of the grid; in a batched call the 16 largest such instances
                                    are split by the whole grid one after another, then the
                                    others by the warps of one CTA each.  Cost and masks are
                                    those of the one-warp search (the first minimum-cost leaf);
                                    node counts depend on timing; the clique bound is not
                                    applied inside split instances.  Read by the search calls
                                    except mpld_search_instance_noalloc (MPLD_E_INVALID) and the
                                    server (ignored). */
#define MPLD_SPLIT_BUDGET 128u   /* budgeted split search: the node budget B of each instance is
                                    spent by many independent searches instead of one (the task
                                    parallelism of Sec. 1 / Sec. 2.3 inside one sub-graph).  The
                                    instance's tree is cut at depth D, the first depth with
                                    k^D >= 64 (at most n and 8), into S = k^D subtrees numbered in
                                    depth-first order (subtree s takes, at level i < D, the row
                                    at place digit i of s in base k of the ascending (added cost,
                                    mask) order).  Every search gets b = ceil(B / (S + 1)) nodes.
                                    A first search of the whole tree runs with budget b; if it
                                    ends on its own its answer stands.  Otherwise its incumbent
                                    (cost c1 at subtree s1) seeds S subtree searches, each with
                                    budget b, counting the nodes on its forced path, taking a
                                    leaf only if it beats (c1, s1) in the order (cost, subtree);
                                    these run on every warp of the GPU at once.  The result is
                                    the smallest (cost, subtree) found, its masks, the nodes of
                                    all searches, and status MPLD_BUDGET if a subtree search
                                    stopped on its budget (else the answer is exact).  The result
                                    does not depend on timing or launch shape.  An instance of
                                    more than 4096 segments is not split: one search with the
                                    whole budget.  node_budget 0: the exhaustive search.  Read
                                    by the search calls and by mpld_server_create; not with
                                    MPLD_PARALLEL_EXACT, nor on problems built (or layouts
                                    submitted) with MPLD_CLIQUE_BOUND (MPLD_E_INVALID); not
                                    available to mpld_search_instance_noalloc
                                    (MPLD_E_INVALID). */
#define MPLD_DENSITY_BALANCE 256u  /* balance mask usage over the layout (a reading of the density
                                    balance the paper names only in passing): renaming the masks
                                    of one component keeps its cost, so after the search each
                                    instance in instance order takes the permutation that pairs
                                    its masks by decreasing segment count (lower mask first on
                                    ties) with the layout's masks so far by increasing count
                                    (lower first), and the recovery gives a removed unit the least
                                    used of the masks its coloured conflict neighbours leave free
                                    (lowest on ties).  Cost, conflicts and stitches are those
                                    without the flag.  Read by mpld_build_matrix (and
                                    mpld_server_submit); not with MPLD_BICONNECTED
                                    (MPLD_E_INVALID). */
#define MPLD_HOST_ONLY 4u        /* build the host side only (no device memory): for inspection with
                                    mpld_problem_info / mpld_component_results / mpld_export_matrix;
                                    the solve calls then return MPLD_E_STATE */

/* Largest search instance (segments of one sub-graph). */
#define MPLD_MAX_INSTANCE_SEGMENTS 65535

/*
 * Layout graph (Sec. 2.1: G = {V, E}, E = CE u SE).  Caller-owned, read only
 * during mpld_build_matrix.
 *   n_seg        segments (nodes), ids 0..n_seg-1;
 *   k            masks, 2 <= k <= 8;
 *   conf_u/v     n_conf conflict edges; duplicates and (v,u) repeats are
 *                merged; self-loops and ids outside [0,n_seg) are errors;
 *   st_u/v       n_stitch stitch edges, same rules;
 *   polygon_of   segment -> polygon id in [0,n_seg), or NULL (each segment
 *                its own polygon).  A polygon together with everything joined
 *                to it by stitch edges is one unit of simplification;
 *   cost_conflict, cost_stitch   integer weights in [0, 10000].
 */
typedef struct {
  int32_t n_seg, k;
  int32_t n_conf;
  const int32_t *conf_u, *conf_v;
  int32_t n_stitch;
  const int32_t *st_u, *st_v;
  const int32_t *polygon_of;
  int32_t cost_conflict, cost_stitch;
} mpld_graph;

/*
 * Search parameters.
 *   node_budget    per search instance; 0 = unlimited.  A node is one step
 *                  of Algorithm 1 (one recursive call); once an instance has
 *                  an incumbent and has counted node_budget nodes, its
 *                  search stops with status MPLD_BUDGET;
 *   time_limit_ms  per search instance, measured on the device from the
 *                  start of its search; 0 = 60000.  An instance still
 *                  searching when it runs out stops with status MPLD_TIMEOUT
 *                  and keeps its incumbent (the layout status is then
 *                  MPLD_BUDGET);
 *   flags          MPLD_NO_SIMPLIFY | MPLD_SINGLE_INSTANCE | MPLD_HOST_ONLY |
 *                  MPLD_BICONNECTED | MPLD_CLIQUE_BOUND | MPLD_DENSITY_BALANCE (used by
 *                  mpld_build_matrix); MPLD_COLUMN_BFS | MPLD_PARALLEL_EXACT |
 *                  MPLD_SPLIT_BUDGET (used by the search calls);
 *   warps_per_cta, slot_bytes   launch shape of the batched kernel; 0 = the
 *                  tuned or default shape (see mpld_autotune); at most 16
 *                  warps (larger values are clamped);
 *   cta_segments   instances of at least this many segments are searched by
 *                  all threads of a CTA together (at least 8 warps) instead
 *                  of one warp; 0 = 4096, negative = never.  Same search and
 *                  results; large instances go faster.
 */
typedef struct {
  int64_t node_budget;
  int64_t time_limit_ms;
  uint32_t flags;
  int32_t warps_per_cta;
  int32_t slot_bytes;
  int32_t cta_segments;
} mpld_params;

/* Layout-level result (Sec. 3: st# and cn# are n_stitches and n_conflicts). */
typedef struct {
  int32_t status;               /* MPLD_OK / MPLD_BUDGET (worst over instances) */
  int32_t n_components;         /* search instances */
  int64_t n_conflicts, n_stitches;
  int64_t cost;                 /* cost_conflict*n_conflicts + cost_stitch*n_stitches */
  int64_t nodes;                /* search nodes over all instances */
  int64_t n_removed_segments;   /* removed by simplification, recovered after the search */
  int32_t max_component;        /* segments in the largest instance */
  int32_t n_budget_components;  /* instances that stopped on budget or time */
  int64_t work;                 /* algorithmic integer operations of the search: 2 per
                                   uncovered column per node, k per neighbour of each
                                   expanded segment, 5 per column of each covered row */
} mpld_result;

typedef struct mpld_problem mpld_problem;

/*
 * Build the EC matrices of a layout (Sec. 2.2 simplification and sub-graph
 * split; Sec. 2.3 "homogeneous graph to binary matrix"; Algorithm 1 steps
 * that split the DG into sub-graphs) and upload them to the device.
 * Rows of instance i are (segment v, mask c); primary column P_v; secondary
 * column S_{e,c} per conflict edge e and mask c.  The matrices and search
 * stacks live in one device arena owned by the returned handle.
 *   graph   caller-owned, read during the call only;
 *   params  only `flags` is read; NULL = defaults;
 *   stream  the upload is enqueued on it; the call returns once the host
 *           staging buffer may be reused (it synchronises the stream);
 *   out     receives the handle; free it with mpld_free.
 * Errors: MPLD_E_INVALID, MPLD_E_TOO_LARGE (a sub-graph with more than
 * MPLD_MAX_INSTANCE_SEGMENTS segments), MPLD_E_OOM, MPLD_E_CUDA.
 */
int mpld_build_matrix(const mpld_graph *graph, const mpld_params *params, void *stream,
                      mpld_problem **out);

/*
 * Plain path: one kernel launch per search instance (Sec. 3: "one block for
 * each sub-graph"), one after the other on `stream`, then the copy back,
 * recovery of the removed segments (Sec. 2.2) and the counts.
 *   mask_out  host, n_seg int8 masks (may be NULL);
 *   result    host (may be NULL).
 * Synchronous with respect to the host outputs.
 */
int mpld_solve(mpld_problem *p, const mpld_params *params, int8_t *mask_out, mpld_result *result,
               void *stream);

/*
 * Batched path: the instances of all `n` problems in ONE persistent launch
 * fed by a device work queue ordered largest first (Sec. 2.3 task
 * parallelism over sub-graphs), replayed from a captured CUDA graph; then
 * the copy back, recovery and counts per problem.
 *   ps         n problem handles (distinct);
 *   masks_out  n host pointers (each n_seg of its problem) or NULL / NULL
 *              entries to skip;
 *   results    n host results or NULL.
 * Synchronous with respect to the host outputs.
 */
int mpld_solve_batch(mpld_problem *const *ps, int32_t n, const mpld_params *params,
                     int8_t *const *masks_out, mpld_result *results, void *stream);

/*
 * Device-only halves of mpld_solve_batch, for callers that keep the work on
 * the device: mpld_search_batch_async enqueues the batched search on
 * `stream` and returns without waiting; the per-instance results stay in
 * device memory until mpld_fetch copies them back (it synchronises
 * `stream`), recovers the removed segments and counts.
 */
int mpld_search_batch_async(mpld_problem *const *ps, int32_t n, const mpld_params *params,
                            void *stream);
int mpld_fetch(mpld_problem *p, int8_t *mask_out, mpld_result *result, void *stream);

/* Device-only half of mpld_solve (one launch per instance, enqueued only). */
int mpld_search_plain_async(mpld_problem *p, const mpld_params *params, void *stream);

/* Release every host and device resource of the handle.  NULL is a no-op.
 * The caller must make sure no work of the handle is still in flight. */
void mpld_free(mpld_problem *p);

/* Static string for a status or error code. */
const char *mpld_status_string(int code);

/* Sizes of a built problem. */
typedef struct {
  int32_t n_seg, k, n_components, max_component;
  int64_t n_removed_segments;
  int64_t arena_bytes;          /* device bytes of EC matrices and graph data */
  int64_t state_bytes;          /* device bytes reserved for search stacks */
  int64_t instance_segments;    /* segments inside search instances */
} mpld_info;
int mpld_problem_info(const mpld_problem *p, mpld_info *info);

/*
 * Per-instance results of the last fetch (instance order = ascending lowest
 * segment id).  Each array holds n_components entries; any may be NULL.
 * comp_of (n_seg entries): instance of each segment, -1 if removed.
 */
int mpld_component_results(const mpld_problem *p, int64_t *nodes, int64_t *cost, int32_t *status,
                           int32_t *comp_of);

/*
 * EC matrix of instance `comp` as a dense 0/1 array, row-major
 * [n*k][1 + n + k*|E_c|]: column 0 unused, column 1+v = P_v, column
 * 1+n+e*k+c = S_{e,c} with conflict edges e sorted by (min,max) local id.
 * Rebuilt on the host from the handle's packed form, for inspection;
 * `dense` must hold n*k*(1+n+k*|E_c|) bytes; query the sizes with
 * dims = {n, k, n_conf_edges} first by passing dense = NULL.
 */
int mpld_export_matrix(const mpld_problem *p, int32_t comp, uint8_t *dense, int32_t *dims);

/*
 * Launch shape of the batched kernel.  mpld_autotune times the candidate
 * shapes on the given problems (results are the same for every shape) and
 * stores the fastest in a process-wide cache keyed by (k, size histogram),
 * which mpld_solve_batch uses when params leave the shape at 0.
 */
typedef struct {
  int32_t warps_per_cta;
  int32_t slot_bytes;
  int32_t ctas_per_sm;
  int32_t n_instances_spilled;  /* instances whose state did not fit the slot */
  float ms;                     /* measured time of the chosen shape */
} mpld_tune;
int mpld_autotune(mpld_problem *const *ps, int32_t n, const mpld_params *params, void *stream,
                  mpld_tune *best);

/*
 * One layout over several GPUs (one process per GPU).  The layout's search
 * instances are independent (Sec. 1, task parallelism over sub-graphs), so
 * every rank builds the same problem, searches its share of the instances,
 * and the ranks' per-instance results are gathered (by the caller, e.g. with
 * an all-gather) before the recovery of the removed segments and the counts.
 *
 * mpld_shard_instances: the share of each instance, longest processing time
 *   first: instances by decreasing estimated work (segments + adjacency
 *   entries, ties to the lower index), each to the rank with the least work
 *   so far (ties to the lower rank).  owner_out: n_components entries in
 *   [0, world).  Deterministic: every rank computes the same shares.
 * mpld_instance_sizes: segments of each instance (n_components entries); the
 *   masks of instance c start at the sum of the sizes of the instances
 *   before it in the arrays below.
 * mpld_search_subset_async: the batched search (mpld_search_batch_async's
 *   kernel and launch shape) of the listed distinct instances only; the
 *   others are not searched.  MPLD_PARALLEL_EXACT is refused (MPLD_E_INVALID).
 * mpld_fetch_instances: the last search's per-instance results, copied back
 *   (synchronises `stream`): nodes, cost, status (-1 for an instance that
 *   was not searched) and the masks of every instance (instance_segments
 *   bytes, instance after instance, each in ascending segment id); any
 *   pointer may be NULL.  MPLD_E_STATE before a search.
 * mpld_finish_from: scatter per-instance results given by the caller (the
 *   arrays of mpld_fetch_instances, merged over the ranks), recover the
 *   removed segments and count, as mpld_fetch does; every status must be
 *   MPLD_OK, MPLD_BUDGET or MPLD_TIMEOUT (else MPLD_E_STATE).  Works on
 *   MPLD_HOST_ONLY handles.
 */
int mpld_shard_instances(const mpld_problem *p, int32_t world, int32_t *owner_out);
int mpld_instance_sizes(const mpld_problem *p, int32_t *sizes);
int mpld_search_subset_async(mpld_problem *p, const mpld_params *params, const int32_t *inst,
                             int32_t n, void *stream);
int mpld_fetch_instances(mpld_problem *p, int64_t *nodes, int64_t *cost, int32_t *status,
                         int8_t *inst_masks, void *stream);
int mpld_finish_from(mpld_problem *p, const int64_t *nodes, const int64_t *cost,
                     const int32_t *status, const int8_t *inst_masks, int8_t *mask_out,
                     mpld_result *result);

/*
 * Serving: continuous batching of whole layouts on one GPU.
 *
 * The paper runs the sub-graphs of one layout in parallel (Sec. 1, "task
 * parallelism"; Sec. 3, one block per sub-graph).  A server extends that
 * to a stream of layouts:
 *   - mpld_server_submit copies the layout and queues it; host worker
 *     threads simplify, split and pack it (as mpld_build_matrix);
 *   - mpld_server_poll admits built layouts in submission order (a layout
 *     still being built holds back none behind it; one waiting for device
 *     memory holds back the layouts after it) while their device bytes (packed matrices, search state, descriptors, results)
 *     fit the server's arena and fewer than max_in_flight layouts are on
 *     the device; each admitted layout is uploaded and searched by one
 *     persistent launch of the batched kernel on one of the server's
 *     streams, so layouts admitted at different times run side by side;
 *   - finished layouts (their stream passed the copy-back) give their
 *     device bytes back, which admits waiting layouts, and worker threads
 *     recover the removed segments and count (Sec. 2.2);
 *   - mpld_server_result hands out a finished layout's masks and counts and
 *     forgets the ticket.
 * Each layout's result equals mpld_solve_batch's on that layout alone with
 * the same search parameters: instances are searched independently.
 * submit / poll / result / stats may be called from one thread at a time.
 */
typedef struct mpld_server mpld_server;

typedef struct {
  int64_t arena_bytes;        /* device bytes for admitted layouts; 0 = 1 GiB */
  int64_t result_pool_bytes;  /* pinned host bytes for results of admitted layouts; 0 = 256 MiB */
  int32_t max_in_flight;      /* layouts on the device at once; 0 = 64 */
  int32_t streams;            /* CUDA streams the launches rotate over; 0 = 8 */
  int32_t warps_per_cta;      /* batched kernel shape; 0 = 4 */
  int32_t worker_threads;     /* host build / recovery threads; 0 = three quarters of the hardware threads */
} mpld_server_config;

typedef struct {
  int64_t submitted, built, admitted, completed, failed;
  int64_t waiting;            /* built, not yet admitted */
  int64_t in_flight;          /* admitted, not yet finished */
  int64_t arena_used_bytes, arena_peak_bytes;
  int64_t instances_launched;
  int64_t kernel_launches;
  int64_t max_concurrent;     /* most layouts on the device at one time */
} mpld_server_stats;

/* Create a server on the current device: allocates the device arena, the pinned result pool
 * and the streams, starts the worker threads.  search: node_budget, time_limit_ms and the
 * flags MPLD_COLUMN_BFS and MPLD_SPLIT_BUDGET for every layout (NULL = defaults; with
 * MPLD_SPLIT_BUDGET each layout's device bytes include the split search's lists, contexts and
 * up to 64 MiB of per-warp state).  Errors: MPLD_E_INVALID, MPLD_E_OOM, MPLD_E_CUDA. */
int mpld_server_create(const mpld_server_config *cfg, const mpld_params *search,
                       mpld_server **out);

/* Queue a layout (copied; `graph` may be reused at once).  flags as mpld_params.flags for
 * mpld_build_matrix (MPLD_NO_SIMPLIFY, MPLD_SINGLE_INSTANCE, MPLD_BICONNECTED,
 * MPLD_CLIQUE_BOUND, MPLD_DENSITY_BALANCE; other bits are ignored).  Returns MPLD_OK and a ticket, or
 * MPLD_E_INVALID for MPLD_CLIQUE_BOUND on a server with MPLD_SPLIT_BUDGET.  Input errors
 * surface later as the ticket's result code. */
int mpld_server_submit(mpld_server *s, const mpld_graph *graph, uint32_t flags, int64_t *ticket);

/* Non-blocking progress: admit, upload, launch, detect finished layouts.  Writes up to
 * max_done finished tickets (any order) to `done` and their number to *n_done (done may be
 * NULL when max_done is 0). */
int mpld_server_poll(mpld_server *s, int64_t *done, int32_t max_done, int32_t *n_done);

/* Result of a finished ticket: n_seg masks (host) and the counts; releases the ticket.
 * Returns the layout's status (MPLD_OK / MPLD_BUDGET) or its error; MPLD_E_STATE if the
 * ticket is unknown or not finished. */
int mpld_server_result(mpld_server *s, int64_t ticket, int8_t *mask_out, mpld_result *result);

int mpld_server_stats_get(const mpld_server *s, mpld_server_stats *stats);

/* Wait for the work on the device, join the workers and free everything.  Unfinished tickets
 * are dropped.  NULL is a no-op. */
void mpld_server_destroy(mpld_server *s);

/*
 * Search of one instance that allocates no memory.
 *
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate GPU memory themselves.  Examples are a plug-in running inside
 * a host application whose caching allocator already owns the device's
 * memory, and a latency-bound caller that cannot accept the device-wide
 * synchronisation cudaMalloc / cudaFree can cause.  Such a caller passes the
 * instance and the outputs in device buffers it already has; everything
 * else the search needs (the packed EC matrix and the search stacks) lives
 * in one fixed array inside the library, MPLD_NOALLOC_SCRATCH_BYTES bytes,
 * which every GPU that loads the library holds until the process exits.
 *
 * The instance is the whole given graph (no simplification, no split into
 * sub-graphs), searched exactly as mpld_solve searches an instance: the same
 * column and row order, node budget and time limit, so mask, cost and node
 * count equal those of mpld_solve on the same graph built with
 * MPLD_NO_SIMPLIFY | MPLD_SINGLE_INSTANCE.
 *
 *   inst        host struct holding sizes and DEVICE pointers: conflict and
 *               stitch adjacency in CSR form (ptr[n+1], nbr[ptr[n]]), each
 *               list in ascending order, both directions of every edge, no
 *               self-loops or duplicates;
 *   params      node_budget and time_limit_ms are used; NULL = defaults;
 *   mask_out    DEVICE, n int8: best assignment found;
 *   result_out  DEVICE: cost, node count and status.  The kernel checks the
 *               CSR before searching: a neighbour id out of range, a
 *               self-loop, a list out of order, a bad offset, or an edge
 *               listed from one end only give status MPLD_E_INVALID, and
 *               the mask is then not written.  device_error is 0, or
 *               MPLD_E_TIMEOUT when the copy of the packed instance into
 *               shared memory did not land in time (the search then ran
 *               from the library's array and its result stands);
 *   stream      all work is enqueued on it; the call does not wait.
 * Returns MPLD_E_INVALID for bad sizes, k or costs, MPLD_E_TOO_LARGE when the
 * instance needs more than MPLD_NOALLOC_SCRATCH_BYTES bytes or has more than
 * MPLD_MAX_INSTANCE_SEGMENTS segments (nothing is launched then),
 * MPLD_E_CUDA on a failed launch, or when a CUDA error left by earlier work
 * of the caller is still pending (nothing is launched, and that error is
 * left pending for the caller).
 *
 * The first call on a device (the device current at the call) looks up the
 * array's device address and sets the kernel's shared-memory limit; make
 * that first call before any stream capture on that device.  Every call
 * shares the one array and leaves its contents behind (each call rewrites
 * what it reads, and clears its status word); calls whose GPU work overlaps
 * (on different streams, or from different host threads) race on the array
 * and give wrong results, so order them on one stream.
 */
#define MPLD_NOALLOC_SCRATCH_BYTES (8u << 20)

typedef struct {
  int32_t n, k;
  int32_t n_conf_entries;       /* conf_ptr[n] */
  int32_t n_stitch_entries;     /* st_ptr[n] */
  const int32_t *conf_ptr, *conf_nbr;
  const int32_t *st_ptr, *st_nbr;
  int32_t cost_conflict, cost_stitch;
} mpld_device_instance;

typedef struct {
  int64_t cost;
  int64_t nodes;
  int32_t status;               /* MPLD_OK, MPLD_BUDGET, MPLD_TIMEOUT or MPLD_E_INVALID */
  int32_t device_error;         /* 0, or MPLD_E_TIMEOUT (see above) */
  int64_t work;                 /* as mpld_result.work */
} mpld_instance_result;

int mpld_search_instance_noalloc(const mpld_device_instance *inst, const mpld_params *params,
                                 int8_t *mask_out, mpld_instance_result *result_out,
                                 void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MPLD_H */
