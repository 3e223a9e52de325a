/*
 * hytg -- hybrid host-to-GPU transfer graph engine for one GB300 (sm_103a).
 *
 * The engine runs vertex-centric push algorithms (BFS, SSSP, connected
 * components, delta-PageRank) over a CSR graph whose edge arrays live in
 * pinned host memory, because they exceed a capped device budget.  Vertex
 * data (row offsets, values, frontier) stays on the GPU and edge data in host
 * memory, as stated in the paper's problem setting (Sec. I; Sec. II-A, last
 * paragraph; Sec. IV).  Each iteration, a per-partition cost model (Sec. V-A,
 * Eq. 1-3) picks one of four routes for each partition's active edges:
 *   CACHE  the partition is resident in a device region carved from the budget;
 *   F      explicit copy of the whole partition (ExpTM-filter, Eq. 1);
 *   C      GPU compaction of only the active adjacency lists (ExpTM-compaction,
 *          Eq. 2), gathered from mapped host memory into a device buffer;
 *   Z      zero-copy: the relax kernel reads mapped host memory (ImpTM-ZC, Eq. 3);
 * partitions are then combined into tasks (Sec. V-B, Alg. 1) and relaxed by
 * push kernels on several streams (Sec. VI-B).
 *
 * Conventions for every call:
 *   - every function returns an hytg_status; no exception crosses the ABI;
 *   - host pointers are plain host memory owned by the caller and are only
 *     read (inputs) or written (outputs) during the call;
 *   - after any error other than HYTG_ERR_CUDA the context stays usable;
 *     after HYTG_ERR_CUDA only hytg_destroy is meaningful;
 *   - one context is driven by one host thread at a time;
 *   - hytg_last_error() returns a message for the last failed call.
 */
#ifndef HYTG_H
#define HYTG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hytg_ctx hytg_ctx;

typedef enum {
    HYTG_OK = 0,
    HYTG_ERR_ARG = 1,       /* invalid argument (bad CSR, source out of range, bad key) */
    HYTG_ERR_CUDA = 2,      /* a CUDA call failed; the context is no longer usable */
    HYTG_ERR_BUDGET = 3,    /* device budget below one staging slot plus compaction buffer */
    HYTG_ERR_HOSTMEM = 4,   /* pinned host allocation failed */
    HYTG_ERR_OVERFLOW = 5,  /* an SSSP distance reached 0xFFFFFFFE (does not fit 32 bits) */
    HYTG_ERR_TIMEOUT = 6,   /* hytg_run passed its "run_timeout_ms" deadline */
    HYTG_ERR_STATE = 7      /* call out of order (no graph loaded, no completed run) */
} hytg_status;

typedef enum {
    HYTG_BFS = 0,       /* level[v]: hops from the source (Sec. VII-A)            */
    HYTG_SSSP = 1,      /* dist[v]: min sum of uint32 weights (Sec. II-A, Fig. 1)  */
    HYTG_CC = 2,        /* label[v]: min vertex id of v's component; needs a symmetric CSR
                           (see hytg_run) */
    HYTG_PAGERANK = 3,  /* delta-based PageRank (Sec. VI-A), ranks normalised to sum 1 */
    HYTG_PPR = 4        /* personalised PageRank from one seed, normalised to sum 1 */
} hytg_algo;

typedef enum {
    HYTG_ROUTE_NONE = 0,   /* partition has no active out-edge this iteration */
    HYTG_ROUTE_CACHE = 1,
    HYTG_ROUTE_F = 2,
    HYTG_ROUTE_C = 3,
    HYTG_ROUTE_Z = 4
} hytg_route;

#define HYTG_UNREACHED 0xFFFFFFFFu

/* Totals of the last hytg_run.  Index [r] of the per-route arrays is a
 * hytg_route value. */
typedef struct hytg_stats {
    uint32_t iterations;
    uint32_t status;                  /* hytg_status of the run */
    uint64_t edges_relaxed;           /* sum over iterations of active out-edges (TEPS numerator) */
    uint64_t vertices_processed;      /* sum over iterations of active vertices */
    uint64_t route_partitions[5];     /* partition-iterations per route */
    uint64_t route_vertices[5];       /* active vertices (degree > 0) per route */
    uint64_t route_edges[5];          /* active edges per route */
    uint64_t link_bytes[5];           /* host-link bytes per route: F whole partitions,
                                         C and Z 128-byte lines spanned (C with
                                         "compact_host": the active edge bytes plus 16 B of
                                         list index per vertex), cache 0 */
    uint64_t cache_fill_bytes;        /* bytes copied to fill the resident cache this run */
    uint64_t f_tasks;                 /* F copy tasks after combination (Sec. V-B) */
    uint64_t kernel_launches;         /* kernels launched by the run */
    double wall_ms;                   /* host wall time of hytg_run */
    double kernel_ms[12];             /* device time per kernel kind (CUDA events), when
                                         the "timing" parameter is 1; see HYTG_K_*.
                                         Host-issued launches only: iterations run in the
                                         device loop are not split by kind */
    uint64_t kernel_count[12];        /* launches per kernel kind (timing on) */
    double pr_residual_sum;           /* PageRank/PPR: sum of |delta| left at convergence */
    double pr_rank_sum;               /* PageRank/PPR: sum of raw ranks */
    double device_ms;                 /* CUDA-event time of the run on its main stream, which
                                         joins every other stream of the run */
    uint64_t source_edges;            /* batched runs: sum over sources of the edges relaxed
                                         for that source; else edges_relaxed */
    uint32_t n_sources;               /* sources of the run (1 unless batched) */
    uint32_t pad_;
    uint64_t extra_edges;             /* edges relaxed by second passes over resident
                                         partitions ("two_pass", Sec. VI-A; batched PPR:
                                         summed over seeds); not in edges_relaxed */
    double host_compact_ms;           /* host wall time spent compacting the C route on
                                         host threads ("compact_host" > 0), else 0 */
    uint64_t graph_launches;          /* launches of the device-loop graph ("device_loop") */
    uint64_t graph_iterations;        /* iterations run entirely inside those launches */
    double second_pass_ms;            /* device time of the second passes (timing on) */
    uint64_t second_pass_count;       /* second-pass launches timed */
    uint64_t second_pass_vertices;    /* vertices scanned by host-issued second passes */
    double route_busy_ms[5];          /* timing on: wall time during which the route's
                                         transfers were in flight (union over streams of the
                                         F copies, the C gathers, the Z relaxes); with
                                         link_bytes it gives the link rate while a route
                                         transfers.  Index: hytg_route */
    double kernel_busy_ms[13];        /* timing on: union over streams of the launches of
                                         each HYTG_K_* kind (index 12: the second pass), i.e.
                                         the wall time during which that kind was running */
    uint64_t link_sector_bytes[5];    /* host-link bytes read, counted by the kernels that
                                         read mapped host memory (Z relaxes, C gathers): in
                                         each 2,048-edge tile, the distinct 32-byte sectors
                                         its edges occupy, times 32 and the arrays read; F
                                         (and C with "compact_host"): the bytes copied;
                                         cache 0.  Index: hytg_route */
    uint64_t link_line_bytes[5];      /* the same count at 128-byte lines, times 128 */
    uint64_t f_reused_tasks;          /* F tasks run from a staging slot that still held
                                         their partitions ("slot_reuse"): no copy */
    uint64_t f_reused_bytes;          /* the bytes those tasks did not copy (not in
                                         link_bytes) */
    uint64_t f_ahead_tasks;           /* F tasks copied ahead at the end of an iteration for
                                         the next one ("f_ahead"); their bytes are in
                                         link_bytes whether or not the next iteration used them */
    uint64_t f_ahead_hits;            /* tasks that ran from such a copy instead of copying */
} hytg_stats;

/* kernel kinds indexing kernel_ms / kernel_count */
enum {
    HYTG_K_INIT = 0, HYTG_K_COUNT = 1, HYTG_K_BIN = 2, HYTG_K_RELAX_CACHE = 3,
    HYTG_K_RELAX_F = 4, HYTG_K_GATHER_C = 5, HYTG_K_RELAX_C = 6, HYTG_K_RELAX_Z = 7,
    HYTG_K_COPY_F = 8, HYTG_K_FINAL = 9, HYTG_K_CACHE_FILL = 10, HYTG_K_OTHER = 11,
    HYTG_K_SECOND_PASS = 12           /* timeline only: a second pass (Sec. VI-A) */
};

/* Sizes and placement after load / budget / the last plan. */
typedef struct hytg_info {
    uint64_t V, E;
    uint32_t weighted;
    uint32_t n_parts;                 /* partitions of the edge arrays (Sec. IV) */
    uint64_t part_edges;              /* target edges per partition */
    uint64_t slot_edges;              /* edges per staging slot (k partitions) */
    uint32_t n_slots;                 /* staging slots (F streams plus "prefetch_slots") */
    uint32_t n_cached;                /* partitions [0, n_cached) resident for the last algo */
    uint64_t budget_bytes;            /* device budget for edge-side data */
    uint64_t budget_used_bytes;       /* cache + staging + compaction buffer */
    uint64_t compact_edges;           /* capacity of the compaction buffer, in edges */
    uint64_t vertex_state_bytes;      /* device bytes held for vertex-side data */
    uint64_t pinned_host_bytes;       /* pinned host bytes held for edge arrays */
} hytg_info;

/* Create a context on CUDA device `device`.  *out receives an owned handle. */
hytg_status hytg_create(hytg_ctx **out, int device);

/* Release every device and pinned host allocation of the context. */
hytg_status hytg_destroy(hytg_ctx *ctx);

/* Load a CSR graph (Sec. IV: the neighbour index stays on the GPU, the
 * neighbour and weight arrays in host memory).  offsets: V+1 uint64, with
 * offsets[0] = 0, offsets[V] = E, non-decreasing; dst: E uint32, each < V;
 * weights: E uint32 or NULL for an unweighted graph.  The arrays are copied
 * into library-owned pinned, device-mapped host memory; the caller keeps
 * ownership of its arrays.  V must be in [1, 2^32 - 1].  Replaces any earlier
 * graph.  Errors: HYTG_ERR_ARG (bad CSR), HYTG_ERR_HOSTMEM, HYTG_ERR_CUDA. */
hytg_status hytg_load_csr(hytg_ctx *ctx, uint64_t V, uint64_t E, const uint64_t *offsets,
                          const uint32_t *dst, const uint32_t *weights);

/* Hard cap on device bytes for edge-side data: resident cache, staging slots
 * for explicit copies and the compaction buffer.  Vertex-side data is not
 * counted (it is reported by hytg_get_info).  A budget that cannot hold one
 * staging slot of the largest partition plus one partition's worth of
 * compaction buffer returns HYTG_ERR_BUDGET. */
hytg_status hytg_set_device_budget(hytg_ctx *ctx, uint64_t bytes);

/* Set a tunable.  Keys: "alpha", "beta", "gamma" (Sec. V-A selection and
 * RTT_zc, stored as multiples of 1e-6), "m" (request bytes), "MR" (outstanding
 * requests), "k" (partitions per F task, Sec. V-B), "part_bytes" (partition
 * size in bytes of 4-byte entries, Sec. V-B), "streams" (F compute streams),
 * "prefetch_slots" (staging slots beyond one per F stream, default 4: each
 * slot has its own copy stream, so later tasks' copies run while earlier
 * tasks still hold their slots),
 * "staging_frac", "compact_frac" (shares of the budget), "force_route"
 * (-1 cost model, 1 cache, 2 F, 3 C, 4 Z, 5 random per partition per
 * iteration), "seed" (for force_route 5), "pr_damping", "pr_eps" (FP32
 * residual threshold), "max_iters", "run_timeout_ms" (a deadline for each
 * hytg_run, counted from its start; 0, the default: none; see hytg_run),
 * "slot_reuse" (1: an F task whose partitions a staging slot still holds
 * from an earlier iteration or run runs from it without a copy, counted in
 * f_reused_tasks / f_reused_bytes; 0, the default: every F task is copied),
 * "f_ahead" (n in 1..15 and below the number of staging slots: at the end
 * of each host-issued iteration of a single-source run, copy that
 * iteration's first n F tasks into the least
 * recently used staging slots, as a guess at the next iteration's first
 * tasks, while the link would otherwise idle through the iteration's last
 * relaxes and the next planning; a next-iteration task found among them runs
 * from its slot, in its place in the order; counted in f_ahead_tasks /
 * f_ahead_hits; when on, "slot_reuse" is not applied; 0: off),
 * "f_copy" (0, default: F copies by the copy engine, cudaMemcpyAsync; n in
 * 1..32: by a kernel with n blocks per SM that reads the task's edges from
 * mapped host memory with 16-byte loads, starting at the 16-byte boundary
 * at or below the first edge when the slot has room for the up to 3 extra
 * words read, else by the copy engine),
 * "timing" (1: CUDA-event time per kernel
 * kind), "hub_frac" (fraction of vertices moved to the front by hub sorting
 * at the next hytg_load_csr, Sec. VI-A; 0 disables it; default 0.08),
 * "hub_replicas" (how many of the first hub ids get per-SM PageRank
 * accumulators, applied at the next load; default 4096), "sssp_delta"
 * (delta-stepping bucket width for SSSP: -1 automatic, 0 off), "two_pass"
 * (after relaxing a resident F task or the cache, process once more the
 * vertices of that range that became active again, Sec. VI-A: 0 off,
 * 1 PageRank/PPR only (default), 2 every algorithm; batched runs and
 * serving: PPR only), "two_pass_min_degree"
 * (an F task's range gets its second pass only if it holds at least this
 * many edges per vertex; default 4), "compact_host"
 * (0: the C route's active lists are gathered by a GPU kernel over mapped
 * host memory (default); n in 1..256: n host threads compact them into a
 * pinned staging chunk that one explicit copy moves to the device, the
 * CPU-compaction form of ExpTM-C of Sec. III-B; pinned staging of twice the
 * compaction buffer is allocated outside the device budget), "priority"
 * (Sec. VI-A delta-driven priority: 1 (default) issues the F tasks of a
 * PageRank/PPR iteration in decreasing order of the pending |delta| their
 * partitions hold, 0 in partition order; other algorithms always use
 * partition order, which hub sorting makes hub-first), "device_loop" (1,
 * default: runs replay one iteration (planning, binning, cache and zero-copy
 * relax) inside a CUDA graph with a WHILE node; a single-source iteration
 * that needs the F or C route goes to the host, which issues its copies,
 * while batched runs keep F and C iterations in the graph too: one IF node
 * per partition copies it into a staging slot and relaxes it, one IF node
 * gathers and relaxes the C route, each F copy moves one partition (no task
 * combination, partition order), and only a C route larger than the
 * compaction buffer goes to the host; 2: single-source runs keep F and C
 * iterations in the graph as well; 0: the host drives every iteration.
 * Iterations run in the graph report no per-iteration device time and are
 * not in kernel_ms or the timeline; if the installed CUDA driver cannot build
 * the graph, the context keeps using the host loop and graph_launches stays
 * 0 (and if it cannot hold the F and C nodes, those iterations go to the
 * host as at 1), "loop_after_fc" (0, default: in single-source PageRank and
 * PPR runs whose graph holds no F and C nodes, the iteration after one with
 * F or C work is planned by the host at once, and the device loop takes
 * over after an iteration without such work; 1, and always for the other
 * algorithms: the device loop is entered after every host-issued iteration),
 * "z_blocks" (blocks per SM of a host-issued zero-copy relax, 1..32,
 * default 12: more blocks than fit at once keep more host-link reads in
 * flight beside the other streams' kernels), "serve_frames" (serving:
 * cap on the query frames hytg_serve_begin plans, 0 (default): as many as
 * the slots can use; see hytg_serve_get_info), "batch_sparse_below" (batched
 * SSSP relax: a warp whose 32 edges carry fewer active sources per edge
 * than this on average walks the sources of each lane's own edge; otherwise
 * it walks its edges with a lane per source; 0 never, 65 always; -1
 * (default): 16, the best of a sweep on R-MAT 24; batched PPR always keeps a
 * lane per edge and pushes each frame of 8 seeds with two vector
 * reductions),
 * "host_huge" (0, default: hytg_load_csr places the edge arrays in
 * cudaHostAlloc(Mapped|Portable) memory; 1: in anonymous memory advised for
 * transparent huge pages, registered with the driver, falling back to
 * cudaHostAlloc if that fails).
 * Changing "part_bytes" re-partitions the loaded graph.
 * Unknown key or value out of range: HYTG_ERR_ARG. */
hytg_status hytg_set_param(hytg_ctx *ctx, const char *key, double value);
hytg_status hytg_get_param(hytg_ctx *ctx, const char *key, double *value);

/* Run `algo` to convergence (Sec. IV: cost-aware task generation and task
 * scheduling alternate until no vertex is active).  sources: n_sources
 * vertex ids (host memory); BFS and SSSP take 1..64 sources, PPR 1..32
 * seeds, CC/PAGERANK ignore them (pass NULL, 0).  With more than one source
 * the run is batched: the planner works on the union of the sources'
 * frontiers, so every partition transfer serves all sources at once (BFS:
 * 64-bit source masks per vertex; SSSP and PPR: one warp per edge with a lane
 * per source); delta-stepping is not used in batched SSSP.  The result stays
 * on the device until hytg_fetch_result.  CC computes weakly connected
 * components and needs a symmetric CSR: every edge u->v has a reverse v->u
 * with the same multiplicity (a self-loop is its own reverse); the first CC
 * run after a load checks this on the host (O(E) plus a sort of each row,
 * cached with the graph) and an asymmetric graph gives HYTG_ERR_ARG.
 * With "run_timeout_ms" > 0 a run that has not converged by then stops at
 * the next iteration boundary: the host checks the deadline before it issues
 * an iteration, and inside the device loop it sets a word of mapped host
 * memory that the loop's decision kernel reads before each iteration.  The
 * call then waits for the work already issued (at most one more iteration),
 * returns HYTG_ERR_TIMEOUT, and leaves the context idle and usable, with no
 * result (hytg_fetch_result gives HYTG_ERR_STATE).
 * Errors: HYTG_ERR_ARG, HYTG_ERR_STATE (no graph or no budget),
 * HYTG_ERR_OVERFLOW (SSSP), HYTG_ERR_TIMEOUT, HYTG_ERR_CUDA. */
hytg_status hytg_run(hytg_ctx *ctx, hytg_algo algo, const uint32_t *sources, uint32_t n_sources);

/* Copy the last run's result into caller-owned host memory `out` of
 * out_bytes >= 4*V*n_sources bytes, source-major (out[s * V + v]): uint32 per
 * vertex (BFS level, SSSP distance, CC label; HYTG_UNREACHED when unreached)
 * or float per vertex (PageRank/PPR, normalised to sum 1 per source).
 * HYTG_ERR_STATE if no run completed. */
hytg_status hytg_fetch_result(hytg_ctx *ctx, void *out, uint64_t out_bytes);

/* Raw delta-PageRank state of the last PageRank/PPR run: rank and the
 * residual delta per vertex (float, V entries each; either may be NULL). */
hytg_status hytg_fetch_pagerank_state(hytg_ctx *ctx, float *rank, float *delta, uint64_t V);

hytg_status hytg_get_stats(hytg_ctx *ctx, hytg_stats *out);
hytg_status hytg_get_info(hytg_ctx *ctx, hytg_info *out);

/* Hub sorting (Sec. VI-A), a pure host function (no GPU needed): the
 * floor(frac * V) vertices with the largest H(v) = D_o(v) * D_i(v) (the
 * paper's normalisation by D_omax * D_imax does not change the order; ties
 * go to the smaller id) come first in decreasing H, then every other vertex
 * in increasing id.  offsets: V+1 uint64; dst: offsets[V] uint32 (host).
 * perm receives V uint32: perm[n] = original id of internal vertex n.
 * *n_hubs (may be NULL) receives floor(frac * V). */
hytg_status hytg_hub_order(uint64_t V, const uint64_t *offsets, const uint32_t *dst, double frac,
                           uint32_t *perm, uint64_t *n_hubs);

/* The internal vertex order of the loaded graph: perm[n] = original id of
 * internal vertex n (identity when hub sorting is off).  Partitions, the
 * frontier of hytg_plan_noalloc and the routes refer to internal ids; every
 * other call takes and returns original ids. */
hytg_status hytg_get_permutation(hytg_ctx *ctx, uint32_t *perm, uint64_t V);

/* Partition table (Sec. IV): vertex bounds, n_parts + 1 uint64 entries.
 * Partitions start on multiples of 32 vertices; each is the longest run with
 * at most part_edges edges, or a single 32-vertex run if that run alone has
 * more.  cap: entries available in vbounds. */
hytg_status hytg_get_partitions(hytg_ctx *ctx, uint64_t *vbounds, uint32_t cap, uint32_t *n_parts);

/* Cost analysis and engine selection alone (Sec. V-A, Alg. 1 cost part) for
 * a caller-given frontier: active (V bytes indexed by original id, nonzero =
 * active) is uploaded,
 * the count and selection kernels run on the device, and the per-partition
 * results come back: routes[n_parts] (hytg_route), and, if non-NULL,
 * counts[3 * n_parts] = {|A_i|, active edges, 128-byte lines} per partition.
 * The resident set is the cache plan for `algo` under the current budget. */
hytg_status hytg_plan(hytg_ctx *ctx, hytg_algo algo, const uint8_t *active, uint8_t *routes,
                      uint64_t *counts, uint32_t cap);

/* Host-link probe (the measured denominators of the link roofline): pinned
 * host-to-device cudaMemcpyAsync bandwidth over `bytes`, best of `reps`, and
 * a zero-copy kernel reading the same pinned buffer in 128-byte lines.
 * Results in GB/s (1e9 bytes/s). */
hytg_status hytg_probe_link(hytg_ctx *ctx, uint64_t bytes, uint32_t reps, double *memcpy_gbs,
                            double *zerocopy_gbs);

/* L2 reduction probe (the ceiling of the relax kernels, which push with
 * fire-and-forget float/integer reductions into L2-resident vertex arrays):
 * n random `red.global.add.f32` into 2^24 floats, with uniform targets and
 * with R-MAT-skewed targets (each of 24 index bits set with probability 0.24),
 * best of `reps`; results in 1e9 updates/s.  Allocates device memory. */
hytg_status hytg_probe_atomics(hytg_ctx *ctx, uint64_t n, uint32_t reps, double *uniform_gops,
                               double *skewed_gops);

/* The same reduction probe with the R-MAT in-degree skew after hub sorting
 * (ids ordered by probability, hot ids first, as hytg_load_csr relabels
 * them): additions straight into the 2^24 floats (*plain_gops), and with the
 * relax kernels' scheme, where additions to ids below n_rep go to the
 * issuing SM's row of per-SM replicas (*replica_gops; the rows are not
 * folded).  n in [1024, 2^30], n_rep <= 2^20.  Allocates device memory. */
hytg_status hytg_probe_atomics_hub(hytg_ctx *ctx, uint64_t n, uint32_t reps, uint32_t n_rep,
                                   double *plain_gops, double *replica_gops);

/* The roof of the batched PPR push: n pushes of a frame of 8 floats (one
 * 32-byte sector) to uniform random vertices of 2^24 frames (512 MiB, more
 * than the L2 holds, like the frames of a large batched run), each push as
 * 8 / width reductions of `width` floats (1: red.global.add.f32; 2 or 4:
 * the .v2 / .v4 vector forms).  Best of `reps`; *frame_gops in 1e9 frame
 * pushes/s (seed updates/s = 8 x that).  n in [1024, 2^30].  Allocates
 * device memory (n * 4 + 512 MiB). */
hytg_status hytg_probe_frame_push(hytg_ctx *ctx, uint64_t n, uint32_t reps, uint32_t width,
                                  double *frame_gops);

/* Per-iteration record of the last run (up to cap records). */
typedef struct hytg_iter_record {
    uint64_t active_vertices;
    uint64_t active_edges;
    uint32_t route_partitions[5];
    uint32_t f_tasks;
    uint64_t route_edges[5];
    uint64_t link_bytes;
    double device_ms;                 /* CUDA-event time from this iteration's planning to
                                         the next one's (timing parameter 1), else 0 */
} hytg_iter_record;
hytg_status hytg_get_iterations(hytg_ctx *ctx, hytg_iter_record *out, uint32_t cap, uint32_t *n);

/* One timed launch or copy of the last hytg_run ("timing" parameter 1), in
 * issue order.  Host-issued work only: iterations inside the device-loop
 * graph are not split into launches.  The second-pass entries, in order, are
 * the process's k_second_pass launches of that run, so a profiler's launch
 * index can be matched to its edge count when the device loop is off. */
typedef struct hytg_timed_launch {
    uint32_t kind;                    /* HYTG_K_* (HYTG_K_SECOND_PASS for a second pass) */
    uint32_t stream;                  /* 0 main stream, 1 compaction stream, 2 + i F stream i,
                                         10 + j copy stream of staging slot j */
    double start_ms, end_ms;          /* CUDA-event times from the run's start event */
    uint64_t bytes;                   /* HYTG_K_COPY_F, host-compaction chunks: bytes copied */
    uint64_t edges;                   /* HYTG_K_RELAX_F: active edges of the task;
                                         HYTG_K_SECOND_PASS: edges it relaxed (UINT64_MAX when
                                         more than 16,382 second passes ran and the later ones
                                         share a counter) */
    uint64_t vertices;                /* HYTG_K_SECOND_PASS: vertices of the range it scanned */
    uint32_t part_first, part_last;   /* HYTG_K_COPY_F, HYTG_K_RELAX_F, HYTG_K_SECOND_PASS of an F
                                         task: the task's partitions [part_first, part_last]
                                         (task combination, Sec. V-B); else 0, 0 */
} hytg_timed_launch;
hytg_status hytg_get_timeline(hytg_ctx *ctx, hytg_timed_launch *out, uint32_t cap, uint32_t *n);

/* ------------------------------------------------------------------------
 * Serving: continuous batching over a batched run.  hytg_serve_begin opens a
 * batched run of n_slots query slots (BFS/SSSP 1..64, PPR 1..32) with empty
 * state; hytg_serve_admit places a query (its source or seed, original id)
 * in a free slot at the next iteration boundary; hytg_serve_step runs one
 * iteration for every busy slot at once (one planning pass and one set of
 * partition transfers serve them all) and reports, as bit masks over slots,
 * the busy slots and the busy slots whose query has converged (no frontier
 * left); hytg_serve_fetch copies a converged slot's result (V values,
 * original vertex order: BFS level from its source, SSSP distance, PPR rank
 * normalised to sum 1) and frees the slot; hytg_serve_end closes the run.
 * Queries admitted while others are running join them at the next
 * iteration, so their work overlaps on the device; a query's result does not
 * depend on the others.  hytg_run is refused while serving. */
hytg_status hytg_serve_begin(hytg_ctx *ctx, hytg_algo algo, uint32_t n_slots);
/* hytg_serve_admit: HYTG_ERR_BUDGET when the slot's group of 8 has no frame
 * of device memory and none is free (see hytg_serve_get_info). */
hytg_status hytg_serve_admit(hytg_ctx *ctx, uint32_t slot, uint32_t source);
hytg_status hytg_serve_step(hytg_ctx *ctx, uint64_t *finished, uint64_t *busy);
hytg_status hytg_serve_fetch(hytg_ctx *ctx, uint32_t slot, void *out, uint64_t out_bytes);
hytg_status hytg_serve_end(hytg_ctx *ctx);

/* Device memory of the open serving run.  A serving run's budget (the one
 * hytg_set_device_budget set) holds both the edge-side data (cache, staging,
 * compaction buffer) and the queries' per-source state, in frames of 8
 * queries: slots [8 g, 8 g + 8) share frame memory (BFS/SSSP V * 32 bytes,
 * PPR V * 96 bytes), attached when the group's first query is admitted and
 * released when its last one is fetched.  hytg_serve_begin plans as many
 * frames as the slots can use (at most the "serve_frames" parameter, when it
 * is nonzero), fewer if the budget cannot hold them beside the smallest
 * edge-side carve (HYTG_ERR_BUDGET if it holds none); the edge side gets the
 * rest.  hytg_serve_admit returns HYTG_ERR_BUDGET, and admits nothing, when
 * the slot's group has no frame and none is free: the query waits for memory
 * even though the slot is free.  Masks and list arrays that do not grow with
 * the number of queries are vertex-side data, outside the budget. */
typedef struct hytg_serve_info {
    uint32_t frames;                  /* frames the budget holds */
    uint32_t frames_free;             /* frames attached to no group */
    uint32_t slots_per_frame;         /* 8 */
    uint32_t pad_;
    uint64_t frame_bytes;             /* device bytes of one frame */
    uint64_t edge_budget_bytes;       /* budget left to cache, staging and compaction */
    uint64_t busy_slots;              /* bit s: slot s holds a query */
} hytg_serve_info;
hytg_status hytg_serve_get_info(hytg_ctx *ctx, hytg_serve_info *out);

const char *hytg_status_str(hytg_status s);
const char *hytg_last_error(hytg_ctx *ctx);

/* ------------------------------------------------------------------------
 * Allocation-free planning (this entry point has no counterpart in the paper).
 *
 * Some callers cannot call cudaMalloc: code that runs while a stream is being
 * captured into a CUDA graph (allocation is not a capturable operation),
 * code embedded in a framework whose caching allocator owns all device
 * memory, or a service that must not change its device footprint once it has
 * started.  hytg_plan_noalloc gives them the per-partition counting and
 * engine selection of hytg_plan (Sec. V-A, Eq. 1-3) without any allocation:
 * no context, no cudaMalloc/cudaFree and no allocating library call.  Its only
 * scratch is a static device array of HYTG_NOALLOC_MAX_PARTS + 1 partition
 * bounds (about 768 KiB), which every GPU that loads the library holds until
 * the process exits.
 *
 * All pointers are device pointers owned by the caller:
 *   frontier      ceil(V / 32) uint32 words, bit v % 32 of word v / 32 set
 *                 when vertex v is active; bits at or beyond V are ignored;
 *   offsets       V + 1 uint64 CSR row offsets;
 *   part_vbounds  n_parts + 1 uint64 vertex bounds of the partitions, from 0
 *                 to V, on multiples of 32 except the last (the layout that
 *                 hytg_get_partitions returns);
 *   routes        n_parts uint8 outputs (hytg_route);
 *   counts        3 * n_parts uint64 outputs {|A_i|, active edges, 128-byte
 *                 lines} per partition (zeroed by the call itself).
 * Partitions [0, n_cached) count as resident.  params may be NULL for the
 * paper's constants (alpha 0.8, beta 0.4, gamma 0.625, m 128, MR 256).
 * stream is a cudaStream_t (NULL: the default stream); the work is queued on
 * it and the call returns without waiting.
 *
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the one array, so calls that
 * overlap on the GPU (on different streams, or from several threads) race:
 * order them on one stream.  Errors: HYTG_ERR_ARG for a NULL pointer, an
 * unknown algorithm, V outside [1, 2^32 - 1], n_parts of 0 or above
 * HYTG_NOALLOC_MAX_PARTS, n_cached > n_parts or bad params; HYTG_ERR_CUDA if
 * the address lookup or a launch fails, or if a CUDA error left by earlier
 * work is already pending when the call starts (nothing is queued then, and
 * that error is left pending for its owner to read). */
#define HYTG_NOALLOC_MAX_PARTS 65536u

typedef struct hytg_cost_params {
    double alpha, beta, gamma;   /* selection thresholds and RTT_zc factor */
    uint32_t m, MR;              /* request bytes, outstanding requests */
} hytg_cost_params;

hytg_status hytg_plan_noalloc(hytg_algo algo, const uint32_t *frontier, const uint64_t *offsets,
                              uint64_t V, const uint64_t *part_vbounds, uint32_t n_parts,
                              uint32_t n_cached, const hytg_cost_params *params, uint8_t *routes,
                              uint64_t *counts, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HYTG_H */
