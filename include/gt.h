/*
 * gt.h -- C-ABI of libgt: edge-tree BFS on one GB300 (sm_103a), after
 * C. Zhang, "A New Perspective of Graph Data and A Generic and Efficient Method for
 * Large Scale Graph Data Traversal" (arXiv 2009.07463).
 *
 * The library splits a graph into a core subgraph and the edge trees of low-degree
 * vertices (Sec. 4, Alg. 8), runs direction-optimizing BFS (Alg. 1: top-down queue
 * expansion, bottom-up scan of unvisited vertices with early exit, a frontier-size
 * switch) on the core only (Alg. 9, BFS_CORE), then gives every edge-tree vertex its
 * level and parent from the vertex its tree hangs off (Alg. 10 / Alg. 7).
 *
 * Conventions shared by every entry point:
 *  - Return 0 on success or a negative GT_E* code; gt_strerror() names it and
 *    gt_last_error() gives a one-line detail of the last failure on this thread.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Work is stream-ordered;
 *    the library never calls cudaDeviceSynchronize. Calls that must read a device
 *    count back (graph build) synchronise the given stream and say so.
 *  - Vertex ids are int64 at the boundary and must lie in [0, n); n <= 2^31 - 1.
 *  - BFS output (Alg. 1 initialisation; Graph500 spanning-tree rule, Sec. 5.3):
 *    level[v] = hop distance from the root, parent[root] = root, and for every other
 *    reached v, parent[v] = the smallest vertex id u adjacent to v with
 *    level[u] = level[v] - 1. Unreached vertices get -1 in both arrays. Self-loops are
 *    ignored and duplicate tuples merged.
 *  - The caller owns every buffer it passes; the library owns graph handles and the
 *    device memory behind them. Handles may be used from one host thread at a time.
 */
#ifndef GT_H
#define GT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GT_API __attribute__((visibility("default")))

/* Status codes. */
#define GT_OK 0
#define GT_EINVAL (-1)   /* bad argument: null pointer, id out of range, bad size */
#define GT_ENOMEM (-2)   /* device or host allocation failed */
#define GT_ETIMEOUT (-3) /* a bounded wait ran out */
#define GT_EBUSY (-4)    /* resource in use */
#define GT_EDEVICE (-5)  /* CUDA error (detail in gt_last_error) */
#define GT_ENOTSUP (-6)  /* not supported on this device / build */
#define GT_EIO (-7)      /* a file could not be read or written, or is not a saved graph */

/* Vertex classes of Sec. 4.2 (codes of gt_graph_vertex_type). */
#define GT_CORE_INTERNAL 0 /* CI */
#define GT_CORE_EDGE 1     /* CE */
#define GT_TREE_INTERNAL 2 /* TI */
#define GT_TREE_LEAF 3     /* TL */
#define GT_VERTEX_ZERO 4   /* VZ */

/* Build-time options. */
typedef struct gt_config {
  int32_t mh;         /* maximum edge-tree height MH of Alg. 8: 0 = leaves only (default,
                         the paper's choice in Sec. 6.2), -1 = peel to the fixpoint */
  int32_t keep_plain; /* 1 (default): keep the unsplit CSR and its BFS state so
                         gt_bfs_plain works; 0: free them after the split */
} gt_config;

/* Run-time tuning of the traversal; results never depend on it. */
typedef struct gt_tuning {
  int32_t alpha;        /* top-down -> bottom-up when m_f * alpha > m_u (default 32) */
  int32_t beta;         /* bottom-up -> top-down when n_f * beta < n and shrinking (256) */
  int32_t td_warp_min;  /* top-down: degree above which a whole warp takes a vertex (32) */
  int32_t td_cta_min;   /* top-down: degree above which a whole CTA takes a vertex (256) */
  int32_t td_grid_min;  /* top-down: degree above which the vertex's edges join one flat
                           edge space shared by the whole grid (2048) */
  int32_t bu_thread_scan; /* bottom-up: neighbours a lane checks alone before the warp
                             takes the vertex over (24) */
  int32_t blocks_per_sm;  /* CTAs per SM of the traversal kernels (8) */
  int32_t force_direction; /* 0 = switch heuristic, 1 = top-down only, 2 = bottom-up only */
  int32_t launch_mode;  /* 0 = whole level loop in one CUDA graph with device-side
                           control (default), 1 = host-driven loop (one readback per level) */
  int32_t count_work;   /* 1: count examined edges per level (slower; for the trace) */
  int32_t time_kernels; /* 1: time the phases of each traversal (gt_bfs_timing) and, with
                           launch_mode = 1, each level's step kernels (gt_bfs_trace), with
                           CUDA events on the caller's stream; each call then synchronises */
  int32_t batch_alpha;  /* gt_bfs_batch: lane word goes bottom-up when the next frontier's
                           summed degree * batch_alpha > core edges (default 14) */
  int32_t batch_beta;   /* gt_bfs_batch: back to top-down when frontier * batch_beta < core
                           vertices and shrinking (default 24) */
  int32_t bu_hub_first; /* 1: degree-aware bottom-up (Alg. 3): each unvisited vertex first
                           tests its highest-degree neighbour; a vertex found that way gets
                           its min-id parent from one ascending pass after the level loop.
                           Default 0 (measured slower; results are the same either way) */
} gt_tuning;

typedef struct gt_stats {
  int64_t n;          /* vertices */
  int64_t m;          /* input tuples */
  int64_t nnz;        /* directed adjacency entries after cleanup (2 x undirected edges) */
  int64_t n_core;     /* CI + CE */
  int64_t nnz_core;   /* directed core-to-core entries */
  int64_t n_class[5]; /* counts of CI, CE, TI, TL, VZ */
  int32_t mh;         /* MH used */
  int32_t height;     /* largest height h at which Alg. 8 marked a tree-internal vertex */
  int64_t device_bytes; /* device memory held by the handle */
} gt_stats;

/* One level of the last traversal on a handle (bfs trace). */
typedef struct gt_level_info {
  int32_t level;        /* level of the frontier this step expanded */
  int32_t direction;    /* 0 top-down, 1 bottom-up over the gathered list of unvisited
                           vertices, 2 bottom-up streaming over all vertices (used while
                           more than a sixth of them are unvisited), 3 the same with a
                           shared-memory filter of a small frontier (after a top-down step) */
  int64_t frontier;     /* frontier vertices n_f */
  int64_t frontier_edges; /* sum of their degrees m_f */
  int64_t unvisited_edges; /* m_u before the step */
  int64_t discovered;   /* vertices found by the step */
  int64_t examined;     /* adjacency entries read by the step (count_work = 1), else -1 */
  double step_ms;       /* duration of the step's kernels (time_kernels = 1), else -1 */
} gt_level_info;

typedef struct gt_graph* gt_graph_t;

GT_API void gt_config_default(gt_config* cfg);
GT_API void gt_tuning_default(gt_tuning* t);

/* Build a graph handle from m tuples (edges[2i], edges[2i+1]), host or device memory
 * (int64, 16-byte aligned if on the device), over vertices [0, n).
 * Steps (all on the device): symmetrise, radix-sort the packed (u, v) keys, drop
 * self-loops and duplicates, row offsets by scan (Sec. 5.1.1 CSR); classify vertices
 * with Alg. 8 at MH = cfg->mh (Sec. 4.3); relabel the core (CI + CE) monotonically in
 * vertex id (the core-left layout of Sec. 5.1.1) and compact core-to-core edges into a
 * dense int32 CSR; lay out the edge-tree edge list (Sec. 5.1.2).
 * cfg may be NULL (defaults). Synchronises `stream`. Returns GT_EINVAL if a tuple has
 * an id outside [0, n) (nothing is kept), GT_ENOMEM if device memory runs out. */
GT_API int gt_graph_build(const int64_t* edges, int64_t m, int64_t n, const gt_config* cfg, void* stream,
                          gt_graph_t* out);
GT_API void gt_graph_free(gt_graph_t g);
/* Checkpoint of a built graph (no counterpart in the paper): gt_graph_save writes what the
 * build derived from the tuples (CSR, Alg. 8 classes and tree parents, core relabel and
 * core CSR, edge-tree lists, batched work lists, configuration, tuning and statistics) to
 * the file at `path`; gt_graph_load reads such a file into a new handle on the current
 * device (or the device of `stream`), allocating the per-traversal state as a build does,
 * so the graph need not be rebuilt from its tuples. Both synchronise `stream`. GT_EINVAL
 * for a null argument, GT_EIO if the file cannot be written or read, is truncated or was
 * not written by this version (a failed save removes the file; a failed load keeps
 * nothing), GT_ENOMEM if device memory runs out. */
GT_API int gt_graph_save(gt_graph_t g, const char* path, void* stream);
GT_API int gt_graph_load(const char* path, void* stream, gt_graph_t* out);
GT_API int gt_graph_stats(gt_graph_t g, gt_stats* out);
/* Copy Alg. 8's vertex_type[n] (GT_* class codes) into out (host or device). */
GT_API int gt_graph_vertex_type(gt_graph_t g, uint8_t* out, void* stream);
/* Copy the cleaned degree of every vertex (int32[n]) into out (host or device). */
GT_API int gt_graph_degree(gt_graph_t g, int32_t* out, void* stream);
GT_API int gt_graph_get_tuning(gt_graph_t g, gt_tuning* out);
GT_API int gt_graph_set_tuning(gt_graph_t g, const gt_tuning* t);

/* Edge-tree BFS from `root` (Alg. 9): root-in-tree walk to its core vertex, BFS on the
 * core only, then edge-tree resolution. parent and level are int32[n], both device or
 * both host memory. With page-locked host memory (cudaHostAlloc / registered) the output
 * pass writes the result straight into it; with pageable host memory the result is
 * staged on the device and copied back. With host memory the call returns after `stream`
 * has finished. */
GT_API int gt_bfs(gt_graph_t g, int64_t root, int32_t* parent, int32_t* level, void* stream);
/* k edge-tree BFS (as gt_bfs, Alg. 9) from roots[0..k-1] (host array), in that order on
 * `stream`; root i writes parent[i] and level[i] (int32[n] each, both device or both host
 * memory; roots may differ). Host results are staged on the device (two staging pairs,
 * 16 B x n, allocated on first use and kept with the handle) and copied to the host on a
 * stream of the handle (by a 12-CTA copy kernel into page-locked memory, by the copy
 * engine into pageable memory) while the next root is traversed, so the host-link
 * transfer of one result overlaps the traversal of the next. Returns after
 * every host result is in place (device results: stream-ordered on `stream`). GT_EINVAL
 * for a null argument, k < 0, a root outside [0, n) or a root whose two outputs are in
 * different memories (nothing is run then). */
GT_API int gt_bfs_roots(gt_graph_t g, const int64_t* roots, int32_t k, int32_t* const* parent,
                        int32_t* const* level, void* stream);
/* The same contract on the unsplit graph (plain direction-optimizing BFS, Alg. 1); the
 * comparison baseline. GT_ENOTSUP if the handle was built with keep_plain = 0. */
GT_API int gt_bfs_plain(gt_graph_t g, int64_t root, int32_t* parent, int32_t* level, void* stream);
/* Batched BFS (multi-source BFS over 64-root lane words; no counterpart in the paper,
 * which runs one root at a time): for every graph i and each of its roots_per_graph[i]
 * roots (taken in order from `roots`), writes the same level and parent arrays gt_bfs
 * would, as rows of parent[i] / level[i]: device int32 [roots_per_graph[i]][n_i], row r
 * for root r. Roots are packed 64 to a lane word; the words of all graphs advance level
 * by level in one persistent cooperative launch that shares every adjacency read among
 * the word's roots. Per-graph lane-word storage (about 420 bytes per core vertex per 64
 * roots) is allocated on first use and kept in the handle. At most 16384 roots per call.
 * All graphs must live on one device. Synchronises `stream`. GT_ETIMEOUT if a bounded
 * grid-barrier wait ran out, GT_ENOTSUP if a traversal is deeper than 65533 levels. */
GT_API int gt_bfs_batch(const gt_graph_t* graphs, int32_t ngraphs, const int64_t* roots,
                        const int32_t* roots_per_graph, int32_t* const* parent, int32_t* const* level,
                        void* stream);
/* Work of the last gt_bfs_batch call whose first graph was g, summed over its lane words:
 * out[0] adjacency entries read by bottom-up (pull) phases, out[1] adjacency entries read
 * by top-down (push) phases, out[2] core vertices scanned by pull phases, out[3] vertices
 * discovered (a vertex counts once per lane word and level that discovers it). For the
 * algorithmic-bytes roofline of the batched launch. */
GT_API int gt_bfs_batch_work(gt_graph_t g, int64_t* out);
/* Failure detection of the batched launches (no counterpart in the paper). Every wait of
 * the persistent kernel at a grid barrier is bounded: after `polls` polls (default 2^26,
 * seconds) the waiting CTA raises an error flag, every CTA leaves the kernel, and the call
 * returns GT_ETIMEOUT with the device still usable. For tests of that path, this call sets
 * the bound of later batched launches (gt_bfs_batch and the server's) and makes each
 * barrier also wait for `extra` arrivals that never come, so that with extra > 0 every
 * launch gives up at its first barrier after `polls` polls. polls = 0, extra = 0 restores
 * the default. Process-wide; not for use while other threads launch batches. */
GT_API void gt_test_batch_barrier(uint32_t polls, uint32_t extra);
/* Allocation-failure injection for tests (no counterpart in the paper): once `after` more
 * device allocations of graph construction (the handle's arrays and the build's
 * temporaries) have succeeded, the next one fails as if device memory had run out, so
 * gt_graph_build returns GT_ENOMEM and frees what it had allocated; after < 0 disables
 * it. Process-wide; not for use while other threads build graphs. */
GT_API void gt_test_fail_alloc(int32_t after);
/* Autotuner: times edge-tree BFS from nsample seeded roots of degree >= 1 (and one batch
 * of up to 64 of them) under settings of gt_tuning, walking one parameter at a time, and
 * keeps the fastest in the handle (also copied to *best if non-null). Results do not
 * depend on the setting. Synchronises `stream`; allocates temporary device buffers. */
GT_API int gt_autotune(gt_graph_t g, int32_t nsample, uint64_t seed, gt_tuning* best, void* stream);
/* Phase times of the last traversal run with time_kernels = 1: start (state reset, root
 * walk), the level loop, and the output pass (tree resolution and scatter); -1 if none. */
typedef struct gt_bfs_timing_t {
  double start_ms, loop_ms, output_ms;
} gt_bfs_timing_t;
GT_API int gt_bfs_timing(gt_graph_t g, gt_bfs_timing_t* out);
/* Per-level trace of the last gt_bfs / gt_bfs_plain on g (synchronises the stream it
 * ran on). Writes up to cap entries, *nlevels = levels run. */
GT_API int gt_bfs_trace(gt_graph_t g, gt_level_info* out, int32_t cap, int32_t* nlevels);

/* Graph500 TEPS numerator: number of tuples (device int64[m][2], 16-byte aligned) whose
 * two ends both have level >= 0 (device int32 level[n]). Synchronises `stream`.
 * GT_EINVAL if a tuple holds an id outside [0, n) (nothing is read out of bounds). */
GT_API int gt_count_traversed(const int64_t* edges, int64_t m, const int32_t* level, int64_t n, int64_t* out,
                              void* stream);

/* ---- Serving: continuous batching over resident graphs (no counterpart in the paper) ----
 * A server keeps graph handles resident and queues single-root queries per graph. A
 * scheduler thread dispatches the pending roots of a graph, whenever one of its streams is
 * free, in the form its running per-graph cost estimates say is cheaper: up to 64
 * single-root traversals back to back (one such flight per graph at a time), or one
 * batched launch (64 roots per lane word, as gt_bfs_batch) whose cost hardly depends on
 * how many lanes are filled. A batched launch goes at once when the GPU is idle,
 * otherwise after up to window_us to fill lane words (only where batching pays); queries
 * that arrive while a batched launch of their graph runs join its free lanes at one of its
 * first level boundaries (join_levels); in a lane word that took joined roots, each lane's
 * results are written, and its query completes, when that lane's traversal ends, even
 * while the launch goes on. Flights on different streams overlap on the device. Each
 * result equals gt_bfs from that root.
 * While a graph is added to a running server, the caller must not traverse it through
 * gt_bfs, gt_bfs_plain, gt_bfs_trace or gt_autotune: those share its traversal state. */
typedef struct gt_serve_config {
  int64_t hbm_budget_bytes; /* graphs + batch storage admitted up to this (default 48 GiB) */
  int32_t streams;          /* flights at once, at most two of them batched launches, each on
                               half of the SMs (default 4) */
  int32_t max_batch_roots;  /* roots per launch (default 256) */
  double window_us;         /* wait to fill lane words while other batches run (default 200) */
  int32_t policy;           /* GT_SERVE_ADAPTIVE (default), GT_SERVE_BATCHED or GT_SERVE_SINGLE */
  int32_t join_levels;      /* a batched launch takes newly submitted roots of its graph into
                               free lanes at its first join_levels level boundaries (default 0:
                               roots join only new launches) */
} gt_serve_config;

enum { GT_SERVE_ADAPTIVE = 0, GT_SERVE_BATCHED = 1, GT_SERVE_SINGLE = 2 };

typedef struct gt_serve_stats {
  int64_t submitted, completed, failed, batches, inflight, pending; /* batches: batched launches */
  double p50_us, p99_us, mean_us, max_us; /* submit -> results in the caller's buffers */
  double qps;                             /* completed / (last completion - first submit) */
  int64_t device_bytes;                   /* graphs + batch storage held against the budget */
  int64_t joined;                         /* queries admitted into a running batched launch */
  int64_t early;                          /* queries completed before their batched launch ended */
} gt_serve_stats;

typedef struct gt_server* gt_server_t;

GT_API void gt_serve_config_default(gt_serve_config* cfg);
/* Starts a server (and its scheduler thread) on the current device. cfg may be NULL. */
GT_API int gt_serve_create(const gt_serve_config* cfg, gt_server_t* out);
/* Makes a built graph resident for queries; GT_ENOMEM if its device memory plus one lane
 * word of batch storage would exceed the budget. The server does not own the handle,
 * which must outlive the server and must not be freed while queries are pending. */
GT_API int gt_serve_add_graph(gt_server_t s, gt_graph_t g, int32_t* gid);
/* Queues a BFS from `root` on graph gid. parent and level are caller-owned device
 * int32[n] buffers that receive the result; they must stay valid until gt_serve_poll
 * reports completion. Thread-safe. */
GT_API int gt_serve_submit(gt_server_t s, int32_t gid, int64_t root, int32_t* parent, int32_t* level,
                           uint64_t* ticket);
/* Waits up to timeout_ms for the query: 0 when its results are in the buffers (the ticket
 * is then released), GT_ETIMEOUT if not yet done (the ticket stays valid), another status
 * if it failed (GT_EBUSY: the server was stopped before it ran). */
GT_API int gt_serve_poll(gt_server_t s, uint64_t ticket, int32_t timeout_ms);
GT_API int gt_serve_get_stats(gt_server_t s, gt_serve_stats* out);
GT_API int gt_serve_reset_stats(gt_server_t s);
/* Stops admitting, finishes the batches in flight, fails queries never dispatched, and
 * frees the server (not the graphs). */
GT_API int gt_serve_destroy(gt_server_t s);

/* ---- Traversal that allocates nothing (the paper has no counterpart) ----
 * For callers that cannot allocate device memory when they need a traversal: a service
 * whose memory plan is fixed at start-up and forbids allocation on the request path (an
 * allocation can block, synchronise the device or fail once memory is fragmented), or a
 * plug-in inside a framework that owns all device memory and passes only inputs and
 * outputs. Runs the plain direction-optimizing BFS (same results as gt_bfs_plain) on the
 * caller's device CSR: row int64[n+1], col int32[row[n]] (sorted, symmetric, no
 * self-loops), writing the device int32[n] parent and level arrays. All scratch lives in
 * one file-scope device array of about 12 MB, reserved on every device that loads the
 * library until the process exits, so n is limited to 262,144 vertices (GT_EINVAL above).
 * No cudaMalloc, cudaFree or allocating library routine is called. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and caches it. Every
 * call uses the same array, so calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller. The call reads nnz and, once per
 * level, the control block back to the host and synchronises `stream` each time, so it
 * returns with the results in place and cannot be called on a stream that is being
 * captured. GT_EINVAL for a null pointer, n < 1 or above the limit, a root outside
 * [0, n), or a buffer that is not memory of the current device. */
GT_API int gt_bfs_csr_noalloc(const int64_t* row, const int32_t* col, int64_t n, int64_t root, int32_t* parent,
                              int32_t* level, void* stream);

GT_API const char* gt_strerror(int code);
GT_API const char* gt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GT_H */
