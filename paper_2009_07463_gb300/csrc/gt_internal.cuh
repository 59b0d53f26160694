// gt_internal.cuh -- definitions shared by the translation units of libgt.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "gt.h"

namespace gt {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint64_t UNVISITED = ~0ull;   // packed (level << 32 | parent) of an unvisited vertex
constexpr int DIR_TD = 0, DIR_BU = 1;
constexpr int MAX_TRACE = 4096;
constexpr int BFS_THREADS = 256;
constexpr int BU_CHUNK_WORDS = 128;     // bitmap words one warp takes per step (4096 vertices)
// Frontier queues are split by degree when a vertex is discovered, so the top-down step
// can give each vertex the right amount of the machine: packed lanes (bin 0), a warp
// (bin 1), a CTA (bin 2) or the whole grid (bin 3).
constexpr int NBINS = 4;
// Batched traversal work split: core vertices of degree <= BATCH_LANE_DEG are scanned by
// one lane each; on graphs with at least BATCH_MID_MIN_CORE core vertices, those of degree
// up to BATCH_MID_DEG are scanned 32 to a warp as one flattened sequence; longer
// adjacencies are cut into chunks of BATCH_CHUNK entries, each a work item for a warp.
constexpr int BATCH_LANE_DEG = 32;
constexpr int BATCH_MID_DEG = 128;
constexpr int64_t BATCH_MID_MIN_CORE = 1 << 19;
constexpr int BATCH_CHUNK = 2048;
// A long-row work item: entries [b, b + (meta & BATCH_ITEM_LEN)) of core vertex w's
// adjacency (a chunk of at most BATCH_CHUNK entries); meta also flags a chunk that is the
// whole row and a chunk that is the row's first.
struct BatchItem {
  int64_t b;
  int32_t w;
  uint32_t meta;
};
static_assert(sizeof(BatchItem) == 16, "one 16-byte load per item");
constexpr uint32_t BATCH_ITEM_LEN = 0xFFFFu;
constexpr uint32_t BATCH_ITEM_FIRST = 1u << 30;
constexpr uint32_t BATCH_ITEM_WHOLE = 1u << 31;

// Per-traversal control block in device memory. Kernels read the direction and buffer
// selectors from here, so the level loop can run without the host (CUDA graph with a
// device-set while condition) or with one small readback per level.
struct BfsCtl {
  int32_t level;      // level of the current frontier
  int32_t dir;        // direction of the step now due
  int32_t done;       // 1 when the frontier is empty
  int32_t cur;        // queue set holding the current frontier (0/1)
  int32_t vcur;       // visited bitmap that is current (0/1)
  int32_t need_mark;  // 1: set visited bits of the current queue before a bottom-up step
  int32_t need_queue; // 1: rebuild the current queue from the bitmaps before a top-down step
  int32_t bu_hash;    // 1: the bottom-up step may probe a shared-memory copy of the frontier
  int32_t bu_stream;  // 1: the bottom-up step streams all vertices (most are unvisited)
  int32_t bu_bloom;   // 1: ... and probes a shared-memory filter of a small frontier first
  int32_t nlevels;    // steps taken
  int64_t n_visited;  // vertices visited so far
  int64_t n_f;        // current frontier vertices
  int64_t m_f;        // their summed degree
  int64_t prev_n_f;
  int64_t m_u;        // summed degree of unvisited vertices
  int64_t bin_n[NBINS];       // current frontier, per degree bin
  int64_t next_bin_n[NBINS];  // next frontier being built, per degree bin
  int64_t next_n;             // vertices of the next frontier
  int64_t next_m;             // summed degree of the next frontier
  int64_t examined;
  int64_t ulist_n;            // bottom-up: unvisited vertices gathered this step
  // traversal start (set by the start kernel)
  int32_t start;      // start vertex in the traversed graph's ids (-1: nothing to traverse)
  int32_t start_level;
  int32_t alpha, beta, force;
  int32_t err;        // nonzero: a kernel found an inconsistency
  gt_level_info trace[MAX_TRACE];
};

// A graph the level loop traverses: the core CSR (edge-tree BFS) or the full CSR (plain).
struct View {
  int64_t n = 0;        // vertices
  int64_t nnz = 0;      // directed entries
  int64_t nwords = 0;   // bitmap words, padded to a multiple of BU_CHUNK_WORDS
  int64_t* row = nullptr;
  int32_t* col = nullptr;
  uint64_t* state = nullptr;   // packed level/parent per vertex
  uint32_t* vis[2] = {nullptr, nullptr};
  int32_t* queues = nullptr;   // 2 x NBINS queues of n entries: [set][bin][n]
  int32_t* ulist = nullptr;    // bottom-up: ascending list of unvisited vertices
  // per vertex {degree, first three neighbours in ascending order (-1 past the degree)}:
  // one sequential 16-byte read answers most bottom-up probes (null: probe the CSR only)
  int4* pre = nullptr;
  int32_t* hub = nullptr;  // per vertex its highest-degree neighbour (degree-aware bottom-up; built on first use)
  const int32_t* new2old = nullptr;  // view id -> vertex id (core view); null when ids agree
  BfsCtl* ctl = nullptr;
};

struct LaunchCfg {
  int sms = 152;
  int grid = 608;
};

// A reusable launch context of the batched traversal. The launch tables (slot
// descriptors, control words, resolution segments) are written into pinned staging memory
// and uploaded by the first node of a captured CUDA graph of the whole launch; the graph
// is kept and replayed while its shape (slots, resolution heights, grid) stays the same.
struct BatchCtx {
  void* dev = nullptr;       // device copy of the tables
  void* stage = nullptr;     // pinned host staging of the tables
  size_t cap_bytes = 0;
  int* h_err = nullptr;      // pinned status word, read back by the graph's last node
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  int key_ns = -1, key_maxh = -1, key_grid = -1, key_ogrid = -1;
  size_t key_bytes = 0;
};

}  // namespace gt

struct gt_graph {
  int device = 0;
  int64_t n = 0, m = 0, nnz = 0;
  gt_config cfg{};
  gt_tuning tuning{};
  gt_stats stats{};
  gt::LaunchCfg launch{};
  // full CSR (Sec. 5.1.1)
  int64_t* row = nullptr;
  int32_t* col = nullptr;
  int32_t* deg = nullptr;       // cleaned degree per vertex
  uint8_t* vtype = nullptr;     // Alg. 8 classes
  int32_t* up = nullptr;        // edge-tree vertex -> the neighbour it hangs from (-1 top / none)
  int32_t* vinfo = nullptr;     // >= 0 core id; -2 - k: tree vertex hanging from anchor k;
                                // INT32_MIN: tree vertex hanging from a tree vertex; -1 other
  // anchors: the core vertices that edge-tree vertices hang from, in core-id order
  int64_t n_anchor = 0;
  int32_t* anchor_cid = nullptr;  // anchor -> core id
  int32_t* anchor_vid = nullptr;  // anchor -> vertex id
  uint64_t* anchor_out = nullptr; // per traversal: (level + 1) << 32 | vertex id, for its tree children
  // batched traversal work lists over the core (built with the graph)
  int64_t n_batch_lane = 0;
  int32_t* batch_lane = nullptr;    // core vertices of degree 1..BATCH_LANE_DEG
  int64_t n_batch_mid = 0;
  int32_t* batch_mid = nullptr;     // core vertices of degree BATCH_LANE_DEG+1..BATCH_MID_DEG (large cores)
  int64_t n_batch_item = 0;
  gt::BatchItem* batch_item = nullptr;  // chunks of the longer adjacencies
  int32_t* new2old = nullptr;   // core id -> vertex id
  int32_t* old2core = nullptr;  // vertex id -> core id or -1
  int32_t* resolve_list = nullptr;  // tree vertices whose up is a tree vertex, by height desc
  int32_t* resolve_up = nullptr;
  int64_t* resolve_ptr_host = nullptr;  // segment starts per height (host copy), nheights + 1
  int32_t resolve_heights = 0;
  int64_t resolve_n = 0;
  gt::View core;   // core CSR + traversal state
  gt::View plain;  // full CSR + traversal state (keep_plain)
  int32_t* scratch_out = nullptr;  // device staging when the caller passes host outputs
  // gt_bfs_roots with host outputs: two device staging pairs (parent, level; 4n int32), the
  // stream their copies to the host run on, and events (output written / copied, per pair)
  int32_t* pipe_out = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t pipe_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t last_stream = nullptr;
  gt::BfsCtl* last_ctl = nullptr;
  // CUDA graphs of the level loop, one per view, instantiated lazily
  cudaGraphExec_t loop_exec[2] = {nullptr, nullptr};
  // step timing (time_kernels): one event pair per level, host copy of the durations
  std::vector<cudaEvent_t> step_events;
  std::vector<double> step_ms;
  cudaEvent_t phase_events[4] = {nullptr, nullptr, nullptr, nullptr};
  double phase_ms[3] = {-1.0, -1.0, -1.0};  // start, level loop, output (time_kernels)
  // batched traversal: per-slot device storage (SLOT_BUFS buffers per slot) and the slot table
  std::vector<void*> batch_mem;
  int batch_slots_alloc = 0;
  gt::BatchCtx* batch_ctx = nullptr;
  int64_t batch_work[4] = {0, 0, 0, 0};  // work counts of the last gt_bfs_batch led by this graph
  int64_t device_bytes = 0;
};

namespace gt {

// error reporting (capi.cu)
void set_error(const std::string& s);
int cuda_fail(cudaError_t e, const char* what);

// build.cu
int build_graph(gt_graph* g, const int64_t* edges, int64_t m, int64_t n, cudaStream_t s);
int alloc_view_state(gt_graph* g, View& v, cudaStream_t s);
int ensure_hub(gt_graph* g, View& v, cudaStream_t s);
void free_graph(gt_graph* g);
int device_malloc(gt_graph* g, void** p, size_t bytes);
// Allocation-failure injection (tests): the allocation after `after` more successful ones
// fails with GT_ENOMEM; after < 0 disables it.
void set_alloc_test(int after);
// Entries a column array of nnz entries is allocated with (whole 16-byte pieces).
int64_t col_alloc(int64_t nnz);

// persist.cu: a built graph to an open file and back (see gt_graph_save / gt_graph_load)
int save_graph(const gt_graph* g, FILE* f, cudaStream_t s);
int load_graph(gt_graph* g, FILE* f, cudaStream_t s);

// scan.cu
// out[i] = sum_{j < i} in[j] for i in [0, n]; out has n + 1 entries.
int scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s, void* tmp, size_t tmp_bytes);
size_t scan_tmp_bytes(int64_t n);
// as above for u8 flags -> int32 exclusive positions (n + 1 entries), total < 2^31
int scan_u8_to_i32(const uint8_t* in, int32_t* out, int64_t n, cudaStream_t s, void* tmp, size_t tmp_bytes);

// radix.cu
size_t radix_tmp_bytes(int64_t nkeys, int grid);
// LSD radix sort of u64 keys on their low `bits` bits; result ends in *keys (ping-pong with alt).
int radix_sort_u64(uint64_t** keys, uint64_t** alt, int64_t nkeys, int bits, int grid, void* tmp,
                   cudaStream_t s);

// bfs.cu
int run_bfs(gt_graph* g, View& v, bool et, int64_t root, int32_t* parent, int32_t* level, cudaStream_t s);

// batch.cu
// One lane word (up to 64 roots of one graph) of a batched launch.
struct SlotSpec {
  gt_graph* g;
  void* const* mem;         // SLOT_BUFS slot buffers from the graph's pool (ensure_slots)
  int nlanes;
  const int64_t* roots;     // nlanes roots
  int32_t* const* outp;     // nlanes parent arrays (device, n entries)
  int32_t* const* outl;     // nlanes level arrays
};

// Roots that join a running batched launch at a level boundary (serving). The host
// publishes entries and then raises `count`; at each level boundary up to `join_max` the
// launch moves published entries into free lanes of the slots that share the mailbox,
// raises `taken`, and sets `closed` once it will take no more. Lives in page-locked host
// memory mapped into the device.
// The same mailbox carries the launch's early completions: a lane whose traversal ended
// while others continue has its results written at the next level boundary, and its bit
// is then set in done[lane word].
constexpr int MAILBOX_CAP = 256;
constexpr int MAILBOX_WORDS = 256;  // lane words of one launch
struct BatchMailbox {
  int32_t count;   // host: entries published
  int32_t taken;   // device: entries admitted into lanes
  int32_t closed;  // device: 1 when no more entries will be admitted
  int32_t pad;
  struct Entry {
    int64_t root;
    int32_t* outp;    // device int32[n]
    int32_t* outl;
    int32_t lane_id;  // device: lane word * 64 + lane the entry was admitted into
    int32_t pad;
  } e[MAILBOX_CAP];
  uint64_t done[MAILBOX_WORDS];  // device: lanes whose results are in their buffers
};
int run_batch(gt_graph* const* graphs, int ngraphs, const int64_t* roots, const int32_t* roots_per_graph,
              int32_t* const* parent, int32_t* const* level, cudaStream_t s);
int ensure_slots(gt_graph* g, int need);
// A lane word's device buffers: visit, front x 2, parents, levels, frontier lists x 2,
// top-down chunk queue.
constexpr int SLOT_BUFS = 8;
void slot_sizes(const gt_graph* g, size_t sz[SLOT_BUFS]);
size_t slot_bytes(const gt_graph* g);
// Enqueues a whole batched traversal on `st` (cooperative kernel on sm_share SMs' worth of
// CTAs, 0 = all); batch_status() reads its outcome once the stream has passed it.
// mb (device address of a mapped mailbox, or null): roots may join the launch mid-flight,
// up to level boundary join_max.
int batch_launch(BatchCtx* ctx, const SlotSpec* specs, int nspecs, int sm_share, cudaStream_t st,
                 BatchMailbox* mb = nullptr, int join_max = 0);
int batch_status(const BatchCtx* ctx);
// Barrier bounds of later batched launches (failure tests): polls = 0 restores the default.
void set_barrier_test(unsigned int polls, unsigned int extra);
void batch_ctx_free(BatchCtx* c);
void free_batch_mem(gt_graph* g);

// tune.cu
int autotune(gt_graph* g, int nsample, uint64_t seed, cudaStream_t s, gt_tuning* out);

}  // namespace gt
