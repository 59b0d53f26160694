// build.cu -- graph build: CSR (Sec. 5.1.1), edge-tree classification (Alg. 8),
// monotone core relabel + core CSR (core-left layout, Sec. 5.1.1) and the edge-tree
// edge list (Sec. 5.1.2). Runs once per graph; not part of the timed traversal.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "gt_device.cuh"
#include "gt_internal.cuh"

namespace gt {
namespace {

constexpr int BT = 256;
constexpr int32_t UNPEELED = 0x7FFFFFFF;
constexpr int32_t NOT_TREE = -2;  // peel round of a zero-degree vertex

int grid_for(const gt_graph* g, int64_t work, int per_thread = 1) {
  int64_t want = (work + (int64_t)BT * per_thread - 1) / ((int64_t)BT * per_thread);
  int64_t cap = (int64_t)g->launch.sms * 16;
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

// ---- a1: keys, sort, dedupe, row offsets -------------------------------------------

__global__ void keygen(const int64_t* __restrict__ edges, int64_t m, int64_t n, int b, uint64_t sent,
                       uint64_t* __restrict__ keys, int* __restrict__ err) {
  for (int64_t i = gtid(); i < m; i += gthreads()) {
    const longlong2 e = reinterpret_cast<const longlong2*>(edges)[i];
    const int64_t u = e.x, v = e.y;
    if (u < 0 || u >= n || v < 0 || v >= n) {
      atomicOr(err, 1);
      keys[2 * i] = sent;
      keys[2 * i + 1] = sent;
      continue;
    }
    if (u == v) {
      keys[2 * i] = sent;
      keys[2 * i + 1] = sent;
    } else {
      keys[2 * i] = ((uint64_t)u << b) | (uint64_t)v;
      keys[2 * i + 1] = ((uint64_t)v << b) | (uint64_t)u;
    }
  }
}

constexpr int UT = 256, UI = 16, UTILE = UT * UI;

__device__ __forceinline__ bool uniq_flag(const uint64_t* keys, int64_t j, int64_t K, uint64_t sent) {
  if (j >= K) return false;
  const uint64_t k = keys[j];
  return k != sent && (j == 0 || keys[j - 1] != k);
}

__global__ void __launch_bounds__(UT) uniq_count(const uint64_t* __restrict__ keys, int64_t K, uint64_t sent,
                                                 int32_t* __restrict__ tilecnt) {
  __shared__ int32_t ws[UT / 32];
  const int64_t base = (int64_t)blockIdx.x * UTILE;
  int32_t c = 0;
  for (int i = threadIdx.x; i < UTILE; i += UT) c += uniq_flag(keys, base + i, K, sent);
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int w = 0; w < UT / 32; ++w) t += ws[w];
    tilecnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(UT) uniq_write(const uint64_t* __restrict__ keys, int64_t K, uint64_t sent, int b,
                                                 const int64_t* __restrict__ tileoff, int32_t* __restrict__ col,
                                                 int32_t* __restrict__ deg) {
  __shared__ int32_t ws[UT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * UTILE + w * (UI * 32);
  int32_t ex[UI];
  int32_t run = 0;
  unsigned fl = 0;
#pragma unroll
  for (int j = 0; j < UI; ++j) {
    const bool f = uniq_flag(keys, base + j * 32 + lane, K, sent);
    const unsigned bal = __ballot_sync(FULL, f);
    ex[j] = run + __popc(bal & lanemask_lt());
    run += __popc(bal);
    fl |= (unsigned)f << j;
  }
  if (lane == 0) ws[w] = run;
  __syncthreads();
  int64_t pre = tileoff[blockIdx.x];
  for (int i = 0; i < w; ++i) pre += ws[i];
  const uint64_t vmask = (1ull << b) - 1;
#pragma unroll
  for (int j = 0; j < UI; ++j) {
    const bool f = (fl >> j) & 1;
    uint64_t k = 0;
    if (f) {
      k = keys[base + j * 32 + lane];
      col[pre + ex[j]] = (int32_t)(k & vmask);
    }
    // degree count, aggregated over lanes with the same source (keys are sorted)
    const uint32_t u = f ? (uint32_t)(k >> b) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(FULL, u);
    if (f && lane == __ffs(peers) - 1) atomicAdd(&deg[u], __popc(peers));
  }
}

// ---- a2: Alg. 8 -------------------------------------------------------------------

__global__ void peel_init(const int64_t* __restrict__ row, int64_t n, int32_t* __restrict__ deg,
                          int32_t* __restrict__ res, uint8_t* __restrict__ vtype, int32_t* __restrict__ round,
                          int32_t* __restrict__ up) {
  for (int64_t v = gtid(); v < n; v += gthreads()) {
    const int32_t d = (int32_t)(row[v + 1] - row[v]);
    deg[v] = d;
    res[v] = d;
    up[v] = -1;
    vtype[v] = d == 0 ? GT_VERTEX_ZERO : (d == 1 ? GT_TREE_LEAF : GT_CORE_INTERNAL);
    round[v] = d == 0 ? NOT_TREE : (d == 1 ? 0 : UNPEELED);
  }
}

// Height 0: every degree-1 vertex is a leaf and hangs from its one neighbour. Two
// adjacent leaves (a K2 component): the smaller id is the tree's top.
__global__ void peel_leaves(const int64_t* __restrict__ row, const int32_t* __restrict__ col, int64_t n,
                            const int32_t* __restrict__ deg, int32_t* __restrict__ res, int32_t* __restrict__ up) {
  for (int64_t v = gtid(); v < n; v += gthreads()) {
    if (deg[v] != 1) continue;
    const int32_t w = col[row[v]];
    if (deg[w] == 1) {
      up[v] = v < w ? -1 : w;
    } else {
      up[v] = w;
      atomicSub(&res[w], 1);
    }
  }
}

// Height r >= 1 (Jacobi: reads the counts as they stood when the height began). A
// vertex still in the core whose count is 0 or 1 becomes tree-internal; it hangs from
// its one remaining neighbour, unless that neighbour is peeled at the same height too
// (then the smaller id is the top), and has no up at count 0.
__global__ void peel_height(const int64_t* __restrict__ row, const int32_t* __restrict__ col, int64_t n, int32_t r,
                            const int32_t* __restrict__ pre, int32_t* __restrict__ res, uint8_t* __restrict__ vtype,
                            int32_t* __restrict__ round, int32_t* __restrict__ up,
                            unsigned long long* __restrict__ peeled) {
  for (int64_t v = gtid(); v < n; v += gthreads()) {
    if (round[v] != UNPEELED || pre[v] > 1) continue;
    int32_t w = -1;
    if (pre[v] == 1) {
      for (int64_t e = row[v]; e < row[v + 1]; ++e) {
        const int32_t x = col[e];
        // not peeled before height r: round is UNPEELED, or r if it is being peeled now
        if (*(volatile int32_t*)&round[x] >= r) {
          w = x;
          break;
        }
      }
    }
    if (w >= 0) {
      if (pre[w] <= 1) {
        up[v] = v < w ? -1 : w;
      } else {
        up[v] = w;
        atomicSub(&res[w], 1);
      }
    } else {
      up[v] = -1;
    }
    round[v] = r;
    vtype[v] = GT_TREE_INTERNAL;
    atomicAdd(peeled, 1ull);
  }
}

__global__ void peel_finish(int64_t n, const int32_t* __restrict__ deg, const int32_t* __restrict__ res,
                            uint8_t* __restrict__ vtype, const int32_t* __restrict__ round,
                            uint8_t* __restrict__ is_core, unsigned long long* __restrict__ cls) {
  __shared__ unsigned long long h[5];
  if (threadIdx.x < 5) h[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t v = gtid(); v < n; v += gthreads()) {
    uint8_t t = vtype[v];
    if (round[v] == UNPEELED) {
      t = res[v] != deg[v] ? GT_CORE_EDGE : GT_CORE_INTERNAL;
      vtype[v] = t;
    }
    is_core[v] = t <= GT_CORE_EDGE;
    atomicAdd(&h[t], 1ull);
  }
  __syncthreads();
  if (threadIdx.x < 5) atomicAdd(&cls[threadIdx.x], h[threadIdx.x]);
}

// ---- a3: monotone core relabel + core CSR -------------------------------------------

__global__ void relabel(int64_t n, const uint8_t* __restrict__ is_core, const int32_t* __restrict__ pos,
                        int32_t* __restrict__ old2core, int32_t* __restrict__ new2old) {
  for (int64_t v = gtid(); v < n; v += gthreads()) {
    if (is_core[v]) {
      old2core[v] = pos[v];
      new2old[pos[v]] = (int32_t)v;
    } else {
      old2core[v] = -1;
    }
  }
}

__global__ void core_degree(const int64_t* __restrict__ row, const int32_t* __restrict__ col,
                            const uint8_t* __restrict__ is_core, const int32_t* __restrict__ new2old, int64_t nc,
                            int32_t* __restrict__ cdeg) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = gtid() >> 5, nw = gthreads() >> 5;
  for (int64_t c = wid; c < nc; c += nw) {
    const int32_t v = new2old[c];
    int32_t cnt = 0;
    for (int64_t e = row[v] + lane; e < row[v + 1]; e += 32) cnt += is_core[col[e]];
    cnt = warp_sum(cnt);
    if (lane == 0) cdeg[c] = cnt;
  }
}

__global__ void core_fill(const int64_t* __restrict__ row, const int32_t* __restrict__ col,
                          const uint8_t* __restrict__ is_core, const int32_t* __restrict__ new2old,
                          const int32_t* __restrict__ old2core, int64_t nc, const int64_t* __restrict__ crow,
                          int32_t* __restrict__ ccol) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = gtid() >> 5, nw = gthreads() >> 5;
  for (int64_t c = wid; c < nc; c += nw) {
    const int32_t v = new2old[c];
    int64_t out = crow[c];
    const int64_t b = row[v], e = row[v + 1];
    for (int64_t k0 = b; k0 < e; k0 += 32) {
      const int64_t k = k0 + lane;
      int32_t w = -1;
      bool keep = false;
      if (k < e) {
        w = col[k];
        keep = is_core[w];
      }
      const unsigned bal = __ballot_sync(FULL, keep);
      if (keep) ccol[out + __popc(bal & lanemask_lt())] = old2core[w];
      out += __popc(bal);
    }
  }
}

// ---- a4: edge-tree layout -----------------------------------------------------------

// Anchors: core vertices that some edge-tree vertex hangs from (up[] is a core vertex).
__global__ void mark_anchors(int64_t n, const uint8_t* __restrict__ vtype, const int32_t* __restrict__ up,
                             const int32_t* __restrict__ old2core, uint8_t* __restrict__ aflag) {
  for (int64_t v = gtid(); v < n; v += gthreads()) {
    const uint8_t t = vtype[v];
    if (t != GT_TREE_LEAF && t != GT_TREE_INTERNAL) continue;
    const int32_t u = up[v];
    if (u < 0) continue;
    const int32_t cu = old2core[u];
    if (cu >= 0) aflag[cu] = 1;
  }
}

__global__ void list_anchors(int64_t nc, const uint8_t* __restrict__ aflag, const int32_t* __restrict__ apos,
                             const int32_t* __restrict__ new2old, int32_t* __restrict__ anchor_cid,
                             int32_t* __restrict__ anchor_vid) {
  for (int64_t c = gtid(); c < nc; c += gthreads()) {
    if (!aflag[c]) continue;
    anchor_cid[apos[c]] = (int32_t)c;
    anchor_vid[apos[c]] = new2old[c];
  }
}

// Work lists of the batched traversal: short adjacencies one per lane, medium ones (large
// cores only: mid_max > BATCH_LANE_DEG) 32 to a warp, long ones in chunks.
__global__ void batch_work_count(int64_t nc, const int64_t* __restrict__ crow, int mid_max,
                                 uint8_t* __restrict__ short_flag, uint8_t* __restrict__ mid_flag,
                                 int32_t* __restrict__ nchunks) {
  for (int64_t v = gtid(); v < nc; v += gthreads()) {
    const int64_t d = crow[v + 1] - crow[v];
    short_flag[v] = d > 0 && d <= BATCH_LANE_DEG;
    mid_flag[v] = d > BATCH_LANE_DEG && d <= mid_max;
    nchunks[v] = d > mid_max ? (int32_t)((d + BATCH_CHUNK - 1) / BATCH_CHUNK) : 0;
  }
}

__global__ void batch_work_fill(int64_t nc, const int64_t* __restrict__ crow, const uint8_t* __restrict__ short_flag,
                                const int32_t* __restrict__ lpos, const uint8_t* __restrict__ mid_flag,
                                const int32_t* __restrict__ mpos, const int32_t* __restrict__ nchunks,
                                const int64_t* __restrict__ ipos, int32_t* __restrict__ lanes,
                                int32_t* __restrict__ mids, BatchItem* __restrict__ items) {
  for (int64_t v = gtid(); v < nc; v += gthreads()) {
    if (short_flag[v]) lanes[lpos[v]] = (int32_t)v;
    if (mid_flag[v]) mids[mpos[v]] = (int32_t)v;
    const int32_t nch = nchunks[v];
    const int64_t rb = crow[v], re = crow[v + 1];
    for (int32_t c = 0; c < nch; ++c) {
      BatchItem it;
      it.b = rb + (int64_t)c * BATCH_CHUNK;
      it.w = (int32_t)v;
      it.meta = (uint32_t)min((int64_t)BATCH_CHUNK, re - it.b) | (c == 0 ? BATCH_ITEM_FIRST : 0u) |
                (nch == 1 ? BATCH_ITEM_WHOLE : 0u);
      items[ipos[v] + c] = it;
    }
  }
}

// vinfo: core id for core vertices; -2 - (anchor index of up) for tree vertices hanging
// from a core vertex; INT32_MIN for tree vertices hanging from another tree vertex
// (resolved height by height, listed through rflag); -1 for the rest (zero-degree
// vertices, tops).
__global__ void tree_info(int64_t n, const uint8_t* __restrict__ vtype, const int32_t* __restrict__ up,
                          const int32_t* __restrict__ old2core, const int32_t* __restrict__ apos,
                          int32_t* __restrict__ vinfo, uint8_t* __restrict__ rflag) {
  for (int64_t v = gtid(); v < n; v += gthreads()) {
    const uint8_t t = vtype[v];
    int32_t info = -1;
    uint8_t f = 0;
    if (t <= GT_CORE_EDGE) {
      info = old2core[v];
    } else if (t == GT_TREE_LEAF || t == GT_TREE_INTERNAL) {
      const int32_t u = up[v];
      if (u >= 0) {
        const int32_t cu = old2core[u];
        if (cu >= 0) {
          info = -2 - apos[cu];
        } else {
          info = INT32_MIN;
          f = 1;
        }
      }
    }
    vinfo[v] = info;
    rflag[v] = f;
  }
}

__global__ void resolve_keys(int64_t n, const uint8_t* __restrict__ rflag, const int32_t* __restrict__ pos,
                             const int32_t* __restrict__ round, int32_t maxr, uint64_t* __restrict__ keys,
                             unsigned long long* __restrict__ per_round) {
  for (int64_t v = gtid(); v < n; v += gthreads()) {
    if (!rflag[v]) continue;
    const int32_t r = round[v];
    keys[pos[v]] = ((uint64_t)(maxr - r) << 31) | (uint64_t)v;
    atomicAdd(&per_round[maxr - r], 1ull);
  }
}

__global__ void resolve_split(int64_t k, const uint64_t* __restrict__ keys, const int32_t* __restrict__ up,
                              int32_t* __restrict__ list, int32_t* __restrict__ lup) {
  for (int64_t i = gtid(); i < k; i += gthreads()) {
    const int32_t v = (int32_t)(keys[i] & 0x7FFFFFFFull);
    list[i] = v;
    lup[i] = up[v];
  }
}

__global__ void reduce_max_i32(int64_t n, const int32_t* __restrict__ a, const uint8_t* __restrict__ mask,
                               int* __restrict__ out) {
  int m = -1;
  for (int64_t v = gtid(); v < n; v += gthreads())
    if (mask[v]) m = max(m, a[v]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void class_hist(int64_t n, const uint8_t* vtype, unsigned long long* h) {
  __shared__ unsigned long long s[5];
  if (threadIdx.x < 5) s[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t v = gtid(); v < n; v += gthreads()) atomicAdd(&s[vtype[v]], 1ull);
  __syncthreads();
  if (threadIdx.x < 5) atomicAdd(&h[threadIdx.x], s[threadIdx.x]);
}


int bits_for(int64_t n) {
  int b = 1;
  while ((1ll << b) < n) ++b;
  return b;
}

}  // namespace

// Column arrays are allocated in whole 16-byte pieces (the entries past nnz are never
// used), so a kernel may read them as aligned vectors.
int64_t col_alloc(int64_t nnz) { return (std::max<int64_t>(nnz, 1) + 3) / 4 * 4; }

// Allocation-failure injection for tests (gt_test_fail_alloc): once `after` more graph
// allocations have succeeded, the next one fails as if device memory had run out.
std::atomic<int> g_fail_after{-1};

static bool injected_alloc_failure() {
  int k = g_fail_after.load();
  while (k >= 0) {
    if (g_fail_after.compare_exchange_weak(k, k - 1)) return k == 0;
  }
  return false;
}

void set_alloc_test(int after) { g_fail_after.store(after < 0 ? -1 : after); }

int device_malloc(gt_graph* g, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (injected_alloc_failure()) {
    *p = nullptr;
    set_error("device allocation failed (injected by gt_test_fail_alloc)");
    return GT_ENOMEM;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    return GT_ENOMEM;
  }
  g->device_bytes += (int64_t)bytes;
  return GT_OK;
}

// Adjacency prefix records of a view: {degree, col[row[v]], col[row[v] + 1], col[row[v] + 2]},
// -1 where the degree ends first.
static __global__ void build_prefix(const int64_t* __restrict__ row, const int32_t* __restrict__ col, int64_t n,
                             int4* __restrict__ pre) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = row[v], d = row[v + 1] - b;
    pre[v] = make_int4((int32_t)d, d > 0 ? col[b] : -1, d > 1 ? col[b + 1] : -1, d > 2 ? col[b + 2] : -1);
  }
}

// Highest-degree neighbour of every vertex of a view (ties: the smaller id, the first met
// in the ascending row); -1 for an empty row. The probe order of the degree-aware bottom-up
// step (Alg. 3).
static __global__ void build_hub(const int64_t* __restrict__ row, const int32_t* __restrict__ col, int64_t n,
                                 int32_t* __restrict__ hub) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int32_t best = -1;
    int64_t bd = -1;
    for (int64_t k = row[v]; k < row[v + 1]; ++k) {
      const int32_t u = col[k];
      const int64_t d = row[u + 1] - row[u];
      if (d > bd) {
        bd = d;
        best = u;
      }
    }
    hub[v] = best;
  }
}

int ensure_hub(gt_graph* g, View& v, cudaStream_t s) {
  if (v.hub || v.n <= 0) return GT_OK;
  int rc = device_malloc(g, (void**)&v.hub, sizeof(int32_t) * v.n);
  if (rc) return rc;
  build_hub<<<grid_for(g, v.n), BT, 0, s>>>(v.row, v.col, v.n, v.hub);
  return cuda_fail(cudaGetLastError(), "hub neighbours");
}

int alloc_view_state(gt_graph* g, View& v, cudaStream_t s) {
  const int64_t n = v.n > 0 ? v.n : 1;
  v.nwords = (n + 31) / 32;
  v.nwords = (v.nwords + BU_CHUNK_WORDS - 1) / BU_CHUNK_WORDS * BU_CHUNK_WORDS;
  int rc;
  if ((rc = device_malloc(g, (void**)&v.state, sizeof(uint64_t) * n))) return rc;
  for (int i = 0; i < 2; ++i)
    if ((rc = device_malloc(g, (void**)&v.vis[i], sizeof(uint32_t) * v.nwords))) return rc;
  if ((rc = device_malloc(g, (void**)&v.queues, sizeof(int32_t) * n * 2 * NBINS))) return rc;
  if ((rc = device_malloc(g, (void**)&v.ulist, sizeof(int32_t) * n))) return rc;
  if ((rc = device_malloc(g, (void**)&v.ctl, sizeof(BfsCtl)))) return rc;
  if ((rc = device_malloc(g, (void**)&v.pre, sizeof(int4) * n))) return rc;
  if (v.n > 0) build_prefix<<<grid_for(g, v.n), BT, 0, s>>>(v.row, v.col, v.n, v.pre);
  return cuda_fail(cudaGetLastError(), "prefix records");
}

static void free_view(View& v) {
  cudaFree(v.state);
  for (int i = 0; i < 2; ++i) cudaFree(v.vis[i]);
  cudaFree(v.queues);
  cudaFree(v.ulist);
  cudaFree(v.ctl);
  cudaFree(v.pre);
  cudaFree(v.hub);
  v = View{};
}

void free_graph(gt_graph* g) {
  for (int i = 0; i < 2; ++i)
    if (g->loop_exec[i]) cudaGraphExecDestroy(g->loop_exec[i]);
  for (cudaEvent_t ev : g->step_events) cudaEventDestroy(ev);
  for (cudaEvent_t& ev : g->phase_events)
    if (ev) cudaEventDestroy(ev);
  g->step_events.clear();
  if (g->core.row != g->row) {
    cudaFree(g->core.row);
    cudaFree(g->core.col);
  }
  free_view(g->core);
  free_view(g->plain);
  cudaFree(g->row);
  cudaFree(g->col);
  cudaFree(g->deg);
  cudaFree(g->vtype);
  cudaFree(g->up);
  cudaFree(g->vinfo);
  cudaFree(g->anchor_cid);
  cudaFree(g->anchor_vid);
  cudaFree(g->anchor_out);
  cudaFree(g->batch_lane);
  cudaFree(g->batch_mid);
  cudaFree(g->batch_item);
  cudaFree(g->new2old);
  cudaFree(g->old2core);
  free_batch_mem(g);
  if (g->batch_ctx) {
    batch_ctx_free(g->batch_ctx);
    delete g->batch_ctx;
    g->batch_ctx = nullptr;
  }
  cudaFree(g->resolve_list);
  cudaFree(g->resolve_up);
  cudaFree(g->scratch_out);
  cudaFree(g->pipe_out);
  g->pipe_out = nullptr;
  if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
  g->copy_stream = nullptr;
  for (cudaEvent_t& e : g->pipe_ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  delete[] g->resolve_ptr_host;
  g->resolve_ptr_host = nullptr;
}

// Frees a set of temporaries on scope exit.
struct Temps {
  std::vector<void*> p;
  void* add(void* x) {
    p.push_back(x);
    return x;
  }
  ~Temps() {
    for (void* x : p) cudaFree(x);
  }
};

static int tmp_malloc(Temps& t, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (injected_alloc_failure()) {
    *p = nullptr;
    set_error("device allocation failed (build temporary; injected by gt_test_fail_alloc)");
    return GT_ENOMEM;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes (build temporary) failed");
    return GT_ENOMEM;
  }
  t.add(*p);
  return GT_OK;
}

#define TRY(x)                 \
  do {                         \
    int rc__ = (x);            \
    if (rc__ != GT_OK) return rc__; \
  } while (0)
#define TRYC(x, what) TRY(cuda_fail((x), what))

int build_graph(gt_graph* g, const int64_t* edges, int64_t m, int64_t n, cudaStream_t s) {
  Temps tmp;
  g->n = n;
  g->m = m;
  const int grid_sort = g->launch.sms * 4;

  // ---- input tuples on the device
  const int64_t* d_edges = edges;
  cudaPointerAttributes attr{};
  cudaError_t pe = cudaPointerGetAttributes(&attr, edges);
  if (pe != cudaSuccess) cudaGetLastError();
  const bool on_device = pe == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
  if (!on_device && m > 0) {
    void* p;
    TRY(tmp_malloc(tmp, &p, sizeof(int64_t) * 2 * m));
    TRYC(cudaMemcpyAsync(p, edges, sizeof(int64_t) * 2 * m, cudaMemcpyHostToDevice, s), "copy tuples");
    d_edges = (const int64_t*)p;
  } else if (m > 0 && ((uintptr_t)edges & 15)) {
    set_error("device tuple array must be 16-byte aligned");
    return GT_EINVAL;
  }

  const int b = bits_for(n);
  const uint64_t sent = (b >= 32) ? ~0ull : ((1ull << (2 * b)) - 1);
  const int64_t K = 2 * m;
  int* d_err;
  TRY(tmp_malloc(tmp, (void**)&d_err, sizeof(int) * 4));
  TRYC(cudaMemsetAsync(d_err, 0, sizeof(int) * 4, s), "memset");

  // ---- a1: CSR
  TRY(device_malloc(g, (void**)&g->row, sizeof(int64_t) * (n + 1)));
  TRY(device_malloc(g, (void**)&g->deg, sizeof(int32_t) * n));
  TRYC(cudaMemsetAsync(g->deg, 0, sizeof(int32_t) * n, s), "memset");
  int64_t nnz = 0;
  size_t scan_bytes = std::max(scan_tmp_bytes(n + 1), scan_tmp_bytes(K + 1)) + 1024;
  void* d_scan;
  TRY(tmp_malloc(tmp, &d_scan, scan_bytes));
  if (K > 0) {
    uint64_t *keys, *alt;
    TRY(tmp_malloc(tmp, (void**)&keys, sizeof(uint64_t) * K));
    TRY(tmp_malloc(tmp, (void**)&alt, sizeof(uint64_t) * K));
    keygen<<<grid_for(g, m), BT, 0, s>>>(d_edges, m, n, b, sent, keys, d_err);
    TRYC(cudaGetLastError(), "keygen");
    void* d_radix;
    TRY(tmp_malloc(tmp, &d_radix, radix_tmp_bytes(K, grid_sort)));
    TRY(radix_sort_u64(&keys, &alt, K, 2 * b, grid_sort, d_radix, s));
    const int64_t nt = (K + UTILE - 1) / UTILE;
    int32_t* tilecnt;
    int64_t* tileoff;
    TRY(tmp_malloc(tmp, (void**)&tilecnt, sizeof(int32_t) * nt));
    TRY(tmp_malloc(tmp, (void**)&tileoff, sizeof(int64_t) * (nt + 1)));
    uniq_count<<<(unsigned)nt, UT, 0, s>>>(keys, K, sent, tilecnt);
    TRY(scan_i32_to_i64(tilecnt, tileoff, nt, s, d_scan, scan_bytes));
    TRYC(cudaMemcpyAsync(&nnz, tileoff + nt, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "readback");
    int h_err = 0;
    TRYC(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "readback");
    TRYC(cudaStreamSynchronize(s), "build sync");
    if (h_err) {
      set_error("gt_graph_build: a tuple has a vertex id outside [0, n)");
      return GT_EINVAL;
    }
    TRY(device_malloc(g, (void**)&g->col, sizeof(int32_t) * col_alloc(nnz)));
    uniq_write<<<(unsigned)nt, UT, 0, s>>>(keys, K, sent, b, tileoff, g->col, g->deg);
    TRYC(cudaGetLastError(), "uniq_write");
    // keys are freed with the temporaries
  } else {
    TRY(device_malloc(g, (void**)&g->col, sizeof(int32_t) * col_alloc(0)));
  }
  g->nnz = nnz;
  TRY(scan_i32_to_i64(g->deg, g->row, n, s, d_scan, scan_bytes));

  // ---- a2: Alg. 8
  int32_t *res, *pre, *round;
  uint8_t* is_core;
  TRY(tmp_malloc(tmp, (void**)&res, sizeof(int32_t) * n));
  TRY(tmp_malloc(tmp, (void**)&pre, sizeof(int32_t) * n));
  TRY(tmp_malloc(tmp, (void**)&round, sizeof(int32_t) * n));
  TRY(tmp_malloc(tmp, (void**)&is_core, n));
  TRY(device_malloc(g, (void**)&g->vtype, n));
  TRY(device_malloc(g, (void**)&g->up, sizeof(int32_t) * n));
  unsigned long long* d_cnt;
  TRY(tmp_malloc(tmp, (void**)&d_cnt, sizeof(unsigned long long) * 16));
  TRYC(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * 16, s), "memset");
  const int gn = grid_for(g, n);
  peel_init<<<gn, BT, 0, s>>>(g->row, n, g->deg, res, g->vtype, round, g->up);
  peel_leaves<<<gn, BT, 0, s>>>(g->row, g->col, n, g->deg, res, g->up);
  TRYC(cudaGetLastError(), "peel leaves");
  // Alg. 8 keeps going while the previous height marked something; height 0 marked the
  // leaves, so the height loop starts only if some vertex has degree 1.
  int32_t height = 0;
  const int mh = g->cfg.mh;
  bool prev_marked;
  {
    unsigned long long h[5] = {0, 0, 0, 0, 0};
    unsigned long long* d_h = d_cnt + 8;
    TRYC(cudaMemsetAsync(d_h, 0, sizeof(unsigned long long) * 5, s), "memset");
    class_hist<<<gn, BT, 0, s>>>(n, g->vtype, d_h);
    TRYC(cudaMemcpyAsync(h, d_h, sizeof(h), cudaMemcpyDeviceToHost, s), "readback");
    TRYC(cudaStreamSynchronize(s), "sync");
    prev_marked = h[GT_TREE_LEAF] > 0;
  }
  for (int32_t r = 1; prev_marked && (mh == -1 || r <= mh); ++r) {
    TRYC(cudaMemcpyAsync(pre, res, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s), "copy counts");
    TRYC(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), s), "memset");
    peel_height<<<gn, BT, 0, s>>>(g->row, g->col, n, r, pre, res, g->vtype, round, g->up, d_cnt);
    unsigned long long peeled = 0;
    TRYC(cudaMemcpyAsync(&peeled, d_cnt, sizeof(peeled), cudaMemcpyDeviceToHost, s), "readback");
    TRYC(cudaStreamSynchronize(s), "sync");
    prev_marked = peeled > 0;
    if (prev_marked) height = r;
  }
  TRYC(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * 16, s), "memset");
  peel_finish<<<gn, BT, 0, s>>>(n, g->deg, res, g->vtype, round, is_core, d_cnt);
  unsigned long long cls[5];
  TRYC(cudaMemcpyAsync(cls, d_cnt, sizeof(cls), cudaMemcpyDeviceToHost, s), "readback");

  // ---- a3: relabel + core CSR
  int32_t* pos;
  TRY(tmp_malloc(tmp, (void**)&pos, sizeof(int32_t) * (n + 1)));
  TRY(scan_u8_to_i32(is_core, pos, n, s, d_scan, scan_bytes));
  int32_t nc32 = 0;
  TRYC(cudaMemcpyAsync(&nc32, pos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "readback");
  TRYC(cudaStreamSynchronize(s), "sync");
  const int64_t nc = nc32;
  TRY(device_malloc(g, (void**)&g->old2core, sizeof(int32_t) * n));
  TRY(device_malloc(g, (void**)&g->new2old, sizeof(int32_t) * std::max<int64_t>(nc, 1)));
  relabel<<<gn, BT, 0, s>>>(n, is_core, pos, g->old2core, g->new2old);
  int32_t* cdeg;
  TRY(tmp_malloc(tmp, (void**)&cdeg, sizeof(int32_t) * std::max<int64_t>(nc, 1)));
  View& cv = g->core;
  cv.n = nc;
  cv.new2old = g->new2old;
  TRY(device_malloc(g, (void**)&cv.row, sizeof(int64_t) * (nc + 1)));
  const int gw = grid_for(g, nc * 32);
  if (nc > 0) core_degree<<<gw, BT, 0, s>>>(g->row, g->col, is_core, g->new2old, nc, cdeg);
  TRY(scan_i32_to_i64(cdeg, cv.row, nc, s, d_scan, scan_bytes));
  TRYC(cudaMemcpyAsync(&cv.nnz, cv.row + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "readback");
  TRYC(cudaStreamSynchronize(s), "sync");
  TRY(device_malloc(g, (void**)&cv.col, sizeof(int32_t) * col_alloc(cv.nnz)));
  if (nc > 0) core_fill<<<gw, BT, 0, s>>>(g->row, g->col, is_core, g->new2old, g->old2core, nc, cv.row, cv.col);
  TRYC(cudaGetLastError(), "core csr");

  // ---- batched traversal work lists
  {
    uint8_t *sflag, *mflag;
    int32_t *lpos, *mpos, *nch;
    int64_t* ipos;
    const int64_t nc1 = std::max<int64_t>(nc, 1);
    TRY(tmp_malloc(tmp, (void**)&sflag, nc1));
    TRY(tmp_malloc(tmp, (void**)&mflag, nc1));
    TRY(tmp_malloc(tmp, (void**)&lpos, sizeof(int32_t) * (nc + 1)));
    TRY(tmp_malloc(tmp, (void**)&mpos, sizeof(int32_t) * (nc + 1)));
    TRY(tmp_malloc(tmp, (void**)&nch, sizeof(int32_t) * nc1));
    TRY(tmp_malloc(tmp, (void**)&ipos, sizeof(int64_t) * (nc + 1)));
    // medium list on large cores only: on small ones the flattened scan's serial steps
    // cost more than one warp per vertex (measured at R-MAT scales 16-24)
    const int mid_max = nc >= BATCH_MID_MIN_CORE ? BATCH_MID_DEG : BATCH_LANE_DEG;
    if (nc > 0) batch_work_count<<<grid_for(g, nc), BT, 0, s>>>(nc, cv.row, mid_max, sflag, mflag, nch);
    TRY(scan_u8_to_i32(sflag, lpos, nc, s, d_scan, scan_bytes));
    TRY(scan_u8_to_i32(mflag, mpos, nc, s, d_scan, scan_bytes));
    TRY(scan_i32_to_i64(nch, ipos, nc, s, d_scan, scan_bytes));
    int32_t nl = 0, nm = 0;
    int64_t ni = 0;
    TRYC(cudaMemcpyAsync(&nl, lpos + nc, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "readback");
    TRYC(cudaMemcpyAsync(&nm, mpos + nc, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "readback");
    TRYC(cudaMemcpyAsync(&ni, ipos + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "readback");
    TRYC(cudaStreamSynchronize(s), "sync");
    g->n_batch_lane = nl;
    g->n_batch_mid = nm;
    g->n_batch_item = ni;
    TRY(device_malloc(g, (void**)&g->batch_lane, sizeof(int32_t) * std::max<int64_t>(nl, 1)));
    TRY(device_malloc(g, (void**)&g->batch_mid, sizeof(int32_t) * std::max<int64_t>(nm, 1)));
    TRY(device_malloc(g, (void**)&g->batch_item, sizeof(BatchItem) * std::max<int64_t>(ni, 1)));
    if (nc > 0)
      batch_work_fill<<<grid_for(g, nc), BT, 0, s>>>(nc, cv.row, sflag, lpos, mflag, mpos, nch, ipos,
                                                     g->batch_lane, g->batch_mid, g->batch_item);
    TRYC(cudaGetLastError(), "batch work lists");
  }

  // ---- a4: anchors and tree layout
  uint8_t* aflag;
  int32_t* apos;
  TRY(tmp_malloc(tmp, (void**)&aflag, std::max<int64_t>(nc, 1)));
  TRY(tmp_malloc(tmp, (void**)&apos, sizeof(int32_t) * (nc + 1)));
  TRYC(cudaMemsetAsync(aflag, 0, std::max<int64_t>(nc, 1), s), "memset");
  mark_anchors<<<gn, BT, 0, s>>>(n, g->vtype, g->up, g->old2core, aflag);
  TRY(scan_u8_to_i32(aflag, apos, nc, s, d_scan, scan_bytes));
  int32_t na32 = 0;
  TRYC(cudaMemcpyAsync(&na32, apos + nc, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "readback");
  TRYC(cudaStreamSynchronize(s), "sync");
  g->n_anchor = na32;
  TRY(device_malloc(g, (void**)&g->anchor_cid, sizeof(int32_t) * std::max<int64_t>(na32, 1)));
  TRY(device_malloc(g, (void**)&g->anchor_vid, sizeof(int32_t) * std::max<int64_t>(na32, 1)));
  TRY(device_malloc(g, (void**)&g->anchor_out, sizeof(uint64_t) * std::max<int64_t>(na32, 1)));
  if (nc > 0) list_anchors<<<grid_for(g, nc), BT, 0, s>>>(nc, aflag, apos, g->new2old, g->anchor_cid, g->anchor_vid);
  TRY(device_malloc(g, (void**)&g->vinfo, sizeof(int32_t) * n));
  uint8_t* rflag = is_core;  // is_core is consumed; reuse its storage
  tree_info<<<gn, BT, 0, s>>>(n, g->vtype, g->up, g->old2core, apos, g->vinfo, rflag);
  TRY(scan_u8_to_i32(rflag, pos, n, s, d_scan, scan_bytes));
  int32_t nres = 0;
  TRYC(cudaMemcpyAsync(&nres, pos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "readback");
  int* d_maxr = d_err + 1;
  TRYC(cudaMemsetAsync(d_maxr, 0xFF, sizeof(int), s), "memset");
  reduce_max_i32<<<gn, BT, 0, s>>>(n, round, rflag, d_maxr);
  int maxr = -1;
  TRYC(cudaMemcpyAsync(&maxr, d_maxr, sizeof(int), cudaMemcpyDeviceToHost, s), "readback");
  TRYC(cudaStreamSynchronize(s), "sync");
  g->resolve_n = nres;
  if (nres > 0) {
    const int nh = maxr + 1;
    uint64_t *rk, *rk_alt;
    unsigned long long* per_round;
    TRY(tmp_malloc(tmp, (void**)&rk, sizeof(uint64_t) * nres));
    TRY(tmp_malloc(tmp, (void**)&rk_alt, sizeof(uint64_t) * nres));
    TRY(tmp_malloc(tmp, (void**)&per_round, sizeof(unsigned long long) * nh));
    TRYC(cudaMemsetAsync(per_round, 0, sizeof(unsigned long long) * nh, s), "memset");
    resolve_keys<<<gn, BT, 0, s>>>(n, rflag, pos, round, maxr, rk, per_round);
    void* d_radix2;
    TRY(tmp_malloc(tmp, &d_radix2, radix_tmp_bytes(nres, grid_sort)));
    TRY(radix_sort_u64(&rk, &rk_alt, nres, 31 + bits_for(nh + 1), grid_sort, d_radix2, s));
    TRY(device_malloc(g, (void**)&g->resolve_list, sizeof(int32_t) * nres));
    TRY(device_malloc(g, (void**)&g->resolve_up, sizeof(int32_t) * nres));
    resolve_split<<<grid_for(g, nres), BT, 0, s>>>(nres, rk, g->up, g->resolve_list, g->resolve_up);
    std::vector<unsigned long long> cnt(nh);
    TRYC(cudaMemcpyAsync(cnt.data(), per_round, sizeof(unsigned long long) * nh, cudaMemcpyDeviceToHost, s),
         "readback");
    TRYC(cudaStreamSynchronize(s), "sync");
    g->resolve_heights = nh;
    g->resolve_ptr_host = new int64_t[nh + 1];
    g->resolve_ptr_host[0] = 0;
    for (int i = 0; i < nh; ++i) g->resolve_ptr_host[i + 1] = g->resolve_ptr_host[i] + (int64_t)cnt[i];
  }

  // ---- traversal state
  TRY(alloc_view_state(g, cv, s));
  if (g->cfg.keep_plain) {
    View& pv = g->plain;
    pv.n = n;
    pv.nnz = nnz;
    pv.row = g->row;
    pv.col = g->col;
    TRY(alloc_view_state(g, pv, s));
  }
  TRYC(cudaStreamSynchronize(s), "build sync");

  gt_stats& st = g->stats;
  memset(&st, 0, sizeof(st));
  st.n = n;
  st.m = m;
  st.nnz = nnz;
  st.n_core = nc;
  st.nnz_core = cv.nnz;
  for (int i = 0; i < 5; ++i) st.n_class[i] = (int64_t)cls[i];
  st.mh = g->cfg.mh;
  st.height = height;
  st.device_bytes = g->device_bytes;
  return GT_OK;
}

}  // namespace gt
