// bfs.cu -- direction-optimizing BFS (Alg. 1) on a CSR view, and the edge-tree steps
// around it (Alg. 9: root walk to the core, BFS_CORE, edge-tree resolution).
//
// Per-vertex state is one 64-bit word (level << 32 | parent's view id), UNVISITED = all
// ones; the output pass of the core view maps parents from core ids to vertex ids.
// Top-down (Alg. 1 TOP-DOWN): every frontier edge to a vertex that was not visited at
// the start of the level does atomicMin(state, (L+1) << 32 | v); the smallest packed
// value wins, i.e. level L+1 with the smallest frontier neighbour as parent, and the
// one thread that replaced UNVISITED enqueues the vertex. Bottom-up (Alg. 1 BOTTOM-UP,
// with the block search of Alg. 5): unvisited vertices are gathered from the visited
// bitmap in 128-bit words; each scans its ascending adjacency (the first three entries
// from a 16-byte per-vertex prefix record) and stops at the first visited neighbour
// (visited before this level means "in the frontier" for an unvisited vertex), which is
// the smallest one. Both directions therefore give the same levels and min-id parents,
// whatever the switch does.
#include <algorithm>
#include <mutex>
#include <string>

#include "gt_device.cuh"
#include "gt_internal.cuh"

namespace gt {
namespace {

constexpr int WARPS = BFS_THREADS / 32;

struct BfsArgs {
  int64_t n;
  int64_t nnz;
  int64_t nwords;
  const int64_t* row;
  const int32_t* col;
  uint64_t* state;
  uint32_t* vis0;
  uint32_t* vis1;
  int32_t* queues;  // [2][NBINS][n]
  int32_t* ulist;
  const int4* pre;         // adjacency prefix records (null: none)
  const int32_t* hub;      // highest-degree neighbours (degree-aware bottom-up; null: off)
  int32_t sms;             // SMs of the device (grid of the one-CTA-per-SM kernels)
  BfsCtl* ctl;
  int32_t td_warp_min;
  int32_t td_cta_min;
  int32_t td_grid_min;
  int32_t bu_scan;
  int32_t count_work;
};

BfsArgs make_args(const View& v, const gt_tuning& t, int sms) {
  BfsArgs a;
  a.sms = std::max(1, sms);
  a.n = v.n;
  a.nnz = v.nnz;
  a.nwords = v.nwords;
  a.row = v.row;
  a.col = v.col;
  a.state = v.state;
  a.vis0 = v.vis[0];
  a.vis1 = v.vis[1];
  a.queues = v.queues;
  a.ulist = v.ulist;
  a.pre = v.pre;
  a.hub = t.bu_hub_first ? v.hub : nullptr;
  a.ctl = v.ctl;
  a.td_warp_min = std::max(1, t.td_warp_min);
  a.td_cta_min = std::max(a.td_warp_min, t.td_cta_min);
  a.td_grid_min = std::max(a.td_cta_min, t.td_grid_min);
  a.bu_scan = std::max(0, t.bu_thread_scan);
  a.count_work = t.count_work;
  return a;
}

__device__ __forceinline__ int32_t* queue_of(const BfsArgs& a, int set, int bin) {
  return a.queues + ((int64_t)(set * NBINS + bin)) * (a.n > 0 ? a.n : 1);
}

// The state keeps parents as view ids. The core relabel is monotone, so the smallest
// core id is also the smallest vertex id, and the traversal never needs the mapping.

__device__ __forceinline__ int bin_of(const BfsArgs& a, int64_t d) {
  return d <= a.td_warp_min ? 0 : (d <= a.td_cta_min ? 1 : (d <= a.td_grid_min ? 2 : 3));
}

// Appends the lanes with `disc` set to frontier queue set `set`, each into the queue of
// its degree bin, with one atomic per non-empty bin per warp. All 32 lanes must call.
__device__ __forceinline__ void warp_enqueue(bool disc, int32_t w, int64_t wdeg, const BfsArgs& a, int set,
                                             int64_t* bin_n) {
  const unsigned bal = __ballot_sync(FULL, disc);
  if (!bal) return;
  const int lane = threadIdx.x & 31;
  const int b = disc ? bin_of(a, wdeg) : -1;
#pragma unroll
  for (int k = 0; k < NBINS; ++k) {
    const unsigned mk = __ballot_sync(FULL, b == k);
    if (!mk) continue;
    const int leader = __ffs(mk) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd((unsigned long long*)&bin_n[k], (unsigned long long)__popc(mk));
    base = __shfl_sync(FULL, base, leader);
    if (b == k) queue_of(a, set, k)[base + __popc(mk & lanemask_lt())] = w;
  }
}

// Per-warp staging of discovered vertices in shared memory: a warp collects up to STG
// vertices per degree bin and appends them to the global queue with one atomic per
// flush, instead of one same-address atomic per warp step.
constexpr int STG = 128;

struct StageQ {
  int32_t* buf;     // this warp's shared buffer, [NBINS][STG]
  int cnt[NBINS];   // entries held per bin (the same in every lane)
};

__device__ __forceinline__ void stage_flush(StageQ& sq, int k, const BfsArgs& a, int set, int64_t* bin_n) {
  const int c = sq.cnt[k];
  if (c == 0) return;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd((unsigned long long*)&bin_n[k], (unsigned long long)c);
  base = __shfl_sync(FULL, base, 0);
  __syncwarp();
  int32_t* q = queue_of(a, set, k);
  for (int i = lane; i < c; i += 32) q[base + i] = sq.buf[k * STG + i];
  __syncwarp();
  sq.cnt[k] = 0;
}

// Stages the lanes with `disc` set, each in its degree bin. All 32 lanes must call.
__device__ __forceinline__ void stage_push(StageQ& sq, bool disc, int32_t w, int64_t wdeg, const BfsArgs& a, int set,
                                           int64_t* bin_n) {
  if (!__ballot_sync(FULL, disc)) return;
  const int b = disc ? bin_of(a, wdeg) : -1;
#pragma unroll
  for (int k = 0; k < NBINS; ++k) {
    const unsigned mk = __ballot_sync(FULL, b == k);
    if (!mk) continue;
    if (sq.cnt[k] + __popc(mk) > STG) stage_flush(sq, k, a, set, bin_n);
    if (b == k) sq.buf[k * STG + sq.cnt[k] + __popc(mk & lanemask_lt())] = w;
    sq.cnt[k] += __popc(mk);
  }
  __syncwarp();
}

constexpr int TDK = 4;  // top-down edges a lane keeps in flight

// TDK frontier edges (v -> w) of one lane at once (w < 0: no edge; packed = (L+1) << 32 |
// v): the visited-bit filter (visited before this level; may lag, so only a filter), the
// state pre-check (values only decrease, so an entry already as good needs no atomic),
// the atomicMin and the degree load are each issued for all edges together, so their
// latencies overlap. disc[t]: this edge replaced "unvisited", i.e. discovered w.
__device__ __forceinline__ void td_visit_k(const BfsArgs& a, const uint32_t* vis, const int32_t (&w)[TDK],
                                           const uint64_t (&packed)[TDK], bool (&disc)[TDK],
                                           int64_t (&wd)[TDK]) {
  uint32_t vw[TDK];
#pragma unroll
  for (int t = 0; t < TDK; ++t) vw[t] = w[t] >= 0 ? vis[w[t] >> 5] : ~0u;
  bool cand[TDK];
  uint64_t st[TDK];
#pragma unroll
  for (int t = 0; t < TDK; ++t) {
    cand[t] = w[t] >= 0 && !((vw[t] >> (w[t] & 31)) & 1u);
    st[t] = cand[t] ? a.state[w[t]] : 0ull;
  }
  unsigned long long old[TDK];
#pragma unroll
  for (int t = 0; t < TDK; ++t) {
    cand[t] = cand[t] && st[t] > packed[t];
    old[t] = cand[t] ? atomicMin((unsigned long long*)&a.state[w[t]], (unsigned long long)packed[t]) : 0ull;
  }
#pragma unroll
  for (int t = 0; t < TDK; ++t) disc[t] = cand[t] && old[t] == UNVISITED;
  int64_t r0[TDK], r1[TDK];
#pragma unroll
  for (int t = 0; t < TDK; ++t) {
    r0[t] = disc[t] ? a.row[w[t]] : 0;
    r1[t] = disc[t] ? a.row[w[t] + 1] : 0;
  }
#pragma unroll
  for (int t = 0; t < TDK; ++t) wd[t] = r1[t] - r0[t];
}

// Adds per-thread counts into the control block with one atomic per CTA and counter.
// Every thread of the CTA must call.
template <int NW = WARPS>
__device__ __forceinline__ void block_commit(const BfsArgs& a, int64_t n_found, int64_t m_found, int64_t examined) {
  __shared__ int64_t red[3][NW];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  n_found = warp_sum(n_found);
  m_found = warp_sum(m_found);
  examined = warp_sum(examined);
  if (lane == 0) {
    red[0][w] = n_found;
    red[1][w] = m_found;
    red[2][w] = examined;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t x = 0, y = 0, z = 0;
    for (int i = 0; i < NW; ++i) {
      x += red[0][i];
      y += red[1][i];
      z += red[2][i];
    }
    if (x) atomicAdd((unsigned long long*)&a.ctl->next_n, (unsigned long long)x);
    if (y) atomicAdd((unsigned long long*)&a.ctl->next_m, (unsigned long long)y);
    if (z && a.count_work) atomicAdd((unsigned long long*)&a.ctl->examined, (unsigned long long)z);
  }
}

// Walks the adjacency entries [s, e) of frontier vertex v with `stride` lanes starting at
// lane offset `first`, TDK windows per step; all lanes of the warp take part in every step.
__device__ __forceinline__ void td_edges(const BfsArgs& a, uint32_t* vis, int nxt, int32_t v, uint64_t hi,
                                         int64_t s, int64_t e, int64_t first, int64_t stride, int64_t& nf,
                                         int64_t& mf, StageQ& sq) {
  const uint64_t packed = hi | (uint32_t)v;
  for (int64_t k0 = s + first; k0 < e; k0 += stride * TDK) {
    int32_t w[TDK];
    uint64_t pk[TDK];
    bool disc[TDK];
    int64_t wd[TDK];
#pragma unroll
    for (int t = 0; t < TDK; ++t) {
      const int64_t k = k0 + t * stride + (threadIdx.x & 31);
      w[t] = k < e ? a.col[k] : -1;
      pk[t] = packed;
    }
    td_visit_k(a, vis, w, pk, disc, wd);
#pragma unroll
    for (int t = 0; t < TDK; ++t) {
      if (disc[t]) {
        ++nf;
        mf += wd[t];
      }
      stage_push(sq, disc[t], w[t], wd[t], a, nxt, a.ctl->next_bin_n);
    }
  }
}

constexpr int TD_WIN = 1024;  // bin-3 vertices whose edges one window flattens

// ---- top-down ----------------------------------------------------------------------
// One launch, four phases over the four degree bins of the frontier (no grid barrier
// between them):
//  bin 3 (degree > td_grid_min): the edges of all such vertices form one flat index space
//    (per-CTA prefix sums of their degrees, in windows of TD_WIN vertices); every warp of
//    the grid takes 32 consecutive edges at a time and finds their vertex by binary
//    search, so a few hubs spread over the whole GPU;
//  bin 2: a CTA per vertex;  bin 1: a warp per vertex;
//  bin 0 (degree <= td_warp_min): a warp takes 32 vertices and its lanes share out their
//    edges (lane-to-vertex by a search over the warp's prefix sum of degrees).
__global__ void __launch_bounds__(BFS_THREADS, 4) bfs_td(BfsArgs a) {
  __shared__ int64_t s_pre[TD_WIN + 1];
  __shared__ int64_t s_beg[TD_WIN];
  __shared__ int32_t s_v[TD_WIN];
  __shared__ int64_t s_wsum[WARPS];
  __shared__ int32_t s_stage[WARPS][NBINS * STG];
  BfsCtl* ctl = a.ctl;
  const int cur = ctl->cur, nxt = cur ^ 1;
  StageQ sq;
  sq.buf = s_stage[threadIdx.x >> 5];
#pragma unroll
  for (int k = 0; k < NBINS; ++k) sq.cnt[k] = 0;
  uint32_t* vis = ctl->vcur ? a.vis1 : a.vis0;
  const uint64_t hi = (uint64_t)(uint32_t)(ctl->level + 1) << 32;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t gw = gtid() >> 5, nw = gthreads() >> 5;
  int64_t nf = 0, mf = 0, examined = 0;
  // bin 3: flattened edge space
  {
    const int32_t* q = queue_of(a, cur, 3);
    const int64_t nb = ctl->bin_n[3];
    for (int64_t ws = 0; ws < nb; ws += TD_WIN) {
      const int cnt = (int)min((int64_t)TD_WIN, nb - ws);
      // each thread owns 4 consecutive window slots; block scan of their degree sums
      int64_t d4[4], loc = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int t = threadIdx.x * 4 + k;
        d4[k] = 0;
        if (t < cnt) {
          const int32_t v = q[ws + t];
          const int64_t b = a.row[v];
          d4[k] = a.row[v + 1] - b;
          s_v[t] = v;
          s_beg[t] = b;
          if (blockIdx.x == 0) atomicOr(&vis[v >> 5], 1u << (v & 31));
        }
        loc += d4[k];
      }
      const int64_t incl = warp_incl_scan(loc);
      if (lane == 31) s_wsum[wib] = incl;
      __syncthreads();
      int64_t pre = incl - loc;
      for (int i = 0; i < wib; ++i) pre += s_wsum[i];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int t = threadIdx.x * 4 + k;
        if (t < cnt) s_pre[t] = pre;
        pre += d4[k];
      }
      if (threadIdx.x == BFS_THREADS - 1) s_pre[cnt] = pre;
      __syncthreads();
      const int64_t E = s_pre[cnt];
      if (blockIdx.x == 0 && threadIdx.x == 0) examined += E;
      for (int64_t c0 = gw * 32 * TDK; c0 < E; c0 += nw * 32 * TDK) {
        int32_t w[TDK];
        uint64_t pk[TDK];
        bool disc[TDK];
        int64_t wd[TDK];
#pragma unroll
        for (int t = 0; t < TDK; ++t) {
          const int64_t off = c0 + 32 * t + lane;
          w[t] = -1;
          pk[t] = 0;
          if (off < E) {
            int lo = 0, hi2 = cnt - 1;  // largest idx with s_pre[idx] <= off
            while (lo < hi2) {
              const int mid = (lo + hi2 + 1) >> 1;
              if (s_pre[mid] <= off) lo = mid; else hi2 = mid - 1;
            }
            w[t] = a.col[s_beg[lo] + (off - s_pre[lo])];
            pk[t] = hi | (uint32_t)s_v[lo];
          }
        }
        td_visit_k(a, vis, w, pk, disc, wd);
#pragma unroll
        for (int t = 0; t < TDK; ++t) {
          if (disc[t]) {
            ++nf;
            mf += wd[t];
          }
          stage_push(sq, disc[t], w[t], wd[t], a, nxt, ctl->next_bin_n);
        }
      }
      __syncthreads();
    }
  }
  // bin 2: a CTA per vertex
  {
    const int32_t* q = queue_of(a, cur, 2);
    const int64_t nb = ctl->bin_n[2];
    for (int64_t j = blockIdx.x; j < nb; j += gridDim.x) {
      const int32_t v = q[j];
      const int64_t s = a.row[v], e = a.row[v + 1];
      if (threadIdx.x == 0) {
        atomicOr(&vis[v >> 5], 1u << (v & 31));
        examined += e - s;
      }
      td_edges(a, vis, nxt, v, hi, s, e, (int64_t)wib * 32, (int64_t)WARPS * 32, nf, mf, sq);
    }
  }
  // bin 1: a warp per vertex
  {
    const int32_t* q = queue_of(a, cur, 1);
    const int64_t nb = ctl->bin_n[1];
    for (int64_t j = gw; j < nb; j += nw) {
      const int32_t v = q[j];
      const int64_t s = a.row[v], e = a.row[v + 1];
      if (lane == 0) {
        atomicOr(&vis[v >> 5], 1u << (v & 31));
        examined += e - s;
      }
      td_edges(a, vis, nxt, v, hi, s, e, 0, 32, nf, mf, sq);
    }
  }
  // bin 0: edges of 32 vertices packed across the warp's lanes
  {
    const int32_t* q = queue_of(a, cur, 0);
    const int64_t nb = ctl->bin_n[0];
    for (int64_t base = gw * 32; base < nb; base += nw * 32) {
      const int64_t i = base + lane;
      int32_t v = -1, vo = -1;
      int64_t rs = 0, re = 0;
      if (i < nb) {
        v = q[i];
        rs = a.row[v];
        re = a.row[v + 1];
        vo = v;
        atomicOr(&vis[v >> 5], 1u << (v & 31));
      }
      const int32_t sd = (int32_t)(re - rs);
      const int32_t incl = warp_incl_scan(sd);
      const int32_t total = __shfl_sync(FULL, incl, 31);
      const int32_t excl = incl - sd;
      if (lane == 0) examined += total;
      for (int32_t r0 = 0; r0 < total; r0 += 32 * TDK) {
        int32_t w[TDK];
        uint64_t pk[TDK];
        bool disc[TDK];
        int64_t wd[TDK];
#pragma unroll
        for (int t = 0; t < TDK; ++t) {
          const int32_t idx = r0 + 32 * t + lane;
          int owner = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int cand = owner + step;
            if (__shfl_sync(FULL, excl, cand) <= idx) owner = cand;
          }
          const int32_t ov = __shfl_sync(FULL, vo, owner);
          const int64_t ors = __shfl_sync(FULL, rs, owner);
          const int32_t oex = __shfl_sync(FULL, excl, owner);
          w[t] = idx < total ? a.col[ors + (idx - oex)] : -1;
          pk[t] = hi | (uint32_t)ov;
        }
        td_visit_k(a, vis, w, pk, disc, wd);
#pragma unroll
        for (int t = 0; t < TDK; ++t) {
          if (disc[t]) {
            ++nf;
            mf += wd[t];
          }
          stage_push(sq, disc[t], w[t], wd[t], a, nxt, ctl->next_bin_n);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NBINS; ++k) stage_flush(sq, k, a, nxt, ctl->next_bin_n);
  block_commit(a, nf, mf, examined);
}

// Sets the visited bits of the current frontier (needed before a bottom-up step that
// follows a top-down one: top-down leaves its discoveries unmarked until they expand).
__global__ void bfs_mark(BfsArgs a) {
  BfsCtl* ctl = a.ctl;
  uint32_t* vis = ctl->vcur ? a.vis1 : a.vis0;
  for (int b = 0; b < NBINS; ++b) {
    const int32_t* __restrict__ q = queue_of(a, ctl->cur, b);
    const int64_t nb = ctl->bin_n[b];
    for (int64_t i = gtid(); i < nb; i += gthreads()) {
      const int32_t v = q[i];
      atomicOr(&vis[v >> 5], 1u << (v & 31));
    }
  }
}

// Rebuilds the binned frontier queue of the current level from the two bitmaps (vertices
// visited now but not before the last bottom-up step) when top-down follows bottom-up.
// A lane takes one word; the warp enqueues round by round, each lane contributing its
// next set bit, so a sparse frontier costs one pass over the words.
__global__ void __launch_bounds__(BFS_THREADS) bfs_queue_from_bitmap(BfsArgs a) {
  BfsCtl* ctl = a.ctl;
  const uint32_t* __restrict__ vnew = ctl->vcur ? a.vis1 : a.vis0;
  const uint32_t* __restrict__ vold = ctl->vcur ? a.vis0 : a.vis1;
  const int cur = ctl->cur;
  const int lane = threadIdx.x & 31;
  const int64_t gw = gtid() >> 5, nw = gthreads() >> 5;
  for (int64_t w0 = gw * 32; w0 < a.nwords; w0 += nw * 32) {
    uint32_t f = vnew[w0 + lane] & ~vold[w0 + lane];
    while (__any_sync(FULL, f != 0)) {
      const bool has = f != 0;
      int32_t v = 0;
      int64_t d = 0;
      if (has) {
        v = (int32_t)((w0 + lane) * 32 + __ffs(f) - 1);
        f &= f - 1;
        d = a.row[v + 1] - a.row[v];
      }
      warp_enqueue(has, v, d, a, cur, ctl->bin_n);
    }
  }
}

// ---- bottom-up ---------------------------------------------------------------------
// Gather: a warp reads 128 visited words with one 128-bit load per lane, copies them to
// the next bitmap, and compacts the unvisited vertices (popc + warp sum, one reservation
// per CTA step, then one ballot per word so each word's vertices are written by
// consecutive lanes) into a global list, ascending within each CTA's span (Alg. 5's block
// search: a fully visited block costs one load). One atomic per CTA step instead of one
// per warp: the counter is a single address that every warp would otherwise queue on.
__global__ void __launch_bounds__(BFS_THREADS) bfs_bu_gather(BfsArgs a) {
  __shared__ unsigned long long s_off[WARPS];
  BfsCtl* ctl = a.ctl;
  const uint4* __restrict__ vc = reinterpret_cast<const uint4*>(ctl->vcur ? a.vis1 : a.vis0);
  uint4* __restrict__ vn = reinterpret_cast<uint4*>(ctl->vcur ? a.vis0 : a.vis1);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nchunks = a.nwords / BU_CHUNK_WORDS;
  // a CTA takes WARPS consecutive chunks per step and reserves list space for all of them
  // with one atomic, so the list stays ascending within the CTA's span
  for (int64_t c0 = (int64_t)blockIdx.x * WARPS; c0 < nchunks; c0 += (int64_t)gridDim.x * WARPS) {
    const int64_t c = c0 + wib;
    uint32_t u0 = 0, u1 = 0, u2 = 0, u3 = 0;
    if (c < nchunks) {
      const uint4 w4 = __ldg(vc + c * 32 + lane);
      vn[c * 32 + lane] = w4;
      u0 = ~w4.x;
      u1 = ~w4.y;
      u2 = ~w4.z;
      u3 = ~w4.w;
    }
    const int cnt = __popc(u0) + __popc(u1) + __popc(u2) + __popc(u3);
    const int total = warp_sum(cnt);
    if (lane == 0) s_off[wib] = (unsigned long long)total;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long run = 0;
      for (int i = 0; i < WARPS; ++i) {
        const unsigned long long t = s_off[i];
        s_off[i] = run;
        run += t;
      }
      const unsigned long long base = run ? atomicAdd((unsigned long long*)&ctl->ulist_n, run) : 0ull;
      for (int i = 0; i < WARPS; ++i) s_off[i] += base;
    }
    __syncthreads();
    unsigned long long p = s_off[wib];
    __syncthreads();  // s_off is rewritten in the next step
    if (total == 0) continue;
    unsigned lanes = __ballot_sync(FULL, cnt != 0);
    while (lanes) {
      const int j = __ffs(lanes) - 1;
      lanes &= lanes - 1;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t word = __shfl_sync(FULL, k == 0 ? u0 : k == 1 ? u1 : k == 2 ? u2 : u3, j);
        if (word == 0) continue;
        const bool bit = (word >> lane) & 1u;
        const unsigned m = __ballot_sync(FULL, bit);
        if (bit) a.ulist[p + __popc(m & lanemask_lt())] = (int32_t)((((c * 32 + j) * 4 + k) << 5) + lane);
        p += __popc(m);
      }
    }
  }
}

// Degree-aware bottom-up (Alg. 3), before the scan: every listed vertex tests its
// highest-degree neighbour; one in the frontier settles the level, and the vertex leaves
// the list with its parent left pending (HUB_PENDING): the first hit of this order is
// not the smallest frontier neighbour, which bfs_hub_parents finds after the level loop.
constexpr uint32_t HUB_PENDING = 0xFFFFFFFFu;

__global__ void __launch_bounds__(BFS_THREADS) bfs_bu_hub(BfsArgs a) {
  BfsCtl* ctl = a.ctl;
  const uint32_t* __restrict__ vc = ctl->vcur ? a.vis1 : a.vis0;
  uint32_t* vn = ctl->vcur ? a.vis0 : a.vis1;
  const uint64_t hi = (uint64_t)(uint32_t)(ctl->level + 1) << 32;
  const int64_t nu = ctl->ulist_n;
  const int lane = threadIdx.x & 31;
  int64_t nf = 0, mf = 0, examined = 0;
  for (int64_t base = gtid() & ~(int64_t)31; base < nu; base += gthreads()) {
    const int64_t i = base + lane;
    const int32_t w = i < nu ? a.ulist[i] : -1;
    bool fnd = false;
    if (w >= 0) {
      const int32_t h = a.hub[w];
      if (h >= 0) {
        ++examined;
        fnd = (__ldg(&vc[h >> 5]) >> (h & 31)) & 1u;
      }
      if (fnd) {
        a.state[w] = hi | HUB_PENDING;
        a.ulist[i] = -1;  // the scan skips it
        ++nf;
        mf += a.row[w + 1] - a.row[w];
      }
    }
    const unsigned peers = __match_any_sync(FULL, fnd ? (w >> 5) : -1);
    const unsigned bits = __reduce_or_sync(peers, fnd ? (1u << (w & 31)) : 0u);
    if (fnd && lane == __ffs(peers) - 1) atomicOr(&vn[w >> 5], bits);
  }
  block_commit(a, nf, mf, examined);
}

// Parents left pending by bfs_bu_hub: the first neighbour in ascending order one level up
// (it exists: the highest-degree neighbour is one), i.e. the smallest frontier neighbour.
__global__ void bfs_hub_parents(BfsArgs a) {
  for (int64_t v = gtid(); v < a.n; v += gthreads()) {
    const uint64_t st = a.state[v];
    if (st == UNVISITED || (uint32_t)st != HUB_PENDING) continue;
    const uint32_t lv = (uint32_t)(st >> 32);
    uint32_t p = HUB_PENDING;
    for (int64_t k = a.row[v]; k < a.row[v + 1]; ++k) {
      const int32_t u = a.col[k];
      if ((uint32_t)(a.state[u] >> 32) == lv - 1) {
        p = (uint32_t)u;
        break;
      }
    }
    a.state[v] = ((uint64_t)lv << 32) | p;
  }
}

constexpr int BU_V = 4;  // listed vertices a lane keeps in flight

__device__ __forceinline__ bool visited_bit(const uint32_t* __restrict__ vc, int32_t u) {
  return (__ldg(&vc[u >> 5]) >> (u & 31)) & 1u;
}

// Sparse-frontier variant: right after a top-down step the frontier is still in the queue;
// when it is small, every CTA copies it into a shared-memory hash set (open addressing,
// load <= 3/8) and the scan probes that set instead of the L2-resident bitmap. For an
// unvisited vertex both tests agree: its visited neighbours are exactly its frontier ones.
constexpr int HASH_SLOTS = 16384;
constexpr int HASH_CAP = 6144;

__device__ __forceinline__ uint32_t hash_slot(int32_t u) { return ((uint32_t)u * 2654435761u) >> 18; }

__device__ __forceinline__ bool hash_has(const int32_t* __restrict__ h, int32_t u) {
  for (uint32_t s = hash_slot(u);; s = (s + 1) & (HASH_SLOTS - 1)) {
    const int32_t x = h[s];
    if (x == u) return true;
    if (x < 0) return false;
  }
}

template <bool HASH>
__device__ __forceinline__ bool in_frontier(const uint32_t* __restrict__ vc, const int32_t* __restrict__ h,
                                            int32_t u) {
  if (HASH) return hash_has(h, u);
  return visited_bit(vc, u);
}

// Rows of the lanes in `lm` still open after the lane's own probes, scanned by the whole
// warp: LS rows in flight at once (each a 32-entry window per step, so LS independent
// load-and-probe chains per lane), a row that is settled (first visited neighbour in
// position order, or its end) replaced at once by the next one of `lm`. The slot
// variables are the same in every lane. A vertex found here gets its state and next-bitmap
// bit from lane 0 (or, with OWN_BIT, sets `fj` in its own lane for the caller to write the
// word); lane 0 counts the entries read.
constexpr int LS = 2;

// A filter of the current frontier in shared memory: 2^19 bits, one multiplicative hash of
// the vertex id (a Bloom filter with one hash function). A vertex whose bit is clear is
// certainly not in the frontier, so the bitmap probe in L2 is only made for the rest: the
// frontier itself and about F / 2^19 of the others (a second hash function lowered that
// share but cost more instructions than it saved: 852-855 against 863-866 GTEPS at scale 26).
constexpr int BLOOM_LOG = 19;
constexpr int BLOOM_WORDS = (1 << BLOOM_LOG) / 32;
constexpr int64_t BLOOM_MAX_FRONTIER = 65536;  // frontiers up to this size get a filter

__device__ __forceinline__ uint32_t bloom_h1(int32_t u) { return ((uint32_t)u * 0x9E3779B1u) >> (32 - BLOOM_LOG); }
__device__ __forceinline__ bool bloom_maybe(const uint32_t* bf, int32_t u) {
  const uint32_t h1 = bloom_h1(u);
  return (bf[h1 >> 5] >> (h1 & 31)) & 1u;
}

template <bool HASH, bool OWN_BIT, bool BLOOM = false>
__device__ __forceinline__ void bu_long_rows(const BfsArgs& a, const uint32_t* __restrict__ vc,
                                             const int32_t* __restrict__ s_hash, uint32_t* vn, uint64_t hi,
                                             unsigned lm, int32_t wj, int64_t limj, int64_t ej, int32_t dj, bool& fj,
                                             int64_t& nf, int64_t& mf, int64_t& examined,
                                             const uint32_t* bf = nullptr) {
  const int lane = threadIdx.x & 31;
  int32_t sw[LS], sr[LS], ss[LS];  // slot: vertex (-1 free), entries left, lane it came from
  int64_t sp[LS];                  // slot: next entry
#pragma unroll
  for (int k = 0; k < LS; ++k) {
    sw[k] = -1;
    sr[k] = ss[k] = 0;
    sp[k] = 0;
  }
  for (;;) {
    bool any = false;
#pragma unroll
    for (int k = 0; k < LS; ++k) {
      if (sw[k] < 0 && lm) {
        const int src = __ffs(lm) - 1;
        lm &= lm - 1;
        sw[k] = __shfl_sync(FULL, wj, src);
        sp[k] = __shfl_sync(FULL, limj, src);
        sr[k] = (int32_t)(__shfl_sync(FULL, ej, src) - sp[k]);
        ss[k] = src;
      }
      any |= sw[k] >= 0;
    }
    if (!any) break;
    int32_t uu[LS];
    bool hh[LS];
#pragma unroll
    for (int k = 0; k < LS; ++k) uu[k] = (sw[k] >= 0 && lane < sr[k]) ? a.col[sp[k] + lane] : -1;
#pragma unroll
    for (int k = 0; k < LS; ++k)
      hh[k] = uu[k] >= 0 && (!BLOOM || bloom_maybe(bf, uu[k])) && in_frontier<HASH>(vc, s_hash, uu[k]);
#pragma unroll
    for (int k = 0; k < LS; ++k) {
      if (sw[k] < 0) continue;
      const unsigned hm = __ballot_sync(FULL, hh[k]);
      if (hm) {
        const int32_t par = __shfl_sync(FULL, uu[k], __ffs(hm) - 1);
        if (lane == 0) {
          examined += __ffs(hm);
          a.state[sw[k]] = hi | (uint32_t)par;
          if (!OWN_BIT) atomicOr(&vn[sw[k] >> 5], 1u << (sw[k] & 31));
          ++nf;
          mf += a.row[sw[k] + 1] - a.row[sw[k]];
        }
        if (OWN_BIT && lane == ss[k]) fj = true;
        sw[k] = -1;
      } else {
        if (lane == 0) examined += min(32, sr[k]);
        sp[k] += 32;
        sr[k] -= 32;
        if (sr[k] <= 0) sw[k] = -1;
      }
    }
  }
}

// Scan: a warp takes 32 x BU_V consecutive listed vertices. With prefix records (PRE),
// each lane reads the records of its BU_V vertices (degree and first three neighbours,
// 16 bytes each, in list order) and tests all listed neighbours at once; only a vertex
// with no hit among them and a larger degree goes on into the CSR, from its fourth
// neighbour. Without records, each lane reads the row offsets and first neighbours of its
// vertices together. Either way a lane then checks up to bu_thread_scan neighbours per
// vertex alone (three of them from the record), depth by depth across its vertices, in
// ascending order, stopping at the first visited one (visited before this level = in
// the frontier, for an unvisited vertex). Vertices still open are taken over by the
// whole warp, one at a time, 32 neighbours per step, first hit by ballot. A found vertex
// records (L+1, parent) and sets its bit in the next bitmap (one atomic per distinct
// word); counts are committed once per CTA. The frontier queue is not written here: the
// next bottom-up step reads the bitmap, and a top-down step rebuilds the queue from the
// bitmaps first.
template <bool HASH, bool PRE>
__global__ void __launch_bounds__(BFS_THREADS, 4) bfs_bu_scan(BfsArgs a) {
  extern __shared__ int32_t s_hash[];
  BfsCtl* ctl = a.ctl;
  const uint32_t* __restrict__ vc = ctl->vcur ? a.vis1 : a.vis0;
  uint32_t* vn = ctl->vcur ? a.vis0 : a.vis1;
  if (HASH) {
    for (int i = threadIdx.x; i < HASH_SLOTS; i += BFS_THREADS) s_hash[i] = -1;
    __syncthreads();
    for (int b = 0; b < NBINS; ++b) {
      const int32_t* q = queue_of(a, ctl->cur, b);
      const int64_t nb = ctl->bin_n[b];
      for (int64_t i = threadIdx.x; i < nb; i += BFS_THREADS) {
        const int32_t u = q[i];
        for (uint32_t sl = hash_slot(u);; sl = (sl + 1) & (HASH_SLOTS - 1))
          if (atomicCAS(&s_hash[sl], -1, u) == -1) break;
      }
    }
    __syncthreads();
  }
  const uint64_t hi = (uint64_t)(uint32_t)(ctl->level + 1) << 32;
  const int64_t nu = ctl->ulist_n;
  const int lane = threadIdx.x & 31;
  const int64_t gw = gtid() >> 5, nw = gthreads() >> 5;
  const int64_t span = 32 * BU_V;
  const int alone = PRE ? max(a.bu_scan - 3, 0) : max(a.bu_scan, 1);  // CSR probes per lane and vertex
  int64_t nf = 0, mf = 0, examined = 0;
  for (int64_t base = gw * span; base < nu; base += nw * span) {
    int32_t w[BU_V], par[BU_V], d[BU_V];
    int64_t s[BU_V], e[BU_V];
#pragma unroll
    for (int j = 0; j < BU_V; ++j) {
      const int64_t i = base + j * 32 + lane;
      w[j] = i < nu ? a.ulist[i] : -1;
    }
    if (PRE) {
      int4 r[BU_V];
#pragma unroll
      for (int j = 0; j < BU_V; ++j) r[j] = w[j] >= 0 ? __ldg(&a.pre[w[j]]) : make_int4(0, -1, -1, -1);
      bool h0[BU_V], h1[BU_V], h2[BU_V];
      if (HASH) {
#pragma unroll
        for (int j = 0; j < BU_V; ++j) {
          h0[j] = r[j].y >= 0 && hash_has(s_hash, r[j].y);
          h1[j] = !h0[j] && r[j].z >= 0 && hash_has(s_hash, r[j].z);
          h2[j] = !h0[j] && !h1[j] && r[j].w >= 0 && hash_has(s_hash, r[j].w);
        }
      } else {
        uint32_t b0[BU_V], b1[BU_V], b2[BU_V];
#pragma unroll
        for (int j = 0; j < BU_V; ++j) {
          b0[j] = r[j].y >= 0 ? __ldg(&vc[r[j].y >> 5]) : 0u;
          b1[j] = r[j].z >= 0 ? __ldg(&vc[r[j].z >> 5]) : 0u;
          b2[j] = r[j].w >= 0 ? __ldg(&vc[r[j].w >> 5]) : 0u;
        }
#pragma unroll
        for (int j = 0; j < BU_V; ++j) {
          h0[j] = r[j].y >= 0 && ((b0[j] >> (r[j].y & 31)) & 1u);
          h1[j] = r[j].z >= 0 && ((b1[j] >> (r[j].z & 31)) & 1u);
          h2[j] = r[j].w >= 0 && ((b2[j] >> (r[j].w & 31)) & 1u);
        }
      }
#pragma unroll
      for (int j = 0; j < BU_V; ++j) {
        par[j] = h0[j] ? r[j].y : h1[j] ? r[j].z : h2[j] ? r[j].w : -1;
        d[j] = r[j].x;
        examined += h0[j] ? 1 : h1[j] ? 2 : h2[j] ? 3 : min(r[j].x, 3);
        s[j] = 0;
        e[j] = 0;
        if (w[j] >= 0 && par[j] < 0 && d[j] > 3) {
          s[j] = a.row[w[j]] + 3;
          e[j] = s[j] - 3 + d[j];
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < BU_V; ++j) {
        par[j] = -1;
        s[j] = 0;
        e[j] = 0;
        if (w[j] >= 0) {
          s[j] = a.row[w[j]];
          e[j] = a.row[w[j] + 1];
        }
        d[j] = (int32_t)(e[j] - s[j]);
      }
    }
    // probe depth by depth: at every depth the open vertices of this lane issue their
    // loads together, so BU_V dependent chains overlap
    int64_t nx[BU_V];
#pragma unroll
    for (int j = 0; j < BU_V; ++j) nx[j] = s[j];
    for (int rd = 0; rd < alone; ++rd) {
      int32_t u[BU_V];
      bool any = false;
#pragma unroll
      for (int j = 0; j < BU_V; ++j) {
        u[j] = -1;
        if (par[j] < 0 && nx[j] < e[j] && nx[j] - s[j] < alone) {
          u[j] = a.col[nx[j]];
          any = true;
        }
      }
      if (!any) break;
      if (HASH) {
#pragma unroll
        for (int j = 0; j < BU_V; ++j) {
          if (u[j] >= 0) {
            ++nx[j];
            if (hash_has(s_hash, u[j])) par[j] = u[j];
          }
        }
      } else {
        uint32_t vw[BU_V];
#pragma unroll
        for (int j = 0; j < BU_V; ++j) vw[j] = u[j] >= 0 ? __ldg(&vc[u[j] >> 5]) : 0u;
#pragma unroll
        for (int j = 0; j < BU_V; ++j) {
          if (u[j] >= 0) {
            ++nx[j];
            if ((vw[j] >> (u[j] & 31)) & 1u) par[j] = u[j];
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < BU_V; ++j) examined += nx[j] - s[j];
#pragma unroll
    for (int j = 0; j < BU_V; ++j) {
      const bool fnd = par[j] >= 0;
      if (fnd) {
        a.state[w[j]] = hi | (uint32_t)par[j];
        ++nf;
        mf += d[j];
      }
      const unsigned peers = __match_any_sync(FULL, fnd ? (w[j] >> 5) : -1);
      const unsigned bits = __reduce_or_sync(peers, fnd ? (1u << (w[j] & 31)) : 0u);
      if (fnd && lane == __ffs(peers) - 1) atomicOr(&vn[w[j] >> 5], bits);
      const int64_t lim = min(e[j], s[j] + (int64_t)alone);  // where this lane's own probes stopped
      unsigned lm = __ballot_sync(FULL, w[j] >= 0 && !fnd && lim < e[j]);
      bool unused = false;
      bu_long_rows<HASH, false>(a, vc, s_hash, vn, hi, lm, w[j], lim, e[j], d[j], unused, nf, mf, examined);
    }
  }
  block_commit(a, nf, mf, examined);
}

// Streaming bottom-up step, for a level at which most vertices are still unvisited (the
// dense middle of the traversal). Instead of gathering the unvisited vertices into a list
// and reading their records through it, each warp takes 32 x BU_V consecutive vertices
// (BU_V bitmap words) and loads their visited words and prefix records together: the
// records of consecutive vertices are consecutive, so one 512-byte coalesced load per
// word, with no list in between. Unvisited vertices then go on exactly as in the scan
// above (record probes, lane continuation, whole-warp continuation for long rows). The
// warp owns its words of the next bitmap and writes each one whole (visited bits | bits
// found), so neither the gather pass's copy nor per-word atomics are needed.
// COUNT: also count the adjacency entries read (the trace's `examined`; off in timed runs,
// where the counting would only add instructions).
// BLOOM: the step follows a top-down step with a frontier of at most BLOOM_MAX_FRONTIER
// vertices (all in the queue); every CTA first builds the frontier's filter in shared
// memory and probes the bitmap only for neighbours that pass it. For an unvisited vertex
// both tests agree, since its visited neighbours are exactly its frontier ones. One
// 1024-thread CTA per SM holds one copy of the filter, so L1 keeps most of its capacity.
template <bool COUNT, bool BLOOM, int T, int MINB>
__global__ void __launch_bounds__(T, MINB) bfs_bu_stream(BfsArgs a) {
  extern __shared__ uint32_t s_bloom[];
  BfsCtl* ctl = a.ctl;
  const uint32_t* __restrict__ vc = ctl->vcur ? a.vis1 : a.vis0;
  uint32_t* vn = ctl->vcur ? a.vis0 : a.vis1;
  if (BLOOM) {
    for (int i = threadIdx.x; i < BLOOM_WORDS; i += T) s_bloom[i] = 0u;
    __syncthreads();
    for (int b = 0; b < NBINS; ++b) {
      const int32_t* q = queue_of(a, ctl->cur, b);
      const int64_t nb = ctl->bin_n[b];
      for (int64_t i = threadIdx.x; i < nb; i += T) {
        const int32_t u = q[i];
        const uint32_t h1 = bloom_h1(u);
        atomicOr(&s_bloom[h1 >> 5], 1u << (h1 & 31));
      }
    }
    __syncthreads();
  }
  const uint32_t* bf = s_bloom;
  const uint64_t hi = (uint64_t)(uint32_t)(ctl->level + 1) << 32;
  const int lane = threadIdx.x & 31;
  const int64_t gw = gtid() >> 5, nw = gthreads() >> 5;
  const int alone = max(a.bu_scan - 3, 0);  // CSR probes per lane and vertex after the record
  int64_t nf = 0, mf = 0, examined = 0;
  for (int64_t w0 = gw * BU_V; w0 < a.nwords; w0 += nw * BU_V) {
    uint32_t vw[BU_V];
    int4 r[BU_V];  // prefix record; degree 0 for a visited vertex or one past n
#pragma unroll
    for (int j = 0; j < BU_V; ++j) {
      vw[j] = __ldg(&vc[w0 + j]);
      const int64_t v = (w0 + j) * 32 + lane;
      r[j] = v < a.n ? __ldg(&a.pre[v]) : make_int4(0, 0, 0, 0);
    }
#pragma unroll
    for (int j = 0; j < BU_V; ++j)
      if ((vw[j] >> lane) & 1u) r[j].x = 0;  // visited (padding bits past n are set)
    uint32_t b0[BU_V], b1[BU_V], b2[BU_V];
#pragma unroll
    for (int j = 0; j < BU_V; ++j) {
      b0[j] = (r[j].x > 0 && (!BLOOM || bloom_maybe(bf, r[j].y))) ? __ldg(&vc[r[j].y >> 5]) : 0u;
      b1[j] = (r[j].x > 1 && (!BLOOM || bloom_maybe(bf, r[j].z))) ? __ldg(&vc[r[j].z >> 5]) : 0u;
      b2[j] = (r[j].x > 2 && (!BLOOM || bloom_maybe(bf, r[j].w))) ? __ldg(&vc[r[j].w >> 5]) : 0u;
    }
    int32_t par[BU_V], lr[BU_V];  // parent (-1: none yet); CSR entries left to the lane
    const int32_t* cp[BU_V];       // the vertex's entries after its record
#pragma unroll
    for (int j = 0; j < BU_V; ++j) {
      const bool h0 = (b0[j] >> (r[j].y & 31)) & 1u;
      const bool h1 = (b1[j] >> (r[j].z & 31)) & 1u;
      const bool h2 = (b2[j] >> (r[j].w & 31)) & 1u;
      par[j] = h0 ? r[j].y : h1 ? r[j].z : h2 ? r[j].w : -1;
      if (COUNT) examined += h0 ? 1 : h1 ? 2 : h2 ? 3 : min(r[j].x, 3);
      const bool open = par[j] < 0 && r[j].x > 3;
      lr[j] = open ? min(r[j].x - 3, alone) : 0;
      cp[j] = open ? a.col + a.row[(w0 + j) * 32 + lane] + 3 : a.col;
    }
    // lane continuation, depth by depth: at every depth the open vertices of this lane
    // issue their loads together, so BU_V dependent chains overlap
    for (int t = 0; t < alone; ++t) {
      bool any = false;
      int32_t u[BU_V];
#pragma unroll
      for (int j = 0; j < BU_V; ++j) {
        any |= t < lr[j];
        u[j] = t < lr[j] ? cp[j][t] : 0;
      }
      if (!any) break;
      uint32_t pw[BU_V];
#pragma unroll
      for (int j = 0; j < BU_V; ++j)
        pw[j] = (t < lr[j] && (!BLOOM || bloom_maybe(bf, u[j]))) ? __ldg(&vc[u[j] >> 5]) : 0u;
#pragma unroll
      for (int j = 0; j < BU_V; ++j) {
        if (t < lr[j] && ((pw[j] >> (u[j] & 31)) & 1u)) {
          par[j] = u[j];
          if (COUNT) examined += t + 1;
          lr[j] = 0;  // settled: no more probes
        }
      }
    }
#pragma unroll
    for (int j = 0; j < BU_V; ++j) {
      const int32_t v = (int32_t)((w0 + j) * 32 + lane);
      const int32_t cnt = r[j].x - 3;  // entries after the record
      if (COUNT && par[j] < 0 && cnt > 0) examined += min(cnt, alone);
      bool fj = par[j] >= 0;
      if (fj) {
        a.state[v] = hi | (uint32_t)par[j];
        ++nf;
        mf += r[j].x;
      }
      const bool lng = !fj && cnt > alone;
      const unsigned lm = __ballot_sync(FULL, lng);
      if (lm) {
        const int64_t s0 = lng ? (int64_t)(cp[j] - a.col) : 0;
        bu_long_rows<false, true, BLOOM>(a, vc, nullptr, vn, hi, lm, v, s0 + alone, s0 + cnt, r[j].x, fj, nf,
                                         mf, examined, bf);
      }
      const unsigned fb = __ballot_sync(FULL, fj);
      if (lane == j) vn[w0 + j] = vw[j] | fb;
    }
  }
  block_commit<T / 32>(a, nf, mf, examined);
}

// ---- level control -----------------------------------------------------------------
// After each step: record the trace, swap queue sets (and bitmaps after bottom-up), and
// pick the next direction by the frontier-size rule of Beamer et al. (the paper's
// reference [12]; Alg. 1 calls it is_top_down_direction): top-down -> bottom-up when
// m_f * alpha > m_u, bottom-up -> top-down when n_f * beta < n and the frontier shrank.
__device__ __forceinline__ unsigned step_kind(const BfsCtl* c);

__global__ void bfs_decide(BfsArgs a, cudaGraphConditionalHandle h_loop, cudaGraphConditionalHandle h_dir,
                           int use_handles) {
  BfsCtl* c = a.ctl;
  if (!c->done) {
    const int L = c->level, dir = c->dir;
    const int64_t nn = c->next_n, nm = c->next_m;
    if (c->nlevels < MAX_TRACE) {
      gt_level_info& t = c->trace[c->nlevels];
      t.level = L;
      t.direction = (dir == DIR_BU && c->bu_stream) ? (c->bu_bloom ? 3 : 2) : dir;
      t.frontier = c->n_f;
      t.frontier_edges = c->m_f;
      t.unvisited_edges = c->m_u;
      t.discovered = nn;
      t.examined = a.count_work ? c->examined : -1;
      t.step_ms = -1.0;
    }
    c->nlevels += 1;
    c->m_u -= nm;
    c->prev_n_f = c->n_f;
    c->n_f = nn;
    c->m_f = nm;
    for (int b = 0; b < NBINS; ++b) {
      c->bin_n[b] = dir == DIR_TD ? c->next_bin_n[b] : 0;  // bottom-up fills no queue
      c->next_bin_n[b] = 0;
    }
    c->next_n = 0;
    c->next_m = 0;
    c->ulist_n = 0;
    c->examined = 0;
    c->cur ^= 1;
    if (dir == DIR_BU) c->vcur ^= 1;
    c->level = L + 1;
    int nd = dir;
    if (nn == 0 || c->m_u == 0) {  // no frontier, or no unvisited vertex with an edge left
      c->done = 1;
    } else if (c->force == 1) {
      nd = DIR_TD;
    } else if (c->force == 2) {
      nd = DIR_BU;
    } else if (dir == DIR_TD) {
      if (nm * (int64_t)c->alpha > c->m_u) nd = DIR_BU;
    } else {
      if (nn * (int64_t)c->beta < a.n && nn < c->prev_n_f) nd = DIR_TD;
    }
    c->need_mark = (dir == DIR_TD && nd == DIR_BU);
    c->need_queue = (dir == DIR_BU && nd == DIR_TD);
    c->bu_hash = c->need_mark && nn <= HASH_CAP;
    c->n_visited += nn;
    // stream while more than a sixth of the vertices are unvisited (measured at scale 26:
    // 1/2, 1/3, 1/4, 1/6, 1/10, always; 1/6 to 1/10 best) and records exist (the
    // degree-aware option works on the gathered list)
    c->bu_stream = a.pre && !a.hub && (a.n - c->n_visited) * 6 > a.n;
    // a small frontier right after a top-down step (it is all in the queue): filter it
    c->bu_bloom = c->bu_stream && c->need_mark && nn <= BLOOM_MAX_FRONTIER;
    c->dir = nd;
  }
  if (use_handles) {
    cudaGraphSetConditional(h_loop, c->done ? 0u : 1u);
    if (!c->done) cudaGraphSetConditional(h_dir, step_kind(c));  // routes the next iteration
  }
}

// Which step kernels run next: 0 top-down, 1 bottom-up, 2 mark + bottom-up,
// 3 queue rebuild + top-down, 4 mark + bottom-up probing a shared-memory frontier set,
// 5 streaming bottom-up, 6 mark + streaming bottom-up, 7 mark + streaming bottom-up with a
// Bloom filter of the frontier in shared memory.
__device__ __forceinline__ unsigned step_kind(const BfsCtl* c) {
  if (c->dir == DIR_TD) return c->need_queue ? 3u : 0u;
  if (c->need_mark) return c->bu_bloom ? 7u : c->bu_hash ? 4u : (c->bu_stream ? 6u : 2u);
  return c->bu_stream ? 5u : 1u;
}


// Clears the traversal state: state = UNVISITED, visited bitmap 0 except the padding
// bits past n (kept set so no scan ever takes them for unvisited vertices).
__global__ void bfs_reset(uint64_t* __restrict__ state, uint32_t* __restrict__ vis0, int64_t n, int64_t nwords) {
  const int64_t T = gthreads();
  for (int64_t i = gtid(); i < n; i += T) state[i] = UNVISITED;
  for (int64_t w = gtid(); w < nwords; w += T) {
    const int64_t first = w * 32;
    uint32_t x = 0;
    if (first + 32 <= n) x = 0;
    else if (first >= n) x = 0xFFFFFFFFu;
    else x = ~((1u << (uint32_t)(n - first)) - 1u);
    vis0[w] = x;
  }
}

// Control block for a traversal starting at vertex `start` (view ids) on level
// start_level; start < 0 means there is nothing to traverse.
__device__ void ctl_begin(const BfsArgs& a, int32_t start, int32_t start_level, int32_t alpha, int32_t beta,
                          int32_t force) {
  BfsCtl* c = a.ctl;
  c->cur = 0;
  c->vcur = 0;
  c->nlevels = 0;
  c->err = 0;
  for (int b = 0; b < NBINS; ++b) {
    c->bin_n[b] = 0;
    c->next_bin_n[b] = 0;
  }
  c->next_n = 0;
  c->next_m = 0;
  c->examined = 0;
  c->ulist_n = 0;
  c->need_queue = 0;
  c->bu_hash = 0;
  c->bu_stream = 0;
  c->bu_bloom = 0;
  c->alpha = alpha;
  c->beta = beta;
  c->force = force;
  c->start = start;
  c->start_level = start_level;
  c->level = start_level;
  c->prev_n_f = 0;
  c->need_mark = 0;
  c->dir = force == 2 ? DIR_BU : DIR_TD;
  c->n_visited = 0;
  if (start < 0) {
    c->done = 1;
    c->n_f = 0;
    c->m_f = 0;
    c->m_u = 0;
    return;
  }
  c->done = 0;
  c->n_visited = 1;
  const int64_t d = a.row[start + 1] - a.row[start];
  a.state[start] = ((uint64_t)(uint32_t)start_level << 32) | (uint32_t)start;
  a.vis0[start >> 5] |= 1u << (start & 31);
  const int b = bin_of(a, d);
  queue_of(a, 0, b)[0] = start;
  c->bin_n[b] = 1;
  c->n_f = 1;
  c->m_f = d;
  c->m_u = a.nnz - d;
}

__global__ void bfs_start_plain(BfsArgs a, int32_t root, int32_t alpha, int32_t beta, int32_t force) {
  ctl_begin(a, root, 0, alpha, beta, force);
}

struct EtArgs {
  const int32_t* vinfo;
  const int32_t* up;
  const int32_t* old2core;
  const int32_t* new2old;
  int64_t n;
  const int32_t* anchor_cid;
  const int32_t* anchor_vid;
  uint64_t* anchor_out;
  int64_t n_anchor;
};

// Alg. 9, root in an edge tree: follow up[] from the root to the first core vertex c
// (property 3: unique). The core BFS starts at c on level (hops to c); a walk that ends
// at a tree top without reaching the core leaves nothing for the core BFS.
__global__ void et_start(BfsArgs a, EtArgs e, int32_t root, int32_t alpha, int32_t beta, int32_t force) {
  const int32_t info = e.vinfo[root];
  if (info >= 0) {
    ctl_begin(a, info, 0, alpha, beta, force);
    return;
  }
  int32_t v = root, hops = 0, start = -1;
  for (int64_t guard = 0; guard < e.n; ++guard) {
    const int32_t u = e.up[v];
    if (u < 0) break;
    ++hops;
    const int32_t cu = e.old2core[u];
    if (cu >= 0) {
      start = cu;
      break;
    }
    v = u;
  }
  ctl_begin(a, start, hops, alpha, beta, force);
}

// What the tree children of each anchor (a core vertex that edge-tree vertices hang
// from) inherit: level + 1 and the anchor's vertex id, packed like the state. The
// anchors are a small set spread over the core; gathering them into one dense array
// first lets the output pass read it from L2 instead of hitting the core state at
// random once per tree vertex.
__global__ void et_anchors(EtArgs e, const uint64_t* __restrict__ state) {
  for (int64_t k = gtid(); k < e.n_anchor; k += gthreads()) {
    const uint64_t st = state[e.anchor_cid[k]];
    e.anchor_out[k] = st == UNVISITED ? UNVISITED : (((st >> 32) + 1) << 32) | (uint32_t)e.anchor_vid[k];
  }
}

// Levels and parents of every vertex in vertex-id order: core vertices from the core
// BFS state (parents there are core ids, mapped to vertex ids here), edge-tree vertices
// hanging from a core vertex from their anchor's entry (Alg. 7 / Alg. 10 with levels),
// tree vertices hanging from a tree vertex -2 ("resolve pending", see et_resolve),
// everything else -1. Four consecutive vertices per thread: one 128-bit vinfo load,
// four independent gathers, 128-bit stores (when n and the outputs allow). What streams
// through (vinfo, core state, outputs) is loaded and stored evict-first, which leaves L2
// to the id map and the anchor array that the pass gathers from.
__device__ __forceinline__ uint64_t et_packed(const EtArgs& e, const uint64_t* __restrict__ state, int32_t info) {
  if (info >= 0) return __ldcs(reinterpret_cast<const unsigned long long*>(state) + info);
  if (info != INT32_MIN && info <= -2) return e.anchor_out[-2 - info];
  return UNVISITED;
}

__device__ __forceinline__ int32_t et_parent(const EtArgs& e, uint64_t st, int32_t info) {
  return info >= 0 ? e.new2old[(uint32_t)st] : (int32_t)(uint32_t)st;
}

__global__ void et_output(EtArgs e, const uint64_t* __restrict__ state, int32_t* __restrict__ parent,
                          int32_t* __restrict__ level, int vec) {
  const int64_t n4 = vec ? e.n / 4 : 0;
  for (int64_t i = gtid(); i < n4; i += gthreads()) {
    const int4 in = __ldcs(reinterpret_cast<const int4*>(e.vinfo) + i);
    const int32_t info[4] = {in.x, in.y, in.z, in.w};
    uint64_t st[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) st[k] = et_packed(e, state, info[k]);
    int32_t l[4], p[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool r = st[k] != UNVISITED;
      l[k] = r ? (int32_t)(st[k] >> 32) : (info[k] == INT32_MIN ? -2 : -1);
      p[k] = r ? et_parent(e, st[k], info[k]) : l[k];
    }
    __stcs(reinterpret_cast<int4*>(level) + i, make_int4(l[0], l[1], l[2], l[3]));
    __stcs(reinterpret_cast<int4*>(parent) + i, make_int4(p[0], p[1], p[2], p[3]));
  }
  for (int64_t v = 4 * n4 + gtid(); v < e.n; v += gthreads()) {
    const int32_t info = e.vinfo[v];
    const uint64_t st = et_packed(e, state, info);
    const bool r = st != UNVISITED;
    const int32_t l = r ? (int32_t)(st >> 32) : (info == INT32_MIN ? -2 : -1);
    level[v] = l;
    parent[v] = r ? et_parent(e, st, info) : l;
  }
}

// Root on an edge tree: the vertices on the walk from the root to the core get their
// levels and parents from the walk (direction reversed: parent = the previous vertex),
// and the core vertex reached takes the last tree vertex as parent. Walk vertices then
// hold levels >= 0, so the resolution pass (which only fills -2 entries) leaves them.
__global__ void et_fixup(EtArgs e, int32_t root, int32_t* __restrict__ parent, int32_t* __restrict__ level) {
  if (e.vinfo[root] >= 0) return;
  level[root] = 0;
  parent[root] = root;
  int32_t v = root, k = 0;
  for (int64_t guard = 0; guard < e.n; ++guard) {
    const int32_t u = e.up[v];
    if (u < 0) break;
    if (e.old2core[u] >= 0) {
      parent[u] = v;
      break;
    }
    ++k;
    level[u] = k;
    parent[u] = v;
    v = u;
  }
}

// Tree vertices hanging from another tree vertex, one height at a time from the top:
// level = level(up) + 1 (Alg. 10 with levels), for entries still at -2.
__global__ void et_resolve(const int32_t* __restrict__ list, const int32_t* __restrict__ lup, int64_t b, int64_t e,
                           int32_t* __restrict__ parent, int32_t* __restrict__ level) {
  for (int64_t i = b + gtid(); i < e; i += gthreads()) {
    const int32_t v = list[i];
    if (level[v] != -2) continue;
    const int32_t u = lup[i];
    const int32_t lu = level[u];
    level[v] = lu >= 0 ? lu + 1 : -1;
    parent[v] = lu >= 0 ? u : -1;
  }
}

__global__ void plain_output(const uint64_t* __restrict__ state, int64_t n, int32_t* __restrict__ parent,
                             int32_t* __restrict__ level) {
  for (int64_t v = gtid(); v < n; v += gthreads()) {
    const uint64_t s = state[v];
    const bool r = s != UNVISITED;
    level[v] = r ? (int32_t)(s >> 32) : -1;
    parent[v] = r ? (int32_t)(uint32_t)s : -1;
  }
}

int grid_stream(const gt_graph* g, int64_t work) {
  int64_t want = (work + 255) / 256;
  int64_t cap = (int64_t)g->launch.sms * 8;
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

constexpr int NKINDS = 8;
constexpr size_t HASH_SMEM = sizeof(int32_t) * HASH_SLOTS;
constexpr size_t BLOOM_SMEM = sizeof(uint32_t) * BLOOM_WORDS;

// Lets the shared-memory-set variant of the scan take its 64 KB of dynamic shared memory.
int prepare_kernels() {
  int rc = cuda_fail(cudaFuncSetAttribute(bfs_bu_scan<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)HASH_SMEM),
                     "scan shared memory");
  if (rc == GT_OK)
    rc = cuda_fail(cudaFuncSetAttribute(bfs_bu_scan<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)HASH_SMEM),
                   "scan shared memory");
  if (rc == GT_OK)
    rc = cuda_fail(cudaFuncSetAttribute(bfs_bu_stream<false, true, 1024, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BLOOM_SMEM),
                   "stream shared memory");
  if (rc == GT_OK)
    rc = cuda_fail(cudaFuncSetAttribute(bfs_bu_stream<true, true, 1024, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BLOOM_SMEM),
                   "stream shared memory");
  return rc;
}

// The step kernels of one level: 0 top-down, 1 bottom-up (gather + scan), 2 mark +
// bottom-up, 3 queue rebuild + top-down, 4 mark + bottom-up with the frontier set in
// shared memory, 5 streaming bottom-up, 6 mark + streaming bottom-up, 7 mark + streaming
// bottom-up with a Bloom filter of the frontier.
void launch_step(int kind, const BfsArgs& a, int grid, cudaStream_t s) {
  if (kind == 3) bfs_queue_from_bitmap<<<grid, BFS_THREADS, 0, s>>>(a);
  if (kind == 0 || kind == 3) {
    bfs_td<<<grid, BFS_THREADS, 0, s>>>(a);
    return;
  }
  if (kind == 2 || kind == 4 || kind == 6 || kind == 7) bfs_mark<<<grid, BFS_THREADS, 0, s>>>(a);
  if (kind == 5 || kind == 6) {
    if (a.count_work)
      bfs_bu_stream<true, false, BFS_THREADS, 4><<<grid, BFS_THREADS, 0, s>>>(a);
    else
      bfs_bu_stream<false, false, BFS_THREADS, 4><<<grid, BFS_THREADS, 0, s>>>(a);
    return;
  }
  if (kind == 7) {
    if (a.count_work)
      bfs_bu_stream<true, true, 1024, 1><<<a.sms, 1024, BLOOM_SMEM, s>>>(a);
    else
      bfs_bu_stream<false, true, 1024, 1><<<a.sms, 1024, BLOOM_SMEM, s>>>(a);
    return;
  }
  bfs_bu_gather<<<grid, BFS_THREADS, 0, s>>>(a);
  if (a.hub) bfs_bu_hub<<<grid, BFS_THREADS, 0, s>>>(a);
  if (kind == 4) {
    if (a.pre)
      bfs_bu_scan<true, true><<<grid, BFS_THREADS, HASH_SMEM, s>>>(a);
    else
      bfs_bu_scan<true, false><<<grid, BFS_THREADS, HASH_SMEM, s>>>(a);
  } else {
    if (a.pre)
      bfs_bu_scan<false, true><<<grid, BFS_THREADS, 0, s>>>(a);
    else
      bfs_bu_scan<false, false><<<grid, BFS_THREADS, 0, s>>>(a);
  }
}

unsigned host_step_kind(int dir, int need_mark, int need_queue, int bu_hash, int bu_stream, int bu_bloom) {
  if (dir == DIR_TD) return need_queue ? 3u : 0u;
  if (need_mark) return bu_bloom ? 7u : bu_hash ? 4u : (bu_stream ? 6u : 2u);
  return bu_stream ? 5u : 1u;
}

// Builds the CUDA graph of the level loop for one view:
//   WHILE(loop) { SWITCH(kind) { 0: td | 1: gather, scan | 2: mark, gather, scan |
//                                3: queue, td | 4: mark, gather, scan (frontier set) } -> decide }
// Both handles are created on the top graph with a launch default (loop: 1; kind: the
// first step of a fresh traversal); decide sets them for the next iteration.
int build_loop_graph(gt_graph* g, const View& v, cudaGraphExec_t* out) {
  const BfsArgs a = make_args(v, g->tuning, g->launch.sms);
  const int grid = g->launch.grid;
  cudaGraph_t graph = nullptr;
  cudaStream_t cs = nullptr;
  int rc = GT_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    if (rc == GT_OK) rc = cuda_fail(e, what);
  };
  fail(cudaGraphCreate(&graph, 0), "graph create");
  // both handles live on the top graph and are reset at every launch: the loop runs, and
  // the first step is the one a fresh traversal starts with (top-down, or bottom-up when
  // forced); afterwards decide routes each next iteration
  const unsigned first_kind = g->tuning.force_direction == 2 ? 1u : 0u;
  cudaGraphConditionalHandle h_loop = 0, h_dir = 0;
  if (rc == GT_OK) fail(cudaGraphConditionalHandleCreate(&h_loop, graph, 1, cudaGraphCondAssignDefault), "handle");
  if (rc == GT_OK)
    fail(cudaGraphConditionalHandleCreate(&h_dir, graph, first_kind, cudaGraphCondAssignDefault), "handle");
  if (rc == GT_OK) fail(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream");
  cudaGraph_t body = nullptr;
  if (rc == GT_OK) {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h_loop;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t loop = nullptr;
    fail(cudaGraphAddNode(&loop, graph, nullptr, nullptr, 0, &np), "while node");
    if (rc == GT_OK) body = np.conditional.phGraph_out[0];
  }
  cudaGraph_t branch[NKINDS] = {};
  cudaGraphNode_t sw = nullptr;
  if (rc == GT_OK) rc = prepare_kernels();
  if (rc == GT_OK) {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h_dir;
    np.conditional.type = cudaGraphCondTypeSwitch;
    np.conditional.size = NKINDS;
    fail(cudaGraphAddNode(&sw, body, nullptr, nullptr, 0, &np), "switch node");
    if (rc == GT_OK)
      for (int i = 0; i < NKINDS; ++i) branch[i] = np.conditional.phGraph_out[i];
  }
  for (int i = 0; i < NKINDS && rc == GT_OK; ++i) {
    fail(cudaStreamBeginCaptureToGraph(cs, branch[i], nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "capture");
    if (rc != GT_OK) break;
    launch_step(i, a, grid, cs);
    cudaGraph_t got = nullptr;
    fail(cudaStreamEndCapture(cs, &got), "end capture");
  }
  if (rc == GT_OK) {
    cudaKernelNodeParams kp{};
    int use = 1;
    BfsArgs ac = a;
    void* args[] = {(void*)&ac, (void*)&h_loop, (void*)&h_dir, (void*)&use};
    kp.func = (void*)bfs_decide;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    cudaGraphNode_t dec;
    fail(cudaGraphAddKernelNode(&dec, body, &sw, 1, &kp), "decide node");
  }
  if (rc == GT_OK) fail(cudaGraphInstantiate(out, graph, 0), "instantiate");
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  return rc;
}

int run_level_loop(gt_graph* g, View& v, int which, cudaStream_t s) {
  const gt_tuning& t = g->tuning;
  g->step_ms.clear();
  if (t.launch_mode == 0) {
    if (!g->loop_exec[which]) {
      int rc = build_loop_graph(g, v, &g->loop_exec[which]);
      if (rc != GT_OK) return rc;
    }
    return cuda_fail(cudaGraphLaunch(g->loop_exec[which], s), "graph launch");
  }
  // host-driven: one small readback per level
  const BfsArgs a = make_args(v, t, g->launch.sms);
  const int grid = g->launch.grid;
  struct Head {
    int32_t level, dir, done, cur, vcur, need_mark, need_queue, bu_hash, bu_stream, bu_bloom;
  } h{};
  const cudaGraphConditionalHandle none = 0;
  int timed_steps = 0;
  g->step_ms.clear();
  int rc0 = prepare_kernels();
  if (rc0 != GT_OK) return rc0;
  for (int guard = 0; guard < (1 << 30); ++guard) {
    int rc = cuda_fail(cudaMemcpyAsync(&h, v.ctl, sizeof(h), cudaMemcpyDeviceToHost, s), "ctl readback");
    if (rc == GT_OK) rc = cuda_fail(cudaStreamSynchronize(s), "level sync");
    if (rc != GT_OK) return rc;
    if (h.done) break;
    const bool timed = t.time_kernels && guard < MAX_TRACE;
    if (timed) {
      while ((int)g->step_events.size() < 2 * (guard + 1)) {
        cudaEvent_t ev;
        rc = cuda_fail(cudaEventCreate(&ev), "event create");
        if (rc != GT_OK) return rc;
        g->step_events.push_back(ev);
      }
      cudaEventRecord(g->step_events[2 * guard], s);
    }
    launch_step((int)host_step_kind(h.dir, h.need_mark, h.need_queue, h.bu_hash, h.bu_stream, h.bu_bloom), a, grid, s);
    if (timed) {
      cudaEventRecord(g->step_events[2 * guard + 1], s);
      ++timed_steps;
    }
    bfs_decide<<<1, 1, 0, s>>>(a, none, none, 0);
    rc = cuda_fail(cudaGetLastError(), "level launch");
    if (rc != GT_OK) return rc;
  }
  for (int i = 0; i < timed_steps; ++i) {
    float ms = -1.f;
    if (cudaEventElapsedTime(&ms, g->step_events[2 * i], g->step_events[2 * i + 1]) != cudaSuccess) {
      cudaGetLastError();
      ms = -1.f;
    }
    g->step_ms.push_back(ms);
  }
  return GT_OK;
}

}  // namespace

int run_bfs(gt_graph* g, View& v, bool et, int64_t root, int32_t* parent, int32_t* level, cudaStream_t s) {
  const gt_tuning& t = g->tuning;
  if (t.bu_hub_first) {
    const int rc0 = ensure_hub(g, v, s);
    if (rc0 != GT_OK) return rc0;
  }
  const BfsArgs a = make_args(v, t, g->launch.sms);
  const bool timed = t.time_kernels;
  if (timed && !g->phase_events[0])
    for (int i = 0; i < 4; ++i) cudaEventCreate(&g->phase_events[i]);
  if (timed) cudaEventRecord(g->phase_events[0], s);
  const int gs = grid_stream(g, std::max<int64_t>(v.n, v.nwords));
  bfs_reset<<<gs, 256, 0, s>>>(v.state, v.vis[0], v.n, v.nwords);
  EtArgs e{g->vinfo, g->up, g->old2core, g->new2old, g->n, g->anchor_cid, g->anchor_vid, g->anchor_out, g->n_anchor};
  if (et)
    et_start<<<1, 1, 0, s>>>(a, e, (int32_t)root, t.alpha, t.beta, t.force_direction);
  else
    bfs_start_plain<<<1, 1, 0, s>>>(a, (int32_t)root, t.alpha, t.beta, t.force_direction);
  int rc = cuda_fail(cudaGetLastError(), "bfs start");
  if (rc != GT_OK) return rc;
  if (timed) cudaEventRecord(g->phase_events[1], s);
  rc = run_level_loop(g, v, et ? 0 : 1, s);
  if (rc != GT_OK) return rc;
  if (timed) cudaEventRecord(g->phase_events[2], s);
  if (a.hub) bfs_hub_parents<<<grid_stream(g, v.n), 256, 0, s>>>(a);
  if (et) {
    const int go = grid_stream(g, g->n);
    const int vec = ((uintptr_t)parent % 16 == 0) && ((uintptr_t)level % 16 == 0);
    if (g->n_anchor > 0) et_anchors<<<grid_stream(g, g->n_anchor), 256, 0, s>>>(e, v.state);
    et_output<<<go, 256, 0, s>>>(e, v.state, parent, level, vec);
    et_fixup<<<1, 1, 0, s>>>(e, (int32_t)root, parent, level);
    for (int h = 0; h < g->resolve_heights; ++h) {
      const int64_t b = g->resolve_ptr_host[h], en = g->resolve_ptr_host[h + 1];
      if (en > b)
        et_resolve<<<grid_stream(g, en - b), 256, 0, s>>>(g->resolve_list, g->resolve_up, b, en, parent, level);
    }
  } else {
    plain_output<<<grid_stream(g, v.n), 256, 0, s>>>(v.state, v.n, parent, level);
  }
  g->last_stream = s;
  g->last_ctl = v.ctl;
  rc = cuda_fail(cudaGetLastError(), "bfs output");
  if (timed && rc == GT_OK) {
    cudaEventRecord(g->phase_events[3], s);
    rc = cuda_fail(cudaEventSynchronize(g->phase_events[3]), "timing sync");
    for (int i = 0; i < 3 && rc == GT_OK; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, g->phase_events[i], g->phase_events[i + 1]);
      g->phase_ms[i] = ms;
    }
  }
  return rc;
}

// ---- Traversal that allocates nothing ------------------------------------------------------
// Some callers cannot allocate device memory when they need a traversal: a service that
// fixes its memory plan at start-up and forbids allocation on the request path (an
// allocation can block, synchronise the device, or fail once memory is fragmented), or a
// plug-in running inside a host framework that owns all device memory and hands the
// plug-in only its inputs and outputs. gt_bfs_csr_noalloc serves them: the plain
// direction-optimizing traversal of a caller's device CSR, with every piece of scratch
// (per-vertex state, visited bitmaps, frontier queues, control block) carved from the one
// file-scope array below. That array is reserved on each device when the library's code
// is loaded there and stays reserved until the process exits.
constexpr int64_t NOALLOC_MAX_N = int64_t(1) << 18;       // largest graph: 262,144 vertices
constexpr int64_t NOALLOC_WORDS = NOALLOC_MAX_N / 32;     // a multiple of BU_CHUNK_WORDS
constexpr size_t NOALLOC_CTL_BYTES = (sizeof(BfsCtl) + 255) & ~size_t(255);
constexpr size_t NOALLOC_BYTES = NOALLOC_CTL_BYTES + 8 * NOALLOC_MAX_N          // state
                                 + 2 * 4 * NOALLOC_WORDS                        // two bitmaps
                                 + 4 * NOALLOC_MAX_N * 2 * NBINS                // queue sets
                                 + 4 * NOALLOC_MAX_N;                           // unvisited list
static_assert(NOALLOC_WORDS % BU_CHUNK_WORDS == 0, "bitmap words must fill whole chunks");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device. Host code cannot use the
// array's name as an address (it names a host-side shadow), so the address is looked up
// once per device with that device current and cached.
int noalloc_scratch(void** out) {
  int dev = 0;
  int rc = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    set_error("gt_bfs_csr_noalloc: device index beyond the supported range");
    return GT_ENOTSUP;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    rc = cuda_fail(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress of the traversal scratch");
    if (rc) return rc;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return GT_OK;
}

// True for memory of device `dev` (device or managed); memory of another GPU is refused,
// since the kernels would reach it without peer access.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace
}  // namespace gt

extern "C" GT_API int gt_bfs_csr_noalloc(const int64_t* row, const int32_t* col, int64_t n, int64_t root,
                                         int32_t* parent, int32_t* level, void* stream) {
  using namespace gt;
  if (!row || !col || !parent || !level || n < 1 || root < 0 || root >= n) {
    set_error("gt_bfs_csr_noalloc: null pointer, n < 1 or root outside [0, n)");
    return GT_EINVAL;
  }
  if (n > NOALLOC_MAX_N) {
    set_error("gt_bfs_csr_noalloc: n = " + std::to_string(n) + " exceeds the fixed scratch capacity of " +
              std::to_string(NOALLOC_MAX_N) + " vertices");
    return GT_EINVAL;
  }
  int dev = 0, sms = 1;
  int rc = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (!on_device(row, dev) || !on_device(col, dev) || !on_device(parent, dev) || !on_device(level, dev)) {
    set_error("gt_bfs_csr_noalloc: row, col, parent and level must be memory of the current device");
    return GT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  void* base = nullptr;
  rc = noalloc_scratch(&base);
  if (rc) return rc;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t nnz = 0;
  rc = cuda_fail(cudaMemcpyAsync(&nnz, row + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "read nnz");
  if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "sync");
  if (rc) return rc;
  // carve the views of one traversal out of the array
  unsigned char* p = (unsigned char*)base;
  View v;
  v.n = n;
  v.nnz = nnz;
  v.nwords = ((n + 31) / 32 + BU_CHUNK_WORDS - 1) / BU_CHUNK_WORDS * BU_CHUNK_WORDS;
  v.row = const_cast<int64_t*>(row);
  v.col = const_cast<int32_t*>(col);
  v.ctl = (BfsCtl*)p;
  p += NOALLOC_CTL_BYTES;
  v.state = (uint64_t*)p;
  p += 8 * NOALLOC_MAX_N;
  v.vis[0] = (uint32_t*)p;
  p += 4 * NOALLOC_WORDS;
  v.vis[1] = (uint32_t*)p;
  p += 4 * NOALLOC_WORDS;
  v.queues = (int32_t*)p;
  p += 4 * NOALLOC_MAX_N * 2 * NBINS;
  v.ulist = (int32_t*)p;
  gt_tuning t;
  gt_tuning_default(&t);
  const BfsArgs a = make_args(v, t, sms);
  const int grid = sms * std::max(1, t.blocks_per_sm);
  // state and the first bitmap start cleared; the control block is rewritten by the start
  // kernel; queue and list entries are only read below the counts the kernels set
  bfs_reset<<<std::max(1, (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8)), 256, 0, s>>>(
      v.state, v.vis[0], v.n, v.nwords);
  bfs_start_plain<<<1, 1, 0, s>>>(a, (int32_t)root, t.alpha, t.beta, 0);
  struct Head {
    int32_t level, dir, done, cur, vcur, need_mark, need_queue;
  } h{};
  for (int64_t guard = 0; guard <= n + 1; ++guard) {  // at most one step per level
    rc = cuda_fail(cudaMemcpyAsync(&h, v.ctl, sizeof(h), cudaMemcpyDeviceToHost, s), "ctl readback");
    if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "level sync");
    if (rc) return rc;
    if (h.done) break;
    // step kinds 0-3 only: kind 4 (frontier set in shared memory) needs the kernel
    // attribute that prepare_kernels sets, which this path leaves alone
    launch_step(h.dir == DIR_TD ? (h.need_queue ? 3 : 0) : (h.need_mark ? 2 : 1), a, grid, s);
    bfs_decide<<<1, 1, 0, s>>>(a, 0, 0, 0);
    rc = cuda_fail(cudaGetLastError(), "level launch");
    if (rc) return rc;
  }
  if (!h.done) {  // a BFS has at most n levels; a loop that ran past them found an inconsistency
    set_error("gt_bfs_csr_noalloc: level loop passed n + 2 steps without finishing");
    return GT_EDEVICE;
  }
  plain_output<<<std::max(1, (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8)), 256, 0, s>>>(
      v.state, v.n, parent, level);
  return cuda_fail(cudaGetLastError(), "noalloc output");
}
