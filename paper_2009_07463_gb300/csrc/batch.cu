// batch.cu -- many single-root edge-tree BFS at once (multi-source BFS over lane words).
//
// Roots are packed 64 to a "slot": one uint64 lane word per core vertex holds, for each
// of the slot's roots, whether the vertex is visited (visit), in the current frontier
// (front) or in the next one. Every adjacency read then serves all 64 roots. All slots
// of all graphs advance level by level inside ONE persistent cooperative launch; grid
// barriers separate the three phases of a level:
//   E  expand   top-down slots push front bits along frontier edges (atomicOr) and list
//               each newly reached vertex once; bottom-up slots pull: every vertex still
//               missing some lanes scans its ascending adjacency, the first neighbour
//               carrying a lane's frontier bit is that lane's parent (so min-id).
//   P  commit   for vertices reached top-down, one ascending scan assigns each lane its
//               smallest frontier neighbour; every reached lane gets its level; visit |=.
//   D  decide   clear the old frontier words, swap, pick the next direction per slot.
// Per lane the levels and parents equal those of a single-root gt_bfs (Alg. 9): each
// lane is an ordinary BFS from its root's core vertex, levels are shared iterations, and
// parents are the smallest frontier neighbour by construction. Per-vertex results are
// staged vertex-major (parent int32[64], level uint16[64] per core vertex) and written
// to the callers' root-major arrays by one coalesced pass that also resolves the edge
// trees (Alg. 10 / Alg. 7).
//
// Every wait at a grid barrier is bounded; on timeout the kernel raises an error flag
// and all CTAs return, and the call reports GT_ETIMEOUT.
#include <string.h>

#include <algorithm>
#include <vector>

#include "gt_device.cuh"
#include "gt_internal.cuh"

namespace gt {
namespace {

constexpr int BT = 256;
constexpr int BW = BT / 32;
constexpr int MAX_SLOTS_SMEM = 256;
// Neighbours a lane scans alone (two dependent loads each) before its warp continues the
// scan 32 entries per step; multi-source scans rarely stop early, so most of the work is
// best done by the coalesced warp-wide path.
constexpr int THREAD_SCAN = 4;

struct LaneInit {
  int32_t start;    // core id the lane's BFS starts from (-1: nothing to traverse)
  int32_t base;     // level of the start vertex (hops from the root)
  int32_t sparent;  // parent (vertex id) of the start vertex
  int32_t root;
};

struct SlotDev {
  // graph
  int64_t n, nc, nnz_core;
  const int64_t* crow;
  const int32_t* ccol;
  const int32_t* vinfo;
  const int32_t* new2old;
  const int32_t* anchor_cid;  // anchor -> core id (tree vertices name their anchor in vinfo)
  const int32_t* anchor_vid;  // anchor -> vertex id
  const int32_t* up;
  const int32_t* old2core;
  // state (core ids)
  uint64_t* visit;
  uint64_t* front[2];
  int32_t* P;   // [nc][64] parent vertex ids
  uint16_t* L;  // [nc][64] iteration at which the lane reached the vertex
  int32_t* fl[2];
  // outputs: lane l writes parent / level arrays outp[l] / outl[l] (n entries each)
  int32_t* outp[64];
  int32_t* outl[64];
  int32_t nlanes;
  int32_t alpha, beta;
  int32_t pad;
  uint64_t active;
  LaneInit lane[64];
};

struct SlotCtl {
  int64_t fl_n[2];
  int64_t m_next;  // summed degree of the next frontier
  int32_t cur, dir, done, iter;
};

struct BatchCtl {
  unsigned int bar;  // grid barrier arrivals
  int err;
  int live;          // slots not done
  int pad;
};

__device__ __forceinline__ int64_t deg(const SlotDev& s, int32_t v) { return s.crow[v + 1] - s.crow[v]; }

// Grid-wide barrier for a cooperative launch: arrivals counted on one word, each CTA
// waits for its generation's total. Bounded: after ~2^26 polls (seconds) it raises err.
__device__ bool grid_barrier(BatchCtl* bc, unsigned int& gen) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    ++gen;
    const unsigned int target = gen * gridDim.x;
    __threadfence();
    atomicAdd(&bc->bar, 1u);
    int ok = 1;
    unsigned int spins = 0;
    while (ld_relaxed_u32(&bc->bar) < target) {
      if (*(volatile int*)&bc->err) {
        ok = 0;
        break;
      }
      if (++spins > (1u << 26)) {
        atomicExch(&bc->err, 1);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok;
}

__device__ __forceinline__ void set_lane_levels(const SlotDev& s, int32_t w, uint64_t lanes, uint16_t it) {
  uint16_t* row = s.L + (int64_t)w * 64;
  while (lanes) {
    const int l = __ffsll((long long)lanes) - 1;
    lanes &= lanes - 1;
    row[l] = it;
  }
}

// Ascending scan of w's adjacency assigning, for each lane of `want`, the first
// neighbour whose frontier word carries that lane. One thread. Returns the lanes found.
__device__ __forceinline__ uint64_t first_hits_thread(const SlotDev& s, const uint64_t* __restrict__ fc, int32_t w,
                                                      uint64_t want, int64_t b, int64_t e, int64_t* stop) {
  uint64_t got = 0;
  int32_t* prow = s.P + (int64_t)w * 64;
  int64_t k = b;
  for (; k < e && got != want; ++k) {
    const int32_t u = s.ccol[k];
    uint64_t h = fc[u] & want & ~got;
    if (h) {
      got |= h;
      const int32_t uo = s.new2old[u];
      while (h) {
        const int l = __ffsll((long long)h) - 1;
        h &= h - 1;
        prow[l] = uo;
      }
    }
  }
  *stop = k;
  return got;
}

// Warp-cooperative continuation of the same scan from entry b: 32 neighbours per step;
// an exclusive OR-scan over lanes gives each neighbour the lanes it hits first.
__device__ __forceinline__ uint64_t first_hits_warp(const SlotDev& s, const uint64_t* __restrict__ fc, int32_t w,
                                                    uint64_t want, uint64_t got, int64_t b, int64_t e) {
  const int lane = threadIdx.x & 31;
  int32_t* prow = s.P + (int64_t)w * 64;
  for (int64_t k0 = b; k0 < e && got != want; k0 += 32) {
    const int64_t k = k0 + lane;
    int32_t u = -1;
    uint64_t h = 0;
    if (k < e) {
      u = s.ccol[k];
      h = fc[u] & want & ~got;
    }
    uint64_t before = h;  // inclusive OR-scan, then exclude own
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(FULL, before, o);
      if (lane >= o) before |= y;
    }
    const uint64_t excl = __shfl_up_sync(FULL, before, 1);
    const uint64_t mine = h & ~(lane ? excl : 0ull);
    if (mine) {
      const int32_t uo = s.new2old[u];
      uint64_t x = mine;
      while (x) {
        const int l = __ffsll((long long)x) - 1;
        x &= x - 1;
        prow[l] = uo;
      }
    }
    got |= __shfl_sync(FULL, before, 31);
  }
  return got;
}

__global__ void batch_init(SlotDev* slots, SlotCtl* sctl, int nslots) {
  // one thread per (slot, lane): walk the root to its core vertex (Alg. 9) and seed it
  const int sidx = blockIdx.x;
  if (sidx >= nslots) return;
  SlotDev& s = slots[sidx];
  const int l = threadIdx.x;
  if (l < s.nlanes) {
    const LaneInit& li = s.lane[l];
    if (li.start >= 0) {
      const uint64_t bit = 1ull << l;
      atomicOr((unsigned long long*)&s.visit[li.start], (unsigned long long)bit);
      const unsigned long long old = atomicOr((unsigned long long*)&s.front[0][li.start], (unsigned long long)bit);
      if (old == 0) {
        const unsigned long long p = atomicAdd((unsigned long long*)&sctl[sidx].fl_n[0], 1ull);
        s.fl[0][p] = li.start;
      }
      s.P[(int64_t)li.start * 64 + l] = li.sparent;
      s.L[(int64_t)li.start * 64 + l] = 0;
    }
  }
}

__global__ void __launch_bounds__(BT) batch_run(SlotDev* slots, SlotCtl* sctl, int nslots, BatchCtl* bc,
                                                int32_t count_levels) {
  __shared__ int s_cur[MAX_SLOTS_SMEM], s_dir[MAX_SLOTS_SMEM], s_done[MAX_SLOTS_SMEM], s_it[MAX_SLOTS_SMEM];
  __shared__ int64_t s_ncur[MAX_SLOTS_SMEM];
  const int lane = threadIdx.x & 31;
  const int64_t gw = gtid() >> 5, nw = gthreads() >> 5;
  unsigned int gen = 0;
  for (int iter_guard = 0; iter_guard < 65534; ++iter_guard) {
    // snapshot of the per-slot control words for this level
    for (int i = threadIdx.x; i < nslots; i += BT) {
      s_cur[i] = sctl[i].cur;
      s_dir[i] = sctl[i].dir;
      s_done[i] = sctl[i].done;
      s_it[i] = sctl[i].iter;
      s_ncur[i] = sctl[i].fl_n[sctl[i].cur];
    }
    __syncthreads();
    // ---- E: expand
    for (int si = 0; si < nslots; ++si) {
      if (s_done[si]) continue;
      const SlotDev& s = slots[si];
      const int cur = s_cur[si], nxt = cur ^ 1;
      const uint64_t* fc = s.front[cur];
      uint64_t* fn = s.front[nxt];
      if (s_dir[si] == DIR_TD) {
        const int64_t nf = s_ncur[si];
        for (int64_t j = gw; j < nf; j += nw) {  // a warp per frontier vertex
          const int32_t v = s.fl[cur][j];
          const uint64_t f = fc[v];
          const int64_t b = s.crow[v], e = s.crow[v + 1];
          for (int64_t k0 = b; k0 < e; k0 += 32) {
            const int64_t k = k0 + lane;
            bool first = false;
            int32_t w = 0;
            if (k < e) {
              w = s.ccol[k];
              const uint64_t nb = f & ~s.visit[w];
              if (nb) first = atomicOr((unsigned long long*)&fn[w], (unsigned long long)nb) == 0ull;
            }
            const unsigned bal = __ballot_sync(FULL, first);
            if (bal) {
              unsigned long long p = 0;
              if (lane == __ffs(bal) - 1)
                p = atomicAdd((unsigned long long*)&sctl[si].fl_n[nxt], (unsigned long long)__popc(bal));
              p = __shfl_sync(FULL, p, __ffs(bal) - 1);
              if (first) s.fl[nxt][p + __popc(bal & lanemask_lt())] = w;
            }
          }
        }
      } else {
        const uint64_t act = s.active;
        for (int64_t w0 = gw * 32; w0 < s.nc; w0 += nw * 32) {  // a lane per vertex, warp per 32
          const int32_t w = (int32_t)(w0 + lane);
          uint64_t miss = 0;
          int64_t b = 0, e = 0, stop = 0;
          uint64_t got = 0;
          if (w < s.nc) {
            miss = act & ~s.visit[w];
            if (miss) {
              b = s.crow[w];
              e = s.crow[w + 1];
              got = first_hits_thread(s, fc, w, miss, b, min(e, b + THREAD_SCAN), &stop);
            }
          }
          unsigned lm = __ballot_sync(FULL, miss && got != miss && stop < e);
          while (lm) {  // long adjacency: the warp continues the scan
            const int src = __ffs(lm) - 1;
            lm &= lm - 1;
            const int32_t w2 = __shfl_sync(FULL, w, src);
            const uint64_t want2 = __shfl_sync(FULL, miss, src);
            const uint64_t got2 = __shfl_sync(FULL, got, src);
            const int64_t b2 = __shfl_sync(FULL, stop, src), e2 = __shfl_sync(FULL, e, src);
            const uint64_t g2 = first_hits_warp(s, fc, w2, want2, got2, b2, e2);
            if (lane == src) got = g2;
          }
          const bool first = got != 0;
          if (first) fn[w] = got;
          const unsigned bal = __ballot_sync(FULL, first);
          if (bal) {
            unsigned long long p = 0;
            if (lane == __ffs(bal) - 1)
              p = atomicAdd((unsigned long long*)&sctl[si].fl_n[nxt], (unsigned long long)__popc(bal));
            p = __shfl_sync(FULL, p, __ffs(bal) - 1);
            if (first) s.fl[nxt][p + __popc(bal & lanemask_lt())] = w;
          }
        }
      }
    }
    if (!grid_barrier(bc, gen)) return;
    // ---- P: parents of top-down discoveries, levels, visit
    for (int si = 0; si < nslots; ++si) {
      if (s_done[si]) continue;
      const SlotDev& s = slots[si];
      const int cur = s_cur[si], nxt = cur ^ 1;
      const uint64_t* fc = s.front[cur];
      const uint64_t* fn = s.front[nxt];
      const int64_t nn = sctl[si].fl_n[nxt];
      const uint16_t it = (uint16_t)(s_it[si] + 1);
      int64_t msum = 0;
      for (int64_t j0 = gw * 32; j0 < nn; j0 += nw * 32) {
        const int64_t j = j0 + lane;
        int32_t w = -1;
        uint64_t nb = 0, got = 0;
        int64_t b = 0, e = 0, stop = 0;
        if (j < nn) {
          w = s.fl[nxt][j];
          nb = fn[w];
          b = s.crow[w];
          e = s.crow[w + 1];
          msum += e - b;
          if (s_dir[si] == DIR_TD) got = first_hits_thread(s, fc, w, nb, b, min(e, b + THREAD_SCAN), &stop);
          else got = nb;
        }
        unsigned lm = __ballot_sync(FULL, w >= 0 && got != nb);
        while (lm) {
          const int src = __ffs(lm) - 1;
          lm &= lm - 1;
          const int32_t w2 = __shfl_sync(FULL, w, src);
          const uint64_t want2 = __shfl_sync(FULL, nb, src);
          const uint64_t got2 = __shfl_sync(FULL, got, src);
          const int64_t b2 = __shfl_sync(FULL, stop, src), e2 = __shfl_sync(FULL, e, src);
          const uint64_t g2 = first_hits_warp(s, fc, w2, want2, got2, b2, e2);
          if (lane == src) got = g2;
        }
        if (w >= 0) {
          set_lane_levels(s, w, nb, it);
          s.visit[w] |= nb;
        }
      }
      msum = warp_sum(msum);
      if (lane == 0 && msum) atomicAdd((unsigned long long*)&sctl[si].m_next, (unsigned long long)msum);
    }
    if (!grid_barrier(bc, gen)) return;
    // ---- D: clear the old frontier words, then one thread per slot decides
    for (int si = 0; si < nslots; ++si) {
      if (s_done[si]) continue;
      const SlotDev& s = slots[si];
      const int cur = s_cur[si];
      const int64_t nf = s_ncur[si];
      for (int64_t j = gtid(); j < nf; j += gthreads()) s.front[cur][s.fl[cur][j]] = 0;
    }
    if (blockIdx.x == 0) {
      for (int si = threadIdx.x; si < nslots; si += BT) {
        if (s_done[si]) continue;
        SlotCtl& c = sctl[si];
        const SlotDev& s = slots[si];
        const int cur = s_cur[si], nxt = cur ^ 1;
        const int64_t nn = c.fl_n[nxt];
        c.fl_n[cur] = 0;
        c.cur = nxt;
        c.iter = s_it[si] + 1;
        if (nn == 0 || c.iter >= 65534) {
          c.done = 1;
          if (nn != 0) atomicExch(&bc->err, 2);  // too deep for 16-bit levels
          atomicSub(&bc->live, 1);
        } else if (s_dir[si] == DIR_TD) {
          if (c.m_next * (int64_t)s.alpha > s.nnz_core) c.dir = DIR_BU;
        } else {
          if (nn * (int64_t)s.beta < s.nc && nn < s_ncur[si]) c.dir = DIR_TD;
        }
        c.m_next = 0;
      }
    }
    if (!grid_barrier(bc, gen)) return;
    if (*(volatile int*)&bc->live <= 0) return;
    (void)count_levels;
  }
}

// Root-major outputs in vertex-id order. A CTA takes 32 consecutive vertices; warp k
// writes lanes 8k..8k+7 of the slot, each lane's 32 values coalesced. Core vertices and
// tree vertices hanging from a core vertex are final here; tree vertices hanging from a
// tree vertex get -2 ("resolve pending") for batch_resolve.
__global__ void __launch_bounds__(BT) batch_output(SlotDev* slots, int nslots) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int si = 0; si < nslots; ++si) {
    const SlotDev& s = slots[si];
    const int64_t nchunks = (s.n + 31) / 32;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
      const int64_t v = c * 32 + lane;
      const bool in = v < s.n;
      const int32_t info = in ? s.vinfo[v] : -1;
      int32_t cid = -1, add = 0, fixed_parent = -1;
      if (info >= 0) {
        cid = info;
      } else if (info <= -2 && info != INT32_MIN) {
        cid = s.anchor_cid[-2 - info];
        add = 1;
        fixed_parent = s.anchor_vid[-2 - info];
      }
      const uint64_t vis = cid >= 0 ? s.visit[cid] : 0ull;
      for (int k = 0; k < 8; ++k) {
        const int l = wp * 8 + k;
        if (l >= s.nlanes) break;
        int32_t lv = info == INT32_MIN ? -2 : -1, pa = lv;
        if ((vis >> l) & 1ull) {
          lv = (int32_t)s.L[(int64_t)cid * 64 + l] + s.lane[l].base + add;
          pa = add ? fixed_parent : s.P[(int64_t)cid * 64 + l];
        }
        if (in) {
          s.outl[l][v] = lv;
          s.outp[l][v] = pa;
        }
      }
    }
  }
}

// Root on an edge tree (one thread per lane): levels and parents along the walk from
// the root to the core, direction reversed; the core vertex reached takes the last tree
// vertex as parent.
__global__ void batch_fixup(SlotDev* slots, int nslots) {
  const int si = blockIdx.x;
  if (si >= nslots) return;
  const SlotDev& s = slots[si];
  const int l = threadIdx.x;
  if (l >= s.nlanes) return;
  const int32_t root = s.lane[l].root;
  if (s.vinfo[root] >= 0) return;
  int32_t* lv = s.outl[l];
  int32_t* pa = s.outp[l];
  lv[root] = 0;
  pa[root] = root;
  int32_t v = root, k = 0;
  for (int64_t guard = 0; guard < s.n; ++guard) {
    const int32_t u = s.up[v];
    if (u < 0) break;
    if (s.old2core[u] >= 0) {
      pa[u] = v;
      break;
    }
    ++k;
    lv[u] = k;
    pa[u] = v;
    v = u;
  }
}

struct ResolveSeg {
  const int32_t* list;
  const int32_t* lup;
  int64_t b, e;
};

// One height of the tree-up resolution for every lane of every slot: entries still at -2
// take level(up) + 1 and parent up (Alg. 10 with levels); walk vertices are already set.
__global__ void batch_resolve(SlotDev* slots, const ResolveSeg* segs, int nslots) {
  const int si = blockIdx.y;
  if (si >= nslots) return;
  const SlotDev& s = slots[si];
  const ResolveSeg sg = segs[si];
  const int64_t len = sg.e - sg.b;
  const int64_t total = len * s.nlanes;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(t / len);
    const int64_t i = sg.b + t % len;
    int32_t* lv = s.outl[l];
    int32_t* pa = s.outp[l];
    const int32_t v = sg.list[i];
    if (lv[v] != -2) continue;
    const int32_t u = sg.lup[i];
    const int32_t lu = lv[u];
    lv[v] = lu >= 0 ? lu + 1 : -1;
    pa[v] = lu >= 0 ? u : -1;
  }
}

// Lane setup on the device: the Alg. 9 walk of every root (one thread per lane).
__global__ void batch_lanes(SlotDev* slots, int nslots) {
  const int si = blockIdx.x;
  if (si >= nslots) return;
  SlotDev& s = slots[si];
  const int l = threadIdx.x;
  if (l >= s.nlanes) return;
  LaneInit& li = s.lane[l];
  const int32_t root = li.root;
  const int32_t info = s.vinfo[root];
  if (info >= 0) {
    li.start = info;
    li.base = 0;
    li.sparent = root;
  } else {
    int32_t v = root, hops = 0, start = -1;
    for (int64_t guard = 0; guard < s.n; ++guard) {
      const int32_t u = s.up[v];
      if (u < 0) break;
      ++hops;
      const int32_t cu = s.old2core[u];
      if (cu >= 0) {
        start = cu;
        break;
      }
      v = u;
    }
    li.start = start;
    li.base = hops;
    li.sparent = v;
  }
  const unsigned long long bit = li.start >= 0 ? (1ull << l) : 0ull;
  if (bit) atomicOr((unsigned long long*)&s.active, bit);
}

}  // namespace

void free_batch_mem(gt_graph* g) {
  for (void* p : g->batch_mem) cudaFree(p);
  g->batch_mem.clear();
  g->batch_slots_alloc = 0;
}

// Grows the handle's pool of lane-word storage (7 buffers per 64 roots, core-sized) to
// `need` slots.
int ensure_slots(gt_graph* g, int need) {
  const int64_t nc = std::max<int64_t>(g->core.n, 1);
  while (g->batch_slots_alloc < need) {
    void* p[7];
    const size_t sz[7] = {8 * (size_t)nc, 8 * (size_t)nc, 8 * (size_t)nc, 256 * (size_t)nc, 128 * (size_t)nc,
                          4 * (size_t)nc, 4 * (size_t)nc};
    for (int i = 0; i < 7; ++i) {
      int rc = device_malloc(g, &p[i], sz[i]);
      if (rc) {
        for (int j = 0; j < i; ++j) cudaFree(p[j]);
        return rc;
      }
    }
    for (int i = 0; i < 7; ++i) g->batch_mem.push_back(p[i]);
    g->batch_slots_alloc += 1;
  }
  return GT_OK;
}

size_t slot_bytes(const gt_graph* g) { return (size_t)std::max<int64_t>(g->core.n, 1) * (8 * 3 + 256 + 128 + 8); }

void batch_ctx_free(BatchCtx* c) {
  if (!c) return;
  if (c->dev) cudaFree(c->dev);
  if (c->seg_dev) cudaFree(c->seg_dev);
  if (c->h_err) cudaFreeHost(c->h_err);
  c->dev = nullptr;
  c->seg_dev = nullptr;
  c->h_err = nullptr;
  c->cap = 0;
  c->seg_cap = 0;
}

int batch_launch(BatchCtx* ctx, const SlotSpec* specs, int nspecs, int sm_share, cudaStream_t st) {
  if (nspecs <= 0) return GT_OK;
  if (nspecs > MAX_SLOTS_SMEM) {
    set_error("batched BFS: more than 256 lane words (16384 roots) in one launch");
    return GT_EINVAL;
  }
  const int ns = nspecs;
  const size_t t_slots = (sizeof(SlotDev) * ns + 255) & ~(size_t)255;
  const size_t t_ctl = (sizeof(SlotCtl) * ns + 255) & ~(size_t)255;
  const size_t bytes = t_slots + t_ctl + 256 + sizeof(ResolveSeg) * ns * 2 + 256;
  if (ctx->cap < ns) {
    if (ctx->dev) cudaFree(ctx->dev);
    ctx->dev = nullptr;
    int rc = cuda_fail(cudaMalloc(&ctx->dev, bytes), "batch table");
    if (rc) return rc;
    ctx->cap = ns;
  }
  if (!ctx->h_err) {
    int rc = cuda_fail(cudaHostAlloc((void**)&ctx->h_err, sizeof(int) * 4, cudaHostAllocDefault), "pinned status");
    if (rc) return rc;
  }
  ctx->h_err[0] = 0;
  std::vector<SlotDev> hs(ns);
  int maxh = 0;
  gt_graph* g0 = specs[0].g;
  for (int i = 0; i < ns; ++i) {
    const SlotSpec& sp = specs[i];
    gt_graph* g = sp.g;
    SlotDev& d = hs[i];
    memset(&d, 0, sizeof(d));
    d.n = g->n;
    d.nc = g->core.n;
    d.nnz_core = g->core.nnz;
    d.crow = g->core.row;
    d.ccol = g->core.col;
    d.vinfo = g->vinfo;
    d.new2old = g->new2old;
    d.anchor_cid = g->anchor_cid;
    d.anchor_vid = g->anchor_vid;
    d.up = g->up;
    d.old2core = g->old2core;
    d.visit = (uint64_t*)sp.mem[0];
    d.front[0] = (uint64_t*)sp.mem[1];
    d.front[1] = (uint64_t*)sp.mem[2];
    d.P = (int32_t*)sp.mem[3];
    d.L = (uint16_t*)sp.mem[4];
    d.fl[0] = (int32_t*)sp.mem[5];
    d.fl[1] = (int32_t*)sp.mem[6];
    d.nlanes = sp.nlanes;
    d.alpha = g->tuning.batch_alpha;
    d.beta = g->tuning.batch_beta;
    for (int l = 0; l < sp.nlanes; ++l) {
      const int64_t root = sp.roots[l];
      if (root < 0 || root >= g->n || !sp.outp[l] || !sp.outl[l]) {
        set_error("batched BFS: root outside [0, n) or null output");
        return GT_EINVAL;
      }
      d.lane[l].root = (int32_t)root;
      d.lane[l].start = -1;
      d.outp[l] = sp.outp[l];
      d.outl[l] = sp.outl[l];
    }
    maxh = std::max(maxh, g->resolve_heights);
    const size_t nc = (size_t)std::max<int64_t>(g->core.n, 1);
    cudaMemsetAsync(d.visit, 0, 8 * nc, st);
    cudaMemsetAsync(d.front[0], 0, 8 * nc, st);
    cudaMemsetAsync(d.front[1], 0, 8 * nc, st);
  }
  char* base = (char*)ctx->dev;
  SlotDev* d_slots = (SlotDev*)base;
  SlotCtl* d_ctl = (SlotCtl*)(base + t_slots);
  BatchCtl* d_bc = (BatchCtl*)(base + t_slots + t_ctl);
  ResolveSeg* d_seg = (ResolveSeg*)(base + t_slots + t_ctl + 256);
  int rc = cuda_fail(cudaMemcpyAsync(d_slots, hs.data(), sizeof(SlotDev) * ns, cudaMemcpyHostToDevice, st), "slots");
  if (rc) return rc;
  std::vector<SlotCtl> hc(ns);
  for (int i = 0; i < ns; ++i) hc[i] = SlotCtl{{0, 0}, 0, 0, DIR_TD, 0, 0};
  const BatchCtl hb{0u, 0, ns, 0};
  cudaMemcpyAsync(d_ctl, hc.data(), sizeof(SlotCtl) * ns, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_bc, &hb, sizeof(hb), cudaMemcpyHostToDevice, st);
  batch_lanes<<<ns, 64, 0, st>>>(d_slots, ns);
  batch_init<<<ns, 64, 0, st>>>(d_slots, d_ctl, ns);
  int nb_per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_per_sm, batch_run, BT, 0);
  const int share = std::max(1, std::min(sm_share > 0 ? sm_share : g0->launch.sms, g0->launch.sms));
  const int grid = std::max(1, std::min(nb_per_sm, 4)) * share;
  int32_t cl = 0;
  int nsl = ns;
  void* kargs[] = {(void*)&d_slots, (void*)&d_ctl, (void*)&nsl, (void*)&d_bc, (void*)&cl};
  rc = cuda_fail(cudaLaunchCooperativeKernel((void*)batch_run, dim3(grid), dim3(BT), kargs, 0, st), "batch launch");
  if (rc) return rc;
  batch_output<<<share * 16, BT, 0, st>>>(d_slots, ns);
  batch_fixup<<<ns, 64, 0, st>>>(d_slots, ns);
  if (maxh > 0) {
    // heights are processed top down; each slot walks its own graph's segments
    std::vector<ResolveSeg> segs((size_t)ns * maxh);
    for (int h = 0; h < maxh; ++h)
      for (int i = 0; i < ns; ++i) {
        gt_graph* g = specs[i].g;
        ResolveSeg sg{g->resolve_list, g->resolve_up, 0, 0};
        if (h < g->resolve_heights) {
          sg.b = g->resolve_ptr_host[h];
          sg.e = g->resolve_ptr_host[h + 1];
        }
        segs[(size_t)h * ns + i] = sg;
      }
    if (ctx->seg_cap < (int64_t)segs.size()) {
      if (ctx->seg_dev) cudaFree(ctx->seg_dev);
      ctx->seg_dev = nullptr;
      rc = cuda_fail(cudaMalloc(&ctx->seg_dev, sizeof(ResolveSeg) * segs.size()), "resolve table");
      if (rc) return rc;
      ctx->seg_cap = (int64_t)segs.size();
    }
    ResolveSeg* dseg = (ResolveSeg*)ctx->seg_dev;
    cudaMemcpyAsync(dseg, segs.data(), sizeof(ResolveSeg) * segs.size(), cudaMemcpyHostToDevice, st);
    for (int h = 0; h < maxh; ++h) batch_resolve<<<dim3(64, ns), BT, 0, st>>>(d_slots, dseg + (size_t)h * ns, ns);
  }
  (void)d_seg;
  cudaMemcpyAsync(ctx->h_err, &d_bc->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  return cuda_fail(cudaGetLastError(), "batch kernels");
}

int batch_status(const BatchCtx* ctx) {
  const int err = ctx->h_err ? ctx->h_err[0] : 0;
  if (err == 1) {
    set_error("batched BFS: a grid barrier wait ran out");
    return GT_ETIMEOUT;
  }
  if (err == 2) {
    set_error("batched BFS: traversal deeper than 65533 levels");
    return GT_ENOTSUP;
  }
  return GT_OK;
}

int run_batch(gt_graph* const* graphs, int ngraphs, const int64_t* roots, const int32_t* rpg,
              int32_t* const* parent, int32_t* const* level, cudaStream_t st) {
  std::vector<SlotSpec> specs;
  std::vector<int32_t*> lanes_p, lanes_l;
  int64_t total_words = 0;
  for (int gi = 0; gi < ngraphs; ++gi) total_words += (rpg[gi] + 63) / 64;
  lanes_p.reserve((size_t)total_words * 64);
  lanes_l.reserve((size_t)total_words * 64);
  int64_t ro = 0;
  for (int gi = 0; gi < ngraphs; ++gi) {
    gt_graph* g = graphs[gi];
    const int r = rpg[gi];
    const int nsg = (r + 63) / 64;
    int rc = ensure_slots(g, nsg);
    if (rc) return rc;
    for (int k = 0; k < nsg; ++k) {
      SlotSpec sp;
      sp.g = g;
      sp.mem = &g->batch_mem[7 * k];
      sp.nlanes = std::min(64, r - 64 * k);
      sp.roots = roots + ro + 64 * k;
      const size_t off = lanes_p.size();
      for (int l = 0; l < sp.nlanes; ++l) {
        lanes_p.push_back(parent[gi] + (int64_t)(64 * k + l) * g->n);
        lanes_l.push_back(level[gi] + (int64_t)(64 * k + l) * g->n);
      }
      sp.outp = lanes_p.data() + off;
      sp.outl = lanes_l.data() + off;
      specs.push_back(sp);
    }
    ro += r;
  }
  if (specs.empty()) return GT_OK;
  gt_graph* g0 = graphs[0];
  if (!g0->batch_ctx) g0->batch_ctx = new BatchCtx();
  int rc = batch_launch(g0->batch_ctx, specs.data(), (int)specs.size(), 0, st);
  if (!rc) rc = cuda_fail(cudaStreamSynchronize(st), "batch sync");
  if (!rc) rc = batch_status(g0->batch_ctx);
  return rc;
}

}  // namespace gt
