// bfs.cu -- direction-optimizing BFS (Alg. 1) on a CSR view, and the edge-tree steps
// around it (Alg. 9: root walk to the core, BFS_CORE, edge-tree resolution).
//
// Per-vertex state is one 64-bit word (level << 32 | parent), UNVISITED = all ones.
// Top-down (Alg. 1 TOP-DOWN): every frontier edge to a vertex that was not visited at
// the start of the level does atomicMin(state, (L+1) << 32 | v); the smallest packed
// value wins, i.e. level L+1 with the smallest frontier neighbour as parent, and the
// one thread that replaced UNVISITED enqueues the vertex. Bottom-up (Alg. 1 BOTTOM-UP,
// with the block search of Alg. 5): unvisited vertices are found by scanning the
// visited bitmap in 128-bit words; each scans its ascending adjacency and stops at the
// first visited neighbour (visited before this level means "in the frontier" for an
// unvisited vertex), which is the smallest one. Both directions therefore give the
// same levels and min-id parents, whatever the switch does.
#include <algorithm>

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
  int32_t* q0;
  int32_t* q1;
  int32_t* big;
  BfsCtl* ctl;
  int32_t td_warp_min;
  int32_t td_grid_min;
  int32_t bu_scan;
  int32_t count_work;
};

BfsArgs make_args(const View& v, const gt_tuning& t) {
  BfsArgs a;
  a.n = v.n;
  a.nnz = v.nnz;
  a.nwords = v.nwords;
  a.row = v.row;
  a.col = v.col;
  a.state = v.state;
  a.vis0 = v.vis[0];
  a.vis1 = v.vis[1];
  a.q0 = v.queue[0];
  a.q1 = v.queue[1];
  a.big = v.big;
  a.ctl = v.ctl;
  a.td_warp_min = std::max(1, t.td_warp_min);
  a.td_grid_min = std::max(a.td_warp_min, t.td_grid_min);
  a.bu_scan = std::max(0, t.bu_thread_scan);
  a.count_work = t.count_work;
  return a;
}

// Appends the lanes with `disc` set to the next queue; all 32 lanes must call.
__device__ __forceinline__ void warp_enqueue(bool disc, int32_t w, int64_t wdeg, int32_t* __restrict__ nq,
                                             BfsCtl* ctl) {
  const unsigned bal = __ballot_sync(FULL, disc);
  if (!bal) return;
  const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
  const int64_t dsum = warp_sum<int64_t>(disc ? wdeg : 0);
  unsigned long long base = 0;
  if (lane == leader) {
    base = atomicAdd((unsigned long long*)&ctl->next_n, (unsigned long long)__popc(bal));
    atomicAdd((unsigned long long*)&ctl->next_m, (unsigned long long)dsum);
  }
  base = __shfl_sync(FULL, base, leader);
  if (disc) nq[base + __popc(bal & lanemask_lt())] = w;
}

// One frontier edge (v -> w) of a top-down step; packed = (L+1) << 32 | v.
__device__ __forceinline__ bool td_visit(uint64_t* state, const uint32_t* vis, int32_t w, uint64_t packed) {
  if ((vis[w >> 5] >> (w & 31)) & 1u) return false;  // visited before this level (may lag: only a filter)
  if (state[w] <= packed) return false;               // already as good (values only decrease)
  const unsigned long long old = atomicMin((unsigned long long*)&state[w], (unsigned long long)packed);
  return old == UNVISITED;
}

__device__ __forceinline__ void add_examined(const BfsArgs& a, int64_t x) {
  if (!a.count_work) return;
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0 && x) atomicAdd((unsigned long long*)&a.ctl->examined, (unsigned long long)x);
}

// ---- top-down ----------------------------------------------------------------------
// A warp takes 32 frontier vertices. Degree <= td_warp_min: their edges are packed
// across the warp's lanes (lane-to-vertex by a search over the prefix sum of degrees).
// Up to td_grid_min: the whole warp walks one vertex's adjacency. Above: the vertex is
// handed to bfs_td_grid, where every CTA of the grid takes a slice of it.
__global__ void __launch_bounds__(BFS_THREADS) bfs_td(BfsArgs a) {
  BfsCtl* ctl = a.ctl;
  const int cur = ctl->cur;
  const int32_t* __restrict__ q = cur ? a.q1 : a.q0;
  int32_t* __restrict__ nq = cur ? a.q0 : a.q1;
  uint32_t* vis = ctl->vcur ? a.vis1 : a.vis0;
  const int64_t nf = ctl->n_f;
  const uint64_t hi = (uint64_t)(uint32_t)(ctl->level + 1) << 32;
  const int lane = threadIdx.x & 31;
  const int64_t gw = gtid() >> 5, nw = gthreads() >> 5;
  int64_t examined = 0;
  for (int64_t base = gw * 32; base < nf; base += nw * 32) {
    const int64_t i = base + lane;
    int32_t v = -1;
    int64_t rs = 0, re = 0;
    if (i < nf) {
      v = q[i];
      rs = a.row[v];
      re = a.row[v + 1];
      atomicOr(&vis[v >> 5], 1u << (v & 31));
    }
    const int64_t d = re - rs;
    const bool big = d > a.td_grid_min;
    {
      const unsigned bal = __ballot_sync(FULL, big);
      if (bal) {
        unsigned long long b0 = 0;
        if (lane == __ffs(bal) - 1) b0 = atomicAdd((unsigned long long*)&ctl->big_n, (unsigned long long)__popc(bal));
        b0 = __shfl_sync(FULL, b0, __ffs(bal) - 1);
        if (big) a.big[b0 + __popc(bal & lanemask_lt())] = v;
      }
    }
    unsigned med = __ballot_sync(FULL, !big && d > a.td_warp_min);
    while (med) {
      const int src = __ffs(med) - 1;
      med &= med - 1;
      const int32_t vv = __shfl_sync(FULL, v, src);
      const int64_t s = __shfl_sync(FULL, rs, src), e = __shfl_sync(FULL, re, src);
      const uint64_t packed = hi | (uint32_t)vv;
      for (int64_t k0 = s; k0 < e; k0 += 32) {
        const int64_t k = k0 + lane;
        bool disc = false;
        int32_t w = 0;
        int64_t wd = 0;
        if (k < e) {
          w = a.col[k];
          disc = td_visit(a.state, vis, w, packed);
          if (disc) wd = a.row[w + 1] - a.row[w];
        }
        warp_enqueue(disc, w, wd, nq, ctl);
      }
      if (lane == 0) examined += e - s;
    }
    const int32_t sd = (!big && d <= a.td_warp_min) ? (int32_t)d : 0;
    const int32_t incl = warp_incl_scan(sd);
    const int32_t total = __shfl_sync(FULL, incl, 31);
    const int32_t excl = incl - sd;
    if (lane == 0) examined += total;
    for (int32_t r0 = 0; r0 < total; r0 += 32) {
      const int32_t idx = r0 + lane;
      int owner = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int cand = owner + step;
        if (__shfl_sync(FULL, excl, cand) <= idx) owner = cand;
      }
      const int32_t ov = __shfl_sync(FULL, v, owner);
      const int64_t ors = __shfl_sync(FULL, rs, owner);
      const int32_t oex = __shfl_sync(FULL, excl, owner);
      bool disc = false;
      int32_t w = 0;
      int64_t wd = 0;
      if (idx < total) {
        w = a.col[ors + (idx - oex)];
        disc = td_visit(a.state, vis, w, hi | (uint32_t)ov);
        if (disc) wd = a.row[w + 1] - a.row[w];
      }
      warp_enqueue(disc, w, wd, nq, ctl);
    }
  }
  add_examined(a, examined);
}

__global__ void __launch_bounds__(BFS_THREADS) bfs_td_grid(BfsArgs a) {
  BfsCtl* ctl = a.ctl;
  const int64_t nbig = ctl->big_n;
  if (nbig == 0) return;
  const int cur = ctl->cur;
  int32_t* __restrict__ nq = cur ? a.q0 : a.q1;
  uint32_t* vis = ctl->vcur ? a.vis1 : a.vis0;
  const uint64_t hi = (uint64_t)(uint32_t)(ctl->level + 1) << 32;
  const int lane = threadIdx.x & 31;
  const int64_t gw = gtid() >> 5, nw = gthreads() >> 5;
  int64_t examined = 0;
  for (int64_t j = 0; j < nbig; ++j) {
    const int32_t v = a.big[j];
    const int64_t s = a.row[v], e = a.row[v + 1];
    const uint64_t packed = hi | (uint32_t)v;
    for (int64_t k0 = s + gw * 32; k0 < e; k0 += nw * 32) {
      const int64_t k = k0 + lane;
      bool disc = false;
      int32_t w = 0;
      int64_t wd = 0;
      if (k < e) {
        w = a.col[k];
        disc = td_visit(a.state, vis, w, packed);
        if (disc) wd = a.row[w + 1] - a.row[w];
        ++examined;
      }
      warp_enqueue(disc, w, wd, nq, ctl);
    }
  }
  add_examined(a, examined);
}

// Sets the visited bits of the current frontier (needed before a bottom-up step that
// follows a top-down one: top-down leaves its discoveries unmarked until they expand).
__global__ void bfs_mark(BfsArgs a) {
  BfsCtl* ctl = a.ctl;
  const int32_t* __restrict__ q = ctl->cur ? a.q1 : a.q0;
  uint32_t* vis = ctl->vcur ? a.vis1 : a.vis0;
  const int64_t nf = ctl->n_f;
  for (int64_t i = gtid(); i < nf; i += gthreads()) {
    const int32_t v = q[i];
    atomicOr(&vis[v >> 5], 1u << (v & 31));
  }
}

// ---- bottom-up ---------------------------------------------------------------------
// A warp takes 128 bitmap words (4096 vertices) with one 128-bit load per lane. For each
// of the lane's 4 words in turn, the warp compacts the unvisited vertices (popc + warp
// prefix sum) into a shared list; lanes then take one listed vertex each and check its
// first bu_scan neighbours alone; vertices still open after that are taken over by the
// whole warp, 32 neighbours per step, first hit by ballot. Found vertices set bits in a
// shared copy of the 128 words, written once to the next bitmap (Alg. 5's single write
// per block).
__global__ void __launch_bounds__(BFS_THREADS) bfs_bu(BfsArgs a) {
  __shared__ uint16_t slist[WARPS][1024];
  __shared__ uint32_t sfound[WARPS][BU_CHUNK_WORDS];
  BfsCtl* ctl = a.ctl;
  const uint32_t* __restrict__ vc = ctl->vcur ? a.vis1 : a.vis0;
  uint32_t* __restrict__ vn = ctl->vcur ? a.vis0 : a.vis1;
  int32_t* __restrict__ nq = ctl->cur ? a.q0 : a.q1;
  const uint64_t hi = (uint64_t)(uint32_t)(ctl->level + 1) << 32;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t gw = gtid() >> 5, nw = gthreads() >> 5;
  const int64_t nchunks = a.nwords / BU_CHUNK_WORDS;
  uint16_t* list = slist[wp];
  uint32_t* found = sfound[wp];
  int64_t examined = 0;
  for (int64_t c = gw; c < nchunks; c += nw) {
    const uint4 w4 = __ldg(reinterpret_cast<const uint4*>(vc) + c * 32 + lane);
    found[lane * 4 + 0] = 0;
    found[lane * 4 + 1] = 0;
    found[lane * 4 + 2] = 0;
    found[lane * 4 + 3] = 0;
    const unsigned any = __ballot_sync(FULL, (w4.x & w4.y & w4.z & w4.w) != 0xFFFFFFFFu);
    if (any) {
      __syncwarp();
      const int64_t vbase = c * (BU_CHUNK_WORDS * 32);
#pragma unroll 1
      for (int k = 0; k < 4; ++k) {
        uint32_t un = ~(k == 0 ? w4.x : k == 1 ? w4.y : k == 2 ? w4.z : w4.w);
        const int cnt = __popc(un);
        const int incl = warp_incl_scan(cnt);
        const int total = __shfl_sync(FULL, incl, 31);
        if (total == 0) continue;
        int pos = incl - cnt;
        const int wl = lane * 4 + k;
        while (un) {
          const int b = __ffs(un) - 1;
          un &= un - 1;
          list[pos++] = (uint16_t)(wl * 32 + b);
        }
        __syncwarp();
        for (int t0 = 0; t0 < total; t0 += 32) {
          const int t = t0 + lane;
          const bool act = t < total;
          const int32_t loc = act ? list[t] : 0;
          const int32_t w = (int32_t)(vbase + loc);
          int64_t s = 0, e = 0;
          if (act) {
            s = a.row[w];
            e = a.row[w + 1];
          }
          const int64_t lim = min(e, s + (int64_t)a.bu_scan);
          int32_t par = -1;
          int64_t kk = s;
          for (; kk < lim; ++kk) {
            const int32_t u = a.col[kk];
            if ((__ldg(&vc[u >> 5]) >> (u & 31)) & 1u) {
              par = u;
              break;
            }
          }
          examined += (par >= 0 ? kk + 1 : kk) - s;
          const bool fnd = par >= 0;
          if (fnd) {
            a.state[w] = hi | (uint32_t)par;
            atomicOr(&found[loc >> 5], 1u << (loc & 31));
          }
          warp_enqueue(fnd, w, e - s, nq, ctl);
          unsigned lm = __ballot_sync(FULL, act && !fnd && lim < e);
          while (lm) {
            const int src = __ffs(lm) - 1;
            lm &= lm - 1;
            const int32_t w2 = __shfl_sync(FULL, w, src);
            const int32_t loc2 = __shfl_sync(FULL, loc, src);
            const int64_t s2 = __shfl_sync(FULL, lim, src), e2 = __shfl_sync(FULL, e, src);
            const int64_t d2 = e2 - __shfl_sync(FULL, s, src);
            int32_t par2 = -1;
            for (int64_t b0 = s2; b0 < e2; b0 += 32) {
              const int64_t k2 = b0 + lane;
              int32_t u = 0;
              bool hit = false;
              if (k2 < e2) {
                u = a.col[k2];
                hit = (__ldg(&vc[u >> 5]) >> (u & 31)) & 1u;
              }
              const unsigned hm = __ballot_sync(FULL, hit);
              if (lane == 0) examined += hm ? (__ffs(hm)) : min((int64_t)32, e2 - b0);
              if (hm) {
                par2 = __shfl_sync(FULL, u, __ffs(hm) - 1);
                break;
              }
            }
            if (par2 >= 0 && lane == 0) {
              a.state[w2] = hi | (uint32_t)par2;
              atomicOr(&found[loc2 >> 5], 1u << (loc2 & 31));
              const unsigned long long p = atomicAdd((unsigned long long*)&ctl->next_n, 1ull);
              atomicAdd((unsigned long long*)&ctl->next_m, (unsigned long long)d2);
              nq[p] = w2;
            }
          }
        }
        __syncwarp();
      }
    }
    __syncwarp();
    uint4 o;
    o.x = w4.x | found[lane * 4 + 0];
    o.y = w4.y | found[lane * 4 + 1];
    o.z = w4.z | found[lane * 4 + 2];
    o.w = w4.w | found[lane * 4 + 3];
    reinterpret_cast<uint4*>(vn)[c * 32 + lane] = o;
    __syncwarp();
  }
  add_examined(a, examined);
}

// ---- level control -----------------------------------------------------------------
// After each step: record the trace, swap queues (and bitmaps after bottom-up), and pick
// the next direction by the frontier-size rule of Beamer et al. (the paper's reference
// [12]; Alg. 1 calls it is_top_down_direction): top-down -> bottom-up when
// m_f * alpha > m_u, bottom-up -> top-down when n_f * beta < n and the frontier shrank.
__global__ void bfs_decide(BfsArgs a, cudaGraphConditionalHandle h_loop, int use_handles) {
  BfsCtl* c = a.ctl;
  if (!c->done) {
    const int L = c->level, dir = c->dir;
    const int64_t nn = c->next_n, nm = c->next_m;
    if (c->nlevels < MAX_TRACE) {
      gt_level_info& t = c->trace[c->nlevels];
      t.level = L;
      t.direction = dir;
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
    c->next_n = 0;
    c->next_m = 0;
    c->big_n = 0;
    c->examined = 0;
    c->cur ^= 1;
    if (dir == DIR_BU) c->vcur ^= 1;
    c->level = L + 1;
    int nd = dir;
    if (nn == 0) {
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
    c->dir = nd;
  }
  if (use_handles) cudaGraphSetConditional(h_loop, c->done ? 0u : 1u);
}

// First node of each loop iteration: routes the switch to the step now due.
__global__ void bfs_select(BfsCtl* c, cudaGraphConditionalHandle h_dir) {
  cudaGraphSetConditional(h_dir, c->dir == DIR_TD ? 0u : (c->need_mark ? 2u : 1u));
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
  c->next_n = 0;
  c->next_m = 0;
  c->examined = 0;
  c->big_n = 0;
  c->alpha = alpha;
  c->beta = beta;
  c->force = force;
  c->start = start;
  c->start_level = start_level;
  c->level = start_level;
  c->prev_n_f = 0;
  c->need_mark = 0;
  c->dir = force == 2 ? DIR_BU : DIR_TD;
  if (start < 0) {
    c->done = 1;
    c->n_f = 0;
    c->m_f = 0;
    c->m_u = 0;
    return;
  }
  c->done = 0;
  const int64_t d = a.row[start + 1] - a.row[start];
  a.state[start] = ((uint64_t)(uint32_t)start_level << 32) | (uint32_t)start;
  a.vis0[start >> 5] |= 1u << (start & 31);
  a.q0[0] = start;
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
  int32_t* epoch;
  int64_t n;
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

// Levels and parents of every vertex in vertex-id order: core vertices from the core
// BFS state (parents back to vertex ids), edge-tree vertices hanging from a core vertex
// from that vertex's level (Alg. 7 / Alg. 10 with levels), everything else -1.
__global__ void et_output(EtArgs e, const uint64_t* __restrict__ state, int32_t* __restrict__ parent,
                          int32_t* __restrict__ level) {
  for (int64_t v = gtid(); v < e.n; v += gthreads()) {
    const int32_t info = e.vinfo[v];
    int32_t l = -1, p = -1;
    if (info >= 0) {
      const uint64_t s = state[info];
      if (s != UNVISITED) {
        l = (int32_t)(s >> 32);
        p = e.new2old[(uint32_t)s];
      }
    } else if (info <= -2) {
      const int32_t cu = -2 - info;
      const uint64_t s = state[cu];
      if (s != UNVISITED) {
        l = (int32_t)(s >> 32) + 1;
        p = e.new2old[cu];
      }
    }
    level[v] = l;
    parent[v] = p;
  }
}

// Root on an edge tree: the vertices on the walk from the root to the core get their
// levels and parents from the walk (direction reversed: parent = the previous vertex),
// and the core vertex reached takes the last tree vertex as parent. Walk vertices are
// marked with this traversal's epoch so the tree-up resolution pass leaves them alone.
__global__ void et_fixup(EtArgs e, int32_t root, int32_t ep, int32_t* __restrict__ parent,
                         int32_t* __restrict__ level) {
  if (e.vinfo[root] >= 0) return;
  level[root] = 0;
  parent[root] = root;
  e.epoch[root] = ep;
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
    e.epoch[u] = ep;
    v = u;
  }
}

// Tree vertices hanging from another tree vertex, one height at a time from the top:
// level = level(up) + 1 (Alg. 10 with levels).
__global__ void et_resolve(const int32_t* __restrict__ list, const int32_t* __restrict__ lup, int64_t b, int64_t e,
                           const int32_t* __restrict__ epoch, int32_t ep, int32_t* __restrict__ parent,
                           int32_t* __restrict__ level) {
  for (int64_t i = b + gtid(); i < e; i += gthreads()) {
    const int32_t v = list[i];
    if (epoch[v] == ep) continue;
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

// Builds the CUDA graph of the level loop for one view:
//   WHILE(loop) { select -> SWITCH(dir) { 0: td, td_grid | 1: bu | 2: mark, bu } -> decide }
// The while handle (created on the top graph, default 1) is set by decide; the switch
// handle belongs to the body graph, which holds its node, and is set by select.
int build_loop_graph(gt_graph* g, const View& v, cudaGraphExec_t* out) {
  const BfsArgs a = make_args(v, g->tuning);
  const int grid = g->launch.grid;
  cudaGraph_t graph = nullptr;
  cudaStream_t cs = nullptr;
  int rc = GT_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    if (rc == GT_OK) rc = cuda_fail(e, what);
  };
  fail(cudaGraphCreate(&graph, 0), "graph create");
  cudaGraphConditionalHandle h_loop = 0, h_dir = 0;
  if (rc == GT_OK) fail(cudaGraphConditionalHandleCreate(&h_loop, graph, 1, cudaGraphCondAssignDefault), "handle");
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
  if (rc == GT_OK) fail(cudaGraphConditionalHandleCreate(&h_dir, body, 0, 0), "handle");
  cudaGraphNode_t sel = nullptr;
  if (rc == GT_OK) {
    cudaKernelNodeParams kp{};
    BfsCtl* ctl = a.ctl;
    void* args[] = {(void*)&ctl, (void*)&h_dir};
    kp.func = (void*)bfs_select;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    fail(cudaGraphAddKernelNode(&sel, body, nullptr, 0, &kp), "select node");
  }
  cudaGraph_t branch[3] = {nullptr, nullptr, nullptr};
  cudaGraphNode_t sw = nullptr;
  if (rc == GT_OK) {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h_dir;
    np.conditional.type = cudaGraphCondTypeSwitch;
    np.conditional.size = 3;
    fail(cudaGraphAddNode(&sw, body, &sel, nullptr, 1, &np), "switch node");
    if (rc == GT_OK)
      for (int i = 0; i < 3; ++i) branch[i] = np.conditional.phGraph_out[i];
  }
  for (int i = 0; i < 3 && rc == GT_OK; ++i) {
    fail(cudaStreamBeginCaptureToGraph(cs, branch[i], nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "capture");
    if (rc != GT_OK) break;
    if (i == 0) {
      bfs_td<<<grid, BFS_THREADS, 0, cs>>>(a);
      bfs_td_grid<<<grid, BFS_THREADS, 0, cs>>>(a);
    } else {
      if (i == 2) bfs_mark<<<grid, BFS_THREADS, 0, cs>>>(a);
      bfs_bu<<<grid, BFS_THREADS, 0, cs>>>(a);
    }
    cudaGraph_t got = nullptr;
    fail(cudaStreamEndCapture(cs, &got), "end capture");
  }
  if (rc == GT_OK) {
    cudaKernelNodeParams kp{};
    int use = 1;
    BfsArgs ac = a;
    void* args[] = {(void*)&ac, (void*)&h_loop, (void*)&use};
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
  const BfsArgs a = make_args(v, t);
  const int grid = g->launch.grid;
  struct Head {
    int32_t level, dir, done, cur, vcur, need_mark;
  } h{};
  const cudaGraphConditionalHandle none = 0;
  int timed_steps = 0;
  g->step_ms.clear();
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
    if (h.dir == DIR_TD) {
      bfs_td<<<grid, BFS_THREADS, 0, s>>>(a);
      bfs_td_grid<<<grid, BFS_THREADS, 0, s>>>(a);
    } else {
      if (h.need_mark) bfs_mark<<<grid, BFS_THREADS, 0, s>>>(a);
      bfs_bu<<<grid, BFS_THREADS, 0, s>>>(a);
    }
    if (timed) {
      cudaEventRecord(g->step_events[2 * guard + 1], s);
      ++timed_steps;
    }
    bfs_decide<<<1, 1, 0, s>>>(a, none, 0);
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
  const BfsArgs a = make_args(v, t);
  const int gs = grid_stream(g, std::max<int64_t>(v.n, v.nwords));
  bfs_reset<<<gs, 256, 0, s>>>(v.state, v.vis[0], v.n, v.nwords);
  EtArgs e{g->vinfo, g->up, g->old2core, g->new2old, g->epoch, g->n};
  if (et)
    et_start<<<1, 1, 0, s>>>(a, e, (int32_t)root, t.alpha, t.beta, t.force_direction);
  else
    bfs_start_plain<<<1, 1, 0, s>>>(a, (int32_t)root, t.alpha, t.beta, t.force_direction);
  int rc = cuda_fail(cudaGetLastError(), "bfs start");
  if (rc != GT_OK) return rc;
  rc = run_level_loop(g, v, et ? 0 : 1, s);
  if (rc != GT_OK) return rc;
  if (et) {
    const int go = grid_stream(g, g->n);
    et_output<<<go, 256, 0, s>>>(e, v.state, parent, level);
    if (++g->cur_epoch <= 0) {  // wrapped: clear the marks
      cudaMemsetAsync(g->epoch, 0, sizeof(int32_t) * g->n, s);
      g->cur_epoch = 1;
    }
    et_fixup<<<1, 1, 0, s>>>(e, (int32_t)root, g->cur_epoch, parent, level);
    for (int h = 0; h < g->resolve_heights; ++h) {
      const int64_t b = g->resolve_ptr_host[h], en = g->resolve_ptr_host[h + 1];
      if (en > b)
        et_resolve<<<grid_stream(g, en - b), 256, 0, s>>>(g->resolve_list, g->resolve_up, b, en, g->epoch,
                                                           g->cur_epoch, parent, level);
    }
  } else {
    plain_output<<<grid_stream(g, v.n), 256, 0, s>>>(v.state, v.n, parent, level);
  }
  g->last_stream = s;
  g->last_ctl = v.ctl;
  return cuda_fail(cudaGetLastError(), "bfs output");
}

}  // namespace gt
