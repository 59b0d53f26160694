// batch.cu -- many single-root edge-tree BFS at once (multi-source BFS over lane words).
//
// Roots are packed 64 to a "slot": one uint64 lane word per core vertex holds, for each
// of the slot's roots, whether the vertex is visited (visit), in the current frontier
// (front) or in the next one. Every adjacency read then serves all 64 roots. All slots
// of all graphs advance level by level inside ONE persistent cooperative launch; grid
// barriers separate the phases of a level:
//   E  expand   top-down slots push front bits along frontier edges (atomicOr; the first
//               to reach a vertex lists it) and take, per lane, the smallest frontier
//               neighbour as parent (atomicMin); a long frontier adjacency is cut into
//               chunks, the first pushed by the vertex's warp, the rest queued. Bottom-up
//               slots pull: every vertex still missing some lanes scans its ascending
//               adjacency, and the first neighbour carrying a lane's frontier bit is that
//               lane's parent (so min-id); short adjacencies a lane each, medium ones
//               (on large cores) 32 to a warp as one flattened sequence, long ones in
//               chunks a warp each, chunk results merged by atomicMin.
//   E2 queued   every warp takes queued top-down chunks (only when some slot queued any).
//   P  commit   every reached lane gets its level; visit |= new lanes (vertices a pull
//               scanned whole are committed by that pull already, without a mailbox).
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
#include <atomic>
#include <vector>

#include "gt_device.cuh"
#include "gt_internal.cuh"

namespace gt {
namespace {

constexpr int BT = 256;
constexpr int MAX_SLOTS_SMEM = 256;
constexpr int CW = 4;  // 32-entry windows a warp keeps in flight on one adjacency

// What a level reads once (adjacency entries a warp scans, the work lists, the visit words
// of the vertices it pulls) is loaded evict-first, so that L2 keeps the frontier words that
// the pull gathers at random (8 B per core vertex: 54 MB at R-MAT scale 24). A lane's short
// adjacency (16 B per step from one or two 128 B lines) stays on plain loads: evict-first
// ones measured 0.7 % slower at scale 24.
#define BATCH_STREAM_LD(p) __ldcs(p)


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
  const int32_t* lanes;   // bottom-up work: short adjacencies, a lane each
  const int32_t* mids;    // bottom-up work: medium adjacencies, 32 to a warp (hits_lanes32)
  const BatchItem* items; // bottom-up work: chunks of the long ones, a warp each
  int64_t n_lanes, n_mids, n_items;
  // state (core ids)
  uint64_t* visit;
  uint64_t* front[2];
  int32_t* P;   // [nc][64] parent vertex ids
  uint16_t* L;  // [nc][64] iteration at which the lane reached the vertex
  int32_t* fl[2];
  uint64_t* q;  // top-down: (vertex << 32 | chunk) of long frontier adjacencies, second pass
  // outputs: lane l writes parent / level arrays outp[l] / outl[l] (n entries each)
  int32_t* outp[64];
  int32_t* outl[64];
  int32_t nlanes;
  int32_t alpha, beta;
  int32_t join_max;      // last level boundary at which mailbox roots may join (0: none)
  BatchMailbox* mb;      // mapped mailbox shared by the launch's slots (null: none; with one,
                         // lanes that finish early are written and reported at once)
  uint64_t emitted;      // lanes whose results are already written
  uint64_t joined;       // lanes admitted from the mailbox during the launch
  uint64_t joined_now;   // lanes admitted at the current level boundary
  uint64_t young_prev;   // lanes admitted at the boundary before
  uint64_t young;        // lanes in their first two levels after joining: pushed top-down
                         // even when the slot pulls bottom-up (their frontier is small, and
                         // in the pull they would miss at nearly every vertex)
  uint64_t active;
  LaneInit lane[64];
};

struct SlotCtl {
  int64_t fl_n[2];
  int64_t m_next;  // summed degree of the next frontier
  int64_t q_n;     // top-down chunk queue entries
  int32_t cur, dir, done, iter;
  uint64_t alive;  // lanes present in the next frontier (early completion)
  uint64_t fin;    // lanes whose results are written at this level boundary
  // pull work handed out during a level (long items, medium groups, short groups of 32)
  unsigned grab[3];
};

// Pull work is handed out dynamically: a warp takes a few tasks (items, or groups of 32
// list entries) per atomic on its slot's counter, so that no warp idles at the phase's grid
// barrier while others still hold work (with a fixed round-robin share, the last warp of a
// scale-24 pull level finished 1.0-1.4 ms after the first). A take is about 1/GRAB_ROUNDS
// of a warp's fair share, between 1 and GRAB_MAX tasks.
constexpr int64_t GRAB_ROUNDS = 8;
constexpr int GRAB_MAX = 4;
__device__ __forceinline__ int grab_size(int ntask, int64_t nwarps) {
  return (int)max((int64_t)1, min((int64_t)GRAB_MAX, (int64_t)ntask / (nwarps * GRAB_ROUNDS)));
}

// Issues the atomic that reserves this warp's next n tasks; lane 0 holds the result. Task
// counts of a list fit in 32 bits (items: at most nnz / BATCH_CHUNK + core vertices).
__device__ __forceinline__ unsigned grab_issue(unsigned* cnt, int n) {
  return (threadIdx.x & 31) == 0 ? atomicAdd(cnt, (unsigned)n) : 0u;
}
__device__ __forceinline__ int grab_take(unsigned issued) { return (int)__shfl_sync(FULL, issued, 0); }

struct ResolveSeg {
  const int32_t* list;
  const int32_t* lup;
  int64_t b, e;
};

// Bits of lanes 0 .. nlanes-1.
__device__ __forceinline__ uint64_t lanes_of(int nlanes) { return nlanes >= 64 ? ~0ull : (1ull << nlanes) - 1; }

struct BatchCtl {
  unsigned int bar;    // grid barrier arrivals
  int err;
  int live;            // slots not done
  int emit;            // slots with lanes to write at this level boundary
  unsigned int polls;  // a barrier wait gives up after this many polls
  unsigned int extra;  // arrivals a barrier waits for beyond the grid's (0; failure tests only)
  // work of the launch: adjacency entries read by pull phases and by push phases, core
  // vertices scanned by pull phases, vertices discovered (summed over lane words)
  unsigned long long work[4];
};

// Barrier wait bounds of the batched launches (see gt_test_batch_barrier): the default
// gives up after 2^26 polls (seconds); a test can shorten it and add arrivals that never
// come, so that the wait runs out.
constexpr unsigned int BARRIER_POLLS = 1u << 26;
std::atomic<unsigned int> g_barrier_polls{BARRIER_POLLS};
std::atomic<unsigned int> g_barrier_extra{0};

// Grid-wide barrier for a cooperative launch: arrivals counted on one word, each CTA
// waits for its generation's total. Bounded: after bc->polls polls it raises err, and
// every other waiting CTA sees err and leaves too.
__device__ bool grid_barrier(BatchCtl* bc, unsigned int& gen) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    ++gen;
    const unsigned int target = gen * gridDim.x + bc->extra;
    const unsigned int polls = bc->polls;
    __threadfence();
    atomicAdd(&bc->bar, 1u);
    int ok = 1;
    unsigned int spins = 0;
    while (ld_relaxed_u32(&bc->bar) < target) {
      if (*(volatile int*)&bc->err) {
        ok = 0;
        break;
      }
      if (++spins > polls) {
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

// Sets level `it` for the lanes in `lanes` of w's staged row: per group of 8 lanes (16 B)
// one vector read-modify-write instead of one 2-byte store per lane.
// Group q (lanes 8q .. 8q+7) of that update.
__device__ __forceinline__ void set_lane_levels_q(const SlotDev& s, int32_t w, uint64_t lanes, uint16_t it, int q) {
  const uint32_t m8 = (uint32_t)(lanes >> (8 * q)) & 0xFFu;
  if (!m8) return;
  uint4* row = reinterpret_cast<uint4*>(s.L + (int64_t)w * 64);
  const uint32_t it2 = (uint32_t)it * 0x10001u;
  uint4 x = m8 == 0xFFu ? make_uint4(0, 0, 0, 0) : row[q];
  uint32_t* xw = reinterpret_cast<uint32_t*>(&x);
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const uint32_t keep = ((m8 >> (2 * h)) & 1u ? 0u : 0xFFFFu) | ((m8 >> (2 * h + 1)) & 1u ? 0u : 0xFFFF0000u);
    xw[h] = (xw[h] & keep) | (it2 & ~keep);
  }
  row[q] = x;
}

__device__ __forceinline__ void set_lane_levels(const SlotDev& s, int32_t w, uint64_t lanes, uint16_t it) {
  for (int q = 0; q < 8; ++q) set_lane_levels_q(s, w, lanes, it, q);
}

// Ascending scan of entries [b, e) of w's adjacency by one thread, assigning each lane of
// `want` not yet in `got` the first neighbour whose frontier word carries it (so the
// smallest). Four entries and their frontier words are loaded together per step.
__device__ __forceinline__ uint64_t hits_thread(const SlotDev& s, const uint64_t* __restrict__ fc, int32_t w,
                                                uint64_t want, uint64_t got, int64_t b, int64_t e, int64_t& ne) {
  int32_t* prow = s.P + (int64_t)w * 64;
  int64_t k = b;
  for (; k < e && got != want; k += 4) {
    int32_t u[4];
    uint64_t f[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) u[t] = k + t < e ? s.ccol[k + t] : -1;
#pragma unroll
    for (int t = 0; t < 4; ++t) f[t] = u[t] >= 0 ? fc[u[t]] : 0ull;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      uint64_t h = f[t] & want & ~got;
      if (h) {
        got |= h;
        const int32_t uo = s.new2old[u[t]];
        while (h) {
          const int l = __ffsll((long long)h) - 1;
          h &= h - 1;
          prow[l] = uo;
        }
      }
    }
  }
  ne += min(k, e) - b;
  return got;
}

// 32-entry windows per step of the flattened scan (4 windows spill registers of batch_run:
// 16.16 vs 16.01 ms for 64 roots at scale 24)
constexpr int CWM = 2;

// The medium adjacencies of a warp's 32 list entries (lane i: vertex w with `want` lanes
// missing, d entries from rb; d = 0 for none) scanned as one flattened sequence, 32 * CWM
// entries per step, so that the warp's time follows the entries' total rather than its
// longest row. Each entry's vertex (its owner lane) is found by a binary search over the
// lanes' start offsets; a segmented inclusive OR-scan over the lanes, restarted where the
// owner changes, gives each entry the lanes that an earlier entry of the same vertex already
// carries, and s_got (this warp's 32 words of shared memory) holds per vertex the lanes
// found in earlier windows. So every lane of `want` takes the first entry carrying it (the
// smallest neighbour id), as in the ascending scan of hits_thread. Returns, in lane i, the
// lanes found for lane i's vertex. All 32 threads of the warp must call.
__device__ __forceinline__ uint64_t hits_lanes32(const SlotDev& s, const uint64_t* __restrict__ fc, int32_t w,
                                                 uint64_t want, int64_t rb, int32_t d, uint64_t* s_got,
                                                 int64_t& ne) {
  const int lane = threadIdx.x & 31;
  const int32_t incl = warp_incl_scan(d);
  const int32_t total = __shfl_sync(FULL, incl, 31);
  const int32_t start = incl - d;
  s_got[lane] = 0ull;
  uint64_t got = 0;
  __syncwarp();
  for (int32_t r0 = 0; r0 < total; r0 += 32 * CWM) {
    if (__all_sync(FULL, got == want)) break;  // every vertex has all its lanes
    const uint64_t open = want & ~got;
    int32_t u[CWM], own[CWM];
    uint64_t h[CWM];
#pragma unroll
    for (int t = 0; t < CWM; ++t) {
      const int32_t idx = r0 + 32 * t + lane;
      int o = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int cand = o + step;
        if (__shfl_sync(FULL, start, cand) <= idx) o = cand;
      }
      own[t] = o;
      const int64_t orb = __shfl_sync(FULL, rb, o);
      const int32_t ost = __shfl_sync(FULL, start, o);
      const uint64_t oopen = __shfl_sync(FULL, open, o);
      u[t] = idx < total && oopen ? BATCH_STREAM_LD(&s.ccol[orb + (idx - ost)]) : -1;
      h[t] = oopen;
    }
#pragma unroll
    for (int t = 0; t < CWM; ++t) {
      if (u[t] >= 0) ++ne;
      h[t] = u[t] >= 0 ? fc[u[t]] & h[t] : 0ull;
    }
#pragma unroll
    for (int t = 0; t < CWM; ++t) {
      if (!__any_sync(FULL, h[t] != 0)) continue;
      uint64_t inc = h[t];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(FULL, inc, o);
        const int yo = __shfl_up_sync(FULL, own[t], o);
        if (lane >= o && yo == own[t]) inc |= y;
      }
      const uint64_t ex = __shfl_up_sync(FULL, inc, 1);
      const int po = __shfl_up_sync(FULL, own[t], 1);
      const int no = __shfl_down_sync(FULL, own[t], 1);
      const int32_t ow = __shfl_sync(FULL, w, own[t]);
      const uint64_t prev = s_got[own[t]];
      uint64_t mine = h[t] & ~prev & ~((lane > 0 && po == own[t]) ? ex : 0ull);
      if (mine) {
        int32_t* prow = s.P + (int64_t)ow * 64;
        const int32_t uo = s.new2old[u[t]];
        while (mine) {
          const int l = __ffsll((long long)mine) - 1;
          mine &= mine - 1;
          prow[l] = uo;
        }
      }
      __syncwarp();
      if ((lane == 31 || no != own[t]) && inc) s_got[own[t]] = prev | inc;  // segment end
      __syncwarp();
    }
    got = s_got[lane];
  }
  return got;
}

// The same scan by a whole warp over entries [b, e), CW windows of 32 entries in flight;
// per window an inclusive OR-scan over the lanes gives each entry the lanes it supplies
// first. ATOMIC: other warps scan other chunks of the same adjacency, so a parent is
// taken with atomicMin (ascending entries = ascending ids: the smallest chunk wins).
template <bool ATOMIC>
__device__ __forceinline__ uint64_t hits_warp(const SlotDev& s, const uint64_t* __restrict__ fc, int32_t w,
                                              uint64_t want, uint64_t got, int64_t b, int64_t e, int64_t& ne) {
  const int lane = threadIdx.x & 31;
  int32_t* prow = s.P + (int64_t)w * 64;
  int64_t k0 = b;
  for (; k0 < e && got != want; k0 += 32 * CW) {
    int32_t u[CW];
    uint64_t h[CW];
#pragma unroll
    for (int t = 0; t < CW; ++t) {
      const int64_t k = k0 + 32 * t + lane;
      u[t] = k < e ? BATCH_STREAM_LD(&s.ccol[k]) : -1;
    }
#pragma unroll
    for (int t = 0; t < CW; ++t) h[t] = u[t] >= 0 ? fc[u[t]] & want : 0ull;
#pragma unroll
    for (int t = 0; t < CW; ++t) {
      const uint64_t ht = h[t] & ~got;
      if (!__any_sync(FULL, ht != 0)) continue;
      uint64_t incl = ht;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl |= y;
      }
      const uint64_t excl = __shfl_up_sync(FULL, incl, 1);
      uint64_t mine = ht & ~(lane ? excl : 0ull);
      if (mine) {
        const int32_t uo = s.new2old[u[t]];
        while (mine) {
          const int l = __ffsll((long long)mine) - 1;
          mine &= mine - 1;
          if (ATOMIC)
            atomicMin((unsigned int*)&prow[l], (unsigned int)uo);
          else
            prow[l] = uo;
        }
      }
      got |= __shfl_sync(FULL, incl, 31);
    }
  }
  if (lane == 0) ne += min(k0, e) - b;
  return got;
}

// Appends the lanes with `first` set to a slot's next frontier list (one atomic per warp).
__device__ __forceinline__ void list_append(bool first, int32_t w, int64_t* count, int32_t* list) {
  const unsigned bal = __ballot_sync(FULL, first);
  if (!bal) return;
  const int lane = threadIdx.x & 31;
  unsigned long long p = 0;
  if (lane == __ffs(bal) - 1) p = atomicAdd((unsigned long long*)count, (unsigned long long)__popc(bal));
  p = __shfl_sync(FULL, p, __ffs(bal) - 1);
  if (first) list[p + __popc(bal & lanemask_lt())] = w;
}

// Top-down push along entries [b, e) of frontier vertex v (vertex id vo, frontier word
// f), a warp, CW windows in flight: each neighbour gets the lanes it lacks ORed into its
// next word (the first to give it any lists it) and, per lane, the smallest frontier
// neighbour as parent by atomicMin.
__device__ __forceinline__ void td_push(const SlotDev& s, uint64_t f, int32_t vo, int64_t b, int64_t e,
                                        uint64_t* fn, int64_t* count, int32_t* list, int64_t& ne) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) ne += max(e - b, (int64_t)0);
  for (int64_t k0 = b; k0 < e; k0 += 32 * CW) {
    int32_t w[CW];
    uint64_t vis[CW];
#pragma unroll
    for (int t = 0; t < CW; ++t) {
      const int64_t k = k0 + 32 * t + lane;
      w[t] = k < e ? BATCH_STREAM_LD(&s.ccol[k]) : -1;
    }
#pragma unroll
    for (int t = 0; t < CW; ++t) vis[t] = w[t] >= 0 ? s.visit[w[t]] : ~0ull;
#pragma unroll
    for (int t = 0; t < CW; ++t) {
      uint64_t nb = f & ~vis[t];
      bool first = false;
      if (nb) {
        first = atomicOr((unsigned long long*)&fn[w[t]], (unsigned long long)nb) == 0ull;
        unsigned int* prow = (unsigned int*)(s.P + (int64_t)w[t] * 64);
        while (nb) {
          const int l = __ffsll((long long)nb) - 1;
          nb &= nb - 1;
          atomicMin(&prow[l], (unsigned int)vo);
        }
      }
      list_append(first, w[t], count, list);
    }
  }
}

// Per-launch reset of every slot's lane words (visit, both fronts) and of the staged
// parents (all ones: parents taken by atomicMin start above every id).
__global__ void batch_clear(SlotDev* slots, int nslots) {
  for (int si = 0; si < nslots; ++si) {
    const SlotDev& s = slots[si];
    const int64_t nc = s.nc > 0 ? s.nc : 1;
    for (int64_t i = gtid(); i < nc; i += gthreads()) {
      s.visit[i] = 0ull;
      s.front[0][i] = 0ull;
      s.front[1][i] = 0ull;
    }
    uint4* P = reinterpret_cast<uint4*>(s.P);
    const int64_t np = nc * 16;  // 64 int32 per vertex
    for (int64_t i = gtid(); i < np; i += gthreads()) P[i] = make_uint4(~0u, ~0u, ~0u, ~0u);
  }
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

__device__ void lane_walk(const SlotDev& s, LaneInit& li);
__device__ void write_lanes(const SlotDev& s, uint64_t mask);
__device__ void fixup_lane(const SlotDev& s, int l);
__device__ void resolve_lanes(const SlotDev& s, const ResolveSeg& sg, const int8_t* ls, int nl, int64_t t0,
                              int64_t nt);
__device__ int list_lanes(uint64_t mask, int8_t* ls);

// Level boundary of a launch with a mailbox (one thread): published roots move into free
// lanes of the launch's slots, in slot order. A lane joining a slot at its boundary J
// (the slot's next iteration) starts at its core vertex on iteration J, so its levels are
// iteration - J + hops; the start vertex enters the slot's next frontier. Sets `closed`
// once no slot can take a root at a later boundary.
__device__ void admit_roots(SlotDev* slots, SlotCtl* sctl, int nslots, const int* s_done, const int* s_cur,
                            const int* s_it) {
  BatchMailbox* mb = slots[0].mb;
  if (!mb) return;
  volatile BatchMailbox* vm = mb;
  if (vm->closed) return;
  const int join_max = slots[0].join_max;
  int taken = vm->taken;
  const int count = min(vm->count, MAILBOX_CAP);
  __threadfence_system();  // the entries below were published before this count
  bool later = false;
  for (int si = 0; si < nslots; ++si) {
    if (s_done[si]) continue;
    const int J = s_it[si] + 1;
    if (J > join_max) continue;
    SlotDev& s = slots[si];
    SlotCtl& c = sctl[si];
    const int nxt = s_cur[si] ^ 1;
    while (taken < count && s.nlanes < 64) {
      const int l = s.nlanes;
      LaneInit& li = s.lane[l];
      li.root = (int32_t)vm->e[taken].root;
      s.outp[l] = vm->e[taken].outp;
      s.outl[l] = vm->e[taken].outl;
      vm->e[taken].lane_id = si * 64 + l;
      lane_walk(s, li);
      li.base -= J;
      if (li.start >= 0) {
        const uint64_t bit = 1ull << l;
        s.visit[li.start] |= bit;
        s.P[(int64_t)li.start * 64 + l] = li.sparent;
        s.L[(int64_t)li.start * 64 + l] = (uint16_t)J;
        const uint64_t old = s.front[nxt][li.start];
        s.front[nxt][li.start] = old | bit;
        if (old == 0) {
          s.fl[nxt][c.fl_n[nxt]++] = li.start;
          c.m_next += s.crow[li.start + 1] - s.crow[li.start];
        }
        s.active |= bit;
        s.joined |= bit;
        s.joined_now |= bit;
        c.alive |= bit;
      }
      s.nlanes = l + 1;
      ++taken;
    }
    if (J < join_max && s.nlanes < 64) later = true;
  }
  __threadfence_system();  // lane ids of the admitted entries before the new count
  vm->taken = taken;
  if (!later) vm->closed = 1;
  __threadfence_system();
}

// With a mailbox (roots may join a running launch, so lanes can end many levels apart),
// lanes whose traversal has ended (no discovery at a level) while their slot goes on are
// written out at that level boundary: outputs, root walk and resolution for those lanes
// only, grid barriers between the steps; then their bits are set in the mailbox's done
// words for the host. They also leave the bottom-up miss masks. Not inlined: the
// traversal loop keeps its own register budget.
__device__ __noinline__ bool emit_lanes(SlotDev* slots, SlotCtl* sctl, int nslots, BatchCtl* bc,
                                        const ResolveSeg* segs, int maxh, unsigned int& gen) {
  __shared__ int8_t ls[64];
  __shared__ int nl;
  for (int si = 0; si < nslots; ++si) {
    const uint64_t fin = *(volatile const uint64_t*)&sctl[si].fin;
    if (fin) write_lanes(slots[si], fin);
  }
  if (!grid_barrier(bc, gen)) return false;
  for (int64_t t = gtid(); t < (int64_t)nslots * 64; t += gthreads()) {
    const int si = (int)(t >> 6), l = (int)(t & 63);
    if ((*(volatile const uint64_t*)&sctl[si].fin >> l) & 1ull) fixup_lane(slots[si], l);
  }
  for (int h = 0; h < maxh; ++h) {
    if (!grid_barrier(bc, gen)) return false;
    for (int si = 0; si < nslots; ++si) {
      const uint64_t fin = *(volatile const uint64_t*)&sctl[si].fin;
      if (!fin) continue;
      __syncthreads();
      if (threadIdx.x == 0) nl = list_lanes(fin, ls);
      __syncthreads();
      resolve_lanes(slots[si], segs[(size_t)h * nslots + si], ls, nl, gtid(), gthreads());
    }
  }
  __threadfence_system();  // results reach memory before the host sees the done bits
  if (!grid_barrier(bc, gen)) return false;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    volatile BatchMailbox* vm = slots[0].mb;
    for (int si = 0; si < nslots && si < MAILBOX_WORDS; ++si) {
      const uint64_t fin = *(volatile const uint64_t*)&sctl[si].fin;
      if (fin) vm->done[si] = vm->done[si] | fin;
    }
    __threadfence_system();
  }
  return true;
}

__global__ void __launch_bounds__(BT, 4)
    batch_run(SlotDev* slots, SlotCtl* sctl, int nslots, BatchCtl* bc, const ResolveSeg* segs, int maxh) {
  __shared__ int s_cur[MAX_SLOTS_SMEM], s_dir[MAX_SLOTS_SMEM], s_done[MAX_SLOTS_SMEM], s_it[MAX_SLOTS_SMEM];
  __shared__ int64_t s_ncur[MAX_SLOTS_SMEM];
  __shared__ uint64_t s_got[BT / 32][32];  // per warp: lanes found per vertex (hits_lanes32)
  const bool early = slots[0].mb != nullptr;
  const int lane = threadIdx.x & 31;
  const int64_t gw = gtid() >> 5, nw = gthreads() >> 5;
  unsigned int gen = 0;
  int64_t w_pull = 0, w_push = 0, v_pull = 0, v_disc = 0;  // work of this thread (see BatchCtl)
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
        // push: a warp per frontier vertex; of a long adjacency only the first chunk here,
        // the others are queued for the second pass, where every warp takes chunks
        const int64_t nf = s_ncur[si];
        for (int64_t j = gw; j < nf; j += nw) {
          const int32_t v = s.fl[cur][j];
          const int64_t b = s.crow[v], e = s.crow[v + 1];
          const int64_t nch = (e - b + BATCH_CHUNK - 1) / BATCH_CHUNK;
          if (nch > 1 && lane == 0) {
            const unsigned long long p =
                atomicAdd((unsigned long long*)&sctl[si].q_n, (unsigned long long)(nch - 1));
            for (int64_t c = 1; c < nch; ++c) s.q[p + c - 1] = ((uint64_t)v << 32) | (uint32_t)c;
          }
          td_push(s, fc[v], s.new2old[v], b, min(e, b + BATCH_CHUNK), fn, &sctl[si].fl_n[nxt], s.fl[nxt], w_push);
        }
      } else {
        // pull: every core vertex still missing lanes scans its ascending adjacency for the
        // first neighbour carrying each missing lane (min-id parents). Short adjacencies:
        // a lane each; medium ones (large cores): 32 to a warp, flattened; long ones:
        // chunks, a warp each, parents by atomicMin.
        // Young lanes (joined one or two boundaries ago) are pushed top-down below; while
        // there are any, next-frontier words are set by atomicOr from both sides.
        // Without a mailbox, a vertex whose adjacency one thread or one warp scans whole is
        // committed here (levels, visit word, its degree into m_next): no other reader of
        // its visit word runs in this phase, and the commit phase skips it.
        const uint64_t yg = early ? *(volatile const uint64_t*)&s.young : 0ull;
        const uint64_t act = *(volatile const uint64_t*)&s.active & ~yg;  // lanes may have joined at the last boundary
        const uint16_t it1 = (uint16_t)(s_it[si] + 1);
        int64_t msum = 0;
        // long rows first, then medium, then short ones: the small tasks fill the tail
        {
          const int ntask = (int)s.n_items;
          unsigned* cnt = &sctl[si].grab[0];
          const int gsz = grab_size(ntask, nw);
          int t0 = grab_take(grab_issue(cnt, gsz));
          while (t0 < ntask) {
            const unsigned nx = grab_issue(cnt, gsz);  // next tasks, in flight meanwhile
            for (int task = t0; task < min(t0 + gsz, ntask); ++task) {
              const int64_t it = task;
              const int4 rec = BATCH_STREAM_LD(reinterpret_cast<const int4*>(s.items) + it);
              const int64_t b = (int64_t)(((uint64_t)(uint32_t)rec.y << 32) | (uint32_t)rec.x);
              const int32_t w = rec.z;
              const uint32_t meta = (uint32_t)rec.w;
              const int64_t e = b + (meta & BATCH_ITEM_LEN);
              const uint64_t vw = BATCH_STREAM_LD(&s.visit[w]);
              const uint64_t miss = act & ~vw;
              if (!miss) continue;
              const bool whole = meta & BATCH_ITEM_WHOLE;
              if (lane == 0 && (meta & BATCH_ITEM_FIRST)) ++v_pull;
              const uint64_t got = whole ? hits_warp<false>(s, fc, w, miss, 0ull, b, e, w_pull)
                                         : hits_warp<true>(s, fc, w, miss, 0ull, b, e, w_pull);
              if (got && whole && !early && lane < 8) set_lane_levels_q(s, w, got, it1, lane);
              bool first = false;
              if (got && lane == 0) {
                if (whole && !yg) {
                  fn[w] = got;
                  first = true;
                  if (!early) {
                    s.visit[w] = vw | got;
                    msum += e - b;
                  }
                } else {
                  first = atomicOr((unsigned long long*)&fn[w], (unsigned long long)got) == 0ull;
                }
              }
              list_append(first, w, &sctl[si].fl_n[nxt], s.fl[nxt]);
            }
            t0 = grab_take(nx);
          }
        }
        {
          const int ntask = (int)((s.n_mids + 31) / 32);
          unsigned* cnt = &sctl[si].grab[1];
          const int gsz = grab_size(ntask, nw);
          int t0 = grab_take(grab_issue(cnt, gsz));
          while (t0 < ntask) {
            const unsigned nx = grab_issue(cnt, gsz);  // next tasks, in flight meanwhile
            for (int task = t0; task < min(t0 + gsz, ntask); ++task) {
              const int64_t i0 = (int64_t)task * 32;
              const int64_t i = i0 + lane;
              int32_t w = -1, d = 0;
              int64_t rb = 0;
              uint64_t miss = 0, vw = 0, got = 0;
              if (i < s.n_mids) {
                w = BATCH_STREAM_LD(&s.mids[i]);
                vw = BATCH_STREAM_LD(&s.visit[w]);
                miss = act & ~vw;
                if (miss) {
                  rb = s.crow[w];
                  d = (int32_t)(s.crow[w + 1] - rb);
                  ++v_pull;
                }
              }
              if (__any_sync(FULL, d > 0)) got = hits_lanes32(s, fc, w, miss, rb, d, s_got[threadIdx.x >> 5], w_pull);
              if (got && !early) {
                set_lane_levels(s, w, got, it1);
                s.visit[w] = vw | got;
                msum += d;
              }
              bool first = got != 0;
              if (got) {
                if (yg)
                  first = atomicOr((unsigned long long*)&fn[w], (unsigned long long)got) == 0ull;
                else
                  fn[w] = got;
              }
              list_append(first, w, &sctl[si].fl_n[nxt], s.fl[nxt]);
            }
            t0 = grab_take(nx);
          }
        }
        {
          const int ntask = (int)((s.n_lanes + 31) / 32);
          unsigned* cnt = &sctl[si].grab[2];
          const int gsz = grab_size(ntask, nw);
          int t0 = grab_take(grab_issue(cnt, gsz));
          while (t0 < ntask) {
            const unsigned nx = grab_issue(cnt, gsz);  // next tasks, in flight meanwhile
            for (int task = t0; task < min(t0 + gsz, ntask); ++task) {
              const int64_t i0 = (int64_t)task * 32;
              const int64_t i = i0 + lane;
              int32_t w = -1;
              uint64_t got = 0;
              if (i < s.n_lanes) {
                w = BATCH_STREAM_LD(&s.lanes[i]);
                const uint64_t vw = BATCH_STREAM_LD(&s.visit[w]);
                const uint64_t miss = act & ~vw;
                if (miss) {
                  const int64_t rb = s.crow[w], re = s.crow[w + 1];
                  got = hits_thread(s, fc, w, miss, 0ull, rb, re, w_pull);
                  ++v_pull;
                  if (got && !early) {
                    set_lane_levels(s, w, got, it1);
                    s.visit[w] = vw | got;
                    msum += re - rb;
                  }
                }
              }
              bool first = got != 0;
              if (got) {
                if (yg)
                  first = atomicOr((unsigned long long*)&fn[w], (unsigned long long)got) == 0ull;
                else
                  fn[w] = got;
              }
              list_append(first, w, &sctl[si].fl_n[nxt], s.fl[nxt]);
            }
            t0 = grab_take(nx);
          }
        }
        msum = warp_sum(msum);
        if (lane == 0 && msum) atomicAdd((unsigned long long*)&sctl[si].m_next, (unsigned long long)msum);
        if (yg) {
          // push of the young lanes: frontier entries carrying their bits, found 32 at a time
          // by a ballot; a long adjacency's first chunk here, the others queued for E2
          const int64_t nf = s_ncur[si];
          for (int64_t j0 = gw * 32; j0 < nf; j0 += nw * 32) {
            const int64_t j = j0 + lane;
            int32_t v = -1;
            uint64_t f = 0;
            if (j < nf) {
              v = s.fl[cur][j];
              f = fc[v] & yg;
            }
            unsigned m = __ballot_sync(FULL, f != 0);
            while (m) {
              const int src = __ffs(m) - 1;
              m &= m - 1;
              const int32_t vv = __shfl_sync(FULL, v, src);
              const uint64_t ff = __shfl_sync(FULL, f, src);
              const int64_t b = s.crow[vv], e = s.crow[vv + 1];
              const int64_t nch = (e - b + BATCH_CHUNK - 1) / BATCH_CHUNK;
              if (nch > 1 && lane == 0) {
                const unsigned long long p =
                    atomicAdd((unsigned long long*)&sctl[si].q_n, (unsigned long long)(nch - 1));
                for (int64_t c = 1; c < nch; ++c) s.q[p + c - 1] = ((uint64_t)vv << 32) | (uint32_t)c;
              }
              td_push(s, ff, s.new2old[vv], b, min(e, b + BATCH_CHUNK), fn, &sctl[si].fl_n[nxt], s.fl[nxt],
                      w_push);
            }
          }
        }
      }
    }
    if (!grid_barrier(bc, gen)) return;
    // ---- E2: queued chunks of long top-down adjacencies (all slots, one pass; in a slot
    // pulling bottom-up, the young lanes' chunks)
    bool any_q = false;
    for (int si = 0; si < nslots; ++si) {
      if (s_done[si]) continue;
      const int64_t nq = sctl[si].q_n;
      if (nq == 0) continue;
      any_q = true;
      const SlotDev& s = slots[si];
      const uint64_t lanes = s_dir[si] == DIR_TD ? ~0ull : *(volatile const uint64_t*)&s.young;
      const int cur = s_cur[si], nxt = cur ^ 1;
      for (int64_t j = gw; j < nq; j += nw) {
        const uint64_t item = s.q[j];
        const int32_t v = (int32_t)(item >> 32);
        const int64_t rb = s.crow[v], re = s.crow[v + 1];
        const int64_t b = rb + (int64_t)(uint32_t)item * BATCH_CHUNK;
        td_push(s, s.front[cur][v] & lanes, s.new2old[v], b, min(re, b + BATCH_CHUNK), s.front[nxt],
                &sctl[si].fl_n[nxt], s.fl[nxt], w_push);
      }
    }
    if (any_q && !grid_barrier(bc, gen)) return;
    // ---- P: levels and visit of the discoveries
    for (int si = 0; si < nslots; ++si) {
      if (s_done[si]) continue;
      const SlotDev& s = slots[si];
      const int cur = s_cur[si], nxt = cur ^ 1;
      const uint64_t* fn = s.front[nxt];
      const int64_t nn = sctl[si].fl_n[nxt];
      const uint16_t it = (uint16_t)(s_it[si] + 1);
      int64_t msum = 0;
      uint64_t alive = 0;
      for (int64_t j = gtid(); j < nn; j += gthreads()) {
        ++v_disc;
        const int32_t w = s.fl[nxt][j];
        const uint64_t nb = fn[w];
        const uint64_t vw = s.visit[w];
        if ((vw & nb) == nb) continue;  // committed by the pull that found it
        msum += s.crow[w + 1] - s.crow[w];
        set_lane_levels(s, w, nb, it);
        s.visit[w] = vw | nb;
        alive |= nb;
      }
      msum = warp_sum(msum);
      if (lane == 0 && msum) atomicAdd((unsigned long long*)&sctl[si].m_next, (unsigned long long)msum);
      if (early) {
        const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)alive);
        const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(alive >> 32));
        alive = ((uint64_t)hi << 32) | lo;
        if (lane == 0 && alive) atomicOr((unsigned long long*)&sctl[si].alive, (unsigned long long)alive);
      }
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
      if (threadIdx.x == 0) bc->emit = 0;
      if (threadIdx.x == 0 && early) admit_roots(slots, sctl, nslots, s_done, s_cur, s_it);
      __syncthreads();
      for (int si = threadIdx.x; si < nslots; si += BT) {
        SlotCtl& c = sctl[si];
        c.fin = 0;
        if (s_done[si]) continue;
        SlotDev& s = slots[si];
        const int cur = s_cur[si], nxt = cur ^ 1;
        const int64_t nn = c.fl_n[nxt];
        c.fl_n[cur] = 0;
        c.q_n = 0;
        c.grab[0] = c.grab[1] = c.grab[2] = 0;
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
        const uint64_t alive = c.alive;
        c.alive = 0;
        // lanes ending with their slot are left to the output kernels, and so are all of a
        // slot without joined lanes: lanes started together end a few levels apart
        if (early && !c.done && (s.joined & ~s.emitted)) {
          const uint64_t fin = lanes_of(s.nlanes) & ~s.emitted & ~alive;
          if (fin) {
            c.fin = fin;
            s.emitted |= fin;
            s.active &= ~fin;
            atomicAdd(&bc->emit, 1);
          }
        }
        if (early) {  // young for the two levels after joining
          s.young = (s.joined_now | s.young_prev) & s.active;
          s.young_prev = s.joined_now;
          s.joined_now = 0;
        }
      }
    }
    if (!grid_barrier(bc, gen)) return;
    if (early && *(volatile int*)&bc->emit && !emit_lanes(slots, sctl, nslots, bc, segs, maxh, gen)) return;
    if (*(volatile int*)&bc->live <= 0) break;
  }
  // the launch's work counts: warp sums, one atomic per warp and counter
  w_pull = warp_sum(w_pull);
  w_push = warp_sum(w_push);
  v_pull = warp_sum(v_pull);
  v_disc = warp_sum(v_disc);
  if (lane == 0) {
    if (w_pull) atomicAdd(&bc->work[0], (unsigned long long)w_pull);
    if (w_push) atomicAdd(&bc->work[1], (unsigned long long)w_push);
    if (v_pull) atomicAdd(&bc->work[2], (unsigned long long)v_pull);
    if (v_disc) atomicAdd(&bc->work[3], (unsigned long long)v_disc);
  }
}

// Root-major outputs in vertex-id order for the lanes in `mask`. A CTA takes 32
// consecutive vertices; warp k writes lanes 8k..8k+7 of the slot, each lane's 32 values
// coalesced. Core vertices and tree vertices hanging from a core vertex are final here;
// tree vertices hanging from a tree vertex get -2 ("resolve pending") for the resolution.
// The lanes' output pointers are re-read per chunk (L1 hits), which keeps registers low.
__device__ void write_lanes(const SlotDev& s, uint64_t mask) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const uint32_t wm = (uint32_t)(mask >> (wp * 8)) & 0xFFu;  // lanes of the slot this warp writes
  if (!wm) return;
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
    const uint32_t vis = cid >= 0 ? (uint32_t)(s.visit[cid] >> (wp * 8)) & wm : 0u;
    // this warp's 8 lanes of the vertex's staged row: 16 B of levels, 32 B of parents
    uint4 lv8 = make_uint4(0, 0, 0, 0);
    int4 pa0 = make_int4(0, 0, 0, 0), pa1 = pa0;
    if (vis) {
      lv8 = *reinterpret_cast<const uint4*>(s.L + (int64_t)cid * 64 + wp * 8);
      if (!add) {
        pa0 = *reinterpret_cast<const int4*>(s.P + (int64_t)cid * 64 + wp * 8);
        pa1 = *reinterpret_cast<const int4*>(s.P + (int64_t)cid * 64 + wp * 8 + 4);
      }
    }
    const uint32_t lw[4] = {lv8.x, lv8.y, lv8.z, lv8.w};
    const int32_t pw[8] = {pa0.x, pa0.y, pa0.z, pa0.w, pa1.x, pa1.y, pa1.z, pa1.w};
    const int32_t none = info == INT32_MIN ? -2 : -1;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (!((wm >> k) & 1u) || !in) continue;
      const bool r = (vis >> k) & 1u;
      const int32_t lk = (int32_t)((lw[k >> 1] >> (16 * (k & 1))) & 0xFFFFu);
      int32_t* pk = s.outp[wp * 8 + k];
      int32_t* lq = s.outl[wp * 8 + k];
      const int32_t bk = s.lane[wp * 8 + k].base;
      lq[v] = r ? lk + bk + add : none;
      pk[v] = r ? (add ? fixed_parent : pw[k]) : none;
    }
  }
}

// Root on an edge tree: levels and parents along the walk from the root to the core,
// direction reversed; the core vertex reached takes the last tree vertex as parent.
__device__ void fixup_lane(const SlotDev& s, int l) {
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

// One height of the tree-up resolution for the lanes listed in `ls` (nl of them): entries
// still at -2 take level(up) + 1 and parent up (Alg. 10 with levels); walk vertices are
// already set. Thread t of `nt` starting at t0.
__device__ void resolve_lanes(const SlotDev& s, const ResolveSeg& sg, const int8_t* ls, int nl, int64_t t0,
                              int64_t nt) {
  const int64_t len = sg.e - sg.b;
  const int64_t total = len * nl;
  for (int64_t t = t0; t < total; t += nt) {
    const int l = ls[t / len];
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

__device__ int list_lanes(uint64_t mask, int8_t* ls) {
  int n = 0;
  while (mask) {
    ls[n++] = (int8_t)(__ffsll((long long)mask) - 1);
    mask &= mask - 1;
  }
  return n;
}

// Output pass after the launch, pointers re-read per chunk: 40 registers, six CTAs per SM
// (measured on 64 roots at scale 24: 17.3 ms per batch vs 19.8 ms with the pointers
// hoisted at 88 registers, two CTAs per SM).
__global__ void __launch_bounds__(BT, 6) batch_output(SlotDev* slots, int nslots) {
  for (int si = 0; si < nslots; ++si) {
    const SlotDev& s = slots[si];
    write_lanes(s, lanes_of(s.nlanes) & ~s.emitted);
  }
}

// Roots on an edge tree, one thread per lane (lanes not written during the launch).
__global__ void batch_fixup(SlotDev* slots, int nslots) {
  const int si = blockIdx.x;
  if (si >= nslots) return;
  const SlotDev& s = slots[si];
  const int l = threadIdx.x;
  if (l >= s.nlanes || ((s.emitted >> l) & 1ull)) return;
  fixup_lane(s, l);
}

// One height of the resolution for every lane of every slot not written during the launch.
__global__ void batch_resolve(SlotDev* slots, const ResolveSeg* segs, int nslots) {
  const int si = blockIdx.y;
  if (si >= nslots) return;
  __shared__ int8_t ls[64];
  __shared__ int nl;
  const SlotDev& s = slots[si];
  if (threadIdx.x == 0) nl = list_lanes(lanes_of(s.nlanes) & ~s.emitted, ls);
  __syncthreads();
  resolve_lanes(s, segs[si], ls, nl, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// The Alg. 9 walk of a lane's root to its core vertex: start (core id, -1: nothing to
// traverse), base (hops), sparent (the start vertex's parent).
__device__ void lane_walk(const SlotDev& s, LaneInit& li) {
  const int32_t root = li.root;
  const int32_t info = s.vinfo[root];
  if (info >= 0) {
    li.start = info;
    li.base = 0;
    li.sparent = root;
    return;
  }
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

// Lane setup on the device (one thread per lane).
__global__ void batch_lanes(SlotDev* slots, int nslots) {
  const int si = blockIdx.x;
  if (si >= nslots) return;
  SlotDev& s = slots[si];
  const int l = threadIdx.x;
  if (l >= s.nlanes) return;
  LaneInit& li = s.lane[l];
  lane_walk(s, li);
  const unsigned long long bit = li.start >= 0 ? (1ull << l) : 0ull;
  if (bit) atomicOr((unsigned long long*)&s.active, bit);
}

}  // namespace

void free_batch_mem(gt_graph* g) {
  for (void* p : g->batch_mem) cudaFree(p);
  g->batch_mem.clear();
  g->batch_slots_alloc = 0;
}

void slot_sizes(const gt_graph* g, size_t sz[SLOT_BUFS]) {
  const size_t nc = (size_t)std::max<int64_t>(g->core.n, 1);
  const size_t q = 2 * (size_t)(g->core.nnz / BATCH_CHUNK) + 64;  // chunks of long frontier adjacencies
  const size_t v[SLOT_BUFS] = {8 * nc, 8 * nc, 8 * nc, 256 * nc, 128 * nc, 4 * nc, 4 * nc, 8 * q};
  for (int i = 0; i < SLOT_BUFS; ++i) sz[i] = v[i];
}

size_t slot_bytes(const gt_graph* g) {
  size_t sz[SLOT_BUFS], t = 0;
  slot_sizes(g, sz);
  for (int i = 0; i < SLOT_BUFS; ++i) t += sz[i];
  return t;
}

// Grows the handle's pool of lane-word storage (SLOT_BUFS buffers per 64 roots) to `need`
// slots.
int ensure_slots(gt_graph* g, int need) {
  size_t sz[SLOT_BUFS];
  slot_sizes(g, sz);
  while (g->batch_slots_alloc < need) {
    void* p[SLOT_BUFS];
    for (int i = 0; i < SLOT_BUFS; ++i) {
      int rc = device_malloc(g, &p[i], sz[i]);
      if (rc) {
        for (int j = 0; j < i; ++j) cudaFree(p[j]);
        return rc;
      }
    }
    for (int i = 0; i < SLOT_BUFS; ++i) g->batch_mem.push_back(p[i]);
    g->batch_slots_alloc += 1;
  }
  return GT_OK;
}

void batch_ctx_free(BatchCtx* c) {
  if (!c) return;
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->dev) cudaFree(c->dev);
  if (c->stage) cudaFreeHost(c->stage);
  if (c->h_err) cudaFreeHost(c->h_err);
  *c = BatchCtx{};
}

namespace {

// Enqueues the kernels of one batched traversal on `st` (tables already in `dev`).
void enqueue_batch(SlotDev* d_slots, SlotCtl* d_ctl, BatchCtl* d_bc, ResolveSeg* d_seg, int ns, int maxh, int grid,
                   int ogrid, int* h_err, const void* stage, void* dev, size_t bytes, cudaStream_t st) {
  cudaMemcpyAsync(dev, stage, bytes, cudaMemcpyHostToDevice, st);
  batch_clear<<<ogrid, BT, 0, st>>>(d_slots, ns);
  batch_lanes<<<ns, 64, 0, st>>>(d_slots, ns);
  batch_init<<<ns, 64, 0, st>>>(d_slots, d_ctl, ns);
  int nsl = ns;
  const ResolveSeg* segs = d_seg;
  int mh = maxh;
  void* kargs[] = {(void*)&d_slots, (void*)&d_ctl, (void*)&nsl, (void*)&d_bc, (void*)&segs, (void*)&mh};
  cudaLaunchCooperativeKernel((void*)batch_run, dim3(grid), dim3(BT), kargs, 0, st);
  batch_output<<<ogrid, BT, 0, st>>>(d_slots, ns);
  batch_fixup<<<ns, 64, 0, st>>>(d_slots, ns);
  for (int h = 0; h < maxh; ++h) batch_resolve<<<dim3(64, ns), BT, 0, st>>>(d_slots, d_seg + (size_t)h * ns, ns);
  cudaMemcpyAsync(h_err, &d_bc->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(h_err + 4, d_bc->work, sizeof(d_bc->work), cudaMemcpyDeviceToHost, st);
}

}  // namespace

int batch_launch(BatchCtx* ctx, const SlotSpec* specs, int nspecs, int sm_share, cudaStream_t st, BatchMailbox* mb,
                 int join_max) {
  if (nspecs <= 0) return GT_OK;
  if (nspecs > MAX_SLOTS_SMEM) {
    set_error("batched BFS: more than 256 lane words (16384 roots) in one launch");
    return GT_EINVAL;
  }
  const int ns = nspecs;
  int maxh = 0;
  for (int i = 0; i < ns; ++i) maxh = std::max(maxh, specs[i].g->resolve_heights);
  // table layout: slots | slot control | batch control | resolution segments
  const size_t t_slots = (sizeof(SlotDev) * ns + 255) & ~(size_t)255;
  const size_t t_ctl = (sizeof(SlotCtl) * ns + 255) & ~(size_t)255;
  const size_t t_bc = 256;
  const size_t bytes = t_slots + t_ctl + t_bc + sizeof(ResolveSeg) * (size_t)ns * std::max(maxh, 1);
  if (ctx->cap_bytes < bytes) {
    // the captured graph points at the old buffers: drop it with them
    if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
    ctx->exec = nullptr;
    if (ctx->dev) cudaFree(ctx->dev);
    if (ctx->stage) cudaFreeHost(ctx->stage);
    ctx->dev = ctx->stage = nullptr;
    ctx->cap_bytes = 0;
    int rc = cuda_fail(cudaMalloc(&ctx->dev, bytes), "batch table");
    if (rc == GT_OK) rc = cuda_fail(cudaHostAlloc(&ctx->stage, bytes, cudaHostAllocDefault), "batch staging");
    if (rc) return rc;
    ctx->cap_bytes = bytes;
  }
  if (!ctx->h_err) {
    // status word, then (from int 4 on) the launch's four work counters
    int rc = cuda_fail(cudaHostAlloc((void**)&ctx->h_err, sizeof(int) * 12, cudaHostAllocDefault), "pinned status");
    if (rc) return rc;
  }
  ctx->h_err[0] = 0;
  char* hb = (char*)ctx->stage;
  SlotDev* hs = (SlotDev*)hb;
  SlotCtl* hc = (SlotCtl*)(hb + t_slots);
  BatchCtl* hbc = (BatchCtl*)(hb + t_slots + t_ctl);
  ResolveSeg* hseg = (ResolveSeg*)(hb + t_slots + t_ctl + t_bc);
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
    d.lanes = g->batch_lane;
    d.mids = g->batch_mid;
    d.items = g->batch_item;
    d.n_lanes = g->n_batch_lane;
    d.n_mids = g->n_batch_mid;
    d.n_items = g->n_batch_item;
    d.visit = (uint64_t*)sp.mem[0];
    d.front[0] = (uint64_t*)sp.mem[1];
    d.front[1] = (uint64_t*)sp.mem[2];
    d.P = (int32_t*)sp.mem[3];
    d.L = (uint16_t*)sp.mem[4];
    d.fl[0] = (int32_t*)sp.mem[5];
    d.fl[1] = (int32_t*)sp.mem[6];
    d.q = (uint64_t*)sp.mem[7];
    d.nlanes = sp.nlanes;
    d.alpha = g->tuning.batch_alpha;
    d.beta = g->tuning.batch_beta;
    d.mb = mb;
    d.join_max = mb ? join_max : 0;
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
    hc[i] = SlotCtl{{0, 0}, 0, 0, 0, DIR_TD, 0, 0, 0, 0};
    // heights are processed top down; each slot walks its own graph's segments
    for (int h = 0; h < maxh; ++h) {
      ResolveSeg sg{g->resolve_list, g->resolve_up, 0, 0};
      if (h < g->resolve_heights) {
        sg.b = g->resolve_ptr_host[h];
        sg.e = g->resolve_ptr_host[h + 1];
      }
      hseg[(size_t)h * ns + i] = sg;
    }
  }
  *hbc = BatchCtl{0u, 0, ns, 0, g_barrier_polls.load(), g_barrier_extra.load(), {0ull, 0ull, 0ull, 0ull}};
  char* base = (char*)ctx->dev;
  SlotDev* d_slots = (SlotDev*)base;
  SlotCtl* d_ctl = (SlotCtl*)(base + t_slots);
  BatchCtl* d_bc = (BatchCtl*)(base + t_slots + t_ctl);
  ResolveSeg* d_seg = (ResolveSeg*)(base + t_slots + t_ctl + t_bc);
  int nb_per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_per_sm, batch_run, BT, 0);
  const int share = std::max(1, std::min(sm_share > 0 ? sm_share : g0->launch.sms, g0->launch.sms));
  const int grid = std::max(1, std::min(nb_per_sm, 4)) * share;
  const int ogrid = share * 16;
  const bool same = ctx->exec && ctx->key_ns == ns && ctx->key_maxh == maxh && ctx->key_grid == grid &&
                    ctx->key_ogrid == ogrid && ctx->key_bytes == bytes;
  if (!same) {
    if (ctx->exec) cudaGraphExecDestroy(ctx->exec);
    ctx->exec = nullptr;
    if (!ctx->cap_stream) {
      int rc = cuda_fail(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "capture stream");
      if (rc) return rc;
    }
    int rc = cuda_fail(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "batch capture");
    if (rc) return rc;
    enqueue_batch(d_slots, d_ctl, d_bc, d_seg, ns, maxh, grid, ogrid, ctx->h_err, ctx->stage, ctx->dev, bytes,
                  ctx->cap_stream);
    cudaGraph_t graph = nullptr;
    rc = cuda_fail(cudaStreamEndCapture(ctx->cap_stream, &graph), "batch capture end");
    if (rc == GT_OK) rc = cuda_fail(cudaGraphInstantiate(&ctx->exec, graph, 0), "batch graph instantiate");
    if (graph) cudaGraphDestroy(graph);
    if (rc) return rc;
    ctx->key_ns = ns;
    ctx->key_maxh = maxh;
    ctx->key_grid = grid;
    ctx->key_ogrid = ogrid;
    ctx->key_bytes = bytes;
  }
  return cuda_fail(cudaGraphLaunch(ctx->exec, st), "batch graph launch");
}

void set_barrier_test(unsigned int polls, unsigned int extra) {
  g_barrier_polls.store(polls ? polls : BARRIER_POLLS);
  g_barrier_extra.store(extra);
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
  // lane words per graph (a graph may be listed more than once): grow every pool first, so
  // no pointer into a pool is taken before the pool stops growing
  std::vector<std::pair<gt_graph*, int>> need;
  for (int gi = 0; gi < ngraphs; ++gi) {
    const int nsg = (rpg[gi] + 63) / 64;
    bool seen = false;
    for (auto& u : need)
      if (u.first == graphs[gi]) {
        u.second += nsg;
        seen = true;
      }
    if (!seen) need.emplace_back(graphs[gi], nsg);
  }
  for (auto& u : need) {
    int rc = ensure_slots(u.first, u.second);
    if (rc) return rc;
    u.second = 0;  // from here: lane words handed out so far
  }
  int64_t ro = 0;
  for (int gi = 0; gi < ngraphs; ++gi) {
    gt_graph* g = graphs[gi];
    const int r = rpg[gi];
    const int nsg = (r + 63) / 64;
    int first = 0;
    for (auto& u : need)
      if (u.first == g) {
        first = u.second;
        u.second += nsg;
      }
    for (int k = 0; k < nsg; ++k) {
      SlotSpec sp;
      sp.g = g;
      sp.mem = &g->batch_mem[(size_t)SLOT_BUFS * (first + k)];
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
  if (!rc) memcpy(g0->batch_work, g0->batch_ctx->h_err + 4, sizeof(g0->batch_work));
  return rc;
}

}  // namespace gt
