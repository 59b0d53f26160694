// serve.cu -- continuous-batching BFS server over resident graphs.
//
// Queries (graph, root, caller-owned device outputs) are queued per graph. Whenever one of
// the server's streams is free, a scheduler thread dispatches the pending roots of the
// graph with the oldest query in one of two forms, whichever its running estimates say
// is cheaper: up to 64 single-root edge-tree traversals back to back on the stream (each
// query completes on its own), or one batched launch (64 roots per lane word, batch.cu)
// whose cost hardly depends on how many lanes are filled. A graph runs at most one
// single-root flight at a time (the traversal state is the graph's own). A batched
// launch is dispatched at once when the GPU is idle; otherwise, if batching pays on that
// graph, the scheduler waits up to `window_us` to fill lane words. Flights on different
// streams overlap on the device; at most two are batched launches, each cooperative on
// half of the SMs. Graphs are admitted against an HBM budget
// (graph storage + one lane word of batch storage); more lane-word storage is taken
// while the budget allows. Completion is signalled by a host callback on the stream,
// which stamps every query's latency (submit -> results in the caller's buffers). With
// join_levels > 0, roots submitted while a batched launch of their graph runs are
// published in a page-locked mailbox and join its free lanes at a level boundary; such a
// launch also reports in the mailbox each lane whose results are written before it ends,
// and the scheduler completes those queries at once.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gt_internal.cuh"

namespace gt {
namespace {

using Clock = std::chrono::steady_clock;

double now_us() {
  return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

struct Query {
  uint64_t ticket = 0;
  int32_t gid = 0;
  int64_t root = 0;
  int32_t* parent = nullptr;
  int32_t* level = nullptr;
  double t_submit = 0, t_done = 0;
  bool done = false;
  int rc = GT_OK;
};

struct SlotBuf {
  void* p[SLOT_BUFS];
};

struct GraphEntry {
  gt_graph* g = nullptr;
  std::deque<Query*> pending;
  std::vector<SlotBuf> slots;  // lane-word storage owned by the server
  std::vector<int> free_slots;
  bool single_busy = false;    // a flight is running single-root traversals on this graph
  double est_single_us = 0;    // running estimates (0 = not measured yet): one single-root
  double est_word_us = 0;      // traversal; one 64-root lane word in a batched launch
};

struct Flight;
struct QueryDone {
  Flight* f;
  Query* q;
};

// Work on one stream: either one batched launch over `slots`, or `queries` run as
// single-root traversals one after another (each completes on its own).
struct Flight {
  void* srv = nullptr;
  int stream = 0;
  int gid = 0;
  bool single = false;
  double t_launch = 0, t_prev = 0;
  int remaining = 0;
  std::vector<Query*> queries;
  std::vector<int> slots;
  std::vector<QueryDone> done;
  BatchMailbox* mb = nullptr;  // batched: joining roots and early completions (host address)
  int capacity = 0;            // free lanes the launch can still fill
  std::vector<Query*> late;    // queries published in mb, in mailbox order
  std::vector<Query*> lane_q;  // batched: query of each lane (word * 64 + lane); null once completed
  std::vector<uint64_t> seen;  // done bits already handled, per lane word
  int late_seen = 0;           // mailbox entries already placed in lane_q
};

double ema(double old, double x) { return old > 0 ? 0.8 * old + 0.2 * x : x; }

// Places mailbox entries admitted since the last look into their lanes.
void map_admitted(Flight* f, int taken) {
  volatile BatchMailbox* vm = f->mb;
  taken = std::max(0, std::min(taken, (int)f->late.size()));
  for (; f->late_seen < taken; ++f->late_seen) {
    const int id = vm->e[f->late_seen].lane_id;
    if (id >= 0 && id < (int)f->lane_q.size()) f->lane_q[id] = f->late[f->late_seen];
  }
}

}  // namespace
}  // namespace gt

struct gt_server {
  gt_serve_config cfg{};
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<gt::GraphEntry> graphs;  // stable addresses: the scheduler keeps references
  std::unordered_map<uint64_t, gt::Query*> tickets;
  uint64_t next_ticket = 1;
  std::thread worker;
  bool stop = false;
  int device = 0;
  int sms = 1;
  std::vector<cudaStream_t> streams;
  std::vector<gt::BatchCtx> ctxs;
  std::vector<gt::Flight*> flights;  // per stream, null when free
  std::vector<gt::BatchMailbox*> mbox, mbox_dev;  // per stream: pinned mailbox (host / device address)
  int64_t used_bytes = 0;
  // statistics
  int64_t submitted = 0, completed = 0, failed = 0, batches = 0, joined = 0, early = 0;
  double t_first = 0, t_last = 0;
  std::vector<double> lat_us;
};

namespace gt {
namespace {

void complete(gt_server* s, Query* q, int rc, double t) {
  q->done = true;
  q->rc = rc;
  q->t_done = t;
  s->lat_us.push_back(t - q->t_submit);
  if (rc) s->failed++;
  s->completed++;
  s->t_last = t;
}

// Lanes of a running batched launch whose results are already in their buffers (done
// bits in the mailbox) complete now. Caller holds the lock.
void collect_early(gt_server* s, Flight* f) {
  volatile BatchMailbox* vm = f->mb;
  const int words = (int)f->seen.size();
  std::vector<uint64_t> d(words);
  bool any = false;
  for (int w = 0; w < words; ++w) {
    d[w] = vm->done[w] & ~f->seen[w];
    any |= d[w] != 0;
  }
  if (!any) return;
  std::atomic_thread_fence(std::memory_order_acquire);
  map_admitted(f, vm->taken);  // a lane is admitted before its done bit is set
  std::atomic_thread_fence(std::memory_order_acquire);
  const double t = now_us();
  for (int w = 0; w < words; ++w) {
    f->seen[w] |= d[w];
    for (uint64_t b = d[w]; b; b &= b - 1) {
      const int id = w * 64 + __builtin_ctzll(b);
      Query* q = f->lane_q[id];
      if (!q) continue;
      f->lane_q[id] = nullptr;
      complete(s, q, GT_OK, t);
      s->early++;
    }
  }
  s->cv_done.notify_all();
}

// Host callback after one single-root traversal of a single-mode flight.
void CUDART_CB on_query_done(void* arg) {
  QueryDone* d = (QueryDone*)arg;
  Flight* f = d->f;
  gt_server* s = (gt_server*)f->srv;
  const double t = now_us();
  std::lock_guard<std::mutex> lk(s->mu);
  GraphEntry& ge = s->graphs[f->gid];
  ge.est_single_us = ema(ge.est_single_us, t - f->t_prev);
  f->t_prev = t;
  complete(s, d->q, GT_OK, t);
  if (--f->remaining == 0) {
    ge.single_busy = false;
    s->flights[f->stream] = nullptr;
    delete f;
    s->cv_sched.notify_all();
  }
  s->cv_done.notify_all();
}

void CUDART_CB on_flight_done(void* arg) {
  Flight* f = (Flight*)arg;
  gt_server* s = (gt_server*)f->srv;
  const double t = now_us();
  std::lock_guard<std::mutex> lk(s->mu);
  const int rc = batch_status(&s->ctxs[f->stream]);
  GraphEntry& ge = s->graphs[f->gid];
  if (!f->slots.empty()) ge.est_word_us = ema(ge.est_word_us, (t - f->t_launch) / f->slots.size());
  for (int k : f->slots) ge.free_slots.push_back(k);
  if (f->mb) {
    // the launch has finished: the mailbox is final. Lanes not completed early (all of
    // them if the launch failed before writing them) complete now.
    const int32_t tk = ((volatile BatchMailbox*)f->mb)->taken;
    const size_t taken = (size_t)std::max<int32_t>(0, std::min<int32_t>(tk, (int32_t)f->late.size()));
    map_admitted(f, (int)taken);
    for (size_t i = f->late.size(); i > taken; --i) ge.pending.push_front(f->late[i - 1]);  // not admitted: back in line
    s->joined += (int64_t)taken;
    for (Query*& q : f->lane_q)
      if (q) {
        complete(s, q, rc, t);
        q = nullptr;
      }
  } else {
    for (Query* q : f->queries) complete(s, q, rc, t);
  }
  s->t_last = t;
  s->flights[f->stream] = nullptr;
  delete f;
  s->cv_done.notify_all();
  s->cv_sched.notify_all();
}

// Grows a graph's lane-word pool by one if the budget allows. Caller holds the lock.
bool grow_slots(gt_server* s, GraphEntry& ge) {
  const size_t sb = slot_bytes(ge.g);
  if (s->used_bytes + (int64_t)sb > s->cfg.hbm_budget_bytes) return false;
  size_t sz[SLOT_BUFS];
  slot_sizes(ge.g, sz);
  SlotBuf b{};
  for (int i = 0; i < SLOT_BUFS; ++i) {
    if (cudaMalloc(&b.p[i], sz[i]) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < i; ++j) cudaFree(b.p[j]);
      return false;
    }
  }
  ge.slots.push_back(b);
  ge.free_slots.push_back((int)ge.slots.size() - 1);
  s->used_bytes += (int64_t)sb;
  return true;
}

// Batched launches at once: each takes 1/max_batched of the SMs (cooperative launches
// need their CTAs resident together); the other streams run single-root flights, whose
// kernels share the GPU. Two halves beat more, smaller launches at saturation.
int max_batched(const gt_server* s) { return std::max(1, std::min<int>(2, (int)s->streams.size())); }

// Picks the graph whose oldest pending query is oldest, among graphs without a running
// single-root flight; -1 if none. Caller holds the lock.
int oldest_graph(gt_server* s) {
  int best = -1;
  double t = 0;
  for (size_t i = 0; i < s->graphs.size(); ++i) {
    const GraphEntry& ge = s->graphs[i];
    if (ge.pending.empty() || ge.single_busy) continue;  // a single-root flight drains it first
    if (best < 0 || ge.pending.front()->t_submit < t) {
      best = (int)i;
      t = ge.pending.front()->t_submit;
    }
  }
  return best;
}

void scheduler(gt_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    int free_stream = -1, busy = 0, busy_batched = 0;
    for (size_t i = 0; i < s->flights.size(); ++i) {
      if (s->flights[i]) {
        ++busy;
        busy_batched += s->flights[i]->single ? 0 : 1;
      } else if (free_stream < 0) {
        free_stream = (int)i;
      }
    }
    if (s->stop && busy == 0) break;
    // lanes of running batched launches that have finished complete at once; pending
    // roots of a graph with a batched launch in flight join its free lanes
    for (Flight* f : s->flights)
      if (f && !f->single && f->mb) collect_early(s, f);
    for (Flight* f : s->flights) {
      if (!f || f->single || !f->mb || s->stop) continue;
      volatile BatchMailbox* vm = f->mb;
      if (vm->closed) continue;
      GraphEntry& ge = s->graphs[f->gid];
      while (!ge.pending.empty() && (int)f->late.size() < f->capacity) {
        Query* q = ge.pending.front();
        ge.pending.pop_front();
        const int k = (int)f->late.size();
        vm->e[k].root = q->root;
        vm->e[k].outp = q->parent;
        vm->e[k].outl = q->level;
        vm->e[k].lane_id = -1;
        std::atomic_thread_fence(std::memory_order_release);  // entry before count
        vm->count = k + 1;
        f->late.push_back(q);
      }
    }
    const int gi = oldest_graph(s);
    if (s->stop || gi < 0 || free_stream < 0) {
      s->cv_sched.wait_for(lk, std::chrono::microseconds(200));
      if (s->stop) {
        // drop queries never dispatched
        for (GraphEntry& ge : s->graphs)
          while (!ge.pending.empty()) {
            Query* q = ge.pending.front();
            ge.pending.pop_front();
            q->done = true;
            q->rc = GT_EBUSY;
            s->failed++;
          }
        s->cv_done.notify_all();
      }
      continue;
    }
    GraphEntry& ge = s->graphs[gi];
    const double age = now_us() - ge.pending.front()->t_submit;
    const size_t want = std::min<size_t>(ge.pending.size(), (size_t)s->cfg.max_batch_roots);
    // Mode: k single-root traversals cost k * est_single; a batched launch costs about
    // est_word per 64-root lane word whatever the number of roots in it. Unmeasured modes
    // are tried first (single for a few queries, batch for many).
    const double words_f = (double)((want + 63) / 64);
    bool single;
    if (ge.est_single_us <= 0)
      single = want <= 4 || ge.est_word_us > 0;
    else if (ge.est_word_us <= 0)
      single = want < 8;
    else
      single = want * ge.est_single_us <= words_f * ge.est_word_us;
    if (s->cfg.policy != GT_SERVE_ADAPTIVE) single = s->cfg.policy == GT_SERVE_SINGLE;
    const bool batching_pays = s->cfg.policy == GT_SERVE_BATCHED ||
                               (ge.est_single_us > 0 && ge.est_word_us > 0 && 64 * ge.est_single_us > ge.est_word_us);
    if (!single && busy > 0 && want < 64 && age < s->cfg.window_us && batching_pays) {
      s->cv_sched.wait_for(lk, std::chrono::microseconds((int64_t)std::max(1.0, s->cfg.window_us - age)));
      continue;
    }
    if (!single && busy_batched >= max_batched(s)) {  // the batched share of the SMs is taken
      s->cv_sched.wait_for(lk, std::chrono::microseconds(200));
      continue;
    }
    if (single) {
      Flight* f = new Flight();
      f->srv = s;
      f->stream = free_stream;
      f->gid = gi;
      f->single = true;
      const size_t take = std::min<size_t>(want, 64);
      for (size_t i = 0; i < take; ++i) {
        f->queries.push_back(ge.pending.front());
        ge.pending.pop_front();
      }
      f->done.resize(take);
      for (size_t i = 0; i < take; ++i) f->done[i] = QueryDone{f, f->queries[i]};
      f->remaining = (int)take;
      f->t_launch = f->t_prev = now_us();
      ge.single_busy = true;
      s->flights[free_stream] = f;
      cudaStream_t st = s->streams[free_stream];
      lk.unlock();  // the graph's single-root state is this flight's alone (single_busy)
      size_t launched = 0;
      int rc = GT_OK;
      for (; launched < take && rc == GT_OK; ++launched) {
        Query* q = f->queries[launched];
        rc = run_bfs(ge.g, ge.g->core, true, q->root, q->parent, q->level, st);
        if (rc == GT_OK) rc = cuda_fail(cudaLaunchHostFunc(st, on_query_done, &f->done[launched]), "host callback");
      }
      lk.lock();
      if (rc != GT_OK) {  // queries past the failure will not call back: fail them here
        const size_t ok = launched - 1;
        for (size_t i = ok; i < take; ++i) {
          f->queries[i]->done = true;
          f->queries[i]->rc = rc;
          s->failed++;
        }
        f->remaining -= (int)(take - ok);
        if (f->remaining == 0) {
          ge.single_busy = false;
          s->flights[free_stream] = nullptr;
          delete f;
        }
        s->cv_done.notify_all();
      }
      continue;
    }
    const int words_needed = (int)((want + 63) / 64);
    while ((int)ge.free_slots.size() < words_needed && grow_slots(s, ge)) {
    }
    const int words = std::min<int>(words_needed, (int)ge.free_slots.size());
    if (words == 0) {  // every lane word of this graph is in flight
      s->cv_sched.wait_for(lk, std::chrono::microseconds(200));
      continue;
    }
    Flight* f = new Flight();
    f->srv = s;
    f->stream = free_stream;
    f->gid = gi;
    const size_t take = std::min<size_t>(want, (size_t)words * 64);
    for (size_t i = 0; i < take; ++i) {
      f->queries.push_back(ge.pending.front());
      ge.pending.pop_front();
    }
    for (int w = 0; w < words; ++w) {
      f->slots.push_back(ge.free_slots.back());
      ge.free_slots.pop_back();
    }
    s->flights[free_stream] = f;
    s->batches++;
    f->t_launch = now_us();
    // build the launch outside the lock
    std::vector<int64_t> roots(take);
    std::vector<int32_t*> op(take), ol(take);
    for (size_t i = 0; i < take; ++i) {
      roots[i] = f->queries[i]->root;
      op[i] = f->queries[i]->parent;
      ol[i] = f->queries[i]->level;
    }
    std::vector<SlotSpec> specs(words);
    for (int w = 0; w < words; ++w) {
      SlotSpec& sp = specs[w];
      sp.g = ge.g;
      sp.mem = ge.slots[f->slots[w]].p;
      sp.nlanes = (int)std::min<size_t>(64, take - 64 * (size_t)w);
      sp.roots = roots.data() + 64 * w;
      sp.outp = op.data() + 64 * w;
      sp.outl = ol.data() + 64 * w;
    }
    cudaStream_t st = s->streams[free_stream];
    BatchCtx* ctx = &s->ctxs[free_stream];
    const int share = std::max(1, s->sms / max_batched(s));
    // with free lanes and join_levels > 0 the launch takes roots through the stream's
    // mailbox, and reports there the lanes that end before the launch does
    f->capacity = s->cfg.join_levels > 0 ? std::min<int>(MAILBOX_CAP, words * 64 - (int)take) : 0;
    BatchMailbox* mb_dev = nullptr;
    if (f->capacity > 0) {
      f->mb = s->mbox[free_stream];
      f->lane_q.assign((size_t)words * 64, nullptr);
      for (size_t i = 0; i < take; ++i) f->lane_q[i] = f->queries[i];
      f->seen.assign(words, 0);
      volatile BatchMailbox* vm = f->mb;
      vm->count = 0;
      vm->taken = 0;
      vm->closed = 0;
      for (int w = 0; w < words; ++w) vm->done[w] = 0;
      std::atomic_thread_fence(std::memory_order_release);
      mb_dev = s->mbox_dev[free_stream];
    }
    lk.unlock();
    int rc = batch_launch(ctx, specs.data(), words, share, st, mb_dev, s->cfg.join_levels);
    if (rc == GT_OK) rc = cuda_fail(cudaLaunchHostFunc(st, on_flight_done, f), "host callback");
    lk.lock();
    if (rc != GT_OK) {  // nothing will call back: fail the queries here
      for (int k : f->slots) ge.free_slots.push_back(k);
      for (Query* q : f->queries) {
        q->done = true;
        q->rc = rc;
        s->failed++;
      }
      s->flights[free_stream] = nullptr;
      delete f;
      s->cv_done.notify_all();
    }
  }
  // queries a last launch did not admit came back to the queues: they fail like the rest
  for (GraphEntry& ge : s->graphs)
    while (!ge.pending.empty()) {
      Query* q = ge.pending.front();
      ge.pending.pop_front();
      q->done = true;
      q->rc = GT_EBUSY;
      s->failed++;
    }
  s->cv_done.notify_all();
}

}  // namespace
}  // namespace gt

using namespace gt;

extern "C" {

GT_API void gt_serve_config_default(gt_serve_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->hbm_budget_bytes = (int64_t)48 << 30;
  c->streams = 4;  // two of them batched at most (max_batched)
  c->max_batch_roots = 256;
  c->window_us = 200.0;
  c->policy = GT_SERVE_ADAPTIVE;
  c->join_levels = 0;  // measured: joins lengthen launches more than they save waiting
}

GT_API int gt_serve_create(const gt_serve_config* cfg, gt_server_t* out) {
  if (!out) return GT_EINVAL;
  *out = nullptr;
  gt_server* s = new (std::nothrow) gt_server();
  if (!s) return GT_ENOMEM;
  if (cfg)
    s->cfg = *cfg;
  else
    gt_serve_config_default(&s->cfg);
  if (s->cfg.streams < 1 || s->cfg.streams > 16 || s->cfg.max_batch_roots < 1 || s->cfg.max_batch_roots > 16384 ||
      s->cfg.hbm_budget_bytes < 0 || s->cfg.window_us < 0 || s->cfg.policy < GT_SERVE_ADAPTIVE ||
      s->cfg.policy > GT_SERVE_SINGLE || s->cfg.join_levels < 0 || s->cfg.join_levels > 64) {
    delete s;
    set_error("gt_serve_create: configuration out of range");
    return GT_EINVAL;
  }
  cudaGetDevice(&s->device);
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
  s->streams.resize(s->cfg.streams);
  s->ctxs.resize(s->cfg.streams);
  s->flights.assign(s->cfg.streams, nullptr);
  s->mbox.assign(s->cfg.streams, nullptr);
  s->mbox_dev.assign(s->cfg.streams, nullptr);
  for (int i = 0; i < s->cfg.streams; ++i) {
    void* h = nullptr;
    void* d = nullptr;
    if (cudaHostAlloc(&h, sizeof(BatchMailbox), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
      cudaGetLastError();
      if (h) cudaFreeHost(h);
      for (auto* m : s->mbox)
        if (m) cudaFreeHost(m);
      delete s;
      set_error("gt_serve_create: pinned mailbox allocation failed");
      return GT_ENOMEM;
    }
    memset(h, 0, sizeof(BatchMailbox));
    s->mbox[i] = (BatchMailbox*)h;
    s->mbox_dev[i] = (BatchMailbox*)d;
  }
  for (auto& st : s->streams) {
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (auto& t : s->streams)
        if (t) cudaStreamDestroy(t);
      for (auto* m : s->mbox)
        if (m) cudaFreeHost(m);
      delete s;
      set_error("gt_serve_create: stream creation failed");
      return GT_EDEVICE;
    }
  }
  s->worker = std::thread(scheduler, s);
  *out = s;
  return GT_OK;
}

GT_API int gt_serve_add_graph(gt_server_t s, gt_graph_t g, int32_t* gid) {
  if (!s || !g || !gid) return GT_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (g->device != s->device) {
    set_error("gt_serve_add_graph: graph lives on another device");
    return GT_EINVAL;
  }
  const int64_t need = g->device_bytes + (int64_t)slot_bytes(g);
  if (s->used_bytes + need > s->cfg.hbm_budget_bytes) {
    set_error("gt_serve_add_graph: graph plus one lane word of batch storage exceeds the HBM budget");
    return GT_ENOMEM;
  }
  GraphEntry ge;
  ge.g = g;
  s->graphs.push_back(ge);
  s->used_bytes += g->device_bytes;
  if (!grow_slots(s, s->graphs.back())) {
    s->used_bytes -= g->device_bytes;
    s->graphs.pop_back();
    set_error("gt_serve_add_graph: could not allocate batch storage");
    return GT_ENOMEM;
  }
  *gid = (int32_t)s->graphs.size() - 1;
  return GT_OK;
}

GT_API int gt_serve_submit(gt_server_t s, int32_t gid, int64_t root, int32_t* parent, int32_t* level,
                           uint64_t* ticket) {
  if (!s || !ticket || !parent || !level) return GT_EINVAL;
  cudaPointerAttributes pa{}, la{};
  if (cudaPointerGetAttributes(&pa, parent) != cudaSuccess || cudaPointerGetAttributes(&la, level) != cudaSuccess ||
      pa.type != cudaMemoryTypeDevice || la.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    set_error("gt_serve_submit: parent and level must be device memory");
    return GT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return GT_EBUSY;
  if (gid < 0 || gid >= (int32_t)s->graphs.size() || root < 0 || root >= s->graphs[gid].g->n) {
    set_error("gt_serve_submit: unknown graph id or root outside [0, n)");
    return GT_EINVAL;
  }
  Query* q = new (std::nothrow) Query();
  if (!q) return GT_ENOMEM;
  q->ticket = s->next_ticket++;
  q->gid = gid;
  q->root = root;
  q->parent = parent;
  q->level = level;
  q->t_submit = now_us();
  if (s->submitted == 0) s->t_first = q->t_submit;
  s->submitted++;
  s->graphs[gid].pending.push_back(q);
  s->tickets[q->ticket] = q;
  *ticket = q->ticket;
  s->cv_sched.notify_all();
  return GT_OK;
}

GT_API int gt_serve_poll(gt_server_t s, uint64_t ticket, int32_t timeout_ms) {
  if (!s) return GT_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) {
    set_error("gt_serve_poll: unknown ticket (never issued or already collected)");
    return GT_EINVAL;
  }
  Query* q = it->second;
  const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  while (!q->done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !q->done) return GT_ETIMEOUT;
  }
  const int rc = q->rc;
  s->tickets.erase(it);
  delete q;
  return rc;
}

GT_API int gt_serve_get_stats(gt_server_t s, gt_serve_stats* out) {
  if (!s || !out) return GT_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->batches = s->batches;
  out->joined = s->joined;
  out->early = s->early;
  for (auto* f : s->flights) out->inflight += f ? 1 : 0;
  for (auto& ge : s->graphs) out->pending += (int64_t)ge.pending.size();
  out->device_bytes = s->used_bytes;
  if (!s->lat_us.empty()) {
    std::vector<double> v = s->lat_us;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->max_us = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_us = sum / v.size();
    const double span = s->t_last - s->t_first;
    out->qps = span > 0 ? s->completed / (span * 1e-6) : 0;
  }
  return GT_OK;
}

GT_API int gt_serve_reset_stats(gt_server_t s) {
  if (!s) return GT_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat_us.clear();
  s->submitted = s->completed = s->failed = s->batches = s->joined = s->early = 0;
  s->t_first = s->t_last = 0;
  return GT_OK;
}

GT_API int gt_serve_destroy(gt_server_t s) {
  if (!s) return GT_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto st : s->streams) cudaStreamSynchronize(st);
  // single-root flights left the graphs pointing at the server's streams: all their work
  // is done, so the graphs forget those streams before they are destroyed
  for (auto& ge : s->graphs)
    if (std::find(s->streams.begin(), s->streams.end(), ge.g->last_stream) != s->streams.end())
      ge.g->last_stream = nullptr;
  for (auto st : s->streams) cudaStreamDestroy(st);
  for (auto& c : s->ctxs) batch_ctx_free(&c);
  for (auto* m : s->mbox)
    if (m) cudaFreeHost(m);
  for (auto& ge : s->graphs)
    for (auto& b : ge.slots)
      for (int i = 0; i < SLOT_BUFS; ++i) cudaFree(b.p[i]);
  for (auto& kv : s->tickets) delete kv.second;
  delete s;
  return GT_OK;
}

}  // extern "C"
