// capi.cu -- the extern "C" entry points declared in include/gt.h: argument checks,
// host/device buffer handling, status codes. All compute happens in the kernels of
// build.cu and bfs.cu.
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "gt_device.cuh"
#include "gt_internal.cuh"

namespace gt {

static thread_local std::string g_last_error;

void set_error(const std::string& s) { g_last_error = s; }

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GT_OK;
  cudaGetLastError();
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? GT_ENOMEM : GT_EDEVICE;
}

namespace {

int select_device(cudaStream_t s, int* dev) {
  int d = 0;
  if (s) {
    if (cudaStreamGetDevice(s, &d) != cudaSuccess) {
      cudaGetLastError();
      if (cudaGetDevice(&d) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaGetDevice");
    }
  } else if (cudaGetDevice(&d) != cudaSuccess) {
    return cuda_fail(cudaGetLastError(), "cudaGetDevice");
  }
  if (dev) *dev = d;
  return cuda_fail(cudaSetDevice(d), "cudaSetDevice");
}

// 1: device (or managed) memory, 0: host memory, -1: null
int where(const void* p) {
  if (!p) return -1;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 1 : 0;
}

// Device address of page-locked host memory mapped into the device's address space, or
// null for pageable or unmapped memory.
int32_t* mapped_host(void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return (int32_t*)a.devicePointer;
}

void apply_launch(gt_graph* g) {
  int bpm = g->tuning.blocks_per_sm > 0 ? g->tuning.blocks_per_sm : 8;
  g->launch.grid = g->launch.sms * bpm;
}

__global__ void count_traversed(const int64_t* __restrict__ edges, int64_t m, const int32_t* __restrict__ level,
                                int64_t n, unsigned long long* __restrict__ out, int* __restrict__ bad) {
  unsigned long long c = 0;
  for (int64_t i = gtid(); i < m; i += gthreads()) {
    const longlong2 e = reinterpret_cast<const longlong2*>(edges)[i];
    if (e.x < 0 || e.x >= n || e.y < 0 || e.y >= n) {
      *bad = 1;
      continue;
    }
    c += (level[e.x] >= 0) & (level[e.y] >= 0);
  }
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

int bfs_common(gt_graph_t g, bool et, int64_t root, int32_t* parent, int32_t* level, void* stream) {
  if (!g || !parent || !level) {
    set_error("gt_bfs: null handle or output");
    return GT_EINVAL;
  }
  if (root < 0 || root >= g->n) {
    set_error("gt_bfs: root outside [0, n)");
    return GT_EINVAL;
  }
  if (!et && !g->cfg.keep_plain) {
    set_error("gt_bfs_plain: handle built with keep_plain = 0");
    return GT_ENOTSUP;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int rc = cuda_fail(cudaSetDevice(g->device), "cudaSetDevice");
  if (rc) return rc;
  const int wp = where(parent), wl = where(level);
  if (wp != wl) {
    set_error("gt_bfs: parent and level must both be device or both host memory");
    return GT_EINVAL;
  }
  gt::View& v = et ? g->core : g->plain;
  if (wp == 1) return run_bfs(g, v, et, root, parent, level, s);
  // Pinned (page-locked, device-mapped) host buffers: the output pass writes them directly
  // over the host link, so no device staging or copy is needed.
  int32_t* mp = mapped_host(parent);
  int32_t* ml = mapped_host(level);
  if (mp && ml) {
    rc = run_bfs(g, v, et, root, mp, ml, s);
    if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "bfs sync");
    return rc;
  }
  if (!g->scratch_out) {
    rc = device_malloc(g, (void**)&g->scratch_out, sizeof(int32_t) * 2 * g->n);
    if (rc) return rc;
  }
  int32_t* dp = g->scratch_out;
  int32_t* dl = g->scratch_out + g->n;
  rc = run_bfs(g, v, et, root, dp, dl, s);
  if (rc) return rc;
  rc = cuda_fail(cudaMemcpyAsync(parent, dp, sizeof(int32_t) * g->n, cudaMemcpyDeviceToHost, s), "copy parent");
  if (!rc) rc = cuda_fail(cudaMemcpyAsync(level, dl, sizeof(int32_t) * g->n, cudaMemcpyDeviceToHost, s), "copy level");
  if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "bfs sync");
  return rc;
}

// Copies one staged result (parent, level: n entries each) into page-locked host memory
// from the SMs, the same path as the output pass's direct writes into host memory. Beside
// the next root's traversal the copy needs many bytes in flight but few CTAs, which would
// otherwise slow that traversal: each thread keeps STAGE_COPY_UNROLL 16-byte pairs in
// flight. gt_bfs_roots at scale 26, one pair in flight: 256 / 330 / 347-361 / 338 / 302
// GTEPS with 16 / 32 / 48-80 / 96 / 128 CTAs; 4 in flight: 367-370 (16 CTAs), 357 (24);
// 8 in flight: 372-374 with 8-16 CTAs.
constexpr int STAGE_COPY_UNROLL = 8;
__global__ void stage_to_host(const int32_t* __restrict__ sp, const int32_t* __restrict__ sl, int32_t* hp,
                              int32_t* hl, int64_t n, int vec) {
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, T = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = vec ? n / 4 : 0;
  const int4* sp4 = reinterpret_cast<const int4*>(sp);
  const int4* sl4 = reinterpret_cast<const int4*>(sl);
  for (int64_t i0 = t0; i0 < n4; i0 += T * STAGE_COPY_UNROLL) {
    int4 a[STAGE_COPY_UNROLL], b[STAGE_COPY_UNROLL];
#pragma unroll
    for (int u = 0; u < STAGE_COPY_UNROLL; ++u) {
      const int64_t i = i0 + u * T;
      if (i < n4) {
        a[u] = __ldcs(sp4 + i);
        b[u] = __ldcs(sl4 + i);
      }
    }
#pragma unroll
    for (int u = 0; u < STAGE_COPY_UNROLL; ++u) {
      const int64_t i = i0 + u * T;
      if (i < n4) {
        reinterpret_cast<int4*>(hp)[i] = a[u];
        reinterpret_cast<int4*>(hl)[i] = b[u];
      }
    }
  }
  for (int64_t i = 4 * n4 + t0; i < n; i += T) {
    hp[i] = sp[i];
    hl[i] = sl[i];
  }
}
constexpr int STAGE_COPY_CTAS = 12;

// Device-accessible address of page-locked host memory, or null for pageable memory.
void* pinned_device_ptr(void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// k edge-tree traversals in order on `s`. Roots with device outputs write them directly.
// Roots with host outputs write a device staging pair (two pairs, alternating), which is
// moved to the host on the graph's copy stream while the traversal of the next root
// already runs: by a small copy kernel into page-locked memory, by the copy engine into
// pageable memory. The next root is always enqueued before the copy of the previous one,
// so pageable copies (which block the calling thread) overlap it too.
int bfs_roots(gt_graph_t g, const int64_t* roots, int32_t k, int32_t* const* parent, int32_t* const* level,
              cudaStream_t s) {
  std::vector<char> host(k);
  bool any_host = false;
  for (int32_t i = 0; i < k; ++i) {
    const int wp = where(parent[i]), wl = where(level[i]);
    if (wp < 0 || wl < 0 || wp != wl) {
      set_error("gt_bfs_roots: null output, or parent and level of a root in different memories");
      return GT_EINVAL;
    }
    host[i] = wp == 0;
    any_host |= wp == 0;
  }
  int rc = GT_OK;
  if (any_host) {
    if (!g->pipe_out) rc = device_malloc(g, (void**)&g->pipe_out, sizeof(int32_t) * 4 * g->n);
    if (!rc && !g->copy_stream)
      rc = cuda_fail(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking), "copy stream");
    for (int i = 0; i < 4 && !rc; ++i)
      if (!g->pipe_ev[i]) rc = cuda_fail(cudaEventCreateWithFlags(&g->pipe_ev[i], cudaEventDisableTiming), "event");
    if (rc) return rc;
  }
  cudaStream_t cs = g->copy_stream;
  cudaEvent_t* ev_out = g->pipe_ev;       // staging pair b written
  cudaEvent_t* ev_copied = g->pipe_ev + 2;  // staging pair b copied to the host
  std::vector<int> pair(k, -1);
  bool used[2] = {false, false};
  int next_pair = 0;
  auto launch = [&](int32_t i) -> int {
    if (!host[i]) return run_bfs(g, g->core, true, roots[i], parent[i], level[i], s);
    const int b = next_pair;
    next_pair ^= 1;
    pair[i] = b;
    if (used[b]) {
      const int r = cuda_fail(cudaStreamWaitEvent(s, ev_copied[b], 0), "wait copy");
      if (r) return r;
    }
    used[b] = true;
    int32_t* dp = g->pipe_out + (int64_t)(2 * b) * g->n;
    int r = run_bfs(g, g->core, true, roots[i], dp, dp + g->n, s);
    if (!r) r = cuda_fail(cudaEventRecord(ev_out[b], s), "record output");
    return r;
  };
  auto copy = [&](int32_t i) -> int {
    const int b = pair[i];
    const int32_t* dp = g->pipe_out + (int64_t)(2 * b) * g->n;
    const size_t bytes = sizeof(int32_t) * (size_t)g->n;
    int r = cuda_fail(cudaStreamWaitEvent(cs, ev_out[b], 0), "wait output");
    int32_t* hp = (int32_t*)pinned_device_ptr(parent[i]);
    int32_t* hl = (int32_t*)pinned_device_ptr(level[i]);
    if (!r && hp && hl) {
      const int vec = ((uintptr_t)hp % 16 == 0) && ((uintptr_t)hl % 16 == 0);
      stage_to_host<<<STAGE_COPY_CTAS, 256, 0, cs>>>(dp, dp + g->n, hp, hl, g->n, vec);
      r = cuda_fail(cudaGetLastError(), "copy kernel");
    } else {
      if (!r) r = cuda_fail(cudaMemcpyAsync(parent[i], dp, bytes, cudaMemcpyDeviceToHost, cs), "copy parent");
      if (!r) r = cuda_fail(cudaMemcpyAsync(level[i], dp + g->n, bytes, cudaMemcpyDeviceToHost, cs), "copy level");
    }
    if (!r) r = cuda_fail(cudaEventRecord(ev_copied[b], cs), "record copy");
    return r;
  };
  if (k > 0) rc = launch(0);
  for (int32_t i = 0; i < k && !rc; ++i) {
    if (i + 1 < k) rc = launch(i + 1);
    if (!rc && host[i]) rc = copy(i);
  }
  if (any_host) {
    const int r = cuda_fail(cudaStreamSynchronize(cs), "copy sync");
    if (!rc) rc = r;
  }
  return rc;
}

int copy_out(gt_graph_t g, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  int rc = cuda_fail(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s), "copy");
  if (!rc && where(dst) == 0) rc = cuda_fail(cudaStreamSynchronize(s), "sync");
  (void)g;
  return rc;
}

}  // namespace
}  // namespace gt

using namespace gt;

extern "C" {

GT_API void gt_config_default(gt_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->mh = 0;
  c->keep_plain = 1;
}

GT_API void gt_tuning_default(gt_tuning* t) {
  if (!t) return;
  memset(t, 0, sizeof(*t));
  t->alpha = 32;
  t->beta = 256;
  t->td_warp_min = 32;
  t->td_cta_min = 256;
  t->td_grid_min = 2048;
  t->bu_thread_scan = 24;
  t->blocks_per_sm = 8;
  t->force_direction = 0;
  t->launch_mode = 0;
  t->count_work = 0;
  t->bu_hub_first = 0;
  t->time_kernels = 0;
  t->batch_alpha = 14;
  t->batch_beta = 24;
}

GT_API int gt_graph_build(const int64_t* edges, int64_t m, int64_t n, const gt_config* cfg, void* stream,
                          gt_graph_t* out) {
  if (!out || (m > 0 && !edges) || m < 0 || n < 1 || n > 0x7FFFFFFFLL) {
    set_error("gt_graph_build: need out != NULL, edges != NULL when m > 0, m >= 0, 1 <= n <= 2^31 - 1");
    return GT_EINVAL;
  }
  if (cfg && cfg->mh < -1) {
    set_error("gt_graph_build: mh must be >= -1");
    return GT_EINVAL;
  }
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  int rc = select_device(s, &dev);
  if (rc) return rc;
  gt_graph* g = new (std::nothrow) gt_graph();
  if (!g) return GT_ENOMEM;
  g->device = dev;
  if (cfg)
    g->cfg = *cfg;
  else
    gt_config_default(&g->cfg);
  gt_tuning_default(&g->tuning);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  g->launch.sms = sms > 0 ? sms : 1;
  apply_launch(g);
  rc = build_graph(g, edges, m, n, s);
  if (rc) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    free_graph(g);
    delete g;
    return rc;
  }
  *out = g;
  return GT_OK;
}

GT_API void gt_graph_free(gt_graph_t g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->last_stream) cudaStreamSynchronize(g->last_stream);
  free_graph(g);
  delete g;
}

GT_API int gt_graph_stats(gt_graph_t g, gt_stats* out) {
  if (!g || !out) return GT_EINVAL;
  *out = g->stats;
  out->device_bytes = g->device_bytes;
  return GT_OK;
}

GT_API int gt_graph_vertex_type(gt_graph_t g, uint8_t* out, void* stream) {
  if (!g || !out) return GT_EINVAL;
  cudaSetDevice(g->device);
  return copy_out(g, out, g->vtype, (size_t)g->n, (cudaStream_t)stream);
}

GT_API int gt_graph_degree(gt_graph_t g, int32_t* out, void* stream) {
  if (!g || !out) return GT_EINVAL;
  cudaSetDevice(g->device);
  return copy_out(g, out, g->deg, sizeof(int32_t) * (size_t)g->n, (cudaStream_t)stream);
}

GT_API int gt_graph_get_tuning(gt_graph_t g, gt_tuning* out) {
  if (!g || !out) return GT_EINVAL;
  *out = g->tuning;
  return GT_OK;
}

GT_API int gt_graph_set_tuning(gt_graph_t g, const gt_tuning* t) {
  if (!g || !t) return GT_EINVAL;
  if (t->alpha < 1 || t->beta < 1 || t->td_warp_min < 1 || t->td_cta_min < t->td_warp_min ||
      t->td_grid_min < t->td_cta_min ||
      t->bu_thread_scan < 0 || t->blocks_per_sm < 1 || t->blocks_per_sm > 32 || t->force_direction < 0 ||
      t->force_direction > 2 || t->launch_mode < 0 || t->launch_mode > 1 || t->time_kernels < 0 ||
      t->time_kernels > 1 || t->batch_alpha < 1 ||
      t->batch_beta < 1 || t->bu_hub_first < 0 || t->bu_hub_first > 1) {
    set_error("gt_graph_set_tuning: value out of range");
    return GT_EINVAL;
  }
  cudaSetDevice(g->device);
  if (g->last_stream) cudaStreamSynchronize(g->last_stream);
  g->tuning = *t;
  apply_launch(g);
  for (int i = 0; i < 2; ++i) {
    if (g->loop_exec[i]) cudaGraphExecDestroy(g->loop_exec[i]);
    g->loop_exec[i] = nullptr;
  }
  return GT_OK;
}

GT_API int gt_bfs(gt_graph_t g, int64_t root, int32_t* parent, int32_t* level, void* stream) {
  return bfs_common(g, true, root, parent, level, stream);
}

GT_API int gt_bfs_roots(gt_graph_t g, const int64_t* roots, int32_t k, int32_t* const* parent,
                        int32_t* const* level, void* stream) {
  if (!g || k < 0 || (k > 0 && (!roots || !parent || !level))) {
    set_error("gt_bfs_roots: null argument or k < 0");
    return GT_EINVAL;
  }
  for (int32_t i = 0; i < k; ++i)
    if (roots[i] < 0 || roots[i] >= g->n) {
      set_error("gt_bfs_roots: root outside [0, n)");
      return GT_EINVAL;
    }
  int rc = cuda_fail(cudaSetDevice(g->device), "cudaSetDevice");
  if (rc) return rc;
  return bfs_roots(g, roots, k, parent, level, (cudaStream_t)stream);
}

GT_API int gt_graph_save(gt_graph_t g, const char* path, void* stream) {
  if (!g || !path) {
    set_error("gt_graph_save: null argument");
    return GT_EINVAL;
  }
  int rc = cuda_fail(cudaSetDevice(g->device), "cudaSetDevice");
  if (rc) return rc;
  FILE* f = fopen(path, "wb");
  if (!f) {
    set_error(std::string("gt_graph_save: cannot open ") + path + " for writing");
    return GT_EIO;
  }
  rc = save_graph(g, f, (cudaStream_t)stream);
  if (fclose(f) != 0 && rc == GT_OK) {
    set_error("gt_graph_save: write failed");
    rc = GT_EIO;
  }
  if (rc) remove(path);
  return rc;
}

GT_API int gt_graph_load(const char* path, void* stream, gt_graph_t* out) {
  if (!path || !out) {
    set_error("gt_graph_load: null argument");
    return GT_EINVAL;
  }
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  int rc = select_device(s, &dev);
  if (rc) return rc;
  FILE* f = fopen(path, "rb");
  if (!f) {
    set_error(std::string("gt_graph_load: cannot open ") + path);
    return GT_EIO;
  }
  gt_graph* g = new (std::nothrow) gt_graph();
  if (!g) {
    fclose(f);
    return GT_ENOMEM;
  }
  g->device = dev;
  gt_config_default(&g->cfg);
  gt_tuning_default(&g->tuning);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  g->launch.sms = sms > 0 ? sms : 1;
  rc = load_graph(g, f, s);
  fclose(f);
  if (rc) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    free_graph(g);
    delete g;
    return rc;
  }
  apply_launch(g);
  *out = g;
  return GT_OK;
}

GT_API void gt_test_batch_barrier(uint32_t polls, uint32_t extra) { set_barrier_test(polls, extra); }

GT_API void gt_test_fail_alloc(int32_t after) { set_alloc_test(after); }

GT_API int gt_bfs_batch_work(gt_graph_t g, int64_t* out) {
  if (!g || !out) {
    set_error("gt_bfs_batch_work: null argument");
    return GT_EINVAL;
  }
  for (int i = 0; i < 4; ++i) out[i] = g->batch_work[i];
  return GT_OK;
}

GT_API int gt_bfs_plain(gt_graph_t g, int64_t root, int32_t* parent, int32_t* level, void* stream) {
  return bfs_common(g, false, root, parent, level, stream);
}

GT_API int gt_bfs_batch(const gt_graph_t* graphs, int32_t ngraphs, const int64_t* roots,
                        const int32_t* roots_per_graph, int32_t* const* parent, int32_t* const* level,
                        void* stream) {
  if (!graphs || ngraphs < 1 || !roots_per_graph || !parent || !level) {
    set_error("gt_bfs_batch: null argument or ngraphs < 1");
    return GT_EINVAL;
  }
  int64_t total = 0;
  for (int i = 0; i < ngraphs; ++i) {
    if (!graphs[i] || roots_per_graph[i] < 0 || graphs[i]->device != graphs[0]->device) {
      set_error("gt_bfs_batch: bad graph handle, negative root count or graphs on different devices");
      return GT_EINVAL;
    }
    if (roots_per_graph[i] > 0 && (where(parent[i]) != 1 || where(level[i]) != 1)) {
      set_error("gt_bfs_batch: outputs must be device memory");
      return GT_EINVAL;
    }
    total += roots_per_graph[i];
  }
  if (total > 0 && !roots) return GT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = cuda_fail(cudaSetDevice(graphs[0]->device), "cudaSetDevice");
  if (rc) return rc;
  for (int i = 0; i < ngraphs; ++i)
    if (graphs[i]->last_stream && graphs[i]->last_stream != s) cudaStreamSynchronize(graphs[i]->last_stream);
  rc = run_batch(graphs, ngraphs, roots, roots_per_graph, parent, level, s);
  for (int i = 0; i < ngraphs; ++i) graphs[i]->last_stream = s;
  return rc;
}

GT_API int gt_autotune(gt_graph_t g, int32_t nsample, uint64_t seed, gt_tuning* best, void* stream) {
  if (!g || nsample < 1) return GT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = cuda_fail(cudaSetDevice(g->device), "cudaSetDevice");
  if (rc) return rc;
  if (g->last_stream && g->last_stream != s) cudaStreamSynchronize(g->last_stream);
  rc = autotune(g, nsample, seed, s, best);
  g->last_stream = s;
  return rc;
}

GT_API int gt_bfs_timing(gt_graph_t g, gt_bfs_timing_t* out) {
  if (!g || !out) return GT_EINVAL;
  out->start_ms = g->phase_ms[0];
  out->loop_ms = g->phase_ms[1];
  out->output_ms = g->phase_ms[2];
  return GT_OK;
}

GT_API int gt_bfs_trace(gt_graph_t g, gt_level_info* out, int32_t cap, int32_t* nlevels) {
  if (!g || !nlevels || cap < 0 || (cap > 0 && !out)) return GT_EINVAL;
  *nlevels = 0;
  if (!g->last_ctl) return GT_OK;
  cudaSetDevice(g->device);
  int rc = cuda_fail(cudaStreamSynchronize(g->last_stream), "trace sync");
  if (rc) return rc;
  int32_t nl = 0;
  rc = cuda_fail(cudaMemcpy(&nl, &g->last_ctl->nlevels, sizeof(int32_t), cudaMemcpyDeviceToHost), "trace");
  if (rc) return rc;
  *nlevels = nl;
  int32_t k = nl < cap ? nl : cap;
  if (k > MAX_TRACE) k = MAX_TRACE;
  if (k > 0)
    rc = cuda_fail(cudaMemcpy(out, g->last_ctl->trace, sizeof(gt_level_info) * k, cudaMemcpyDeviceToHost), "trace");
  for (int32_t i = 0; i < k && i < (int32_t)g->step_ms.size(); ++i) out[i].step_ms = g->step_ms[i];
  return rc;
}

GT_API int gt_count_traversed(const int64_t* edges, int64_t m, const int32_t* level, int64_t n, int64_t* out,
                              void* stream) {
  if (!out || m < 0 || n < 0 || (m > 0 && (!edges || !level))) return GT_EINVAL;
  *out = 0;
  if (m == 0) return GT_OK;
  if ((uintptr_t)edges & 15) {
    set_error("gt_count_traversed: tuples must be 16-byte aligned device memory");
    return GT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int rc = select_device(s, nullptr);
  if (rc) return rc;
  unsigned long long* d = nullptr;
  rc = cuda_fail(cudaMallocAsync((void**)&d, 2 * sizeof(unsigned long long), s), "alloc");
  if (rc) return rc;
  cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), s);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  count_traversed<<<sms * 8, 256, 0, s>>>(edges, m, level, n, d, (int*)(d + 1));
  unsigned long long h[2] = {0, 0};
  rc = cuda_fail(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s), "count readback");
  cudaFreeAsync(d, s);
  if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "count sync");
  if (!rc && h[1]) {
    set_error("gt_count_traversed: a tuple has a vertex id outside [0, n)");
    return GT_EINVAL;
  }
  *out = (int64_t)h[0];
  return rc;
}

GT_API const char* gt_strerror(int code) {
  switch (code) {
    case GT_OK: return "ok";
    case GT_EINVAL: return "invalid argument";
    case GT_ENOMEM: return "out of memory";
    case GT_ETIMEOUT: return "timed out";
    case GT_EBUSY: return "busy";
    case GT_EDEVICE: return "CUDA error";
    case GT_ENOTSUP: return "not supported";
    case GT_EIO: return "file error";
    default: return "unknown error";
  }
}

GT_API const char* gt_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
