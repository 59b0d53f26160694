// tune.cu -- per-graph autotuner for the traversal parameters (gt_tuning).
//
// The parameters only move work between threads, warps, CTAs and directions; the
// levels and parents are the same for every setting. The tuner times edge-tree BFS from
// a few sample roots (CUDA events on the caller's stream) and walks the parameters one
// at a time (coordinate descent, two sweeps), keeping a value only if it lowers the
// summed time by more than 2 %. The batch switch constants are tuned the same way on
// one 64-root batch. The best setting is stored in the handle and returned.
#include <algorithm>
#include <vector>

#include "gt_internal.cuh"

namespace gt {
namespace {

uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void reset_graphs(gt_graph* g) {
  for (int i = 0; i < 2; ++i) {
    if (g->loop_exec[i]) cudaGraphExecDestroy(g->loop_exec[i]);
    g->loop_exec[i] = nullptr;
  }
}

int apply(gt_graph* g, const gt_tuning& t) {
  g->tuning = t;
  g->launch.grid = g->launch.sms * std::max(1, t.blocks_per_sm);
  reset_graphs(g);
  return GT_OK;
}

}  // namespace

int autotune(gt_graph* g, int nsample, uint64_t seed, cudaStream_t s, gt_tuning* out) {
  const int64_t n = g->n;
  std::vector<int32_t> deg(n);
  int rc = cuda_fail(cudaMemcpyAsync(deg.data(), g->deg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s), "degrees");
  if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "sync");
  if (rc) return rc;
  std::vector<int64_t> roots;
  for (uint64_t j = 0; (int)roots.size() < nsample && j < (uint64_t)(64 * n + 1024); ++j) {
    const int64_t c = (int64_t)(mix64(seed * 0x100000001B3ull + j) % (uint64_t)n);
    if (deg[c] > 0 && std::find(roots.begin(), roots.end(), c) == roots.end()) roots.push_back(c);
  }
  if (roots.empty()) {
    if (out) *out = g->tuning;
    return GT_OK;
  }
  int32_t *par = nullptr, *lev = nullptr;
  rc = cuda_fail(cudaMallocAsync((void**)&par, sizeof(int32_t) * n * 2, s), "tune buffers");
  if (rc) return rc;
  lev = par + n;
  const int nb = (int)std::min<size_t>(64, roots.size());
  int32_t *bpar = nullptr, *blev = nullptr;
  rc = cuda_fail(cudaMallocAsync((void**)&bpar, sizeof(int32_t) * n * nb * 2, s), "tune buffers");
  if (rc) {
    cudaFreeAsync(par, s);
    return rc;
  }
  blev = bpar + (int64_t)n * nb;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const gt_tuning start = g->tuning;

  auto time_single = [&](const gt_tuning& t, float* ms) -> int {
    apply(g, t);
    int r = run_bfs(g, g->core, true, roots[0], par, lev, s);  // warm (graph instantiation)
    if (r) return r;
    cudaEventRecord(e0, s);
    for (int64_t root : roots)
      if ((r = run_bfs(g, g->core, true, root, par, lev, s))) return r;
    cudaEventRecord(e1, s);
    if ((r = cuda_fail(cudaEventSynchronize(e1), "tune sync"))) return r;
    return cuda_fail(cudaEventElapsedTime(ms, e0, e1), "tune time");
  };
  auto time_batch = [&](const gt_tuning& t, float* ms) -> int {
    apply(g, t);
    gt_graph* gs[1] = {g};
    const int32_t cnt[1] = {nb};
    int32_t* pp[1] = {bpar};
    int32_t* lp[1] = {blev};
    int r = run_batch(gs, 1, roots.data(), cnt, pp, lp, s);
    if (r) return r;
    cudaEventRecord(e0, s);
    if ((r = run_batch(gs, 1, roots.data(), cnt, pp, lp, s))) return r;
    cudaEventRecord(e1, s);
    if ((r = cuda_fail(cudaEventSynchronize(e1), "tune sync"))) return r;
    return cuda_fail(cudaEventElapsedTime(ms, e0, e1), "tune time");
  };

  using Field = int32_t gt_tuning::*;
  struct Knob {
    Field field;
    std::vector<int32_t> values;
    bool batch;
  };
  const std::vector<Knob> knobs = {
      {&gt_tuning::alpha, {8, 14, 20, 32, 48}, false},
      {&gt_tuning::beta, {24, 64, 128, 256, 512}, false},
      {&gt_tuning::td_warp_min, {8, 16, 32, 64}, false},
      {&gt_tuning::td_cta_min, {128, 256, 512, 1024}, false},
      {&gt_tuning::td_grid_min, {1024, 2048, 4096, 16384}, false},
      {&gt_tuning::bu_thread_scan, {8, 16, 24, 32, 48}, false},
      {&gt_tuning::blocks_per_sm, {2, 4, 6, 8}, false},
      {&gt_tuning::batch_alpha, {2, 4, 8, 14, 32}, true},
      {&gt_tuning::batch_beta, {4, 12, 24, 64}, true},
  };
  gt_tuning best = start;
  best.launch_mode = 0;
  best.force_direction = 0;
  best.count_work = 0;
  best.time_kernels = 0;
  float best_single = 0.f, best_batch = 0.f;
  rc = time_single(best, &best_single);
  if (!rc) rc = time_batch(best, &best_batch);
  for (int sweep = 0; sweep < 2 && !rc; ++sweep) {
    for (const Knob& k : knobs) {
      for (int32_t v : k.values) {
        if (best.*k.field == v) continue;
        gt_tuning t = best;
        t.*k.field = v;
        if (t.td_cta_min < t.td_warp_min || t.td_grid_min < t.td_cta_min) continue;
        float ms = 0.f;
        rc = k.batch ? time_batch(t, &ms) : time_single(t, &ms);
        if (rc) break;
        float& ref = k.batch ? best_batch : best_single;
        if (ms < 0.98f * ref) {
          ref = ms;
          best = t;
        }
      }
      if (rc) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(par, s);
  cudaFreeAsync(bpar, s);
  cudaStreamSynchronize(s);
  apply(g, rc ? start : best);
  if (!rc && out) *out = best;
  return rc;
}

}  // namespace gt
