// persist.cu -- a built graph to a file and back (gt_graph_save / gt_graph_load).
//
// The file holds what the build derives from the tuples (Sec. 5.1.1 CSR, Alg. 8 classes
// and tree parents, the core relabel and core CSR, the edge-tree lists, the batched work
// lists) behind a fixed header; loading copies them back to the device and allocates the
// per-traversal state as a build does, so a graph need not be rebuilt from its tuples.
// Arrays are streamed through one page-locked staging buffer in 64 MB pieces.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "gt_internal.cuh"

namespace gt {
namespace {

constexpr char MAGIC[8] = {'G', 'T', 'G', 'R', 'A', 'P', 'H', '1'};
constexpr uint32_t VERSION = 2;
constexpr size_t PIECE = size_t(64) << 20;

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t n, m, nnz, n_core, nnz_core, n_anchor, n_batch_lane, n_batch_mid, n_batch_item, resolve_n;
  int32_t resolve_heights, pad;
  gt_config cfg;
  gt_tuning tuning;
  gt_stats stats;
};

// Page-locked staging buffer of one save or load.
struct Staging {
  void* p = nullptr;
  ~Staging() {
    if (p) cudaFreeHost(p);
  }
};

int io_error(const std::string& what) {
  set_error(what);
  return GT_EIO;
}

// Device array -> file, `bytes` long, through the staging buffer.
int write_array(FILE* f, const void* dev, size_t bytes, void* stage, cudaStream_t s) {
  const int64_t len = (int64_t)bytes;
  if (fwrite(&len, sizeof(len), 1, f) != 1) return io_error("gt_graph_save: write failed");
  for (size_t off = 0; off < bytes; off += PIECE) {
    const size_t k = std::min(PIECE, bytes - off);
    int rc = cuda_fail(cudaMemcpyAsync(stage, (const char*)dev + off, k, cudaMemcpyDeviceToHost, s), "save copy");
    if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "save sync");
    if (rc) return rc;
    if (fwrite(stage, 1, k, f) != k) return io_error("gt_graph_save: write failed");
  }
  return GT_OK;
}

// File -> new device array of exactly `bytes` (the length recorded in the file must match).
int read_array(FILE* f, gt_graph* g, void** dev, size_t bytes, size_t alloc_bytes, void* stage, cudaStream_t s) {
  int64_t len = -1;
  if (fread(&len, sizeof(len), 1, f) != 1 || len != (int64_t)bytes)
    return io_error("gt_graph_load: the file is truncated or does not match its header");
  int rc = device_malloc(g, dev, std::max(alloc_bytes, bytes));
  if (rc) return rc;
  for (size_t off = 0; off < bytes; off += PIECE) {
    const size_t k = std::min(PIECE, bytes - off);
    if (fread(stage, 1, k, f) != k) return io_error("gt_graph_load: the file is truncated");
    rc = cuda_fail(cudaMemcpyAsync((char*)*dev + off, stage, k, cudaMemcpyHostToDevice, s), "load copy");
    if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "load sync");
    if (rc) return rc;
  }
  return GT_OK;
}

}  // namespace

int save_graph(const gt_graph* g, FILE* f, cudaStream_t s) {
  FileHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, MAGIC, sizeof(MAGIC));
  h.version = VERSION;
  h.header_bytes = sizeof(FileHeader);
  h.n = g->n;
  h.m = g->m;
  h.nnz = g->nnz;
  h.n_core = g->core.n;
  h.nnz_core = g->core.nnz;
  h.n_anchor = g->n_anchor;
  h.n_batch_lane = g->n_batch_lane;
  h.n_batch_mid = g->n_batch_mid;
  h.n_batch_item = g->n_batch_item;
  h.resolve_n = g->resolve_n;
  h.resolve_heights = g->resolve_heights;
  h.cfg = g->cfg;
  h.tuning = g->tuning;
  h.stats = g->stats;
  if (fwrite(&h, sizeof(h), 1, f) != 1) return io_error("gt_graph_save: write failed");
  Staging st;
  int rc = cuda_fail(cudaHostAlloc(&st.p, PIECE, cudaHostAllocDefault), "save staging");
  const int64_t n = g->n, nc = g->core.n;
  struct Part {
    const void* p;
    size_t bytes;
  } parts[] = {
      {g->row, sizeof(int64_t) * (n + 1)},
      {g->col, sizeof(int32_t) * g->nnz},
      {g->deg, sizeof(int32_t) * n},
      {g->vtype, n},
      {g->up, sizeof(int32_t) * n},
      {g->vinfo, sizeof(int32_t) * n},
      {g->old2core, sizeof(int32_t) * n},
      {g->new2old, sizeof(int32_t) * nc},
      {g->core.row, sizeof(int64_t) * (nc + 1)},
      {g->core.col, sizeof(int32_t) * g->core.nnz},
      {g->anchor_cid, sizeof(int32_t) * g->n_anchor},
      {g->anchor_vid, sizeof(int32_t) * g->n_anchor},
      {g->batch_lane, sizeof(int32_t) * g->n_batch_lane},
      {g->batch_mid, sizeof(int32_t) * g->n_batch_mid},
      {g->batch_item, sizeof(BatchItem) * g->n_batch_item},
      {g->resolve_list, sizeof(int32_t) * g->resolve_n},
      {g->resolve_up, sizeof(int32_t) * g->resolve_n},
  };
  for (const Part& pt : parts) {
    if (rc) break;
    rc = write_array(f, pt.p, pt.bytes, st.p, s);
  }
  if (!rc && g->resolve_heights > 0) {
    const size_t k = sizeof(int64_t) * (size_t)(g->resolve_heights + 1);
    if (fwrite(g->resolve_ptr_host, 1, k, f) != k) rc = io_error("gt_graph_save: write failed");
  }
  return rc;
}

int load_graph(gt_graph* g, FILE* f, cudaStream_t s) {
  FileHeader h;
  if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, MAGIC, sizeof(MAGIC)) != 0 || h.version != VERSION ||
      h.header_bytes != sizeof(FileHeader))
    return io_error("gt_graph_load: not a graph saved by this version of gt_graph_save");
  if (h.n < 1 || h.n > 0x7FFFFFFFLL || h.nnz < 0 || h.n_core < 0 || h.n_core > h.n || h.nnz_core < 0 ||
      h.nnz_core > h.nnz || h.n_anchor < 0 || h.n_anchor > h.n_core || h.resolve_n < 0 || h.resolve_n > h.n ||
      h.resolve_heights < 0 || h.resolve_heights > 1 << 20 || h.n_batch_lane < 0 || h.n_batch_mid < 0 || h.n_batch_item < 0)
    return io_error("gt_graph_load: the header's sizes are inconsistent");
  g->n = h.n;
  g->m = h.m;
  g->nnz = h.nnz;
  g->cfg = h.cfg;
  g->tuning = h.tuning;
  g->n_anchor = h.n_anchor;
  g->n_batch_lane = h.n_batch_lane;
  g->n_batch_mid = h.n_batch_mid;
  g->n_batch_item = h.n_batch_item;
  g->resolve_n = h.resolve_n;
  const int64_t n = h.n, nc = h.n_core;
  Staging st;
  int rc = cuda_fail(cudaHostAlloc(&st.p, PIECE, cudaHostAllocDefault), "load staging");
  View& cv = g->core;
  cv.n = nc;
  cv.nnz = h.nnz_core;
  struct Part {
    void** p;
    size_t bytes, alloc;
  } parts[] = {
      {(void**)&g->row, sizeof(int64_t) * (n + 1), 0},
      {(void**)&g->col, sizeof(int32_t) * h.nnz, sizeof(int32_t) * col_alloc(h.nnz)},
      {(void**)&g->deg, sizeof(int32_t) * n, 0},
      {(void**)&g->vtype, (size_t)n, 0},
      {(void**)&g->up, sizeof(int32_t) * n, 0},
      {(void**)&g->vinfo, sizeof(int32_t) * n, 0},
      {(void**)&g->old2core, sizeof(int32_t) * n, 0},
      {(void**)&g->new2old, sizeof(int32_t) * nc, 0},
      {(void**)&cv.row, sizeof(int64_t) * (nc + 1), 0},
      {(void**)&cv.col, sizeof(int32_t) * h.nnz_core, sizeof(int32_t) * col_alloc(h.nnz_core)},
      {(void**)&g->anchor_cid, sizeof(int32_t) * h.n_anchor, 0},
      {(void**)&g->anchor_vid, sizeof(int32_t) * h.n_anchor, 0},
      {(void**)&g->batch_lane, sizeof(int32_t) * h.n_batch_lane, 0},
      {(void**)&g->batch_mid, sizeof(int32_t) * h.n_batch_mid, 0},
      {(void**)&g->batch_item, sizeof(BatchItem) * h.n_batch_item, 0},
      {(void**)&g->resolve_list, sizeof(int32_t) * h.resolve_n, 0},
      {(void**)&g->resolve_up, sizeof(int32_t) * h.resolve_n, 0},
  };
  for (const Part& pt : parts) {
    if (rc) break;
    rc = read_array(f, g, pt.p, pt.bytes, pt.alloc, st.p, s);
  }
  if (rc) return rc;
  g->resolve_heights = h.resolve_heights;
  if (h.resolve_heights > 0) {
    g->resolve_ptr_host = new int64_t[h.resolve_heights + 1];
    const size_t k = sizeof(int64_t) * (size_t)(h.resolve_heights + 1);
    if (fread(g->resolve_ptr_host, 1, k, f) != k) return io_error("gt_graph_load: the file is truncated");
  }
  cv.new2old = g->new2old;
  rc = device_malloc(g, (void**)&g->anchor_out, sizeof(uint64_t) * std::max<int64_t>(h.n_anchor, 1));
  if (!rc) rc = alloc_view_state(g, cv, s);
  if (!rc && g->cfg.keep_plain) {
    View& pv = g->plain;
    pv.n = n;
    pv.nnz = h.nnz;
    pv.row = g->row;
    pv.col = g->col;
    rc = alloc_view_state(g, pv, s);
  }
  if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "load sync");
  if (rc) return rc;
  g->stats = h.stats;
  g->stats.device_bytes = g->device_bytes;
  return GT_OK;
}

}  // namespace gt
