// scan.cu -- device-wide exclusive prefix sums (row offsets, relabels, compaction).
// Three steps: per-tile sums, one CTA scans the tile sums, per-tile local scans.
#include "gt_device.cuh"
#include "gt_internal.cuh"

namespace gt {
namespace {

constexpr int ST = 256;              // threads per CTA
constexpr int SI = 16;               // items per thread
constexpr int STILE = ST * SI;       // 4096 items per tile
constexpr int SWARPS = ST / 32;

template <typename TI, typename TO>
__global__ void __launch_bounds__(ST) tile_sums(const TI* __restrict__ in, int64_t n, TO* __restrict__ sums) {
  __shared__ TO ws[SWARPS];
  const int64_t base = (int64_t)blockIdx.x * STILE;
  TO s = 0;
  for (int i = threadIdx.x; i < STILE; i += ST) {
    int64_t k = base + i;
    if (k < n) s += (TO)in[k];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    TO t = 0;
    for (int w = 0; w < SWARPS; ++w) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

// One CTA: in-place exclusive scan of p values; the total goes to *total.
template <typename TO>
__global__ void __launch_bounds__(1024) scan_sums(TO* __restrict__ p, int64_t np, TO* __restrict__ total) {
  __shared__ TO ws[32];
  const int64_t seg = (np + 1023) / 1024;
  const int64_t b = threadIdx.x * seg, e = b + seg < np ? b + seg : np;
  TO s = 0;
  for (int64_t i = b; i < e; ++i) s += p[i];
  TO incl = warp_incl_scan(s);
  if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = incl;
  __syncthreads();
  if (threadIdx.x < 32) {
    TO x = ws[threadIdx.x];
    TO y = warp_incl_scan(x);
    ws[threadIdx.x] = y - x;
  }
  __syncthreads();
  TO run = ws[threadIdx.x >> 5] + incl - s;
  for (int64_t i = b; i < e; ++i) {
    TO x = p[i];
    p[i] = run;
    run += x;
  }
  if (threadIdx.x == 1023) *total = run;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(ST) tile_scan(const TI* __restrict__ in, int64_t n, const TO* __restrict__ offs,
                                                TO* __restrict__ out) {
  __shared__ TO ws[SWARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * STILE + w * (SI * 32);
  TO ex[SI];
  TO run = 0;
#pragma unroll
  for (int j = 0; j < SI; ++j) {
    int64_t k = base + j * 32 + lane;
    TO x = k < n ? (TO)in[k] : (TO)0;
    TO incl = warp_incl_scan(x);
    ex[j] = run + incl - x;
    run += __shfl_sync(FULL, incl, 31);
  }
  if (lane == 0) ws[w] = run;
  __syncthreads();
  TO pre = offs[blockIdx.x];
  for (int i = 0; i < w; ++i) pre += ws[i];
#pragma unroll
  for (int j = 0; j < SI; ++j) {
    int64_t k = base + j * 32 + lane;
    if (k < n) out[k] = pre + ex[j];
  }
}

template <typename TI, typename TO>
int scan_impl(const TI* in, TO* out, int64_t n, cudaStream_t s, void* tmp, size_t tmp_bytes) {
  int64_t nt = (n + STILE - 1) / STILE;
  if (nt < 1) nt = 1;
  if (tmp_bytes < (size_t)(nt + 1) * sizeof(TO)) return GT_EINVAL;
  TO* sums = (TO*)tmp;
  tile_sums<TI, TO><<<(unsigned)nt, ST, 0, s>>>(in, n, sums);
  scan_sums<TO><<<1, 1024, 0, s>>>(sums, nt, out + n);
  tile_scan<TI, TO><<<(unsigned)nt, ST, 0, s>>>(in, n, sums, out);
  return cuda_fail(cudaGetLastError(), "scan");
}

}  // namespace

size_t scan_tmp_bytes(int64_t n) { return (size_t)((n + STILE - 1) / STILE + 2) * sizeof(int64_t); }

int scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s, void* tmp, size_t tmp_bytes) {
  return scan_impl<int32_t, int64_t>(in, out, n, s, tmp, tmp_bytes);
}

int scan_u8_to_i32(const uint8_t* in, int32_t* out, int64_t n, cudaStream_t s, void* tmp, size_t tmp_bytes) {
  return scan_impl<uint8_t, int32_t>(in, out, n, s, tmp, tmp_bytes);
}

}  // namespace gt
