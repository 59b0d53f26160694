// radix.cu -- stable LSD radix sort of 64-bit keys (packed (u << b) | v edge keys).
//
// Each pass sorts on one 8-bit digit. The keys are split into G contiguous ranges, one
// per CTA. Pass structure ("reduce then scan"):
//   1. radix_hist: every CTA counts the digits of its range -> hist[digit][cta];
//   2. radix_offsets: one CTA turns hist into exclusive offsets, digit-major then CTA;
//   3. radix_scatter: every CTA walks its range in 4096-key tiles, ranks each key among
//      equal digits (warp match + per-warp counters, so the rank is stable), stages the
//      tile in shared memory sorted by digit and writes each digit run to its offset.
#include "gt_device.cuh"
#include "gt_internal.cuh"

namespace gt {
namespace {

constexpr int RT = 256;
constexpr int RI = 16;
constexpr int RTILE = RT * RI;
constexpr int RW = RT / 32;
constexpr int RBINS = 256;

__global__ void __launch_bounds__(RT) radix_hist(const uint64_t* __restrict__ keys, int64_t n, int64_t per,
                                                 int shift, int G, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[RW][RBINS];
  const int w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RW * RBINS; i += RT) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t b = (int64_t)blockIdx.x * per, e = b + per < n ? b + per : n;
  for (int64_t i = b + threadIdx.x; i < e; i += RT) atomicAdd(&h[w][(keys[i] >> shift) & 255], 1u);
  __syncthreads();
  uint32_t s = 0;
  for (int ww = 0; ww < RW; ++ww) s += h[ww][threadIdx.x];
  hist[(int64_t)threadIdx.x * G + blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) radix_offsets(const uint32_t* __restrict__ hist, int64_t ne,
                                                      int64_t* __restrict__ offs) {
  __shared__ int64_t ws[32];
  const int64_t seg = (ne + 1023) / 1024;
  const int64_t b = threadIdx.x * seg, e = b + seg < ne ? b + seg : ne;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += hist[i];
  int64_t incl = warp_incl_scan(s);
  if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = incl;
  __syncthreads();
  if (threadIdx.x < 32) {
    int64_t x = ws[threadIdx.x];
    ws[threadIdx.x] = warp_incl_scan(x) - x;
  }
  __syncthreads();
  int64_t run = ws[threadIdx.x >> 5] + incl - s;
  for (int64_t i = b; i < e; ++i) {
    offs[i] = run;
    run += hist[i];
  }
}

__global__ void __launch_bounds__(RT) radix_scatter(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                    int64_t n, int64_t per, int shift, int G,
                                                    const int64_t* __restrict__ offs) {
  __shared__ uint32_t wcnt[RW][RBINS];
  __shared__ uint64_t skeys[RTILE];
  __shared__ uint32_t tcnt[RBINS], toff[RBINS];
  __shared__ int64_t run[RBINS];
  __shared__ uint32_t wsum[RW];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, t = threadIdx.x;
  run[t] = offs[(int64_t)t * G + blockIdx.x];
  const int64_t b = (int64_t)blockIdx.x * per, e = b + per < n ? b + per : n;
  for (int64_t tb = b; tb < e; tb += RTILE) {
    for (int i = t; i < RW * RBINS; i += RT) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    uint64_t k[RI];
    uint32_t rk[RI];
#pragma unroll
    for (int j = 0; j < RI; ++j) {
      const int64_t idx = tb + w * (RI * 32) + j * 32 + lane;
      const bool valid = idx < e;
      k[j] = valid ? in[idx] : 0ull;
      const uint32_t d = valid ? (uint32_t)((k[j] >> shift) & 255) : 256u;
      const unsigned peers = __match_any_sync(FULL, d);
      const uint32_t before = valid ? wcnt[w][d] : 0u;
      rk[j] = before + __popc(peers & lanemask_lt());
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {  // per digit: exclusive over warps, tile total
      uint32_t s = 0;
      for (int ww = 0; ww < RW; ++ww) {
        uint32_t c = wcnt[ww][t];
        wcnt[ww][t] = s;
        s += c;
      }
      tcnt[t] = s;
      uint32_t incl = warp_incl_scan(s);
      if (lane == 31) wsum[w] = incl;
      __syncthreads();
      uint32_t pre = 0;
      for (int ww = 0; ww < w; ++ww) pre += wsum[ww];
      toff[t] = pre + incl - s;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RI; ++j) {
      const int64_t idx = tb + w * (RI * 32) + j * 32 + lane;
      if (idx < e) {
        const uint32_t d = (uint32_t)((k[j] >> shift) & 255);
        skeys[toff[d] + wcnt[w][d] + rk[j]] = k[j];
      }
    }
    __syncthreads();
    const int cnt = (int)(e - tb < RTILE ? e - tb : RTILE);
    for (int i = t; i < cnt; i += RT) {
      const uint64_t key = skeys[i];
      const uint32_t d = (uint32_t)((key >> shift) & 255);
      out[run[d] + (i - toff[d])] = key;
    }
    __syncthreads();
    run[t] += tcnt[t];
    __syncthreads();
  }
}

int64_t per_cta(int64_t n, int grid) {
  int64_t per = (n + grid - 1) / grid;
  per = (per + RTILE - 1) / RTILE * RTILE;
  return per < RTILE ? RTILE : per;
}

}  // namespace

size_t radix_tmp_bytes(int64_t nkeys, int grid) {
  (void)nkeys;
  return (size_t)RBINS * grid * sizeof(uint32_t) + ((size_t)RBINS * grid + 1) * sizeof(int64_t) + 256;
}

int radix_sort_u64(uint64_t** keys, uint64_t** alt, int64_t n, int bits, int grid, void* tmp, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return GT_OK;
  const int64_t per = per_cta(n, grid);
  const int G = (int)((n + per - 1) / per);
  uint32_t* hist = (uint32_t*)tmp;
  int64_t* offs = (int64_t*)(((uintptr_t)(hist + (size_t)RBINS * grid) + 255) & ~(uintptr_t)255);
  const int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    radix_hist<<<G, RT, 0, s>>>(*keys, n, per, shift, G, hist);
    radix_offsets<<<1, 1024, 0, s>>>(hist, (int64_t)RBINS * G, offs);
    radix_scatter<<<G, RT, 0, s>>>(*keys, *alt, n, per, shift, G, offs);
    uint64_t* t = *keys;
    *keys = *alt;
    *alt = t;
  }
  return cuda_fail(cudaGetLastError(), "radix sort");
}

}  // namespace gt
