// gen_device.cu -- device side of the seeded input generator (see graphgen.h).
// Produces the same tuples as gen_host.c for the same arguments, directly in HBM,
// so large graphs (2^30 tuples at scale 26) need no host round trip.
#include <cuda_runtime.h>
#include <stdint.h>

#include "graphgen.h"

#define GG_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

__global__ void rmat_fill_kernel(uint64_t kd, gg_rmat_thresholds t, int scale, gg_perm_keys p, int permute,
                                 int64_t begin, int64_t count, int64_t* __restrict__ out) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride) {
    int64_t u, v;
    gg_rmat_tuple(kd, &t, scale, permute ? &p : nullptr, (uint64_t)(begin + j), &u, &v);
    reinterpret_cast<longlong2*>(out)[j] = make_longlong2(u, v);
  }
}

__global__ void uniform_fill_kernel(uint64_t ku, uint64_t n, int64_t begin, int64_t count,
                                    int64_t* __restrict__ out) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count; j += stride) {
    int64_t u, v;
    gg_uniform_tuple(ku, n, (uint64_t)(begin + j), &u, &v);
    reinterpret_cast<longlong2*>(out)[j] = make_longlong2(u, v);
  }
}

int grid_for(int64_t count) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (count + 255) / 256;
  int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

// Device-resident R-MAT tuples; out is a device pointer to count * 2 int64 (16-byte aligned).
// Returns 0, or the cudaError_t of the launch.
GG_EXPORT int gg_rmat_fill_device(uint64_t seed, int scale, int64_t begin, int64_t count, uint32_t a_ppm,
                                  uint32_t b_ppm, uint32_t c_ppm, int permute, int64_t* out, void* stream) {
  if (count <= 0) return 0;
  gg_rmat_thresholds t = gg_rmat_make_thresholds(a_ppm, b_ppm, c_ppm);
  gg_perm_keys p = gg_make_perm_keys(seed, scale);
  rmat_fill_kernel<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(gg_key(seed, GG_PURPOSE_RMAT), t, scale, p,
                                                                       permute, begin, count, out);
  return (int)cudaGetLastError();
}

// Device-resident uniform tuples over [0, n).
GG_EXPORT int gg_uniform_fill_device(uint64_t seed, int64_t n, int64_t begin, int64_t count, int64_t* out,
                                     void* stream) {
  if (count <= 0) return 0;
  uniform_fill_kernel<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(gg_key(seed, GG_PURPOSE_UNIFORM),
                                                                          (uint64_t)n, begin, count, out);
  return (int)cudaGetLastError();
}
