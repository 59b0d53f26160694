/*
 * gen_host.c -- host side of the seeded input generator (see graphgen.h for the
 * definitions). Plain C, no threads: callers split [begin, begin + count) into
 * chunks to fill in parallel.
 */
#include "graphgen.h"

#define GG_EXPORT __attribute__((visibility("default")))

/* Tuples i in [begin, begin + count) of an R-MAT graph with 2^scale vertices, written
 * as out[2*(i-begin)] = u, out[2*(i-begin)+1] = v. permute != 0 scrambles the ids. */
GG_EXPORT void gg_rmat_fill(uint64_t seed, int scale, int64_t begin, int64_t count, uint32_t a_ppm,
                            uint32_t b_ppm, uint32_t c_ppm, int permute, int64_t* out) {
  gg_rmat_thresholds t = gg_rmat_make_thresholds(a_ppm, b_ppm, c_ppm);
  gg_perm_keys p = gg_make_perm_keys(seed, scale);
  uint64_t kd = gg_key(seed, GG_PURPOSE_RMAT);
  for (int64_t j = 0; j < count; ++j)
    gg_rmat_tuple(kd, &t, scale, permute ? &p : 0, (uint64_t)(begin + j), &out[2 * j], &out[2 * j + 1]);
}

/* Tuples i in [begin, begin + count) of a uniform random multigraph on n vertices. */
GG_EXPORT void gg_uniform_fill(uint64_t seed, int64_t n, int64_t begin, int64_t count, int64_t* out) {
  uint64_t ku = gg_key(seed, GG_PURPOSE_UNIFORM);
  for (int64_t j = 0; j < count; ++j)
    gg_uniform_tuple(ku, (uint64_t)n, (uint64_t)(begin + j), &out[2 * j], &out[2 * j + 1]);
}

/* Root candidates j in [begin, begin + count) over [0, n). */
GG_EXPORT void gg_root_candidates(uint64_t seed, int64_t n, int64_t begin, int64_t count, int64_t* out) {
  uint64_t kr = gg_key(seed, GG_PURPOSE_ROOTS);
  for (int64_t j = 0; j < count; ++j) out[j] = gg_root_candidate_at(kr, (uint64_t)n, (uint64_t)(begin + j));
}

/* The scrambling bijection itself, exposed so tests can check it is a permutation. */
GG_EXPORT void gg_perm_fill(uint64_t seed, int scale, int64_t begin, int64_t count, int64_t* out) {
  gg_perm_keys p = gg_make_perm_keys(seed, scale);
  for (int64_t j = 0; j < count; ++j) out[j] = (int64_t)gg_perm(&p, (uint64_t)(begin + j));
}
