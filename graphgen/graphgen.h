/*
 * graphgen.h -- seeded synthetic graph inputs (edge tuples and BFS roots).
 *
 * This module only makes inputs. It holds none of the BFS / edge-tree arithmetic,
 * and both the CPU oracle side (through gen_host.c) and the GPU side (through
 * gen_device.cu) draw their inputs from these inline definitions, so the same
 * seed gives bit-identical tuples on host and device.
 *
 * Definitions (all integer-exact):
 *  - Counter-based generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 *    pseudorandom number generators", OOPSLA 2014): value at counter c of the
 *    stream with key k is the SplitMix64 finaliser of k + (c + 1) * golden gamma.
 *  - R-MAT tuples (Chakrabarti, Zhan, Faloutsos, SDM 2004), the recursive
 *    quadrant model the paper's Kronecker inputs use (Sec. 6.1: initiator
 *    A=0.57, B=C=0.19, D=0.05, 2^scale vertices, 2^scale * edgefactor tuples).
 *    Tuple i draws one 32-bit word per recursion level; the word is compared
 *    against integer thresholds floor(p * 2^32) for A, A+B, A+B+C.
 *  - Vertex-id scrambling: a keyed bijection on scale-bit integers (four rounds
 *    of odd multiply, xor-shift, add, each modulo 2^scale), applied to both ends.
 *  - Uniform tuples: both ends uniform over [0, n) from one 64-bit draw
 *    (multiply-high mapping of each 32-bit half).
 *  - Root candidates: candidate j is the multiply-high map of draw j to [0, n);
 *    callers keep the distinct candidates of degree >= 1, in candidate order.
 */
#ifndef GRAPHGEN_H
#define GRAPHGEN_H
#include <stdint.h>

#if defined(__CUDACC__)
#define GG_FN __host__ __device__ __forceinline__
#else
#define GG_FN static inline
#endif

/* Stream purposes: each gets its own key derived from the user seed. */
#define GG_PURPOSE_RMAT 1u
#define GG_PURPOSE_PERM 2u
#define GG_PURPOSE_UNIFORM 3u
#define GG_PURPOSE_ROOTS 4u

GG_FN uint64_t gg_splitmix64(uint64_t key, uint64_t ctr) {
  uint64_t z = key + (ctr + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Key of one purpose's stream under a user seed. */
GG_FN uint64_t gg_key(uint64_t seed, uint32_t purpose) {
  return gg_splitmix64(seed ^ 0x6A09E667F3BCC909ull, (uint64_t)purpose);
}

/* Integer thresholds of the R-MAT initiator, probabilities in parts per million. */
typedef struct gg_rmat_thresholds {
  uint32_t t_a, t_ab, t_abc;
} gg_rmat_thresholds;

GG_FN gg_rmat_thresholds gg_rmat_make_thresholds(uint32_t a_ppm, uint32_t b_ppm, uint32_t c_ppm) {
  gg_rmat_thresholds t;
  uint64_t a = a_ppm, ab = (uint64_t)a_ppm + b_ppm, abc = (uint64_t)a_ppm + b_ppm + c_ppm;
  uint64_t ta = (a << 32) / 1000000u, tab = (ab << 32) / 1000000u, tabc = (abc << 32) / 1000000u;
  t.t_a = ta > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)ta;
  t.t_ab = tab > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)tab;
  t.t_abc = tabc > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)tabc;
  return t;
}

/* Round keys of the id scrambling: k[0..3] odd multipliers, k[4..7] addends (mod 2^scale). */
typedef struct gg_perm_keys {
  uint64_t k[8];
  uint64_t mask;
  int shift;
} gg_perm_keys;

GG_FN gg_perm_keys gg_make_perm_keys(uint64_t seed, int scale) {
  gg_perm_keys p;
  uint64_t key = gg_key(seed, GG_PURPOSE_PERM);
  p.mask = scale >= 64 ? ~0ull : ((1ull << scale) - 1u);
  p.shift = (scale + 1) / 2;
  for (int r = 0; r < 4; ++r) {
    p.k[r] = (gg_splitmix64(key, (uint64_t)(2 * r)) & p.mask) | 1u;
    p.k[4 + r] = gg_splitmix64(key, (uint64_t)(2 * r + 1)) & p.mask;
  }
  return p;
}

/* Keyed bijection on [0, 2^scale). Each step (odd multiply, x ^= x >> s with s >= 1,
 * add) is invertible modulo 2^scale, so the composition is a permutation. */
GG_FN uint64_t gg_perm(const gg_perm_keys* p, uint64_t x) {
  for (int r = 0; r < 4; ++r) {
    x = (x * p->k[r]) & p->mask;
    x ^= x >> p->shift;
    x = (x + p->k[4 + r]) & p->mask;
  }
  return x;
}

/* R-MAT tuple i: one 32-bit draw per level, most significant bit first. Quadrants:
 * [0, t_a) -> (0,0); [t_a, t_ab) -> (0,1); [t_ab, t_abc) -> (1,0); [t_abc, 2^32) -> (1,1). */
GG_FN void gg_rmat_tuple(uint64_t key_draw, const gg_rmat_thresholds* t, int scale,
                         const gg_perm_keys* perm, uint64_t i, int64_t* u_out, int64_t* v_out) {
  uint64_t u = 0, v = 0, word = 0;
  for (int l = 0; l < scale; ++l) {
    if ((l & 1) == 0) word = gg_splitmix64(key_draw, i * 16u + (uint64_t)(l >> 1));
    uint32_t r = (l & 1) ? (uint32_t)(word >> 32) : (uint32_t)word;
    uint64_t bu = r >= t->t_ab;
    uint64_t bv = (r >= t->t_a && r < t->t_ab) || r >= t->t_abc;
    u = (u << 1) | bu;
    v = (v << 1) | bv;
  }
  if (perm) {
    u = gg_perm(perm, u);
    v = gg_perm(perm, v);
  }
  *u_out = (int64_t)u;
  *v_out = (int64_t)v;
}

/* Uniform tuple i over [0, n), n <= 2^32. */
GG_FN void gg_uniform_tuple(uint64_t key_uni, uint64_t n, uint64_t i, int64_t* u_out, int64_t* v_out) {
  uint64_t w = gg_splitmix64(key_uni, i);
  *u_out = (int64_t)(((w & 0xFFFFFFFFull) * n) >> 32);
  *v_out = (int64_t)(((w >> 32) * n) >> 32);
}

/* Root candidate j over [0, n), n <= 2^32. */
GG_FN int64_t gg_root_candidate_at(uint64_t key_roots, uint64_t n, uint64_t j) {
  uint64_t w = gg_splitmix64(key_roots, j);
  return (int64_t)(((w >> 32) * n) >> 32);
}

#endif /* GRAPHGEN_H */
