/*
 * oracle.h -- serial CPU oracle for edge-tree BFS. TEST INFRASTRUCTURE ONLY: used by
 * the test suite, the smoke check and the benchmark's CPU-baseline leg, never by the
 * GPU library, with which it shares no code.
 */
#ifndef GT_ORACLE_H
#define GT_ORACLE_H
#include <stdint.h>

#define OR_EXPORT __attribute__((visibility("default")))

/* Vertex classes of Sec. 4.2, numbered in the paper's order of listing. */
enum {
  OR_CORE_INTERNAL = 0, /* CI */
  OR_CORE_EDGE = 1,     /* CE */
  OR_TREE_INTERNAL = 2, /* TI */
  OR_TREE_LEAF = 3,     /* TL */
  OR_VERTEX_ZERO = 4    /* VZ */
};

typedef struct or_graph or_graph;

/* Simple undirected graph of m tuples edges[2i], edges[2i+1] over [0, n), built with
 * nthreads threads (same result for any count). NULL on a vertex id outside [0, n) or on
 * allocation failure. */
OR_EXPORT or_graph* or_graph_build(const int64_t* edges, int64_t m, int64_t n, int nthreads);
OR_EXPORT void or_graph_free(or_graph* g);
OR_EXPORT int64_t or_graph_n(const or_graph* g);
OR_EXPORT int64_t or_graph_nnz(const or_graph* g);
/* Copies row[n+1] and col[nnz] out. */
OR_EXPORT void or_graph_csr(const or_graph* g, int64_t* row, int32_t* col);
/* level[n], parent[n] as defined in oracle.c. 0 on success, -1 bad root, -2 no memory. */
OR_EXPORT int or_bfs(const or_graph* g, int64_t root, int32_t* level, int32_t* parent);
/* Alg. 8 with maximum height `height` (0: leaves only, -1: to the fixpoint).
 * vertex_type[n]; peel_height[n] (nullable): 0 for leaves, h for a vertex marked
 * tree-internal at height h, -1 otherwise; height_reached: largest h that marked a vertex. */
OR_EXPORT int or_classify(const or_graph* g, int height, uint8_t* vertex_type, int32_t* peel_height,
                          int32_t* height_reached);
/* Number of tuples with both endpoints reached (level >= 0). */
OR_EXPORT int64_t or_traversed_tuples(const int64_t* edges, int64_t m, const int32_t* level);

#endif
