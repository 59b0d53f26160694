/*
 * oracle.c -- plain, slow, serial CPU oracle for edge-tree BFS (arXiv 2009.07463).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this code; the GPU library never calls it and shares no
 * code with it. Everything here is written for a reader to check against the paper
 * by eye: no blocking, no fusion, no reordering.
 *
 * What it computes:
 *  - or_graph_build: the simple undirected graph of an edge-tuple list (Sec. 5.1.1:
 *    CSR row + col arrays). Self-loops are dropped, duplicate tuples merged, each
 *    adjacency list sorted ascending.
 *  - or_bfs: the plain definition the whole method must reproduce exactly.
 *    level[v] = hop distance from root (-1 if unreachable); parent[root] = root
 *    (Alg. 1, initialisation); for every other reached v, parent[v] = the smallest
 *    vertex id u adjacent to v with level[u] = level[v] - 1 (the min-id tie-break
 *    that makes the BFS tree unique; any such u satisfies the Graph500 rule quoted in
 *    Sec. 5.3 that every parent lies on the root's spanning tree). Levels come from a
 *    serial first-in-first-out top-down BFS (Alg. 1, TOP-DOWN only, no parallelism);
 *    parents from one scan of each reached vertex's sorted neighbours.
 *  - or_classify: Alg. 8 (edge-tree vertex classification, Sec. 4.3) in the paper's
 *    order and notation, with the Jacobi-style copy of the neighbour counts at the
 *    start of every height (vertex_num_pre / vertex_num_new).
 *  - or_traversed_tuples: the Graph500 TEPS numerator, the number of input tuples
 *    whose two endpoints are both reached.
 */
#include "oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

struct or_graph {
  int64_t n;
  int64_t nnz;
  int64_t* row; /* n + 1 */
  int32_t* col; /* nnz */
};

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Graph construction is not part of what the oracle times (only or_bfs is), so its
 * three passes are split across `nthreads` POSIX threads. Each pass is order-independent:
 * the fill order within a row is arbitrary and every row is sorted afterwards, so the
 * result is the same for any thread count. */
typedef struct build_job {
  const int64_t* edges;
  int64_t lo, hi; /* tuple range (count, fill) or vertex range (sort) */
  int64_t* cnt;
  int64_t* start;
  int64_t* fill;
  int32_t* adj;
  int pass;
} build_job;

static void* build_worker(void* arg) {
  build_job* j = (build_job*)arg;
  if (j->pass == 0) { /* degree counts with duplicates, self-loops skipped */
    for (int64_t i = j->lo; i < j->hi; ++i) {
      int64_t u = j->edges[2 * i], v = j->edges[2 * i + 1];
      if (u == v) continue;
      __atomic_fetch_add(&j->cnt[u], 1, __ATOMIC_RELAXED);
      __atomic_fetch_add(&j->cnt[v], 1, __ATOMIC_RELAXED);
    }
  } else if (j->pass == 1) { /* bucket the directed entries by source */
    for (int64_t i = j->lo; i < j->hi; ++i) {
      int64_t u = j->edges[2 * i], v = j->edges[2 * i + 1];
      if (u == v) continue;
      j->adj[j->start[u] + __atomic_fetch_add(&j->fill[u], 1, __ATOMIC_RELAXED)] = (int32_t)v;
      j->adj[j->start[v] + __atomic_fetch_add(&j->fill[v], 1, __ATOMIC_RELAXED)] = (int32_t)u;
    }
  } else { /* each row: sort ascending, keep one copy of each neighbour */
    for (int64_t v = j->lo; v < j->hi; ++v) {
      int32_t* a = j->adj + j->start[v];
      int64_t k = j->start[v + 1] - j->start[v], w = 0;
      qsort(a, (size_t)k, sizeof(int32_t), cmp_i32);
      for (int64_t t = 0; t < k; ++t)
        if (t == 0 || a[t] != a[t - 1]) a[w++] = a[t];
      j->cnt[v] = w; /* deduplicated degree */
    }
  }
  return NULL;
}

static void run_pass(build_job* proto, int pass, int64_t total, int nthreads) {
  pthread_t tid[64];
  build_job jobs[64];
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 64) nthreads = 64;
  int64_t chunk = (total + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = *proto;
    jobs[t].pass = pass;
    jobs[t].lo = t * chunk < total ? t * chunk : total;
    jobs[t].hi = (t + 1) * chunk < total ? (t + 1) * chunk : total;
    if (nthreads == 1 || pthread_create(&tid[t], NULL, build_worker, &jobs[t]) != 0) {
      build_worker(&jobs[t]);
      tid[t] = 0;
    }
  }
  for (int t = 0; t < nthreads; ++t)
    if (nthreads > 1 && tid[t]) pthread_join(tid[t], NULL);
}

or_graph* or_graph_build(const int64_t* edges, int64_t m, int64_t n, int nthreads) {
  if (n < 0 || n > 2147483647LL || m < 0) return NULL;
  for (int64_t i = 0; i < 2 * m; ++i)
    if (edges[i] < 0 || edges[i] >= n) return NULL;

  int64_t* cnt = calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* start = malloc(((size_t)n + 1) * sizeof(int64_t));
  int64_t* fill = calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt || !start || !fill) { free(cnt); free(start); free(fill); return NULL; }
  build_job job = {edges, 0, 0, cnt, start, fill, NULL, 0};
  run_pass(&job, 0, m, nthreads);
  start[0] = 0;
  for (int64_t v = 0; v < n; ++v) start[v + 1] = start[v] + cnt[v];
  int32_t* adj = malloc((size_t)(start[n] > 0 ? start[n] : 1) * sizeof(int32_t));
  if (!adj) { free(cnt); free(start); free(fill); return NULL; }
  job.adj = adj;
  run_pass(&job, 1, m, nthreads);
  run_pass(&job, 2, n, nthreads);
  int64_t* deg = cnt;

  or_graph* g = malloc(sizeof(or_graph));
  if (!g) { free(cnt); free(start); free(adj); free(fill); return NULL; }
  g->n = n;
  g->row = malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!g->row) { free(g); free(cnt); free(start); free(adj); free(fill); return NULL; }
  g->row[0] = 0;
  for (int64_t v = 0; v < n; ++v) g->row[v + 1] = g->row[v] + deg[v];
  g->nnz = g->row[n];
  g->col = malloc((size_t)(g->nnz > 0 ? g->nnz : 1) * sizeof(int32_t));
  if (!g->col) { free(g->row); free(g); free(cnt); free(start); free(adj); free(fill); return NULL; }
  for (int64_t v = 0; v < n; ++v)
    memcpy(g->col + g->row[v], adj + start[v], (size_t)deg[v] * sizeof(int32_t));
  free(cnt);
  free(start);
  free(adj);
  free(fill);
  return g;
}

void or_graph_free(or_graph* g) {
  if (!g) return;
  free(g->row);
  free(g->col);
  free(g);
}

int64_t or_graph_n(const or_graph* g) { return g->n; }
int64_t or_graph_nnz(const or_graph* g) { return g->nnz; }

void or_graph_csr(const or_graph* g, int64_t* row, int32_t* col) {
  memcpy(row, g->row, ((size_t)g->n + 1) * sizeof(int64_t));
  memcpy(col, g->col, (size_t)g->nnz * sizeof(int32_t));
}

int or_bfs(const or_graph* g, int64_t root, int32_t* level, int32_t* parent) {
  if (root < 0 || root >= g->n) return -1;
  int64_t n = g->n;
  for (int64_t v = 0; v < n; ++v) { level[v] = -1; parent[v] = -1; }
  int32_t* queue = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!queue) return -2;
  int64_t head = 0, tail = 0;
  level[root] = 0;
  queue[tail++] = (int32_t)root;
  while (head < tail) { /* Alg. 1 top-down, one vertex at a time */
    int32_t v = queue[head++];
    for (int64_t e = g->row[v]; e < g->row[v + 1]; ++e) {
      int32_t w = g->col[e];
      if (level[w] < 0) {
        level[w] = level[v] + 1;
        queue[tail++] = w;
      }
    }
  }
  free(queue);
  parent[root] = (int32_t)root;
  for (int64_t v = 0; v < n; ++v) { /* smallest neighbour one level up */
    if (v == root || level[v] < 0) continue;
    for (int64_t e = g->row[v]; e < g->row[v + 1]; ++e) {
      int32_t u = g->col[e];
      if (level[u] == level[v] - 1) { parent[v] = u; break; }
    }
  }
  return 0;
}

int or_classify(const or_graph* g, int height, uint8_t* vertex_type, int32_t* peel_height,
                int32_t* height_reached) {
  int64_t n = g->n;
  int32_t* vertex_num = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t)); /* G.vertex_num */
  int32_t* vertex_num_pre = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t* vertex_num_new = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!vertex_num || !vertex_num_pre || !vertex_num_new) {
    free(vertex_num); free(vertex_num_pre); free(vertex_num_new);
    return -2;
  }
  for (int64_t v = 0; v < n; ++v) {
    vertex_num[v] = (int32_t)(g->row[v + 1] - g->row[v]);
    vertex_type[v] = OR_CORE_INTERNAL;
    if (peel_height) peel_height[v] = -1;
  }
  memcpy(vertex_num_pre, vertex_num, (size_t)n * sizeof(int32_t));
  memcpy(vertex_num_new, vertex_num, (size_t)n * sizeof(int32_t));
  int flag = 0;

  for (int64_t v = 0; v < n; ++v) { /* zero-degree and leaf vertices */
    if (vertex_num_pre[v] == 0) {
      vertex_type[v] = OR_VERTEX_ZERO;
    } else if (vertex_num_pre[v] == 1) {
      vertex_type[v] = OR_TREE_LEAF;
      if (peel_height) peel_height[v] = 0;
      for (int64_t e = g->row[v]; e < g->row[v + 1]; ++e) vertex_num_new[g->col[e]] -= 1;
      flag = 1;
    }
  }

  int height_current = 1, reached = 0;
  while (flag == 1 && (height == -1 || height_current <= height)) { /* tree-internal vertices */
    flag = 0;
    memcpy(vertex_num_pre, vertex_num_new, (size_t)n * sizeof(int32_t));
    for (int64_t v = 0; v < n; ++v) {
      if (vertex_type[v] == OR_CORE_INTERNAL && (vertex_num_pre[v] == 0 || vertex_num_pre[v] == 1)) {
        vertex_type[v] = OR_TREE_INTERNAL;
        if (peel_height) peel_height[v] = height_current;
        for (int64_t e = g->row[v]; e < g->row[v + 1]; ++e) vertex_num_new[g->col[e]] -= 1;
        flag = 1;
      }
    }
    if (flag) reached = height_current;
    height_current += 1;
  }

  for (int64_t v = 0; v < n; ++v) /* core-edge vertices: degree changed */
    if (vertex_type[v] == OR_CORE_INTERNAL && vertex_num_new[v] != vertex_num[v]) vertex_type[v] = OR_CORE_EDGE;

  if (height_reached) *height_reached = reached;
  free(vertex_num);
  free(vertex_num_pre);
  free(vertex_num_new);
  return 0;
}

int64_t or_traversed_tuples(const int64_t* edges, int64_t m, const int32_t* level) {
  int64_t c = 0;
  for (int64_t i = 0; i < m; ++i)
    if (level[edges[2 * i]] >= 0 && level[edges[2 * i + 1]] >= 0) c++;
  return c;
}
