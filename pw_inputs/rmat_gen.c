/*
 * Seeded R-MAT/Kronecker graph generator for large scales (2^24 nodes and
 * beyond), in C with OpenMP.  Input generation only: nothing here is part of
 * the estimator.
 *
 * Edge e (0 <= e < edge_factor * 2^scale) descends `scale` levels of the
 * 2x2 recursive matrix with probabilities (a, b, c, 1-a-b-c); the uniform draw
 * of level l is a counter-based hash (splitmix64 finaliser) of (seed, e, l), so
 * the graph does not depend on the number of threads.  The edges are
 * symmetrised, self-loops and duplicates dropped, rows sorted, and the
 * component of the highest-degree node kept (relabelled in increasing order)
 * when it holds a majority of the non-isolated nodes; otherwise every
 * component is labelled and the largest kept.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static inline double uniform01(uint64_t seed, uint64_t e, uint32_t level) {
  uint64_t h = mix64(seed ^ mix64(e * 64ull + level));
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

static inline void rmat_edge(uint64_t seed, uint64_t e, int scale, double a, double b, double c, uint32_t* u,
                             uint32_t* v) {
  uint32_t x = 0, y = 0;
  for (int l = 0; l < scale; ++l) {
    const double r = uniform01(seed, e, (uint32_t)l);
    const uint32_t bit = 1u << (scale - 1 - l);
    if (r >= a + b) x |= bit;                          /* lower half: quadrants c, d */
    if ((r >= a && r < a + b) || r >= a + b + c) y |= bit; /* right half: quadrants b, d */
  }
  *u = x;
  *v = y;
}

static int cmp_u32(const void* p, const void* q) {
  const uint32_t a = *(const uint32_t*)p, b = *(const uint32_t*)q;
  return (a > b) - (a < b);
}

void pwgen_free(void* p) { free(p); }

/* Returns 0, or -1 on allocation failure.  *row_ptr (n+1 int64) and *col_idx
 * (nnz int32) are malloc'ed; release them with pwgen_free. */
int pwgen_rmat(int scale, int edge_factor, double a, double b, double c, uint64_t seed, int threads, int64_t* n_out,
               int64_t* nnz_out, int64_t** row_ptr_out, int32_t** col_out) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#endif
  const int64_t n = (int64_t)1 << scale;
  const int64_t E = (int64_t)edge_factor << scale;
  int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!deg) return -1;
  /* pass 1: directed degrees (both directions, self-loops dropped) */
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    uint32_t u, v;
    rmat_edge(seed, (uint64_t)e, scale, a, b, c, &u, &v);
    if (u == v) continue;
#pragma omp atomic
    deg[u]++;
#pragma omp atomic
    deg[v]++;
  }
  int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!rp) { free(deg); return -1; }
  rp[0] = 0;
  for (int64_t i = 0; i < n; ++i) rp[i + 1] = rp[i] + deg[i];
  const int64_t m2 = rp[n];
  uint32_t* col = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m2 > 0 ? m2 : 1));
  if (!col) { free(deg); free(rp); return -1; }
  memcpy(deg, rp, sizeof(int64_t) * (size_t)n); /* deg becomes the fill cursor */
  /* pass 2: fill */
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    uint32_t u, v;
    rmat_edge(seed, (uint64_t)e, scale, a, b, c, &u, &v);
    if (u == v) continue;
    int64_t pu, pv;
#pragma omp atomic capture
    pu = deg[u]++;
#pragma omp atomic capture
    pv = deg[v]++;
    col[pu] = v;
    col[pv] = u;
  }
  /* sort each row and drop duplicates; new degrees into deg */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    uint32_t* r = col + rp[i];
    const int64_t d = rp[i + 1] - rp[i];
    if (d > 1) qsort(r, (size_t)d, sizeof(uint32_t), cmp_u32);
    int64_t k = 0;
    for (int64_t j = 0; j < d; ++j)
      if (j == 0 || r[j] != r[j - 1]) r[k++] = r[j];
    deg[i] = k;
  }
  /* component of the highest-degree node by breadth-first search */
  int64_t root = 0;
  for (int64_t i = 1; i < n; ++i)
    if (deg[i] > deg[root]) root = i;
  int32_t* label = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!label || !queue) { free(deg); free(rp); free(col); free(label); free(queue); return -1; }
  for (int64_t i = 0; i < n; ++i) label[i] = -1;
  int64_t nonisolated = 0;
  for (int64_t i = 0; i < n; ++i) nonisolated += deg[i] > 0;
  int32_t best = 0;
  int64_t best_size = 0;
  int32_t comp = 0;
  for (int64_t start = root;; ) {
    int64_t head = 0, tail = 0;
    queue[tail++] = start;
    label[start] = comp;
    while (head < tail) {
      const int64_t x = queue[head++];
      for (int64_t j = rp[x]; j < rp[x] + deg[x]; ++j) {
        const uint32_t y = col[j];
        if (label[y] < 0) {
          label[y] = comp;
          queue[tail++] = y;
        }
      }
    }
    if (tail > best_size) { best_size = tail; best = comp; }
    ++comp;
    if (2 * best_size > nonisolated) break; /* a majority component is the largest */
    int64_t next = -1;
    for (int64_t i = 0; i < n; ++i)
      if (label[i] < 0 && deg[i] > 0) { next = i; break; }
    if (next < 0) break;
    start = next;
  }
  free(queue);
  /* relabel kept nodes in increasing order and rebuild */
  int64_t* new_id = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!new_id) { free(deg); free(rp); free(col); free(label); return -1; }
  int64_t n2 = 0, m = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (label[i] == best && deg[i] > 0) {
      new_id[i] = n2++;
      m += deg[i];
    } else {
      new_id[i] = -1;
    }
  }
  int64_t* rp2 = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n2 + 1));
  int32_t* col2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  if (!rp2 || !col2) { free(deg); free(rp); free(col); free(label); free(new_id); free(rp2); free(col2); return -1; }
  rp2[0] = 0;
  {
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i)
      if (new_id[i] >= 0) { rp2[k + 1] = rp2[k] + deg[i]; ++k; }
  }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    if (new_id[i] < 0) continue;
    const int64_t dst = rp2[new_id[i]];
    for (int64_t j = 0; j < deg[i]; ++j) col2[dst + j] = (int32_t)new_id[col[rp[i] + j]];
  }
  free(deg);
  free(rp);
  free(col);
  free(label);
  free(new_id);
  *n_out = n2;
  *nnz_out = m;
  *row_ptr_out = rp2;
  *col_out = col2;
  return 0;
}
