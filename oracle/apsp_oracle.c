/*
 * CPU oracle for all-pairs shortest paths (APSP) -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this file.  The CUDA library never links, includes or calls it, and it
 * shares no code with the CUDA library.
 *
 * What it computes (the paper, Sec. 3 "Preliminaries"): for an undirected
 * graph with non-negative weights, the length of the shortest path between
 * every pair of vertices; no paths.  Conventions: d(i,i) = 0, a missing edge
 * is the sentinel INF, and d(i,j) = INF exactly when i and j are in different
 * components.
 *
 * Routines:
 *   oracle_fw_i64 / oracle_fw_f64   textbook Floyd-Warshall (the sequential
 *                                   solver the paper's Table 1 "FloydWarshall"
 *                                   delegates to; Sec. 3 cites it as the
 *                                   standard O(n^3) method), int64 / double,
 *                                   INF kept as a checked sentinel.
 *   oracle_minplus_i64 / _f64       C = min(C, A (x) B), the min-plus product of
 *                                   Table 1 "MatProd" followed by "MatMin".
 *   oracle_dijkstra_i64 / _f64      Dijkstra with a binary heap from a list of
 *                                   sources on a CSR graph (the other standard
 *                                   route named in Sec. 3); used as an
 *                                   independent cross-check and at sizes where
 *                                   O(n^3) is out of reach.
 *
 * All loops are written in the order of the definitions, with no blocking,
 * fusion or reordering.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Floyd-Warshall over outer indices k in [k_begin, k_end).  A full solve is
 * k_begin = 0, k_end = n.  Row-major d[i*n + j].  Entries equal to `inf` mean
 * "no path"; a relaxation through such an entry is skipped, so INF never takes
 * part in a sum.  Returns 0, or -1 on a bad argument. */
int oracle_fw_i64(int64_t *d, int64_t n, int64_t inf, int64_t k_begin, int64_t k_end) {
  if (!d || n < 0 || k_begin < 0 || k_end > n || k_begin > k_end) return -1;
  for (int64_t k = k_begin; k < k_end; ++k) {
    for (int64_t i = 0; i < n; ++i) {
      int64_t dik = d[i * n + k];
      if (dik == inf) continue;
      for (int64_t j = 0; j < n; ++j) {
        int64_t dkj = d[k * n + j];
        if (dkj == inf) continue;
        int64_t via = dik + dkj;
        if (via < d[i * n + j]) d[i * n + j] = via;
      }
    }
  }
  return 0;
}

/* Same in double precision; a missing edge is +infinity. */
int oracle_fw_f64(double *d, int64_t n, int64_t k_begin, int64_t k_end) {
  if (!d || n < 0 || k_begin < 0 || k_end > n || k_begin > k_end) return -1;
  for (int64_t k = k_begin; k < k_end; ++k) {
    for (int64_t i = 0; i < n; ++i) {
      double dik = d[i * n + k];
      if (isinf(dik)) continue;
      for (int64_t j = 0; j < n; ++j) {
        double dkj = d[k * n + j];
        if (isinf(dkj)) continue;
        double via = dik + dkj;
        if (via < d[i * n + j]) d[i * n + j] = via;
      }
    }
  }
  return 0;
}

/* C[i][j] = min(C[i][j], min_t A[i][t] + B[t][j]) for an m x kk matrix A, a
 * kk x nn matrix B and an m x nn matrix C, all row-major and dense. */
int oracle_minplus_i64(const int64_t *A, const int64_t *B, int64_t *C, int64_t m, int64_t kk, int64_t nn,
                       int64_t inf) {
  if (!A || !B || !C || m < 0 || kk < 0 || nn < 0) return -1;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < nn; ++j) {
      int64_t best = C[i * nn + j];
      for (int64_t t = 0; t < kk; ++t) {
        int64_t a = A[i * kk + t], b = B[t * nn + j];
        if (a == inf || b == inf) continue;
        if (a + b < best) best = a + b;
      }
      C[i * nn + j] = best;
    }
  return 0;
}

int oracle_minplus_f64(const double *A, const double *B, double *C, int64_t m, int64_t kk, int64_t nn) {
  if (!A || !B || !C || m < 0 || kk < 0 || nn < 0) return -1;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < nn; ++j) {
      double best = C[i * nn + j];
      for (int64_t t = 0; t < kk; ++t) {
        double a = A[i * kk + t], b = B[t * nn + j];
        if (isinf(a) || isinf(b)) continue;
        if (a + b < best) best = a + b;
      }
      C[i * nn + j] = best;
    }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Dijkstra from many sources.  CSR graph: neighbours of v are
 * col[rowptr[v] .. rowptr[v+1]) with weights w[...] (both directions of an
 * undirected edge are present).  out is nsrc x n, row s = distances from
 * sources[s]; unreachable vertices get `inf` (double version: +infinity).
 * A binary min-heap with lazy deletion holds (distance, vertex) pairs.
 * ------------------------------------------------------------------------- */
typedef struct {
  double key;
  int64_t ikey;
  int64_t v;
} heap_item;

typedef struct {
  heap_item *a;
  int64_t size, cap;
  int use_double;
} heap_t;

static int item_less(const heap_t *h, const heap_item *x, const heap_item *y) {
  return h->use_double ? (x->key < y->key) : (x->ikey < y->ikey);
}

static int heap_push(heap_t *h, heap_item it) {
  if (h->size == h->cap) {
    int64_t nc = h->cap ? 2 * h->cap : 1024;
    heap_item *na = (heap_item *)realloc(h->a, (size_t)nc * sizeof(heap_item));
    if (!na) return -1;
    h->a = na;
    h->cap = nc;
  }
  int64_t i = h->size++;
  h->a[i] = it;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!item_less(h, &h->a[i], &h->a[p])) break;
    heap_item t = h->a[i];
    h->a[i] = h->a[p];
    h->a[p] = t;
    i = p;
  }
  return 0;
}

static heap_item heap_pop(heap_t *h) {
  heap_item top = h->a[0];
  h->a[0] = h->a[--h->size];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < h->size && item_less(h, &h->a[l], &h->a[m])) m = l;
    if (r < h->size && item_less(h, &h->a[r], &h->a[m])) m = r;
    if (m == i) break;
    heap_item t = h->a[i];
    h->a[i] = h->a[m];
    h->a[m] = t;
    i = m;
  }
  return top;
}

typedef struct {
  int64_t n;
  const int64_t *rowptr, *col;
  const int64_t *wi;
  const double *wd;
  const int64_t *sources;
  int64_t nsrc;
  int64_t *outi;
  double *outd;
  int64_t inf;
  int64_t first, step; /* this worker handles sources first, first+step, ... */
  int status;
} dj_job;

static void *dijkstra_worker(void *arg) {
  dj_job *J = (dj_job *)arg;
  int dbl = J->wd != NULL;
  heap_t h = {NULL, 0, 0, dbl};
  char *done = (char *)malloc((size_t)J->n);
  if (!done && J->n) {
    J->status = -1;
    return NULL;
  }
  for (int64_t s = J->first; s < J->nsrc; s += J->step) {
    int64_t src = J->sources[s];
    int64_t *di = dbl ? NULL : J->outi + s * J->n;
    double *dd = dbl ? J->outd + s * J->n : NULL;
    for (int64_t v = 0; v < J->n; ++v) {
      if (dbl) dd[v] = INFINITY;
      else di[v] = J->inf;
    }
    memset(done, 0, (size_t)J->n);
    h.size = 0;
    heap_item it = {0.0, 0, src};
    if (dbl) dd[src] = 0.0;
    else di[src] = 0;
    if (heap_push(&h, it)) { J->status = -1; break; }
    while (h.size > 0) {
      heap_item u = heap_pop(&h);
      if (done[u.v]) continue;
      done[u.v] = 1;
      for (int64_t e = J->rowptr[u.v]; e < J->rowptr[u.v + 1]; ++e) {
        int64_t v = J->col[e];
        if (done[v]) continue;
        if (dbl) {
          double nd = u.key + J->wd[e];
          if (nd < dd[v]) {
            dd[v] = nd;
            heap_item x = {nd, 0, v};
            if (heap_push(&h, x)) { J->status = -1; goto out; }
          }
        } else {
          int64_t nd = u.ikey + J->wi[e];
          if (nd < di[v]) {
            di[v] = nd;
            heap_item x = {0.0, nd, v};
            if (heap_push(&h, x)) { J->status = -1; goto out; }
          }
        }
      }
    }
  }
out:
  free(h.a);
  free(done);
  return NULL;
}

static int run_dijkstra(dj_job proto, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  dj_job jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = proto;
    jobs[t].first = t;
    jobs[t].step = nthreads;
    jobs[t].status = 0;
  }
  if (nthreads == 1) {
    dijkstra_worker(&jobs[0]);
    return jobs[0].status;
  }
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, dijkstra_worker, &jobs[t]) != 0) break;
    ++started;
  }
  /* any worker that could not start is run on this thread */
  for (int t = started; t < nthreads; ++t) dijkstra_worker(&jobs[t]);
  int st = 0;
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  for (int t = 0; t < nthreads; ++t) st |= jobs[t].status;
  return st;
}

int oracle_dijkstra_i64(int64_t n, const int64_t *rowptr, const int64_t *col, const int64_t *w,
                        const int64_t *sources, int64_t nsrc, int64_t *out, int64_t inf, int nthreads) {
  if (n < 0 || !rowptr || !sources || !out || nsrc < 0) return -1;
  for (int64_t s = 0; s < nsrc; ++s)
    if (sources[s] < 0 || sources[s] >= n) return -1;
  dj_job p = {n, rowptr, col, w, NULL, sources, nsrc, out, NULL, inf, 0, 1, 0};
  return run_dijkstra(p, nthreads);
}

int oracle_dijkstra_f64(int64_t n, const int64_t *rowptr, const int64_t *col, const double *w,
                        const int64_t *sources, int64_t nsrc, double *out, int nthreads) {
  if (n < 0 || !rowptr || !sources || !out || nsrc < 0 || !w) return -1;
  for (int64_t s = 0; s < nsrc; ++s)
    if (sources[s] < 0 || sources[s] >= n) return -1;
  dj_job p = {n, rowptr, col, NULL, w, sources, nsrc, NULL, out, 0, 0, 1, 0};
  return run_dijkstra(p, nthreads);
}
