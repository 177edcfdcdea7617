/*
 * Betweenness-centrality oracle: plain, slow, single-purpose CPU code.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * What it computes (arxiv 1701.05975, Sec. 2.1, Eq. 1 and the Brandes
 * recursion stated after it):
 *
 *   BC(v) = scale * sum_{s in Q} delta_s(v),
 *   delta_s(v) = sum_{t != s, v} sigma_st(v) / sigma_st
 *             = sum_{u : v in P_s(u)} sigma_sv / sigma_su * (1 + delta_s(u)),
 *
 * over an undirected weighted graph stored as CSR plus a weight array (Sec.
 * 3.1).  With Q = V and scale = 1 this is Eq. 1 over ordered pairs; scale =
 * 1/2 gives the usual undirected value.
 *
 * Algorithm: the sequential method the paper uses as its CPU baseline (Sec.
 * 4.1: Brandes with a binary-heap Dijkstra).  Per source: Dijkstra with lazy
 * deletion, counting shortest paths (sigma) at relaxation time and recording
 * the settle order S; then S is walked in reverse, each vertex pushing its
 * dependency share to its predecessors P_s(w) = {p : d(p) + w(p, w) = d(w)}.
 *
 * Conventions (readings of points the paper leaves open):
 *   - weights must be >= 1 (a weight of 0 is rejected with ORACLE_EINVAL);
 *   - every CSR entry is a distinct edge (multigraph semantics: parallel
 *     equal-weight edges each count as a shortest path);
 *   - unreachable pairs contribute nothing (sigma_st = 0 pairs are skipped);
 *   - distances are uint64, sigma / delta / BC are IEEE double.
 *
 * The second entry point, oracle_phased(), replays the paper's own parallel
 * algorithm (Algorithms 1, 2 and 3, node-parallel form) sequentially, in the
 * paper's notation, with a switch between the settle conditions of Eq. 3
 * (D(v) <= Delta_i) and Eq. 4 (D(v) < Delta_i) and a switch for the order in
 * which the frontier's "parallel" iterations are replayed.  It exists to pin
 * the Sec. 3.2 argument that Eq. 3 breaks sigma while Eq. 4 does not.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOMEM 2

#define INF_DIST UINT64_MAX

/* ------------------------------------------------------------------------ */
/* input validation                                                          */

static int check_csr(uint32_t n, const uint64_t *row_ptr, const uint32_t *col,
                     const uint32_t *w) {
  if (n == 0 || row_ptr == NULL) return ORACLE_EINVAL;
  if (row_ptr[0] != 0) return ORACLE_EINVAL;
  for (uint32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return ORACLE_EINVAL;
  uint64_t nnz = row_ptr[n];
  if (nnz > 0 && (col == NULL || w == NULL)) return ORACLE_EINVAL;
  for (uint64_t e = 0; e < nnz; ++e) {
    if (col[e] >= n) return ORACLE_EINVAL;
    if (w[e] == 0) return ORACLE_EINVAL;
  }
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* binary min-heap of (distance, vertex) with lazy deletion                  */

typedef struct {
  uint64_t key;
  uint32_t v;
} heap_item;

typedef struct {
  heap_item *a;
  uint64_t len, cap;
} heap;

static int heap_push(heap *h, uint64_t key, uint32_t v) {
  if (h->len == h->cap) {
    uint64_t nc = h->cap ? 2 * h->cap : 1024;
    heap_item *na = (heap_item *)realloc(h->a, nc * sizeof(heap_item));
    if (!na) return ORACLE_ENOMEM;
    h->a = na;
    h->cap = nc;
  }
  uint64_t i = h->len++;
  while (i > 0) {
    uint64_t parent = (i - 1) / 2;
    if (h->a[parent].key <= key) break;
    h->a[i] = h->a[parent];
    i = parent;
  }
  h->a[i].key = key;
  h->a[i].v = v;
  return ORACLE_OK;
}

static heap_item heap_pop(heap *h) {
  heap_item top = h->a[0];
  heap_item last = h->a[--h->len];
  uint64_t i = 0;
  for (;;) {
    uint64_t l = 2 * i + 1, r = l + 1, m = i;
    uint64_t mk = last.key;
    if (l < h->len && h->a[l].key < mk) { m = l; mk = h->a[l].key; }
    if (r < h->len && h->a[r].key < mk) { m = r; }
    if (m == i) break;
    h->a[i] = h->a[m];
    i = m;
  }
  if (h->len > 0) h->a[i] = last;
  return top;
}

/* ------------------------------------------------------------------------ */
/* per-source workspace                                                      */

typedef struct {
  uint64_t *d;
  double *sigma;
  double *delta;
  uint32_t *S;
  unsigned char *done;
  heap h;
} work;

static int work_init(work *wk, uint32_t n) {
  memset(wk, 0, sizeof(*wk));
  wk->d = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  wk->sigma = (double *)malloc((size_t)n * sizeof(double));
  wk->delta = (double *)malloc((size_t)n * sizeof(double));
  wk->S = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  wk->done = (unsigned char *)malloc(n);
  if (!wk->d || !wk->sigma || !wk->delta || !wk->S || !wk->done) return ORACLE_ENOMEM;
  return ORACLE_OK;
}

static void work_free(work *wk) {
  free(wk->d);
  free(wk->sigma);
  free(wk->delta);
  free(wk->S);
  free(wk->done);
  free(wk->h.a);
}

/*
 * Single-source shortest paths with path counting (Dijkstra, Sec. 2.2; the
 * sigma bookkeeping is Brandes' first phase, Sec. 2.1).  Fills d, sigma and
 * the settle order S; returns the number of settled (reachable) vertices.
 */
static int64_t sssp_count(uint32_t n, const uint64_t *row_ptr, const uint32_t *col,
                          const uint32_t *w, uint32_t s, work *wk) {
  for (uint32_t v = 0; v < n; ++v) {
    wk->d[v] = INF_DIST;
    wk->sigma[v] = 0.0;
    wk->done[v] = 0;
  }
  wk->h.len = 0;
  wk->d[s] = 0;
  wk->sigma[s] = 1.0;
  if (heap_push(&wk->h, 0, s)) return -1;
  uint32_t settled = 0;
  while (wk->h.len > 0) {
    heap_item it = heap_pop(&wk->h);
    uint32_t u = it.v;
    if (wk->done[u] || it.key > wk->d[u]) continue; /* stale entry */
    wk->done[u] = 1;
    wk->S[settled++] = u;
    for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      uint32_t x = col[e];
      uint64_t alt = wk->d[u] + (uint64_t)w[e];
      if (alt < wk->d[x]) {
        /* strictly shorter path: x's count restarts from u's */
        wk->d[x] = alt;
        wk->sigma[x] = wk->sigma[u];
        if (heap_push(&wk->h, alt, x)) return -1;
      } else if (alt == wk->d[x]) {
        /* another shortest path through u */
        wk->sigma[x] += wk->sigma[u];
      }
    }
  }
  return (int64_t)settled;
}

/*
 * Brandes' dependency accumulation (Sec. 2.1 recursion, Algorithm 3's
 * formula): walk S backwards; every predecessor p of w gets
 * sigma_p / sigma_w * (1 + delta_w).  Adds delta_s(w) into acc for w != s.
 */
static void accumulate(const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                       uint32_t s, uint32_t settled, work *wk, double *acc) {
  for (uint32_t i = 0; i < settled; ++i) wk->delta[wk->S[i]] = 0.0;
  for (uint32_t i = settled; i-- > 0;) {
    uint32_t x = wk->S[i];
    for (uint64_t e = row_ptr[x]; e < row_ptr[x + 1]; ++e) {
      uint32_t p = col[e];
      if (wk->d[p] != INF_DIST && wk->d[p] + (uint64_t)w[e] == wk->d[x])
        wk->delta[p] += wk->sigma[p] / wk->sigma[x] * (1.0 + wk->delta[x]);
    }
    if (x != s) acc[x] += wk->delta[x];
  }
}

/*
 * oracle_sssp: exact distances (UINT64_MAX = unreachable) and shortest-path
 * counts from one source.  Optional outputs may be NULL.
 */
int oracle_sssp(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                uint32_t s, uint64_t *out_dist, double *out_sigma, uint32_t *out_order,
                uint32_t *out_reached) {
  int rc = check_csr(n, row_ptr, col, w);
  if (rc) return rc;
  if (s >= n) return ORACLE_EINVAL;
  work wk;
  if (work_init(&wk, n)) { work_free(&wk); return ORACLE_ENOMEM; }
  int64_t settled = sssp_count(n, row_ptr, col, w, s, &wk);
  if (settled < 0) { work_free(&wk); return ORACLE_ENOMEM; }
  if (out_dist) memcpy(out_dist, wk.d, (size_t)n * sizeof(uint64_t));
  if (out_sigma) memcpy(out_sigma, wk.sigma, (size_t)n * sizeof(double));
  if (out_order) memcpy(out_order, wk.S, (size_t)settled * sizeof(uint32_t));
  if (out_reached) *out_reached = (uint32_t)settled;
  work_free(&wk);
  return ORACLE_OK;
}

/* per-source dependencies delta_s(v) for one source (tests only) */
int oracle_delta(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                 uint32_t s, double *out_delta) {
  int rc = check_csr(n, row_ptr, col, w);
  if (rc) return rc;
  if (s >= n) return ORACLE_EINVAL;
  work wk;
  if (work_init(&wk, n)) { work_free(&wk); return ORACLE_ENOMEM; }
  int64_t settled = sssp_count(n, row_ptr, col, w, s, &wk);
  if (settled < 0) { work_free(&wk); return ORACLE_ENOMEM; }
  for (uint32_t v = 0; v < n; ++v) out_delta[v] = 0.0;
  accumulate(row_ptr, col, w, s, (uint32_t)settled, &wk, out_delta);
  work_free(&wk);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Brandes over a source list, optionally split over threads                 */

typedef struct {
  uint32_t n;
  const uint64_t *row_ptr;
  const uint32_t *col, *w, *sources;
  uint32_t k, tid, nthreads;
  double *acc; /* private partial sums, n doubles */
  int rc;
} job;

static void *run_job(void *arg) {
  job *j = (job *)arg;
  work wk;
  if (work_init(&wk, j->n)) { work_free(&wk); j->rc = ORACLE_ENOMEM; return NULL; }
  for (uint32_t i = j->tid; i < j->k; i += j->nthreads) {
    int64_t settled = sssp_count(j->n, j->row_ptr, j->col, j->w, j->sources[i], &wk);
    if (settled < 0) { j->rc = ORACLE_ENOMEM; break; }
    accumulate(j->row_ptr, j->col, j->w, j->sources[i], (uint32_t)settled, &wk, j->acc);
  }
  work_free(&wk);
  return NULL;
}

/*
 * oracle_bc: out_bc[v] = scale * sum_{s in sources} delta_s(v).  Duplicate
 * sources count twice.  nthreads <= 1 runs single-threaded; otherwise the
 * source list is dealt round-robin to nthreads POSIX threads, each with its
 * own partial sum, and the partials are added in thread order.
 */
int oracle_bc(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
              const uint32_t *sources, uint32_t k, double scale, double *out_bc,
              int nthreads) {
  int rc = check_csr(n, row_ptr, col, w);
  if (rc) return rc;
  for (uint32_t i = 0; i < k; ++i)
    if (sources[i] >= n) return ORACLE_EINVAL;
  if (nthreads < 1) nthreads = 1;
  if ((uint32_t)nthreads > k && k > 0) nthreads = (int)k;
  job *jobs = (job *)calloc((size_t)nthreads, sizeof(job));
  double *parts = (double *)calloc((size_t)nthreads * n, sizeof(double));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !parts || !th) { free(jobs); free(parts); free(th); return ORACLE_ENOMEM; }
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = (job){n, row_ptr, col, w, sources, k, (uint32_t)t, (uint32_t)nthreads,
                    parts + (size_t)t * n, ORACLE_OK};
  }
  if (nthreads == 1) {
    run_job(&jobs[0]);
  } else {
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, run_job, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  }
  rc = ORACLE_OK;
  for (int t = 0; t < nthreads; ++t)
    if (jobs[t].rc) rc = jobs[t].rc;
  for (uint32_t v = 0; v < n; ++v) {
    double sum = 0.0;
    for (int t = 0; t < nthreads; ++t) sum += parts[(size_t)t * n + v];
    out_bc[v] = scale * sum;
  }
  free(jobs);
  free(parts);
  free(th);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Directed graphs (Sec. 2.1: the method extends to them).  Dependencies are */
/* pulled from successors over out-edges, Algorithm 3's formula: walking the */
/* settle order backwards, delta(a) = sum over entries (a -> b, w) with       */
/* d(a) + w = d(b) of sigma_a / sigma_b * (1 + delta_b).  It needs no        */
/* in-edges, so it is correct for any CSR, symmetric or not.                 */

int oracle_bc_pull(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                   const uint32_t *sources, uint32_t k, double scale, double *out_bc) {
  int rc = check_csr(n, row_ptr, col, w);
  if (rc) return rc;
  for (uint32_t i = 0; i < k; ++i)
    if (sources[i] >= n) return ORACLE_EINVAL;
  for (uint32_t v = 0; v < n; ++v) out_bc[v] = 0.0;
  work wk;
  if (work_init(&wk, n)) { work_free(&wk); return ORACLE_ENOMEM; }
  for (uint32_t i = 0; i < k; ++i) {
    uint32_t s = sources[i];
    int64_t settled = sssp_count(n, row_ptr, col, w, s, &wk);
    if (settled < 0) { work_free(&wk); return ORACLE_ENOMEM; }
    for (int64_t j = settled; j-- > 0;) {
      uint32_t a = wk.S[j];
      double dep = 0.0;
      for (uint64_t e = row_ptr[a]; e < row_ptr[a + 1]; ++e) {
        uint32_t b = col[e];
        if (wk.d[b] != INF_DIST && wk.d[a] + (uint64_t)w[e] == wk.d[b])
          dep += wk.sigma[a] / wk.sigma[b] * (1.0 + wk.delta[b]);
      }
      wk.delta[a] = dep;
      if (a != s) out_bc[a] += dep;
    }
  }
  work_free(&wk);
  for (uint32_t v = 0; v < n; ++v) out_bc[v] *= scale;
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Edge betweenness (the paper's tool reports node and edge BC, Sec. 1).    */
/* Per CSR entry e = (a -> b, w): the pair-dependency share that crosses it  */
/* in the direction a -> b, i.e. when a is a shortest-path predecessor of b  */
/* (d(a) + w = d(b)): sigma_a / sigma_b * (1 + delta_b), summed over the      */
/* sources and times scale.  The undirected edge {a, b} carries the sum of   */
/* its two entries.  Dependencies are pulled from successors as in           */
/* Algorithm 3, walking the settle order backwards.                          */

int oracle_edge_bc(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                   const uint32_t *sources, uint32_t k, double scale, double *out_ebc) {
  int rc = check_csr(n, row_ptr, col, w);
  if (rc) return rc;
  for (uint32_t i = 0; i < k; ++i)
    if (sources[i] >= n) return ORACLE_EINVAL;
  uint64_t nnz = row_ptr[n];
  for (uint64_t e = 0; e < nnz; ++e) out_ebc[e] = 0.0;
  work wk;
  if (work_init(&wk, n)) { work_free(&wk); return ORACLE_ENOMEM; }
  for (uint32_t i = 0; i < k; ++i) {
    uint32_t s = sources[i];
    int64_t settled = sssp_count(n, row_ptr, col, w, s, &wk);
    if (settled < 0) { work_free(&wk); return ORACLE_ENOMEM; }
    for (int64_t j = settled; j-- > 0;) {
      uint32_t a = wk.S[j];
      double dep = 0.0;
      for (uint64_t e = row_ptr[a]; e < row_ptr[a + 1]; ++e) {
        uint32_t b = col[e];
        if (wk.d[b] != INF_DIST && wk.d[a] + (uint64_t)w[e] == wk.d[b]) {
          double share = wk.sigma[a] / wk.sigma[b] * (1.0 + wk.delta[b]);
          dep += share;
          out_ebc[e] += share;
        }
      }
      wk.delta[a] = dep;
    }
  }
  work_free(&wk);
  for (uint64_t e = 0; e < nnz; ++e) out_ebc[e] *= scale;
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* The paper's node-parallel algorithm, replayed sequentially.               */

/*
 * oracle_phased: Algorithm 1 (initialisation), Algorithm 2 (parallel
 * Dijkstra with sigma counting and the Delta_i settle test of Eq. 2 with
 * Eq. 4, or Eq. 3 when nonstrict != 0) and Algorithm 3 (dependency
 * accumulation over the recorded levels), for one source s.
 *
 * Every "for ... do in parallel" over vertices is replayed one vertex at a
 * time, in increasing vertex id, or decreasing when reverse != 0: the order
 * decides the outcome of the races Sec. 3.2 discusses.  Delta_node(v) is the
 * minimum weight incident to v (Sec. 3.2, before Eq. 2).
 *
 * Outputs (each may be NULL): d, sigma, the level (settle batch) of each
 * vertex (UINT32_MAX if never settled), delta (Algorithm 3's delta[w]), and
 * the number of levels.
 */
int oracle_phased(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                  uint32_t s, int nonstrict, int reverse, uint64_t *out_dist, double *out_sigma,
                  uint32_t *out_level, double *out_delta, uint32_t *out_nlevels) {
  int rc = check_csr(n, row_ptr, col, w);
  if (rc) return rc;
  if (s >= n) return ORACLE_EINVAL;
  unsigned char *U = (unsigned char *)malloc(n);
  unsigned char *F = (unsigned char *)malloc(n);
  unsigned char *Fnext = (unsigned char *)malloc(n);
  uint64_t *d = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  double *sigma = (double *)malloc((size_t)n * sizeof(double));
  double *delta = (double *)malloc((size_t)n * sizeof(double));
  uint64_t *dnode = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  uint32_t *S = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
  uint32_t *ends = (uint32_t *)malloc(((size_t)n + 2) * sizeof(uint32_t));
  if (!U || !F || !Fnext || !d || !sigma || !delta || !dnode || !S || !ends) {
    free(U); free(F); free(Fnext); free(d); free(sigma); free(delta); free(dnode); free(S); free(ends);
    return ORACLE_ENOMEM;
  }
  /* Delta_node v = min incident weight (infinite for an isolated vertex) */
  for (uint32_t v = 0; v < n; ++v) {
    uint64_t m = INF_DIST;
    for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
      if ((uint64_t)w[e] < m) m = w[e];
    dnode[v] = m;
  }
  /* Algorithm 1 */
  for (uint32_t v = 0; v < n; ++v) {
    U[v] = 1;
    F[v] = 0;
    d[v] = INF_DIST;
    sigma[v] = 0.0;
    delta[v] = 0.0;
  }
  d[s] = 0;
  sigma[s] = 1.0;
  U[s] = 0;
  F[s] = 1;
  S[0] = s;
  uint32_t S_len = 1;
  ends[0] = 0;
  ends[1] = 1;
  uint32_t ends_len = 2;
  uint64_t Delta = 0;

  /* Algorithm 2 */
  while (Delta != INF_DIST) {
    /* inspect the frontier: relax distances, count paths */
    for (uint32_t i = 0; i < n; ++i) {
      uint32_t v = reverse ? n - 1 - i : i;
      if (!F[v]) continue;
      for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        uint32_t x = col[e];
        uint64_t alt = d[v] + (uint64_t)w[e];
        if (U[x] && alt < d[x]) {
          d[x] = alt;
          sigma[x] = 0.0;
        }
        if (d[x] == alt) sigma[x] += sigma[v];
      }
    }
    /* Eq. 2: Delta_i = min over unsettled reached u of D(u) + Delta_node(u) */
    Delta = INF_DIST;
    for (uint32_t v = 0; v < n; ++v)
      if (U[v] && d[v] != INF_DIST && d[v] + dnode[v] < Delta) Delta = d[v] + dnode[v];
    /* settle with Eq. 4 (strict) or Eq. 3 (non-strict) */
    uint32_t cnt = 0;
    for (uint32_t i = 0; i < n; ++i) {
      uint32_t v = reverse ? n - 1 - i : i;
      Fnext[v] = 0;
      int take = nonstrict ? (U[v] && d[v] != INF_DIST && d[v] <= Delta)
                           : (U[v] && d[v] < Delta);
      if (take) {
        U[v] = 0;
        Fnext[v] = 1;
        S[S_len++] = v;
        ++cnt;
      }
    }
    memcpy(F, Fnext, n);
    if (cnt > 0) {
      ends[ends_len] = ends[ends_len - 1] + cnt;
      ++ends_len;
    }
  }

  /* Algorithm 3: levels in reverse, pull from successors */
  for (uint32_t depth = ends_len - 1; depth > 0; --depth) {
    uint32_t start = ends[depth - 1], end = ends[depth];
    for (uint32_t i = start; i < end; ++i) {
      uint32_t x = S[i];
      double dsw = 0.0;
      for (uint64_t e = row_ptr[x]; e < row_ptr[x + 1]; ++e) {
        uint32_t v = col[e];
        if (d[v] != INF_DIST && d[v] == d[x] + (uint64_t)w[e])
          dsw += sigma[x] / sigma[v] * (1.0 + delta[v]);
      }
      delta[x] = dsw;
    }
  }

  if (out_dist) memcpy(out_dist, d, (size_t)n * sizeof(uint64_t));
  if (out_sigma) memcpy(out_sigma, sigma, (size_t)n * sizeof(double));
  if (out_delta) memcpy(out_delta, delta, (size_t)n * sizeof(double));
  if (out_level) {
    for (uint32_t v = 0; v < n; ++v) out_level[v] = UINT32_MAX;
    for (uint32_t l = 0; l + 1 < ends_len; ++l)
      for (uint32_t i = ends[l]; i < ends[l + 1]; ++i) out_level[S[i]] = l;
  }
  if (out_nlevels) *out_nlevels = ends_len - 1;
  free(U); free(F); free(Fnext); free(d); free(sigma); free(delta); free(dnode); free(S); free(ends);
  return ORACLE_OK;
}
