/* A C caller of libbcgpu (no Python): BC of a weighted path graph, whose
 * exact value is BC(v_i) = i (n - 1 - i) for undirected BC (scale 0.5 over
 * all sources), through bc_compute, a step graph and edge BC.
 * Exit status 0 when every check passes. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "bcgpu.h"

#define N 9

static int check(int rc, const char *what) {
  if (rc != BC_OK) {
    fprintf(stderr, "%s failed: %d (%s)\n", what, rc, bc_last_error());
    exit(1);
  }
  return rc;
}

int main(void) {
  /* path v0 - v1 - ... - v8, weights 1 + i % 3, both directions stored */
  uint64_t row_ptr[N + 1];
  uint32_t col[2 * (N - 1)], w[2 * (N - 1)];
  uint64_t e = 0;
  for (uint32_t v = 0; v < N; ++v) {
    row_ptr[v] = e;
    if (v > 0) {
      col[e] = v - 1;
      w[e++] = 1 + (v - 1) % 3;
    }
    if (v + 1 < N) {
      col[e] = v + 1;
      w[e++] = 1 + v % 3;
    }
  }
  row_ptr[N] = e;
  bc_graph_t g;
  check(bc_graph_create(row_ptr, col, w, N, e, BC_UNDIRECTED_CHECK, &g), "bc_graph_create");
  uint32_t src[N];
  for (uint32_t v = 0; v < N; ++v) src[v] = v;
  double out[N];
  check(bc_compute(g, src, N, 0.5, out), "bc_compute");
  int bad = 0;
  for (uint32_t v = 0; v < N; ++v) {
    const double want = (double)v * (double)(N - 1 - v);
    if (fabs(out[v] - want) > 1e-12 * (want > 1 ? want : 1)) {
      fprintf(stderr, "bc[%u] = %.17g, want %.17g\n", v, out[v], want);
      bad = 1;
    }
  }
  /* edge BC: edge {v, v+1} separates v + 1 vertices from N - 1 - v */
  double ebc[2 * (N - 1)], vbc[N];
  check(bc_edge_compute(g, src, N, 0.5, ebc, vbc), "bc_edge_compute");
  for (uint32_t v = 0; v + 1 < N; ++v) {
    double sum = 0;
    for (uint64_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k)
      if (col[k] == v + 1) sum += ebc[k];
    for (uint64_t k = row_ptr[v + 1]; k < row_ptr[v + 2]; ++k)
      if (col[k] == v) sum += ebc[k];
    const double want = (double)(v + 1) * (double)(N - 1 - v);
    if (fabs(sum - want) > 1e-12 * want) {
      fprintf(stderr, "edge {%u,%u} = %.17g, want %.17g\n", v, v + 1, sum, want);
      bad = 1;
    }
  }
  bc_run_stats st;
  check(bc_last_run_stats(g, &st), "bc_last_run_stats");
  if (st.sources != N) {
    fprintf(stderr, "stats: %llu sources\n", (unsigned long long)st.sources);
    bad = 1;
  }
  /* errors come back as codes with a message */
  uint32_t oob = N;
  if (bc_compute(g, &oob, 1, 1.0, out) != BC_ERR_INVALID || bc_last_error()[0] == 0) {
    fprintf(stderr, "out-of-range source not rejected\n");
    bad = 1;
  }
  check(bc_graph_destroy(g), "bc_graph_destroy");
  if (!bad) printf("ok\n");
  return bad;
}
