/*
 * The C ABI driven from plain C (no Python): set-up of a brick mesh and of a
 * general tetrahedral mesh of orders 2 and 3, the plane-wave RHS, the
 * problem counts and a structure export.  Host calls only (d3m_setup makes
 * no CUDA call), so it runs without a GPU.  Prints "key value" lines that the
 * test compares with the Python binding's view of the same problems.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "d3m.h"

static int report(const char *tag, d3m_ctx *ctx) {
  d3m_stats st;
  if (d3m_stats_get(ctx, &st) != D3M_OK) return 1;
  printf("%s_n_edges %lld\n", tag, (long long)st.n_edges);
  printf("%s_n_lm %lld\n", tag, (long long)st.n_lm);
  printf("%s_n_m %lld\n", tag, (long long)st.n_m);
  printf("%s_n_fronts %lld\n", tag, (long long)st.n_fronts);
  size_t bytes = 0;
  if (d3m_structure(ctx, D3M_M_MAP, NULL, &bytes) != D3M_OK) return 1;
  printf("%s_m_map_bytes %zu\n", tag, bytes);
  /* one plane wave along +z polarised along x */
  const double kp[9] = {0, 0, 1, 1, 0, 0, 0, 0, 0};
  double *rhs = calloc(2 * (size_t)st.n_edges, sizeof(double));
  if (!rhs || d3m_rhs_planewave(ctx, kp, 1, rhs, st.n_edges) != D3M_OK) return 1;
  double s = 0;
  for (int64_t i = 0; i < 2 * st.n_edges; ++i) s += fabs(rhs[i]);
  printf("%s_rhs_l1 %.12e\n", tag, s);
  free(rhs);
  return 0;
}

int main(void) {
  const double k = 2.0 * 3.14159265358979323846;
  /* 4 x 2 x 2 bricks in a 0.4 x 0.2 x 0.2 box, 2 x 1 x 1 subdomains */
  d3m_mesh mesh = {4, 2, 2, 0.4, 0.2, 0.2, D3M_BRICK, NULL, 0, 0, NULL, 0};
  double eps[2 * 16];
  for (int c = 0; c < 16; ++c) {
    eps[2 * c] = 1.0 + 0.1 * c;
    eps[2 * c + 1] = -0.05;
  }
  d3m_materials mat = {eps, NULL};
  const int32_t cx[3] = {0, 2, 4}, cy[2] = {0, 2}, cz[2] = {0, 2};
  d3m_partition part = {2, 1, 1, cx, cy, cz, NULL, NULL, NULL};
  d3m_options opt = {0};
  opt.precision = D3M_FP64;
  d3m_ctx *ctx = NULL;
  if (d3m_setup(&mesh, &mat, k, &part, &opt, &ctx) != D3M_OK) {
    printf("setup_error %s\n", ctx ? d3m_last_error(ctx) : "");
    return 1;
  }
  if (report("brick", ctx)) return 1;
  d3m_free(ctx);

  /* a unit-cell cube of side 0.2 as six tetrahedra, vertex ids i + 2 (j + 2 k) */
  double v[8 * 3];
  for (int n = 0; n < 8; ++n) {
    v[3 * n] = 0.2 * (n & 1);
    v[3 * n + 1] = 0.2 * ((n >> 1) & 1);
    v[3 * n + 2] = 0.2 * ((n >> 2) & 1);
  }
  const int64_t tets[6 * 4] = {0, 1, 3, 7, 0, 1, 5, 7, 0, 2, 3, 7, 0, 2, 6, 7, 0, 4, 5, 7, 0, 4, 6, 7};
  d3m_mesh tm = {0, 0, 0, 0.0, 0.0, 0.0, D3M_TET_MESH, v, 8, 6, tets, 2};
  double teps[2 * 6];
  for (int t = 0; t < 6; ++t) {
    teps[2 * t] = 2.0;
    teps[2 * t + 1] = 0.0;
  }
  d3m_materials tmat = {teps, NULL};
  const double gx[3] = {0.0, 0.1, 0.2}, gy[2] = {0.0, 0.2}, gz[2] = {0.0, 0.2};
  d3m_partition tpart = {2, 1, 1, NULL, NULL, NULL, gx, gy, gz};
  if (d3m_setup(&tm, &tmat, k, &tpart, &opt, &ctx) != D3M_OK) {
    printf("setup_error %s\n", ctx ? d3m_last_error(ctx) : "");
    return 1;
  }
  if (report("mesh", ctx)) return 1;
  d3m_free(ctx);
  tm.order = 3; /* curl-complete second order: two more dofs per face */
  if (d3m_setup(&tm, &tmat, k, &tpart, &opt, &ctx) != D3M_OK) {
    printf("setup_error %s\n", ctx ? d3m_last_error(ctx) : "");
    return 1;
  }
  if (report("mesh3", ctx)) return 1;
  d3m_free(ctx);
  printf("ok 1\n");
  return 0;
}
