/*
 * The C ABI (include/bem.h) used from plain C11: a circle of radius 0.35 on a
 * 256^2 grid, Dirichlet data u = x^2 - y^2 on every boundary cell, the flux q
 * from bem_solve (FP64 plan), then one host apply of the single layer and a
 * check that it reproduces the system's right-hand side c u - D u on the
 * solution (Eq. 15 with c = 1/2: S q = c u - D u).  Prints one line; exit
 * status 0 on success.
 *
 * Boundary cells follow the library's convention: every grid cell the curve
 * passes through (once, in the order the curve first enters it), weighted by
 * the curve's arc length inside the cell, with the outward normal in the mean
 * direction of that arc.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "bem.h"

#define N_GRID 256

static int fail(const char* what, bem_status rc) {
  fprintf(stderr, "%s: %s: %s\n", what, bem_status_string(rc), bem_last_error());
  return 1;
}

int main(void) {
  const double pi = 3.14159265358979323846;
  const double h = 1.0 / N_GRID, R = 0.35, cx = 0.5, cy = 0.5;
  const int64_t M = (int64_t)64 * N_GRID; /* curve samples */
  const double dtheta = 2.0 * pi / (double)M;
  int32_t* cell = malloc(sizeof(int32_t) * 2 * (size_t)M);
  double* w = calloc((size_t)M, sizeof(double));
  double* sc = calloc((size_t)M, sizeof(double));
  double* ss = calloc((size_t)M, sizeof(double));
  int64_t* slot = malloc(sizeof(int64_t) * N_GRID * N_GRID); /* cell -> entry, in first-visit order */
  if (!cell || !w || !sc || !ss || !slot) return 1;
  for (int64_t i = 0; i < (int64_t)N_GRID * N_GRID; ++i) slot[i] = -1;
  int64_t nb = 0;
  for (int64_t k = 0; k < M; ++k) {
    const double t = ((double)k + 0.5) * dtheta;
    const int32_t ix = (int32_t)floor((cx + R * cos(t)) / h), iy = (int32_t)floor((cy + R * sin(t)) / h);
    int64_t* e = &slot[(int64_t)ix * N_GRID + iy];
    if (*e < 0) {
      *e = nb;
      cell[2 * nb] = ix;
      cell[2 * nb + 1] = iy;
      ++nb;
    }
    w[*e] += R * dtheta; /* arc length inside the cell */
    sc[*e] += cos(t);    /* mean direction of the in-cell arc */
    ss[*e] += sin(t);
  }
  double* normal = malloc(sizeof(double) * 2 * (size_t)nb);
  double* data = malloc(sizeof(double) * (size_t)nb);
  uint8_t* bc = calloc((size_t)nb, 1);
  double* u = malloc(sizeof(double) * (size_t)nb);
  double* q = malloc(sizeof(double) * (size_t)nb);
  double* sq = malloc(sizeof(double) * (size_t)nb);
  double* du = malloc(sizeof(double) * (size_t)nb);
  if (!normal || !data || !bc || !u || !q || !sq || !du) return 1;
  for (int64_t j = 0; j < nb; ++j) {
    const double r = hypot(sc[j], ss[j]);
    const double nx = sc[j] / r, ny = ss[j] / r; /* outward normal of a circle = radial direction */
    const double x = cx + R * nx, y = cy + R * ny;
    normal[2 * j] = nx;
    normal[2 * j + 1] = ny;
    data[j] = x * x - y * y;
  }

  bem_plan_t plan = NULL;
  const int64_t n[2] = {N_GRID, N_GRID};
  bem_status rc = bem_plan(&plan, 2, n, h, nb, cell, w, normal, BEM_LAPLACE_2D, 0.0, 0.0, BEM_F64, 0, NULL);
  if (rc != BEM_OK) return fail("bem_plan", rc);
  bem_solve_info info;
  rc = bem_solve(plan, bc, data, 0.5, 1e-10, 2000, 200, NULL, u, q, &info, NULL);
  if (rc != BEM_OK) return fail("bem_solve", rc);
  /* S q = c u - D u on the solution */
  rc = bem_apply_host(plan, BEM_SINGLE, q, sq, NULL);
  if (rc != BEM_OK) return fail("bem_apply_host(single)", rc);
  rc = bem_apply_host(plan, BEM_DOUBLE, u, du, NULL);
  if (rc != BEM_OK) return fail("bem_apply_host(double)", rc);
  double num = 0.0, den = 0.0;
  for (int64_t j = 0; j < nb; ++j) {
    const double b = 0.5 * u[j] - du[j];
    num += (sq[j] - b) * (sq[j] - b);
    den += b * b;
  }
  const double rel = sqrt(num / den);
  printf("nb %lld iters %d rel_residual %.3e check %.3e\n", (long long)nb, info.iters, info.rel_residual, rel);
  bem_destroy(plan);
  free(cell); free(w); free(sc); free(ss); free(slot); free(normal); free(data); free(bc); free(u); free(q);
  free(sq); free(du);
  return rel <= 1e-9 ? 0 : 2;
}
