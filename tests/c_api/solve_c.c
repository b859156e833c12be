/* A plain C client of the library: only include/mg.h and libmg.so, no
 * Python and no torch (the CUDA runtime only for a page-locked buffer).
 * Solves a definite 2D problem (k^2 = -30, Gaussian source, a layer of width
 * 1/3) to a relative residual of 1e-10 with BPX (undamped factors 0.6;
 * the oracle needs 80 cycles on this problem), runs one BPX cycle of a 3D problem from a
 * page-locked host buffer, refines an adaptive 2D grid dynamically (cycles and
 * refinement steps from the regular level-2 grid), and checks the argument
 * validation of mg_create and mg_adapt.
 * Exit status 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "mg.h"

static int check(int rc, const char* what, const mg_ctx* ctx) {
  if (rc != MG_OK) fprintf(stderr, "%s: status %d (%s)\n", what, rc, mg_last_error(ctx));
  return rc;
}

int main(void) {
  /* argument validation happens before any device work */
  mg_ctx* bad = NULL;
  if (mg_create(5, 3, NULL, 0.0, 0.0, &bad) != MG_ERR_INVALID || bad != NULL) return 2;

  const int depth = 4, n = 81, N = n + 1;
  const size_t nv = (size_t)N * N;
  double* k2 = (double*)malloc(nv * sizeof(double));
  mg_c128* f = (mg_c128*)malloc(nv * sizeof(mg_c128));
  for (int y = 0; y < N; ++y)
    for (int x = 0; x < N; ++x) {
      const double dx = (double)x / n - 0.5, dy = (double)y / n - 0.5;
      k2[(size_t)y * N + x] = -30.0;
      f[(size_t)y * N + x].re = exp(-(dx * dx + dy * dy) / (2 * 0.05 * 0.05));
      f[(size_t)y * N + x].im = 0.0;
    }
  mg_ctx* ctx = NULL;
  /* a layer on coarse grid lines (w = 1/3), so the FAS fixed point is the
   * discrete solution */
  if (check(mg_create(2, depth, k2, 0.5235987755982988, 1.0 / 3.0, &ctx), "mg_create", NULL)) return 1;
  if (check(mg_set_rhs(ctx, f, 0), "mg_set_rhs", ctx)) return 1;
  mg_c128 omega[4];
  const mg_c128 ws = {0.6, 0.0};
  if (check(mg_omega_scheme(MG_OMEGA_UCG, ws, depth, 1, 0, omega), "mg_omega_scheme", ctx)) return 1;
  int cycles = 0;
  double rel = 1.0;
  int rc = mg_solve(ctx, MG_BPX, omega, MG_HIERARCHICAL, 1e-10, 2000, &cycles, &rel);
  printf("2D depth %d: status %d after %d cycles, relative residual %.3e\n", depth, rc, cycles, rel);
  double a = 0.0, r = 0.0;
  if (check(mg_residual_norm(ctx, &a, &r), "mg_residual_norm", ctx)) return 1;
  mg_destroy(ctx);
  free(k2);
  free(f);
  if (rc != MG_OK || rel > 1e-10 || r > 1.0001e-10) return 1;

  /* 3D: one BPX cycle from a page-locked host buffer */
  const int d3 = 2, n3 = 9, N3 = n3 + 1;
  const size_t nv3 = (size_t)N3 * N3 * N3;
  double* k3 = (double*)malloc(nv3 * sizeof(double));
  for (size_t i = 0; i < nv3; ++i) k3[i] = 20.0;
  mg_ctx* c3 = NULL;
  if (check(mg_create(3, d3, k3, 0.5235987755982988, 0.2, &c3), "mg_create 3D", NULL)) return 1;
  mg_c128* u = NULL;
  if (cudaMallocHost((void**)&u, nv3 * sizeof(mg_c128)) != cudaSuccess) return 1;
  for (size_t i = 0; i < nv3; ++i) { u[i].re = 1.0; u[i].im = 0.5; }
  if (check(mg_set_rhs(c3, u, 0), "mg_set_rhs 3D", c3)) return 1;
  const mg_c128 om3[2] = {{0.6, 0.0}, {0.6, 0.0}};
  if (check(mg_cycle(c3, MG_BPX, om3, MG_HIERARCHICAL), "mg_cycle 3D", c3)) return 1;
  if (check(mg_get_solution(c3, u, 0), "mg_get_solution 3D", c3)) return 1;
  int finite = 1;
  for (size_t i = 0; i < nv3; ++i) finite = finite && isfinite(u[i].re) && isfinite(u[i].im);
  printf("3D depth %d: one BPX cycle, u[center] = (%.6e, %.6e)\n", d3, u[nv3 / 2].re, u[nv3 / 2].im);
  mg_destroy(c3);
  cudaFreeHost(u);
  free(k3);
  if (!finite) return 1;

  /* adaptive 2D grid, depth 4: level 1 refined, the rest grows by feature-based refinement */
  const int da = 4, na = 81, Na = na + 1;
  const size_t nva = (size_t)Na * Na;
  double* ka = (double*)malloc(nva * sizeof(double));
  mg_c128* fa = (mg_c128*)malloc(nva * sizeof(mg_c128));
  for (int j = 0; j < Na; ++j)
    for (int i = 0; i < Na; ++i) {
      const double x = (double)i / na - 0.3, y = (double)j / na - 0.6;
      ka[(size_t)j * Na + i] = 25.0;
      fa[(size_t)j * Na + i].re = exp(-(x * x + y * y) / (2.0 * 0.05 * 0.05));
      fa[(size_t)j * Na + i].im = 0.0;
    }
  const size_t nflags = 9 + 81 + 729; /* levels 1..3 */
  unsigned char* refine = (unsigned char*)calloc(nflags, 1);
  for (int k = 0; k < 9; ++k) refine[k] = 1;
  mg_ctx* ca = NULL;
  if (check(mg_create_adaptive(2, da, ka, 0.5235987755982988, 0.0, 0.2, 0.2, refine, &ca), "mg_create_adaptive",
            NULL))
    return 1;
  if (check(mg_set_rhs(ca, fa, 0), "mg_set_rhs adaptive", ca)) return 1;
  const mg_c128 oma[4] = {{0.6, 0.0}, {0.6, 0.0}, {0.6, 0.0}, {0.6, 0.0}};
  long long st[4] = {0, 0, 0, 0};
  for (int it = 0; it < 5; ++it) {
    if (check(mg_cycle(ca, MG_BPX, oma, MG_HIERARCHICAL), "mg_cycle adaptive", ca)) return 1;
    if (check(mg_adapt(ca, 0.1, 0.02, 20, 1e-2, it % 2, 2, st), "mg_adapt", ca)) return 1;
  }
  if (check(mg_get_refinement(ca, refine), "mg_get_refinement", ca)) return 1;
  int refined2 = 0;
  for (int k = 9; k < 90; ++k) refined2 += refine[k];
  double rmax = 0.0;
  if (check(mg_residual_max(ca, &rmax), "mg_residual_max adaptive", ca)) return 1;
  printf("adaptive depth %d: 5 steps, %lld fine-grid vertices, finest level %lld, %d refined level-2 cells, "
         "max |r| %.3e\n", da, st[2], st[3], refined2, rmax);
  if (mg_adapt(ca, 0.1, 0.02, 0, 1e-2, 0, 2, st) != MG_ERR_INVALID) return 1; /* bins out of range */
  mg_destroy(ca);
  free(refine);
  free(fa);
  free(ka);
  return (refined2 > 0 && st[2] > 49 && isfinite(rmax)) ? 0 : 1;
}
