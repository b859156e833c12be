/* A plain C client of the library: only include/mg.h and libmg.so, no
 * Python and no torch (the CUDA runtime only for a page-locked buffer).
 * Solves a definite 2D problem (k^2 = -30, Gaussian source, a layer of width
 * 1/3) to a relative residual of 1e-10 with BPX (undamped factors 0.6;
 * the oracle needs 80 cycles on this problem), runs one BPX cycle of a 3D problem from a
 * page-locked host buffer, refines an adaptive 2D grid dynamically (cycles and
 * refinement steps from the regular level-2 grid), repeats the 2D solve with
 * complex64 cycles inside FP64 defect correction and compares the two
 * solutions, solves three problems as one batch, runs the adjoint calls
 * (device k^2, sampling, adjoint right-hand side, gradients) on a small
 * varying-shift problem, runs coupled two-channel cycles, and checks the
 * argument validation of mg_create, mg_adapt and mg_mc_create.
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
  if (rc != MG_OK || rel > 1e-10 || r > 1.0001e-10) return 1;
  /* the same problem with complex64 cycles inside FP64 defect correction */
  mg_c128* u128 = (mg_c128*)malloc(nv * sizeof(mg_c128));
  mg_c128* u64 = (mg_c128*)malloc(nv * sizeof(mg_c128));
  if (check(mg_get_solution(ctx, u128, 0), "mg_get_solution", ctx)) return 1;
  for (size_t i = 0; i < nv; ++i) { u64[i].re = 0.0; u64[i].im = 0.0; }
  if (check(mg_set_solution(ctx, u64, 0), "mg_set_solution", ctx)) return 1;
  if (check(mg_set_precision(ctx, MG_C64_REFINE, 16), "mg_set_precision", ctx)) return 1;
  int rc64 = mg_solve(ctx, MG_BPX, omega, MG_HIERARCHICAL, 1e-10, 4000, &cycles, &rel);
  if (check(mg_get_solution(ctx, u64, 0), "mg_get_solution c64", ctx)) return 1;
  double dn = 0.0, nn = 0.0;
  for (size_t i = 0; i < nv; ++i) {
    const double er = u64[i].re - u128[i].re, ei = u64[i].im - u128[i].im;
    dn += er * er + ei * ei;
    nn += u128[i].re * u128[i].re + u128[i].im * u128[i].im;
  }
  printf("2D depth %d, complex64 refinement: status %d after %d inner cycles, relative residual %.3e, "
         "|u64 - u128| / |u128| = %.3e\n", depth, rc64, cycles, rel, sqrt(dn / nn));
  mg_destroy(ctx);
  free(u128);
  free(u64);
  if (rc64 != MG_OK || sqrt(dn / nn) > 1e-7) return 1;

  /* three problems of different depths as one batch */
  {
    const int nb = 3;
    int bd[3] = {2, 2, 2}, bdepth[3] = {3, 4, 4};
    double bth[3] = {0.5235987755982988, 0.5235987755982988, 0.5235987755982988};
    double bw[3] = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};
    double* bk2[3];
    for (int p = 0; p < nb; ++p) {
      const int Np = (int)pow(3.0, bdepth[p]) + 1;
      bk2[p] = (double*)malloc((size_t)Np * Np * sizeof(double));
      for (int i = 0; i < Np * Np; ++i) bk2[p][i] = -20.0 - 10.0 * p;
    }
    mg_batch* bt = NULL;
    if (check(mg_batch_create(nb, bd, bdepth, (const double* const*)bk2, bth, bw, &bt), "mg_batch_create", NULL))
      return 1;
    mg_c128 bom[3][4];
    const mg_c128* bomp[3];
    for (int p = 0; p < nb; ++p) {
      mg_ctx* cp = NULL;
      if (check(mg_batch_get_ctx(bt, p, &cp), "mg_batch_get_ctx", NULL)) return 1;
      const int Np = (int)pow(3.0, bdepth[p]) + 1;
      mg_c128* fp = (mg_c128*)malloc((size_t)Np * Np * sizeof(mg_c128));
      for (int j = 0; j < Np; ++j)
        for (int i = 0; i < Np; ++i) {
          const double dx = (double)i / (Np - 1) - 0.4 - 0.1 * p, dy = (double)j / (Np - 1) - 0.5;
          fp[(size_t)j * Np + i].re = exp(-(dx * dx + dy * dy) / (2 * 0.05 * 0.05));
          fp[(size_t)j * Np + i].im = 0.0;
        }
      if (check(mg_set_rhs(cp, fp, 0), "mg_set_rhs batch", cp)) return 1;
      free(fp);
      if (check(mg_omega_scheme(MG_OMEGA_EXP, ws, bdepth[p], 1, 0, bom[p]), "mg_omega_scheme", NULL)) return 1;
      bomp[p] = bom[p];
    }
    int bst[3], bcyc[3];
    double brel[3];
    int brc = mg_batch_solve(bt, MG_ADD, bomp, MG_DLINEAR, 1e-8, 200, 16, bst, bcyc, brel);
    printf("batch of %d: status %d (%d %d %d), relative residuals %.2e %.2e %.2e\n", nb, brc, bst[0], bst[1],
           bst[2], brel[0], brel[1], brel[2]);
    mg_batch_destroy(bt);
    for (int p = 0; p < nb; ++p) free(bk2[p]);
    for (int p = 0; p < nb; ++p)
      if (bst[p] != MG_OK || brel[p] > 1e-8) return 1;
  }

  /* adjoint calls on a small varying-shift problem (device k^2) */
  {
    const int dd = 3, nd = 27, Nd = nd + 1;
    const size_t nvd = (size_t)Nd * Nd;
    double* kv = (double*)malloc(nvd * sizeof(double));
    mg_c128* fv = (mg_c128*)malloc(nvd * sizeof(mg_c128));
    for (int j = 0; j < Nd; ++j)
      for (int i = 0; i < Nd; ++i) {
        const double dx = (double)i / nd - 0.5, dy = (double)j / nd - 0.5;
        kv[(size_t)j * Nd + i] = -40.0 - 30.0 * exp(-(dx * dx + dy * dy) / 0.02);
        fv[(size_t)j * Nd + i].re = exp(-(dx * dx + dy * dy) / (2 * 0.05 * 0.05));
        fv[(size_t)j * Nd + i].im = 0.0;
      }
    mg_ctx* ca2 = NULL;
    if (check(mg_create(2, dd, kv, 0.5235987755982988, 1.0 / 3.0, &ca2), "mg_create adjoint", NULL)) return 1;
    double* kdev = NULL;
    mg_c128 *udev = NULL, *ldev = NULL;
    double *gV = NULL, *gf = NULL;
    if (cudaMalloc((void**)&kdev, nvd * sizeof(double)) != cudaSuccess) return 1;
    if (cudaMalloc((void**)&udev, nvd * sizeof(mg_c128)) != cudaSuccess) return 1;
    if (cudaMalloc((void**)&ldev, nvd * sizeof(mg_c128)) != cudaSuccess) return 1;
    if (cudaMalloc((void**)&gV, nvd * sizeof(double)) != cudaSuccess) return 1;
    if (cudaMalloc((void**)&gf, nvd * sizeof(double)) != cudaSuccess) return 1;
    for (size_t i = 0; i < nvd; ++i) kv[i] *= 1.1;
    if (cudaMemcpy(kdev, kv, nvd * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) return 1;
    if (check(mg_set_k2(ca2, kdev, 1), "mg_set_k2 device", ca2)) return 1;
    if (check(mg_set_rhs(ca2, fv, 0), "mg_set_rhs adjoint", ca2)) return 1;
    /* a varying shift moves the plain cycle's FAS fixed point (rediscretisation is
     * not the Galerkin product): solve with FP64 defect correction */
    if (check(mg_set_precision(ca2, MG_C64_REFINE, 16), "mg_set_precision adjoint", ca2)) return 1;
    mg_c128 oma2[3];
    if (check(mg_omega_scheme(MG_OMEGA_EXP, ws, dd, 1, 0, oma2), "mg_omega_scheme", NULL)) return 1;
    int c1 = 0;
    double r1 = 0.0;
    if (check(mg_solve(ca2, MG_ADD, oma2, MG_DLINEAR, 1e-10, 4000, &c1, &r1), "mg_solve forward", ca2)) return 1;
    if (check(mg_get_solution(ca2, udev, 1), "mg_get_solution forward", ca2)) return 1;
    double xyz[2 * 16];
    mg_c128 wq[16], s_val;
    for (int q = 0; q < 16; ++q) {
      const double ph = 2.0 * 3.141592653589793 * q / 16;
      xyz[2 * q] = 0.5 + 0.35 * cos(ph);
      xyz[2 * q + 1] = 0.5 + 0.35 * sin(ph);
      wq[q].re = cos(2 * ph);
      wq[q].im = sin(2 * ph);
    }
    if (check(mg_sample(ca2, 16, xyz, wq, &s_val), "mg_sample", ca2)) return 1;
    if (check(mg_set_rhs_samples(ca2, 16, xyz, wq), "mg_set_rhs_samples", ca2)) return 1;
    mg_c128* z = (mg_c128*)calloc(nvd, sizeof(mg_c128));
    if (check(mg_set_solution(ca2, z, 0), "mg_set_solution adjoint", ca2)) return 1;
    if (check(mg_solve(ca2, MG_ADD, oma2, MG_DLINEAR, 1e-10, 4000, &c1, &r1), "mg_solve adjoint", ca2)) return 1;
    if (check(mg_get_solution(ca2, ldev, 1), "mg_get_solution adjoint", ca2)) return 1;
    if (check(mg_adjoint_grad(ca2, udev, ldev, s_val, gV, gf), "mg_adjoint_grad", ca2)) return 1;
    double* hg = (double*)malloc(nvd * sizeof(double));
    if (cudaMemcpy(hg, gf, nvd * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    double gmax = 0.0;
    int gfin = 1;
    for (size_t i = 0; i < nvd; ++i) {
      gfin = gfin && isfinite(hg[i]);
      if (fabs(hg[i]) > gmax) gmax = fabs(hg[i]);
    }
    printf("adjoint depth %d: s = (%.6e, %.6e), max |dJ/df| = %.3e\n", dd, s_val.re, s_val.im, gmax);
    mg_destroy(ca2);
    cudaFree(kdev);
    cudaFree(udev);
    cudaFree(ldev);
    cudaFree(gV);
    cudaFree(gf);
    free(hg);
    free(z);
    free(kv);
    free(fv);
    if (!gfin || !(gmax > 0.0)) return 1;
  }

  /* coupled multichannel: two channels, the residual falls over cycles */
  {
    mg_mc_ctx* bad_mc = NULL;
    const mg_c128 phi_bad[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    if (mg_mc_create(2, 3, 5, phi_bad, 0.5, 0.1, &bad_mc) != MG_ERR_INVALID || bad_mc != NULL) return 2;
    const mg_c128 phi[4] = {{-40.0, 0.0}, {3.0, 0.0}, {3.0, 0.0}, {-60.0, 0.0}};
    mg_mc_ctx* mc = NULL;
    if (mg_mc_create(2, 4, 2, phi, 0.5235987755982988, 1.0 / 3.0, &mc) != MG_OK) return 1;
    const size_t nvm = (size_t)N * N * 2;
    mg_c128* fm = (mg_c128*)malloc(nvm * sizeof(mg_c128));
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < N; ++x)
        for (int ch = 0; ch < 2; ++ch) {
          const double dx = (double)x / n - 0.5 + 0.1 * ch, dy = (double)y / n - 0.5;
          fm[((size_t)y * N + x) * 2 + ch].re = exp(-(dx * dx + dy * dy) / (2 * 0.05 * 0.05));
          fm[((size_t)y * N + x) * 2 + ch].im = 0.0;
        }
    if (mg_mc_set_rhs(mc, fm, 0) != MG_OK) return 1;
    double m0 = 0.0, mrel = 0.0;
    if (mg_mc_residual_norm(mc, &m0, &mrel) != MG_OK) return 1;
    for (int it = 0; it < 40; ++it)
      if (mg_mc_cycle(mc, MG_BPX, omega, MG_HIERARCHICAL) != MG_OK) return 1;
    double m1 = 0.0;
    if (mg_mc_residual_norm(mc, &m1, &mrel) != MG_OK) return 1;
    printf("multichannel 2 channels, depth 4: relative residual %.3e after 40 BPX cycles\n", mrel);
    mg_mc_destroy(mc);
    free(fm);
    if (!(mrel < 1e-3)) return 1;
  }
  free(k2);
  free(f);

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
