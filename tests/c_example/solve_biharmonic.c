/*
 * The C-ABI from plain C: assemble the 16 x 16-patch biharmonic problem (Example 5.1 with
 * p = 3, 4 levels, 2,560 unknowns), set up a static block-FSAI Chebyshev-4 V(2,2) cycle and
 * solve with PCG to a relative residual of 1e-8.
 *
 * Build:  gcc -std=c99 -I include -I $CUDA/include solve_biharmonic.c \
 *             -L <dir of libpum.so> -lpum -L $CUDA/lib64 -lcudart
 * Exit status: 0 converged, 1 a library call failed, 2 no CUDA device (pum_create failed).
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "pum.h"

#define MODES 8

static int fail(pum_ctx *ctx, const char *what, pum_status st) {
  fprintf(stderr, "%s: status %d: %s\n", what, (int)st, pum_last_error(ctx));
  return 1;
}

int main(void) {
  pum_ctx *ctx = NULL;
  pum_status st = pum_create(&ctx, 0, NULL); /* device 0, a stream of its own */
  if (st != PUM_OK) {
    fprintf(stderr, "pum_create: status %d (no usable CUDA device?)\n", (int)st);
    return 2;
  }

  /* f = sum_ab c_ab (a^2 + b^2)^-1 sin(a pi x) sin(b pi y) with c_ab = 1 / (a + b) */
  double coef[MODES * MODES];
  for (int a = 1; a <= MODES; ++a)
    for (int b = 1; b <= MODES; ++b) coef[(a - 1) * MODES + (b - 1)] = 1.0 / (a + b);
  pum_problem pr = {0};
  pr.equation = 4;
  pr.p = 3;
  pr.finest_m = 16;
  pr.n_levels = 4;
  pr.f_coef = coef;
  pr.f_modes = MODES;
  pr.f_decay = 2.0;

  const size_t n = (size_t)16 * 16 * 10; /* patches x (p+1)(p+2)/2 */
  double *b = NULL, *x = NULL;
  if (cudaMalloc((void **)&b, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void **)&x, n * sizeof(double)) != cudaSuccess ||
      cudaMemset(x, 0, n * sizeof(double)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    fprintf(stderr, "device allocation failed\n");
    return 1;
  }

  pum_hier *h = NULL;
  if ((st = pum_assemble(ctx, &pr, &h, b)) != PUM_OK) return fail(ctx, "pum_assemble", st);

  bfsai_params fp = {PUM_P0_LOWER, /*adaptive*/ 0, /*t_max*/ 0, /*tau*/ 1.0, /*nested*/ 0, /*tie_rel*/ 1e-9};
  smoother_params sp = {/*degree_k*/ 2, /*lanczos_its*/ 100, /*lanczos_safety*/ 1.01, /*lanczos_seed*/ 0,
                        PUM_F64, PUM_F64, /*mixed_levels*/ 64, /*fp32_levels*/ 64, PUM_SMOOTHER_CHEB4,
                        PUM_CYCLE_VKK};
  if ((st = bfsai_setup(ctx, h, &fp, &sp)) != PUM_OK) return fail(ctx, "bfsai_setup", st);

  double hist[101];
  pcg_report rep = {0};
  rep.rtol = 1e-8;
  rep.maxit = 100;
  rep.hist = hist;
  if ((st = pcg_solve(ctx, h, b, x, &rep)) != PUM_OK) return fail(ctx, "pcg_solve", st);
  printf("converged in %d PCG iterations, ||r|| / ||b|| = %.3e\n", (int)rep.iters, rep.final_relres);

  pum_hier_destroy(h);
  pum_destroy(ctx);
  cudaFree(b);
  cudaFree(x);
  return rep.converged ? 0 : 1;
}
