/* A C consumer of the libmb4 ABI (include/mb4.h), with no Python in between: a
 * 16x16 periodic grid with hopping 1, three defects at V = 20, chi = 1 and a
 * Gaussian wavepacket (sigma = 2 sites, wavevector pi/4 along x, normalised), 100
 * MB4 steps of h = 0.01 (Algorithm 1's time loop), and the energy before and after
 * (Sec. 2.1).  Exit status: 0 if |dH/H| <= 1e-13, 2 if not, 3 if mb4_create reports
 * MB4_ERR_CUDA (no GPU), 1 on any other error. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "mb4.h"

int main(void) {
  const int nx = 16, ny = 16, S = nx * ny;
  double* V = calloc((size_t)S, sizeof(double));
  double* re = calloc((size_t)S, sizeof(double));
  double* im = calloc((size_t)S, sizeof(double));
  if (!V || !re || !im) return 1;
  V[17] = V[100] = V[201] = 20.0;
  const double pi = 3.14159265358979323846, sigma = 2.0, k = pi / 4.0;
  double n2 = 0.0;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const double dx = x - nx / 2, dy = y - ny / 2;
      const double a = exp(-(dx * dx + dy * dy) / (4.0 * sigma * sigma));
      re[y * nx + x] = a * cos(k * x);
      im[y * nx + x] = a * sin(k * x);
      n2 += a * a;
    }
  for (int s = 0; s < S; ++s) {
    re[s] /= sqrt(n2);
    im[s] /= sqrt(n2);
  }
  mb4_grid grid = {nx, ny, 1.0, 1.0, 0.0};
  mb4_potential pot = {V, 0};
  mb4_nonlinearity nl = {1.0};
  mb4_options opt;
  mb4_default_options(&opt);
  mb4_ctx* ctx = NULL;
  int rc = mb4_create(&grid, &pot, &nl, 0.01, &opt, &ctx);
  if (rc != MB4_OK) {
    printf("mb4_create: %s (%d)\n", mb4_status_string(rc), rc);
    return rc == MB4_ERR_CUDA ? 3 : 1;
  }
  double H0 = 0.0, H1 = 0.0;
  mb4_stats st;
  if ((rc = mb4_set_state(ctx, re, im, 0)) != MB4_OK || (rc = mb4_energy(ctx, &H0, NULL)) != MB4_OK ||
      (rc = mb4_step(ctx, 100, &st)) != MB4_OK || (rc = mb4_energy(ctx, &H1, NULL)) != MB4_OK ||
      (rc = mb4_get_state(ctx, re, im, 0)) != MB4_OK) {
    printf("error: %s (%d)\n", mb4_status_string(rc), rc);
    mb4_destroy(ctx);
    return 1;
  }
  mb4_destroy(ctx);
  const double drift = fabs(H1 - H0) / fabs(H0);
  printf("steps %lld, Newton iterations %lld, H0 %.17g, |dH/H| %.3e\n", st.steps_done, st.newton_iters_total, H0,
         drift);
  free(V);
  free(re);
  free(im);
  return drift <= 1e-13 ? 0 : 2;
}
