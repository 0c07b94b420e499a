// Host-side MB4 constants (Sec. 2.2; the set-up of Algorithm 1), in long double.
//
// * A_{tau,zeta} = [tau, tau^2/2, tau^3/3] M(alpha1) [1, zeta, zeta^2]^T  (eq. Adefinition)
// * l_j: Lagrange basis on (0, c1, c2, c3)                                   (eq. Lagrange)
// * E_ij = int_0^1 A_{c_i,zeta} l_j(zeta) dzeta, j = 0..3                    (eq. defE, eq. Ei0)
//   evaluated with the 6-node Gauss-Legendre rule, exact here (degree 5).
// * E(1:3,1:3) = T Lambda T^-1 with real eigenvalues (Sec. 2.2): roots of the
//   characteristic cubic by the trigonometric (Viete) form, polished by
//   Newton's method; eigenvectors as cross products of two rows of E - lambda I.
#include <cmath>
#include <cstring>

#include "mb4_internal.h"

namespace mb4 {
namespace {

typedef long double ld;

// Legendre P_n and its derivative by the three-term recurrence.
void legendre(int n, ld x, ld* p, ld* dp) {
  ld p0 = 1, p1 = x;
  if (n == 0) { *p = 1; *dp = 0; return; }
  for (int k = 1; k < n; ++k) {
    ld p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1);
}

// n-point Gauss-Legendre rule on [0, 1] (Newton iteration on the roots of P_n).
void gauss_legendre01(int n, ld* x01, ld* w01) {
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    ld x = std::cos(pi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      legendre(n, x, &p, &dp);
      ld dx = p / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-19L) break;
    }
    ld p, dp;
    legendre(n, x, &p, &dp);
    ld w = 2 / ((1 - x * x) * dp * dp);
    // ascending order on [0, 1]
    x01[n - 1 - i] = (1 + x) / 2;
    w01[n - 1 - i] = w / 2;
  }
}

ld peval(const ld* c, int ncoef, ld z) {
  ld acc = 0;
  for (int k = ncoef - 1; k >= 0; --k) acc = acc * z + c[k];
  return acc;
}

}  // namespace

int compute_constants(double alpha1, double c1, double c2, Constants* out) {
  if (!out) return MB4_ERR_INVALID_ARG;
  if (!(c1 > 0 && c1 < c2 && c2 < 1)) return MB4_ERR_INVALID_ARG;
  if (!(alpha1 < -300.0 * 0.7770503941)) return MB4_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  const ld a = alpha1;
  const ld M[3][3] = {{a + 4, -6 * a - 6, 6 * a},
                      {-6 * a - 6, 36 * a + 12, -36 * a},
                      {6 * a, -36 * a, 36 * a}};
  const ld nodes[4] = {0, (ld)c1, (ld)c2, 1};
  out->alpha1 = alpha1;
  out->c[0] = c1;
  out->c[1] = c2;
  out->c[2] = 1.0;

  // A_{c_i, zeta} coefficients in zeta.
  ld Ac[3][3];
  for (int i = 0; i < 3; ++i) {
    ld t = nodes[i + 1];
    ld row[3] = {t, t * t / 2, t * t * t / 3};
    for (int b = 0; b < 3; ++b) {
      ld s = 0;
      for (int r = 0; r < 3; ++r) s += row[r] * M[r][b];
      Ac[i][b] = s;
      out->Acoef[i][b] = (double)s;
    }
  }
  // Lagrange basis in monomial form: l_j = prod_{m != j} (zeta - c_m) / (c_j - c_m).
  ld lag[4][4];
  for (int j = 0; j < 4; ++j) {
    ld poly[4] = {1, 0, 0, 0};
    int deg = 0;
    for (int m = 0; m < 4; ++m) {
      if (m == j) continue;
      ld inv = 1 / (nodes[j] - nodes[m]);
      ld next[4] = {0, 0, 0, 0};
      for (int k = 0; k <= deg; ++k) {
        next[k] += -nodes[m] * inv * poly[k];
        next[k + 1] += inv * poly[k];
      }
      ++deg;
      for (int k = 0; k < 4; ++k) poly[k] = next[k];
    }
    for (int k = 0; k < 4; ++k) {
      lag[j][k] = poly[k];
      out->lag[j][k] = (double)poly[k];
    }
  }
  ld gx[kGauss], gw[kGauss];
  gauss_legendre01(kGauss, gx, gw);
  for (int q = 0; q < kGauss; ++q) {
    out->gx[q] = (double)gx[q];
    out->gw[q] = (double)gw[q];
  }
  // E_ij by Gauss quadrature (integrand of degree 5).
  ld E[3][4];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 4; ++j) {
      ld s = 0;
      for (int q = 0; q < kGauss; ++q) s += gw[q] * peval(Ac[i], 3, gx[q]) * peval(lag[j], 4, gx[q]);
      E[i][j] = s;
      out->E[i][j] = (double)s;
    }
  // Eigenvalues of E3 = E(1:3, 1:3): x^3 + a2 x^2 + a1 x + a0 with a2 = -tr, a1 = sum of principal
  // 2x2 minors, a0 = -det.
  ld e[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) e[i][j] = E[i][j + 1];
  ld tr = e[0][0] + e[1][1] + e[2][2];
  ld m2 = e[0][0] * e[1][1] - e[0][1] * e[1][0] + e[0][0] * e[2][2] - e[0][2] * e[2][0] +
          e[1][1] * e[2][2] - e[1][2] * e[2][1];
  ld det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
           e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
  ld A2 = -tr, A1 = m2, A0 = -det;
  ld p = A1 - A2 * A2 / 3;
  ld qq = 2 * A2 * A2 * A2 / 27 - A2 * A1 / 3 + A0;
  if (!(p < 0) || 4 * p * p * p + 27 * qq * qq >= 0) return MB4_ERR_INVALID_ARG;  // not 3 real roots
  ld r = 2 * std::sqrt(-p / 3);
  ld arg = (3 * qq / (2 * p)) * std::sqrt(-3 / p);
  if (arg > 1) arg = 1;
  if (arg < -1) arg = -1;
  ld phi = std::acos(arg) / 3;
  const ld twopi3 = 2.094395102393195492308428922186335256L;
  ld lam[3];
  for (int k = 0; k < 3; ++k) {
    ld x = r * std::cos(phi - twopi3 * k) - A2 / 3;
    for (int it = 0; it < 8; ++it) {  // Newton polish on the cubic
      ld f = ((x + A2) * x + A1) * x + A0;
      ld df = (3 * x + 2 * A2) * x + A1;
      if (df == 0) break;
      x -= f / df;
    }
    lam[k] = x;
  }
  // ascending
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (lam[j] < lam[i]) { ld t = lam[i]; lam[i] = lam[j]; lam[j] = t; }
  ld T[3][3];
  for (int k = 0; k < 3; ++k) {
    ld B[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) B[i][j] = e[i][j] - (i == j ? lam[k] : 0);
    // null vector of B: the largest cross product of two of its rows
    ld best[3] = {0, 0, 0}, bestn = -1;
    for (int r1 = 0; r1 < 3; ++r1)
      for (int r2 = r1 + 1; r2 < 3; ++r2) {
        ld v[3] = {B[r1][1] * B[r2][2] - B[r1][2] * B[r2][1], B[r1][2] * B[r2][0] - B[r1][0] * B[r2][2],
                   B[r1][0] * B[r2][1] - B[r1][1] * B[r2][0]};
        ld n = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if (n > bestn) { bestn = n; best[0] = v[0]; best[1] = v[1]; best[2] = v[2]; }
      }
    if (!(bestn > 0)) return MB4_ERR_INVALID_ARG;
    ld nrm = std::sqrt(bestn);
    int imax = 0;
    for (int i = 1; i < 3; ++i)
      if (std::fabs(best[i]) > std::fabs(best[imax])) imax = i;
    ld sgn = best[imax] < 0 ? -1 : 1;
    for (int i = 0; i < 3; ++i) T[i][k] = sgn * best[i] / nrm;
  }
  // Tinv by the adjugate.
  ld dT = T[0][0] * (T[1][1] * T[2][2] - T[1][2] * T[2][1]) - T[0][1] * (T[1][0] * T[2][2] - T[1][2] * T[2][0]) +
          T[0][2] * (T[1][0] * T[2][1] - T[1][1] * T[2][0]);
  if (!(std::fabs(dT) > 1e-12L)) return MB4_ERR_INVALID_ARG;
  ld Ti[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
      Ti[i][j] = (T[i1][j1] * T[i2][j2] - T[i1][j2] * T[i2][j1]) / dT;
    }
  for (int i = 0; i < 3; ++i) {
    out->lam[i] = (double)lam[i];
    for (int j = 0; j < 3; ++j) {
      out->T[i][j] = (double)T[i][j];
      out->Tinv[i][j] = (double)Ti[i][j];
    }
  }
  return MB4_OK;
}

}  // namespace mb4

extern "C" int mb4_constants(double alpha1, double c1, double c2, double* E34, double* lam3, double* T9,
                             double* Tinv9, double* gauss_x6, double* gauss_w6) {
  mb4::Constants k;
  int rc = mb4::compute_constants(alpha1, c1, c2, &k);
  if (rc != MB4_OK) return rc;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 4; ++j)
      if (E34) E34[i * 4 + j] = k.E[i][j];
    if (lam3) lam3[i] = k.lam[i];
    for (int j = 0; j < 3; ++j) {
      if (T9) T9[i * 3 + j] = k.T[i][j];
      if (Tinv9) Tinv9[i * 3 + j] = k.Tinv[i][j];
    }
  }
  for (int q = 0; q < mb4::kGauss; ++q) {
    if (gauss_x6) gauss_x6[q] = k.gx[q];
    if (gauss_w6) gauss_w6[q] = k.gw[q];
  }
  return MB4_OK;
}
