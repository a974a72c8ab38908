/*
 * Natural cubic splines on uniform grids (oracle side of the tabulated
 * embedded-atom potential, App. B of arXiv 1801.10233, whose F(rho), rho(r)
 * and phi(r) come as tables on uniform grids).
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle.
 *
 * The spline S interpolates y_k at x_k = k h, is a cubic on each interval, has
 * continuous first and second derivatives, and zero second derivative at both
 * ends ("natural").  Its knot second derivatives M_k solve
 *   M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1}) / h^2,
 *   k = 1 .. n-2,  M_0 = M_{n-1} = 0,
 * (tridiagonal, solved by plain forward elimination and back substitution),
 * and on [x_k, x_{k+1}], with t = (x - x_k)/h,
 *   S = y_k + t [(y_{k+1} - y_k) - h^2 (2 M_k + M_{k+1})/6]
 *         + t^2 [h^2 M_k / 2] + t^3 [h^2 (M_{k+1} - M_k)/6].
 */
#include <math.h>
#include <stdlib.h>

#include "orc_eam_tab.h"

int orc_spline_build(orc_spline* s, int n, double h, const double* y) {
  s->n = 0;
  s->h = h;
  s->c = NULL;
  if (n < 2 || !(h > 0.0)) return -1;
  double* M = (double*)calloc((size_t)n, sizeof(double));
  double* cp = (double*)calloc((size_t)n, sizeof(double));
  double* dp = (double*)calloc((size_t)n, sizeof(double));
  double* c = (double*)malloc((size_t)(n - 1) * 4 * sizeof(double));
  if (!M || !cp || !dp || !c) {
    free(M); free(cp); free(dp); free(c);
    return -8;
  }
  /* forward elimination over the interior knots 1 .. n-2 */
  for (int k = 1; k <= n - 2; ++k) {
    double rhs = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]) / (h * h);
    double diag = 4.0 - (k > 1 ? cp[k - 1] : 0.0);
    cp[k] = 1.0 / diag;
    dp[k] = (rhs - (k > 1 ? dp[k - 1] : 0.0)) / diag;
  }
  /* back substitution; M_0 = M_{n-1} = 0 */
  for (int k = n - 2; k >= 1; --k) M[k] = dp[k] - cp[k] * M[k + 1];
  for (int k = 0; k < n - 1; ++k) {
    c[4 * k] = y[k];
    c[4 * k + 1] = (y[k + 1] - y[k]) - h * h * (2.0 * M[k] + M[k + 1]) / 6.0;
    c[4 * k + 2] = h * h * M[k] / 2.0;
    c[4 * k + 3] = h * h * (M[k + 1] - M[k]) / 6.0;
  }
  free(M); free(cp); free(dp);
  s->n = n;
  s->c = c;
  return 0;
}

void orc_spline_free(orc_spline* s) {
  free(s->c);
  s->c = NULL;
  s->n = 0;
}

double orc_spline_value(const orc_spline* s, double x, double* dydx) {
  if (s->n < 2) {
    if (dydx) *dydx = 0.0;
    return 0.0;
  }
  double u = x / s->h;
  int k = (int)floor(u);
  if (k < 0) k = 0;
  if (k > s->n - 2) k = s->n - 2;
  double t = u - (double)k;
  const double* c = s->c + 4 * k;
  if (dydx) *dydx = (c[1] + t * (2.0 * c[2] + 3.0 * t * c[3])) / s->h;
  return c[0] + t * (c[1] + t * (c[2] + t * c[3]));
}

/* Build the spline of (n, h, y) and evaluate it at m points (for the pin
 * tests of the spline itself). */
int orc_spline_eval(int n, double h, const double* y, int m, const double* x, double* v, double* dv) {
  orc_spline s;
  int e = orc_spline_build(&s, n, h, y);
  if (e) return e;
  for (int i = 0; i < m; ++i) v[i] = orc_spline_value(&s, x[i], dv ? dv + i : NULL);
  orc_spline_free(&s);
  return 0;
}
