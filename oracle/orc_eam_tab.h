/*
 * Natural cubic splines on uniform grids, for the tabulated embedded-atom
 * mechanical potential of the oracle (sl_eam_tab.c).
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle; nothing in the CUDA
 * library includes or links it.
 */
#ifndef ORC_EAM_TAB_H
#define ORC_EAM_TAB_H

/* Spline through (k h, y_k), k = 0 .. n-1: per interval k the coefficients
 * c[4k .. 4k+3] of y_k + t c1 + t^2 c2 + t^3 c3, t = x/h - k. */
typedef struct {
  int n;
  double h;
  double* c;
} orc_spline;

/* Tables of the embedded-atom potential: F(rho), rho(r), phi(r). */
typedef struct {
  orc_spline F, rho, phi;
  int ready;
} orc_eam_tabs;

int orc_spline_build(orc_spline* s, int n, double h, const double* y);
void orc_spline_free(orc_spline* s);
/* Value at x (>= 0); *dydx (if not NULL) the derivative.  x below the grid
 * uses the first interval's cubic, above it the last one's. */
double orc_spline_value(const orc_spline* s, double x, double* dydx);

#endif
