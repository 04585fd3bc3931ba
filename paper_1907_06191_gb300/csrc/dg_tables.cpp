// dg_tables.cpp -- GLL nodal basis of order p (Eq. 8 on a tensor-product
// grid) and the real-axis stability limit of SSP-RK3, in FP64 on the host.
#include <cmath>

#include "dg_internal.h"

namespace dg {

// P_k(x) and P_k'(x) for k = p by Bonnet's recurrence and
// P_{k+1}' = (k+1) P_k + x P_k'.
static void legendre_pair(int p, double x, double *Pp, double *dPp, double *Pm,
                          double *dPm) {
  double P0 = 1.0, P1 = x, d0 = 0.0, d1 = 1.0;
  if (p == 1) { *Pp = P1; *dPp = d1; *Pm = P0; *dPm = d0; return; }
  for (int k = 1; k < p; ++k) {
    const double P2 = ((2.0 * k + 1.0) * x * P1 - k * P0) / (k + 1.0);
    const double d2 = (k + 1.0) * P1 + x * d1;
    P0 = P1; P1 = P2; d0 = d1; d1 = d2;
  }
  *Pp = P1; *dPp = d1; *Pm = P0; *dPm = d0;
}

// Interior GLL nodes are the zeros of q(x) = P_{p-1}(x) - x P_p(x), which is
// (1 - x^2) P_p'(x) / p; Newton with q' = P_{p-1}' - P_p - x P_p'.
// Weights 2 / (p (p+1) P_p(x_i)^2).  D_ij = P_p(x_i) / (P_p(x_j) (x_i - x_j))
// off the diagonal, -p(p+1)/4 and p(p+1)/4 at the two ends, 0 elsewhere.
bool gll_tables(int p, Gll *g) {
  if (p < 1 || p > kMaxP) return false;
  const int n = p + 1;
  g->p = p;
  g->xi[0] = -1.0;
  g->xi[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double x = -std::cos(M_PI * (double)i / (double)p);
    for (int it = 0; it < 60; ++it) {
      double Pp, dPp, Pm, dPm;
      legendre_pair(p, x, &Pp, &dPp, &Pm, &dPm);
      const double q = Pm - x * Pp;
      const double dq = dPm - Pp - x * dPp;
      const double step = q / dq;
      x -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    g->xi[i] = x;
  }
  double Pv[kMaxN];
  for (int i = 0; i < n; ++i) {
    double Pp, dPp, Pm, dPm;
    legendre_pair(p, g->xi[i], &Pp, &dPp, &Pm, &dPm);
    Pv[i] = Pp;
    g->w[i] = 2.0 / ((double)p * (p + 1.0) * Pp * Pp);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double d = 0.0;
      if (i != j) d = Pv[i] / (Pv[j] * (g->xi[i] - g->xi[j]));
      else if (i == 0) d = -0.25 * p * (p + 1.0);
      else if (i == p) d = 0.25 * p * (p + 1.0);
      g->D[i * n + j] = d;
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += g->D[i * n + k] * g->D[k * n + j];
      g->D2[i * n + j] = s;
    }
  return true;
}

// SSP-RK3 amplification on the real axis is 1 + z + z^2/2 + z^3/6; the step
// stays stable for -x3 <= z <= 0 where the polynomial reaches -1 at z = -x3.
double rk3_real_axis_limit() {
  double z = -2.5;
  for (int it = 0; it < 50; ++it) {
    const double f = 2.0 + z + 0.5 * z * z + z * z * z / 6.0;
    const double df = 1.0 + z + 0.5 * z * z;
    z -= f / df;
  }
  return -z;
}

}  // namespace dg
