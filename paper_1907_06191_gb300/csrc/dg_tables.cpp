// dg_tables.cpp -- GLL nodal basis of order p (Eq. 8 on a tensor-product
// grid) and the real-axis stability limit of SSP-RK3, in FP64 on the host.
#include <algorithm>
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

namespace {

// a + b with its rounding error (Knuth's TwoSum)
inline double two_sum(double a, double b, double *err) {
  const double s = a + b;
  const double bb = s - a;
  *err = (a - (s - bb)) + (b - bb);
  return s;
}

// Exact sum of FP32 values, or false if FP64 cannot hold it exactly.
bool exact_sum(const float *v, int n, int skip, double *out) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    if (k == skip) continue;
    double e;
    s = two_sum(s, (double)v[k], &e);
    if (e != 0.0) return false;
  }
  *out = s;
  return true;
}

float step_ulp(float x, int k) {
  for (; k > 0; --k) x = std::nextafter(x, INFINITY);
  for (; k < 0; ++k) x = std::nextafter(x, -INFINITY);
  return x;
}

double ulp_of(double t) {
  const float f = (float)std::fabs(t);
  return (double)std::nextafter(f, INFINITY) - (double)f;
}

// FP32 row g close to the FP64 row t (n entries) with an exactly zero sum.
// Structural zeros of t stay zero.  mirror = 0: no constraint; +1 / -1: the
// row must satisfy g[n-1-k] = mirror * g[k] (middle row of a centro-symmetric
// / antisymmetric matrix).  One entry (the free one) takes minus the sum of
// the others; at most one other entry (and its mirror partner) moves by one
// ulp.  The candidate with the smallest largest error in ulps wins.
bool zero_sum_row(const double *t_in, int n, int mirror, float *g_out) {
  double t[kMaxN], tmax = 0.0;
  for (int k = 0; k < n; ++k) tmax = std::fmax(tmax, std::fabs(t_in[k]));
  for (int k = 0; k < n; ++k) t[k] = std::fabs(t_in[k]) < 1e-12 * tmax ? 0.0 : t_in[k];
  float f[kMaxN];
  for (int k = 0; k < n; ++k) f[k] = (float)t[k];
  if (mirror != 0)
    for (int k = 0; k < n; ++k) f[n - 1 - k] = (float)mirror * f[k];
  double s0;
  if (exact_sum(f, n, -1, &s0) && s0 == 0.0) {
    for (int k = 0; k < n; ++k) g_out[k] = f[k];
    return true;
  }
  double best = INFINITY;
  for (int m = 0; m < n; ++m) {
    if (t[m] == 0.0) continue;
    if (mirror == 1 && 2 * m != n - 1) continue;  // palindrome: only the centre is free
    if (mirror == -1) continue;                   // antisymmetric rows already sum to zero
    for (int j = -1; j < n; ++j) {
      for (int dir = -1; dir <= 1; dir += 2) {
        if (j == m || (j < 0 && dir > 0)) continue;
        if (j >= 0 && t[j] == 0.0) continue;
        float g[kMaxN];
        for (int k = 0; k < n; ++k) g[k] = f[k];
        if (j >= 0) {
          g[j] = step_ulp(g[j], dir);
          if (mirror == 1) g[n - 1 - j] = g[j];
          if (mirror == 1 && n - 1 - j == m) continue;
        }
        double s;
        if (!exact_sum(g, n, m, &s)) continue;
        if ((double)(float)s != s) continue;
        g[m] = (float)(-s);
        double cost = 0.0;
        for (int k = 0; k < n; ++k)
          if (t[k] != 0.0) cost = std::fmax(cost, std::fabs((double)g[k] - t[k]) / ulp_of(t[k]));
        if (cost < best) {
          best = cost;
          for (int k = 0; k < n; ++k) g_out[k] = g[k];
        }
      }
    }
  }
  return best < 8.0;
}

// mirror = -1: centro-antisymmetric (D), +1: centro-symmetric (D D).
void zero_sum_matrix(const double *M, int n, int mirror, float *out) {
  for (int a = 0; 2 * a < n; ++a) {
    const bool mid = 2 * a == n - 1;
    float g[kMaxN];
    if (!zero_sum_row(M + a * n, n, mid ? mirror : 0, g))
      for (int k = 0; k < n; ++k) g[k] = (float)M[a * n + k];  // plain rounding
    for (int k = 0; k < n; ++k) {
      out[a * n + k] = g[k];
      out[(n - 1 - a) * n + (n - 1 - k)] = (float)mirror * g[k];
    }
  }
}

}  // namespace

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
  // interior nodes of the left half by Newton; the right half mirrors them
  // (x_{p-i} = -x_i exactly, and 0 in the middle for even p), so that the
  // tables below are exactly centro-(anti)symmetric
  for (int i = 1; 2 * i < p; ++i) {
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
    g->xi[p - i] = -x;
  }
  if (p % 2 == 0) g->xi[p / 2] = 0.0;
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
  zero_sum_matrix(g->D, n, -1, g->Df);
  zero_sum_matrix(g->D2, n, 1, g->D2f);
  return true;
}


namespace {

double factorial(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= k;
  return f;
}

// integral of r^a s^b over the reference triangle (0,0), (1,0), (0,1)
double tri_mono(int a, int b) { return factorial(a) * factorial(b) / factorial(a + b + 2); }

// in-place inverse of an n x n row-major matrix (Gauss-Jordan, partial
// pivoting); false if singular
bool invert(double *A, int n) {
  double B[kTriN * kTriN * 2];
  const int w = 2 * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < w; ++j) B[i * w + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(B[i * w + c]) > std::fabs(B[piv * w + c])) piv = i;
    if (B[piv * w + c] == 0.0) return false;
    if (piv != c)
      for (int j = 0; j < w; ++j) std::swap(B[c * w + j], B[piv * w + j]);
    const double d = B[c * w + c];
    for (int j = 0; j < w; ++j) B[c * w + j] /= d;
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      const double f = B[i * w + c];
      if (f == 0.0) continue;
      for (int j = 0; j < w; ++j) B[i * w + j] -= f * B[c * w + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = B[i * w + n + j];
  return true;
}

int tri_index(int p, int i, int j) { return j * (p + 1) - j * (j - 1) / 2 + i; }

int tri_edge_node(int p, int e, int t) {
  if (e == 0) return tri_index(p, t, 0);
  if (e == 1) return tri_index(p, p - t, t);
  return tri_index(p, 0, p - t);
}

}  // namespace

bool tri_tables(int p, TriRef *T) {
  if (p < 1 || p > kTriMaxP) return false;
  const int N = (p + 1) * (p + 2) / 2, NE = p + 1;
  T->p = p;
  T->N = N;
  // nodes and monomials r^ea s^eb (a + b <= p)
  int ea[kTriN], eb[kTriN];
  {
    int k = 0;
    for (int j = 0; j <= p; ++j)
      for (int i = 0; i + j <= p; ++i, ++k) {
        T->r[k] = (double)i / p;
        T->s[k] = (double)j / p;
      }
    k = 0;
    for (int a = 0; a <= p; ++a)
      for (int b = 0; a + b <= p; ++b, ++k) {
        ea[k] = a;
        eb[k] = b;
      }
  }
  // C = V^-1, V[k][m] = r_k^a_m s_k^b_m: basis function j = sum_m C[m][j] mono_m
  double C[kTriN * kTriN];
  for (int k = 0; k < N; ++k)
    for (int m = 0; m < N; ++m) C[k * N + m] = std::pow(T->r[k], ea[m]) * std::pow(T->s[k], eb[m]);
  if (!invert(C, N)) return false;
  // exact integrals of products of basis functions and their derivatives
  double M[kTriN * kTriN], Sr[kTriN * kTriN], Ss[kTriN * kTriN];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double m = 0.0, sr = 0.0, ss = 0.0;
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
          const double cc = C[a * N + i] * C[b * N + j];
          if (cc == 0.0) continue;
          m += cc * tri_mono(ea[a] + ea[b], eb[a] + eb[b]);
          if (ea[b] > 0) sr += cc * ea[b] * tri_mono(ea[a] + ea[b] - 1, eb[a] + eb[b]);
          if (eb[b] > 0) ss += cc * eb[b] * tri_mono(ea[a] + ea[b], eb[a] + eb[b] - 1);
        }
      M[i * N + j] = m;       // int N_i N_j
      Sr[i * N + j] = sr;     // int N_i dN_j/dr
      Ss[i * N + j] = ss;
    }
  double Mi[kTriN * kTriN];
  for (int k = 0; k < N * N; ++k) Mi[k] = M[k];
  if (!invert(Mi, N)) return false;
  // 1D mass matrix of the equispaced Lagrange basis on [0, 1]
  double C1[(kTriMaxP + 1) * (kTriMaxP + 1)], E1[(kTriMaxP + 1) * (kTriMaxP + 1)];
  for (int t = 0; t < NE; ++t)
    for (int a = 0; a < NE; ++a) C1[t * NE + a] = std::pow((double)t / p, a);
  if (!invert(C1, NE)) return false;
  for (int t = 0; t < NE; ++t)
    for (int u = 0; u < NE; ++u) {
      double v = 0.0;
      for (int a = 0; a < NE; ++a)
        for (int b = 0; b < NE; ++b) v += C1[a * NE + t] * C1[b * NE + u] / (a + b + 1.0);
      E1[t * NE + u] = v;
    }
  // the two triangles of a pixel
  const double ij[2][4] = {{1.0, -1.0, 0.0, 1.0}, {1.0, 0.0, -1.0, 1.0}};  // rx ry sx sy (x h)
  const double q = std::sqrt(0.5);
  const double nr[2][3][2] = {{{0.0, -1.0}, {1.0, 0.0}, {-q, q}}, {{q, -q}, {0.0, 1.0}, {-1.0, 0.0}}};
  const double len[2][3] = {{1.0, 1.0, std::sqrt(2.0)}, {std::sqrt(2.0), 1.0, 1.0}};
  for (int t = 0; t < 2; ++t) {
    const double rx = ij[t][0], ry = ij[t][1], sx = ij[t][2], sy = ij[t][3];
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        double gx = 0.0, gy = 0.0;
        for (int k = 0; k < N; ++k) {
          // (rx Sr^T + sx Ss^T)[k][j] = rx Sr[j][k] + sx Ss[j][k]
          gx += Mi[i * N + k] * (rx * Sr[j * N + k] + sx * Ss[j * N + k]);
          gy += Mi[i * N + k] * (ry * Sr[j * N + k] + sy * Ss[j * N + k]);
        }
        T->G[t][0][i * N + j] = -gx;
        T->G[t][1][i * N + j] = -gy;
      }
    for (int e = 0; e < 3; ++e) {
      T->nrm[t][e][0] = nr[t][e][0];
      T->nrm[t][e][1] = nr[t][e][1];
      for (int i = 0; i < N; ++i)
        for (int u = 0; u < NE; ++u) {
          double v = 0.0;
          for (int tt = 0; tt < NE; ++tt) v += Mi[i * N + tri_edge_node(p, e, tt)] * E1[tt * NE + u];
          T->Lf[t][e][i * NE + u] = len[t][e] * v;
        }
    }
  }
  const int mab[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
  for (int q6 = 0; q6 < 6; ++q6)
    for (int j = 0; j < N; ++j) {
      double v = 0.0;
      for (int m = 0; m < N; ++m) v += C[m * N + j] * tri_mono(mab[q6][0] + ea[m], mab[q6][1] + eb[m]);
      T->mono[q6][j] = v;
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
