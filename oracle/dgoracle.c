/*
 * dgoracle.c -- plain FP64 CPU oracle of the DG diffusion step and of the
 * moment reduction behind the displacement covariance Sigma.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file's library.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * Paper: Cervantes, Moreles, Pena, Ramirez-Manzanares, "A GPU implementation
 * of the Discontinuous Galerkin method for simulation of diffusion in brain
 * tissue", arXiv 1907.06191.
 *
 * What is computed (section / equation of the paper in brackets):
 *   u_t = div(k grad u) on the extracellular region, k = k0 there and 0 in the
 *   axons [Eqs. 1 and 5]; reflecting axon walls [Eq. 3]; u = 0 on the outer
 *   edge [Eq. 4].  Mixed form q = grad u, u_t = div(k q) [Eq. 6], element weak
 *   form [Eq. 7] with the central u-flux and the harmonic-mean q-flux
 *   [Sec. 3.2], nodal Lagrange basis [Eq. 8], explicit Runge-Kutta in time
 *   [Sec. 3.1].
 *
 * Readings taken where the paper is silent (each is listed in the design
 * notes of the repository):
 *   - square elements of side h on a uniform grid with a tensor-product
 *     Gauss-Lobatto-Legendre (GLL) nodal basis of order p; the GLL nodes are
 *     also the quadrature points, so the mass matrix is diagonal;
 *   - the weak form of Eq. 7 with GLL quadrature is rewritten by summation by
 *     parts into its equivalent strong form; this file evaluates the strong
 *     form, in two passes: first q at every node, then div(k q);
 *   - axon elements (centre strictly inside a disk) are removed by default:
 *     their faces are walls with u_hat = u^- and q_hat = 0 (wall_mode 0).
 *     wall_mode 1 keeps them with k = 0 as the paper does in Sec. 3.3, so that
 *     u_hat = (u^- + u^+)/2 and the harmonic mean gives q_hat = 0;
 *   - optional interior penalty: h_q gets -tau (u^- - u^+), tau = eta k_h
 *     (p+1)^2 / h; eta = 0 is the paper's flux;
 *   - outer edge (Eq. 4): u_hat = 0, normal flux k q^- . n - tau_D u^-;
 *   - SSP-RK3 (Shu-Osher form) as the Runge-Kutta method;
 *   - moments by GLL nodal quadrature of the numerical solution [Sec. 4.1].
 *
 * Storage: dense grid of nx*ny elements, element e = ey*nx + ex, node (i, j)
 * with i along x and j along y at offset e*n*n + j*n + i, n = p+1.  Elements
 * that are not in the mesh hold zeros.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 8 /* p <= 7 */

/* ------------------------------------------------------------------------ */
/* Nodal basis tables (Eq. 8 on a tensor-product GLL grid).                  */
/* ------------------------------------------------------------------------ */

/* Legendre P_p(x) and its first derivative, by the three-term recurrences
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and P'_{k+1} = P'_{k-1} + (2k+1) P_k. */
static void legendre(int p, double x, double *P, double *dP) {
  double pm1 = 1.0, p0 = x, dpm1 = 0.0, dp0 = 1.0;
  if (p == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < p; ++k) {
    double p1 = ((2.0 * k + 1.0) * x * p0 - k * pm1) / (k + 1.0);
    double dp1 = dpm1 + (2.0 * k + 1.0) * p0;
    pm1 = p0; p0 = p1; dpm1 = dp0; dp0 = dp1;
  }
  *P = p0; *dP = dp0;
}

/* GLL nodes xi[0..p] (ascending), weights w[0..p] and the differentiation
 * matrix D[i*(p+1)+m] = l_m'(xi_i) of the Lagrange basis l_m.
 * Interior nodes are the roots of P_p', found by Newton's method from the
 * Chebyshev-Gauss-Lobatto points; P_p'' comes from Legendre's equation
 * (1-x^2) P'' = 2x P' - p(p+1) P.  Weights 2/(p(p+1) P_p(xi)^2).  D from the
 * barycentric form of the Lagrange basis.  Returns 0, or -1 for p out of
 * range. */
int orc_gll(int p, double *xi, double *w, double *D) {
  if (p < 1 || p > ORC_MAXN - 1) return -1;
  int n = p + 1;
  xi[0] = -1.0; xi[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double x = -cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, x, &P, &dP);
      double d2P = (2.0 * x * dP - p * (p + 1.0) * P) / (1.0 - x * x);
      double dx = dP / d2P;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    xi[i] = x;
  }
  for (int i = 0; i < n; ++i) {
    double P, dP;
    legendre(p, xi[i], &P, &dP);
    w[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
  double lam[ORC_MAXN];
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (xi[j] - xi[k]);
    lam[j] = 1.0 / prod;
  }
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double dij = (lam[j] / lam[i]) / (xi[i] - xi[j]);
      D[i * n + j] = dij;
      diag -= dij;
    }
    D[i * n + i] = diag;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Mesh.                                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int p;                       /* polynomial order, n = p+1 nodes per axis */
  int nx, ny;                  /* elements along x and y */
  double h;                    /* element side (um) */
  double x0, y0;               /* lower-left corner of the domain (um) */
  double k0;                   /* diffusivity of the extracellular region */
  double eta;                  /* penalty factor, 0 = paper's fluxes */
  int wall_mode;               /* 0: axon elements removed, 1: kept, k = 0 */
  int periodic;                /* 0: Eq. 4 on the domain edge, 1: periodic */
  const unsigned char *active; /* [ny*nx], 1 = extracellular element */
} orc_mesh;

enum { F_INTERIOR = 0, F_WALL = 1, F_EDGE = 2 };
enum { DIR_E = 0, DIR_W = 1, DIR_N = 2, DIR_S = 3 };

static int in_mesh(const orc_mesh *M, int e) {
  return M->wall_mode == 1 ? 1 : (M->active[e] != 0);
}

static double kval(const orc_mesh *M, int e) {
  return M->active[e] ? M->k0 : 0.0;
}

/* Kind of the face of element (ex, ey) in direction dir; *nb gets the
 * neighbour element index for interior faces. */
static int face_kind(const orc_mesh *M, int ex, int ey, int dir, int *nb) {
  int qx = ex, qy = ey;
  if (dir == DIR_E) qx++;
  else if (dir == DIR_W) qx--;
  else if (dir == DIR_N) qy++;
  else qy--;
  if (qx < 0 || qx >= M->nx || qy < 0 || qy >= M->ny) {
    if (!M->periodic) return F_EDGE;
    qx = (qx + M->nx) % M->nx;
    qy = (qy + M->ny) % M->ny;
  }
  int e = qy * M->nx + qx;
  *nb = e;
  if (!in_mesh(M, e)) return F_WALL;
  return F_INTERIOR;
}

/* Node offset inside an element: i along x, j along y. */
#define NODE(n, i, j) ((j) * (n) + (i))

/* Face node t of face dir: east face is i = p, west i = 0, north j = p,
 * south j = 0; t runs along the face.  The matching node of the neighbour is
 * the same t on the opposite face. */
static int face_node(int n, int dir, int t) {
  int p = n - 1;
  switch (dir) {
    case DIR_E: return NODE(n, p, t);
    case DIR_W: return NODE(n, 0, t);
    case DIR_N: return NODE(n, t, p);
    default:    return NODE(n, t, 0);
  }
}

static int opposite(int dir) {
  return dir == DIR_E ? DIR_W : dir == DIR_W ? DIR_E : dir == DIR_N ? DIR_S : DIR_N;
}

/* Outward normal of face dir: (+1,0), (-1,0), (0,+1), (0,-1). */
static double nrm_x(int dir) { return dir == DIR_E ? 1.0 : dir == DIR_W ? -1.0 : 0.0; }
static double nrm_y(int dir) { return dir == DIR_N ? 1.0 : dir == DIR_S ? -1.0 : 0.0; }

/* ------------------------------------------------------------------------ */
/* The DG operator L: u -> u_t (Eq. 7 with the fluxes of Sec. 3.2).          */
/* ------------------------------------------------------------------------ */

/* Pass 1 (first line of Eq. 7): q = grad u in every mesh element, with the
 * central flux h_u = (u^- + u^+)/2 n^-.  Strong form at node (a, b):
 *   qx_ab = (1/J) sum_i D_ai u_ib
 *           + [a = p] (uhat_E,b - u_pb) / (J w_p) - [a = 0] (uhat_W,b - u_0b) / (J w_0)
 * and the same along y, J = h/2. */
static void grad_pass(const orc_mesh *M, const double *xi_unused,
                      const double *w, const double *D, const double *u,
                      double *qx, double *qy) {
  (void)xi_unused;
  const int n = M->p + 1, np = n * n;
  const double J = 0.5 * M->h;
#pragma omp parallel for schedule(static)
  for (int ey = 0; ey < M->ny; ++ey) {
    for (int ex = 0; ex < M->nx; ++ex) {
      const int e = ey * M->nx + ex;
      const double *ue = u + (size_t)e * np;
      double *qxe = qx + (size_t)e * np, *qye = qy + (size_t)e * np;
      if (!in_mesh(M, e)) {
        for (int t = 0; t < np; ++t) qxe[t] = qye[t] = 0.0;
        continue;
      }
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          double sx = 0.0, sy = 0.0;
          for (int m = 0; m < n; ++m) {
            sx += D[a * n + m] * ue[NODE(n, m, b)];
            sy += D[b * n + m] * ue[NODE(n, a, m)];
          }
          qxe[NODE(n, a, b)] = sx / J;
          qye[NODE(n, a, b)] = sy / J;
        }
      for (int dir = 0; dir < 4; ++dir) {
        int nb = -1;
        const int kind = face_kind(M, ex, ey, dir, &nb);
        const double wf = w[(dir == DIR_E || dir == DIR_N) ? n - 1 : 0];
        for (int t = 0; t < n; ++t) {
          const int node = face_node(n, dir, t);
          const double um = ue[node];
          double uhat;
          if (kind == F_INTERIOR) {
            const double up = u[(size_t)nb * np + face_node(n, opposite(dir), t)];
            uhat = 0.5 * (um + up);
          } else if (kind == F_WALL) {
            uhat = um;
          } else {
            uhat = 0.0;
          }
          /* surface term (uhat - u^-) n / (J w) */
          qxe[node] += (uhat - um) * nrm_x(dir) / (J * wf);
          qye[node] += (uhat - um) * nrm_y(dir) / (J * wf);
        }
      }
    }
  }
}

/* Pass 2 (second line of Eq. 7): u_t = div(k q) with the harmonic-mean flux
 * h_q = (2 k^- k^+ / (k^- + k^+)) (q^- + q^+)/2 . n^-  (minus tau (u^- - u^+)
 * when eta > 0).  Strong form at node (a, b):
 *   Lu_ab = (k/J) [sum_i D_ai qx_ib + sum_j D_bj qy_aj]
 *           + sum over faces through the node of (h_q - k q^- . n) / (J w_f). */
static void div_pass(const orc_mesh *M, const double *w, const double *D,
                     const double *u, const double *qx, const double *qy,
                     double *Lu) {
  const int n = M->p + 1, np = n * n;
  const double J = 0.5 * M->h;
  const double pen = M->eta * (double)n * (double)n / M->h;
#pragma omp parallel for schedule(static)
  for (int ey = 0; ey < M->ny; ++ey) {
    for (int ex = 0; ex < M->nx; ++ex) {
      const int e = ey * M->nx + ex;
      double *Le = Lu + (size_t)e * np;
      if (!in_mesh(M, e)) {
        for (int t = 0; t < np; ++t) Le[t] = 0.0;
        continue;
      }
      const double k = kval(M, e);
      const double *ue = u + (size_t)e * np;
      const double *qxe = qx + (size_t)e * np, *qye = qy + (size_t)e * np;
      for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
          double s = 0.0;
          for (int m = 0; m < n; ++m) {
            s += D[a * n + m] * qxe[NODE(n, m, b)];
            s += D[b * n + m] * qye[NODE(n, a, m)];
          }
          Le[NODE(n, a, b)] = k * s / J;
        }
      for (int dir = 0; dir < 4; ++dir) {
        int nb = -1;
        const int kind = face_kind(M, ex, ey, dir, &nb);
        const double wf = w[(dir == DIR_E || dir == DIR_N) ? n - 1 : 0];
        const double nx_ = nrm_x(dir), ny_ = nrm_y(dir);
        for (int t = 0; t < n; ++t) {
          const int node = face_node(n, dir, t);
          const double qn_m = qxe[node] * nx_ + qye[node] * ny_;
          double hq;
          if (kind == F_INTERIOR) {
            const int nnode = face_node(n, opposite(dir), t);
            const double kp = kval(M, nb);
            const double kh = (k + kp) > 0.0 ? 2.0 * k * kp / (k + kp) : 0.0;
            const double qn_p = qx[(size_t)nb * np + nnode] * nx_ +
                                qy[(size_t)nb * np + nnode] * ny_;
            const double up = u[(size_t)nb * np + nnode];
            hq = kh * 0.5 * (qn_m + qn_p) - pen * kh * (ue[node] - up);
          } else if (kind == F_WALL) {
            hq = 0.0;
          } else {
            hq = k * qn_m - pen * k * ue[node];
          }
          Le[node] += (hq - k * qn_m) / (J * wf);
        }
      }
    }
  }
}

typedef struct {
  double xi[ORC_MAXN], w[ORC_MAXN], D[ORC_MAXN * ORC_MAXN];
} orc_tables;

static int tables(const orc_mesh *M, orc_tables *T) {
  return orc_gll(M->p, T->xi, T->w, T->D);
}

static size_t field_size(const orc_mesh *M) {
  const size_t n = (size_t)M->p + 1;
  return (size_t)M->nx * M->ny * n * n;
}

/* Lu = L u for one density.  Returns 0, or -1 on bad input / no memory. */
int orc_apply_L(const orc_mesh *M, const double *u, double *Lu) {
  orc_tables T;
  if (tables(M, &T)) return -1;
  const size_t N = field_size(M);
  double *q = (double *)malloc(2 * N * sizeof(double));
  if (!q) return -1;
  grad_pass(M, T.xi, T.w, T.D, u, q, q + N);
  div_pass(M, T.w, T.D, u, q, q + N, Lu);
  free(q);
  return 0;
}

/* nsteps steps of SSP-RK3 (Shu-Osher form) with step dt, in place:
 *   u1 = u + dt L u;  u2 = 3/4 u + 1/4 (u1 + dt L u1);
 *   u <- 1/3 u + 2/3 (u2 + dt L u2).
 * adv (NULL = every element) marks the elements that advance; the others
 * keep their values through all three stages (growing window: elements
 * beyond the window's current radius are held fixed and act as frozen
 * neighbours of the advancing ones). */
int orc_rk3_adv(const orc_mesh *M, double *u, int nsteps, double dt,
                const unsigned char *adv) {
  orc_tables T;
  if (tables(M, &T)) return -1;
  const size_t N = field_size(M);
  const long nn = (long)(M->p + 1) * (M->p + 1);
  double *buf = (double *)malloc(5 * N * sizeof(double));
  if (!buf) return -1;
  double *u1 = buf, *u2 = buf + N, *L = buf + 2 * N, *qx = buf + 3 * N,
         *qy = buf + 4 * N;
#define ORC_ADV(t) (!adv || adv[(t) / nn])
  for (int s = 0; s < nsteps; ++s) {
    grad_pass(M, T.xi, T.w, T.D, u, qx, qy);
    div_pass(M, T.w, T.D, u, qx, qy, L);
#pragma omp parallel for schedule(static)
    for (long t = 0; t < (long)N; ++t) u1[t] = ORC_ADV(t) ? u[t] + dt * L[t] : u[t];
    grad_pass(M, T.xi, T.w, T.D, u1, qx, qy);
    div_pass(M, T.w, T.D, u1, qx, qy, L);
#pragma omp parallel for schedule(static)
    for (long t = 0; t < (long)N; ++t)
      u2[t] = ORC_ADV(t) ? 0.75 * u[t] + 0.25 * (u1[t] + dt * L[t]) : u[t];
    grad_pass(M, T.xi, T.w, T.D, u2, qx, qy);
    div_pass(M, T.w, T.D, u2, qx, qy, L);
#pragma omp parallel for schedule(static)
    for (long t = 0; t < (long)N; ++t)
      if (ORC_ADV(t)) u[t] = u[t] / 3.0 + 2.0 * (u2[t] + dt * L[t]) / 3.0;
  }
#undef ORC_ADV
  free(buf);
  return 0;
}

int orc_rk3(const orc_mesh *M, double *u, int nsteps, double dt) {
  return orc_rk3_adv(M, u, nsteps, dt, NULL);
}

/* ------------------------------------------------------------------------ */
/* Cauchy data (Sec. 4.1) and moments.                                        */
/* ------------------------------------------------------------------------ */

/* Physical coordinates of node (i, j) of element (ex, ey). */
static void node_xy(const orc_mesh *M, const double *xi, int ex, int ey, int i,
                    int j, double *x, double *y) {
  *x = M->x0 + (ex + 0.5) * M->h + 0.5 * M->h * xi[i];
  *y = M->y0 + (ey + 0.5) * M->h + 0.5 * M->h * xi[j];
}

/* Start density: the paper uses a Dirac delta at (xs, ys); a normalised
 * Gaussian of width sigma0 stands in for it, interpolated at the nodes of
 * extracellular elements (zero elsewhere). */
int orc_init_gaussian(const orc_mesh *M, double xs, double ys, double sigma0,
                      double *u) {
  orc_tables T;
  if (tables(M, &T)) return -1;
  const int n = M->p + 1, np = n * n;
  const double c = 1.0 / (2.0 * M_PI * sigma0 * sigma0);
#pragma omp parallel for schedule(static)
  for (int ey = 0; ey < M->ny; ++ey)
    for (int ex = 0; ex < M->nx; ++ex) {
      const int e = ey * M->nx + ex;
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          double x, y;
          node_xy(M, T.xi, ex, ey, i, j, &x, &y);
          const double dx = x - xs, dy = y - ys;
          u[(size_t)e * np + NODE(n, i, j)] =
              M->active[e] ? c * exp(-(dx * dx + dy * dy) / (2.0 * sigma0 * sigma0)) : 0.0;
        }
    }
  return 0;
}

/* Moments by GLL nodal quadrature (Sec. 4.1: "quadrature rules using u_ij at
 * the nodes"), about the start point: out = {M0, Mx, My, Mxx, Mxy, Myy} with
 * M_f = sum_e sum_ij J^2 w_i w_j f(x_ij - xs, y_ij - ys) u_ij.  Summed serially
 * in element order. */
int orc_moments(const orc_mesh *M, const double *u, double xs, double ys,
                double *out) {
  orc_tables T;
  if (tables(M, &T)) return -1;
  const int n = M->p + 1, np = n * n;
  const double J = 0.5 * M->h;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int ey = 0; ey < M->ny; ++ey)
    for (int ex = 0; ex < M->nx; ++ex) {
      const int e = ey * M->nx + ex;
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          double x, y;
          node_xy(M, T.xi, ex, ey, i, j, &x, &y);
          const double dx = x - xs, dy = y - ys;
          const double wu = J * J * T.w[i] * T.w[j] * u[(size_t)e * np + NODE(n, i, j)];
          s[0] += wu;
          s[1] += wu * dx;
          s[2] += wu * dy;
          s[3] += wu * dx * dx;
          s[4] += wu * dx * dy;
          s[5] += wu * dy * dy;
        }
    }
  for (int k = 0; k < 6; ++k) out[k] = s[k];
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Geometry -> element mask (Sec. 2.2 substrate, Sec. 3.3 pixel mesh).        */
/* ------------------------------------------------------------------------ */

/* Element (cx_e, cy_e) centre = ((i + 1/2) L/nc, (j + 1/2) L/nc) of the
 * periodic cell [0, L)^2; active iff, for every disk, the squared periodic
 * minimum-image distance from the centre to the disk centre is >= r^2.
 * Products and sums are rounded one by one (the file is compiled without
 * floating-point contraction). */
void orc_mask_disks(double L, int nc, const double *dcx, const double *dcy,
                    const double *dr, int nd, unsigned char *cell) {
  const double h = L / nc;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < nc; ++j)
    for (int i = 0; i < nc; ++i) {
      const double x = (i + 0.5) * h, y = (j + 0.5) * h;
      unsigned char act = 1;
      for (int d = 0; d < nd; ++d) {
        double dx = x - dcx[d], dy = y - dcy[d];
        if (dx > 0.5 * L) dx -= L;
        if (dx < -0.5 * L) dx += L;
        if (dy > 0.5 * L) dy -= L;
        if (dy < -0.5 * L) dy += L;
        const double d2 = dx * dx + dy * dy;
        if (d2 < dr[d] * dr[d]) { act = 0; break; }
      }
      cell[j * nc + i] = act;
    }
}

/* ------------------------------------------------------------------------ */
/* Spectral radius of L by power iteration (time-step bound).                */
/* ------------------------------------------------------------------------ */

/* splitmix64 (S. Vigna), used as a counter-based generator for the start
 * vector. */
static uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

/* Estimate rho(L) = max |lambda| after iters steps of v <- L v / |L v|,
 * in the GLL-weighted norm; returns |L v| / |v| of the last step, or -1. */
double orc_power_rho(const orc_mesh *M, int iters, uint64_t seed) {
  orc_tables T;
  if (tables(M, &T)) return -1.0;
  const int n = M->p + 1, np = n * n;
  const size_t N = field_size(M);
  double *v = (double *)malloc(4 * N * sizeof(double));
  if (!v) return -1.0;
  double *Lv = v + N, *q = v + 2 * N;
  for (size_t t = 0; t < N; ++t) {
    const size_t e = t / np;
    v[t] = in_mesh(M, (int)e) && M->active[e]
               ? (double)(splitmix64(seed + t) >> 11) * 0x1.0p-53 - 0.5
               : 0.0;
  }
  double rho = 0.0;
  for (int it = 0; it < iters; ++it) {
    grad_pass(M, T.xi, T.w, T.D, v, q, q + N);
    div_pass(M, T.w, T.D, v, q, q + N, Lv);
    double nv = 0.0, nl = 0.0;
    for (size_t t = 0; t < N; ++t) {
      const int node = (int)(t % np);
      const double wt = T.w[node % n] * T.w[node / n];
      nv += wt * v[t] * v[t];
      nl += wt * Lv[t] * Lv[t];
    }
    if (nl == 0.0) { rho = 0.0; break; }
    rho = sqrt(nl / nv);
    const double s = 1.0 / sqrt(nl);
    for (size_t t = 0; t < N; ++t) v[t] = Lv[t] * s;
  }
  free(v);
  return rho;
}

/* Threads of the OpenMP team the element loops above run on (for reporting
 * how many host cores a timing used). */
int orc_threads(void) {
  int n = 1;
#pragma omp parallel
  {
#pragma omp single
    n = omp_get_num_threads();
  }
  return n;
}

/* Size of the OpenMP team of the next element loops (n >= 1); used to time
 * the oracle on one host core as well as on all of them. */
void orc_set_threads(int n) {
  if (n >= 1) omp_set_num_threads(n);
}
