// dg_reduce.cu -- start densities, FP64 moment reduction, covariance of the
// mixture (Sec. 4.1), node layout conversion, power-iteration helpers.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "dg_internal.h"
#include "dg_stage.cuh"

namespace dg {

struct NodeGeo {
  double xi[kMaxN];
  double w[kMaxN];
  double h, x0, y0;
};

static NodeGeo node_geo(const Ctx &c) {
  NodeGeo g;
  for (int i = 0; i <= c.cfg.p; ++i) {
    g.xi[i] = c.gll.xi[i];
    g.w[i] = c.gll.w[i];
  }
  g.h = c.geo.h;
  g.x0 = c.geo.x0;
  g.y0 = c.geo.y0;
  return g;
}

// ---- start densities -------------------------------------------------------
// Normalised Gaussian of width sigma0 about each start point (stand-in for the
// Dirac data of Sec. 4.1), interpolated at the GLL nodes; FP64 arithmetic,
// stored in the state precision.  grid (ceil(nA/256), m).
// ---- start points in element units ------------------------------------------
// For density (g, s): sx = (xs - x0_g)/h_g - 1/2, so that the centre of element
// column ex sits at (ex - sx) h_g from the start point; stored as two floats
// (hi + lo) so that FP32 arithmetic forms ex - sx with an error relative to
// the displacement itself, not to the window size.
__global__ void k_src_rel(const double *__restrict__ src, const int2 *__restrict__ grange,
                          const double4 *__restrict__ gpar, int m, int G,
                          float4 *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G * m) return;
  const int g = i / m;
  const double4 gp = gpar[g];
  const double sx = (src[2 * i] - gp.x) / gp.z - 0.5;
  const double sy = (src[2 * i + 1] - gp.y) / gp.z - 0.5;
  const float sxh = (float)sx, syh = (float)sy;
  out[i] = make_float4(sxh, (float)(sx - (double)sxh), syh, (float)(sy - (double)syh));
}

__device__ __forceinline__ float rel_coord(int e, float hi, float lo, float h) {
  return (((float)e - hi) - lo) * h;
}

template <typename T, int P>
__global__ void k_init(const int2 *__restrict__ exy, const int2 *__restrict__ chunk_tab,
                       const double4 *__restrict__ gpar, long long stride, int m,
                       const double *__restrict__ src, const float4 *__restrict__ srel,
                       double cnorm, double inv2s2, const NodeGeo g, T *__restrict__ u) {
  constexpr int n = P + 1, NP = n * n;
  const int chunk = blockIdx.x;
  const int2 ci = chunk_tab[chunk];
  if ((int)threadIdx.x >= ci.x) return;
  const long long a = (long long)chunk * kBlock + threadIdx.x;
  const int s = blockIdx.y;
  const size_t ds = (size_t)ci.y * m + s;
  const int2 e = exy[a];
  T *out = u + ((size_t)s * stride + a) * NP;
  T v[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) v[k] = (T)0;
  // element-level test: the nearest point of the element to the start point
  // already underflows the state precision -> the element is zero
  const double4 gp = gpar[ci.y];
  const float4 sr = srel[ds];
  const float hf = (float)gp.z;
  const float X = rel_coord(e.x, sr.x, sr.y, hf), Y = rel_coord(e.y, sr.z, sr.w, hf);
  const float dxm = fmaxf(fabsf(X) - 0.5f * hf, 0.0f), dym = fmaxf(fabsf(Y) - 0.5f * hf, 0.0f);
  const float floor_exp = sizeof(T) == 4 ? 110.0f : 760.0f;
  if ((dxm * dxm + dym * dym) * (float)inv2s2 < floor_exp) {
    // exp(-(dx^2 + dy^2)/(2 s^2)) = exp(-dx^2/(2 s^2)) exp(-dy^2/(2 s^2)), FP64
    const double xs = src[2 * ds], ys = src[2 * ds + 1];
    double gx[n], gy[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const double dx = gp.x + (e.x + 0.5) * gp.z + 0.5 * gp.z * g.xi[i] - xs;
      const double dy = gp.y + (e.y + 0.5) * gp.z + 0.5 * gp.z * g.xi[i] - ys;
      gx[i] = exp(-(dx * dx) * inv2s2);
      gy[i] = exp(-(dy * dy) * inv2s2);
    }
#pragma unroll
    for (int j = 0; j < n; ++j)
#pragma unroll
      for (int i = 0; i < n; ++i) v[j * n + i] = (T)(cnorm * (gx[i] * gy[j]));
  }
  store_elem<T, NP>(out, v);
}

// ---- moments -----------------------------------------------------------------
// Per density: M0, Mx, My, Mxx, Mxy, Myy about the start point and the L1 mass
// sum |u| W, with W = J^2 w_i w_j (GLL nodal quadrature, Sec. 4.1).  Pass 1:
// a fixed grid of kMomBlocks blocks per density, each summing a fixed
// element stride, block-reduced in a fixed order -> part[s][block][7].
// Pass 2: one block per density sums the partials in a fixed order.  The
// result does not depend on scheduling.

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of kMomFields values; result valid in thread 0.  blockDim = 256.
__device__ __forceinline__ void block_sum7(double (&v)[kMomFields]) {
  __shared__ double sh[kMomFields][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < kMomFields; ++f) {
    v[f] = warp_sum_d(v[f]);
    if (lane == 0) sh[f][wid] = v[f];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int f = 0; f < kMomFields; ++f) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += sh[f][w];
      v[f] = s;
    }
  }
  __syncthreads();
}

// Element-local moments in reference coordinates, with the GLL weights:
// m_ab = sum_ij w_i w_j xi_i^a xi_j^b u_ij (a + b <= 2) and sum w_i w_j |u_ij|,
// accumulated in the state precision T (tensor product: rows first).
template <typename T, int P>
__device__ __forceinline__ void local_moments(const T *__restrict__ ue, const T (&w)[P + 1],
                                              const T (&wx)[P + 1], const T (&wxx)[P + 1],
                                              T (&lm)[7]) {
  constexpr int n = P + 1;
  for (int k = 0; k < 7; ++k) lm[k] = (T)0;
#pragma unroll
  for (int j = 0; j < n; ++j) {
    T r0 = 0, r1 = 0, r2 = 0, ra = 0;
#pragma unroll
    for (int i = 0; i < n; ++i) {
      const T v = ue[j * n + i];
      r0 += w[i] * v;
      r1 += wx[i] * v;
      r2 += wxx[i] * v;
      ra += w[i] * fabs(v);
    }
    lm[0] += w[j] * r0;    // m00
    lm[1] += w[j] * r1;    // m10
    lm[2] += wx[j] * r0;   // m01
    lm[3] += w[j] * r2;    // m20
    lm[4] += wx[j] * r1;   // m11
    lm[5] += wxx[j] * r0;  // m02
    lm[6] += w[j] * ra;    // |u| mass
  }
}

// Adds the element's contribution to the FP64 moments about the start point:
// node displacement (X + J xi_i, Y + J xi_j) with (X, Y) = element centre - xs.
__device__ __forceinline__ void add_element_moments(double X, double Y, double J,
                                                    const double (&lm)[7],
                                                    double (&acc)[kMomFields]) {
  const double J2 = J * J;
  const double m00 = lm[0], m10 = J * lm[1], m01 = J * lm[2];
  const double m20 = J2 * lm[3], m11 = J2 * lm[4], m02 = J2 * lm[5];
  acc[0] += J2 * m00;
  acc[1] += J2 * (X * m00 + m10);
  acc[2] += J2 * (Y * m00 + m01);
  acc[3] += J2 * (X * X * m00 + 2.0 * X * m10 + m20);
  acc[4] += J2 * (X * Y * m00 + X * m01 + Y * m10 + m11);
  acc[5] += J2 * (Y * Y * m00 + 2.0 * Y * m01 + m02);
  acc[6] += J2 * lm[6];
}

// grid (B, m, G): blocks b of density s of geometry g stride over that
// geometry's elements; partial sums part[((g m + s) B + b)][7].
template <typename T, int P>
__global__ void __launch_bounds__(256)
    k_moments(const int2 *__restrict__ exy, const int2 *__restrict__ grange,
              const double4 *__restrict__ gpar, long long stride, int m,
              const double *__restrict__ src, const float4 *__restrict__ srel, const NodeGeo g,
              const T *__restrict__ u, double *__restrict__ part) {
  constexpr int n = P + 1, NP = n * n;
  const int s = blockIdx.y, gi = blockIdx.z;
  const int2 rg = grange[gi];
  const double4 gp = gpar[gi];
  const double xs = src[2 * ((size_t)gi * m + s)], ys = src[2 * ((size_t)gi * m + s) + 1];
  const double J = 0.5 * gp.z;
  T w[n], wx[n], wxx[n];
#pragma unroll
  for (int i = 0; i < n; ++i) {
    w[i] = (T)g.w[i];
    wx[i] = (T)(g.w[i] * g.xi[i]);
    wxx[i] = (T)(g.w[i] * g.xi[i] * g.xi[i]);
  }
  double acc[kMomFields] = {0, 0, 0, 0, 0, 0, 0};
  const T *U = u + (size_t)s * stride * NP;
  const float4 sr = srel[(size_t)gi * m + s];
  const float hf = (float)gp.z, Jf = 0.5f * hf, J2f = Jf * Jf;
  for (long long k = (long long)blockIdx.x * 256 + threadIdx.x; k < rg.y;
       k += (long long)gridDim.x * 256) {
    const long long a = rg.x + k;
    const int2 e = exy[a];
    T lmT[7];
    local_moments<T, P>(U + (size_t)a * NP, w, wx, wxx, lmT);
    if constexpr (sizeof(T) == 4) {
      // FP32 state: the element's contribution in FP32, accumulated in FP64
      const float X = rel_coord(e.x, sr.x, sr.y, hf), Y = rel_coord(e.y, sr.z, sr.w, hf);
      const float m00 = lmT[0], m10 = Jf * lmT[1], m01 = Jf * lmT[2];
      const float m20 = J2f * lmT[3], m11 = J2f * lmT[4], m02 = J2f * lmT[5];
      acc[0] += (double)(J2f * m00);
      acc[1] += (double)(J2f * (X * m00 + m10));
      acc[2] += (double)(J2f * (Y * m00 + m01));
      acc[3] += (double)(J2f * (X * (X * m00 + 2.0f * m10) + m20));
      acc[4] += (double)(J2f * (X * (Y * m00 + m01) + Y * m10 + m11));
      acc[5] += (double)(J2f * (Y * (Y * m00 + 2.0f * m01) + m02));
      acc[6] += (double)(J2f * lmT[6]);
    } else {
      double lm[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) lm[q] = (double)lmT[q];
      const double X = gp.x + (e.x + 0.5) * gp.z - xs;
      const double Y = gp.y + (e.y + 0.5) * gp.z - ys;
      add_element_moments(X, Y, J, lm, acc);
    }
  }
  block_sum7(acc);
  if (threadIdx.x == 0) {
    double *o = part + (((size_t)gi * m + s) * gridDim.x + blockIdx.x) * kMomFields;
#pragma unroll
    for (int f = 0; f < kMomFields; ++f) o[f] = acc[f];
  }
}

__global__ void __launch_bounds__(256)
    k_moments_final(const double *__restrict__ part, int nblk, double *__restrict__ mom) {
  const int s = blockIdx.x;
  double acc[kMomFields] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblk; b += 256) {
    const double *p = part + ((size_t)s * nblk + b) * kMomFields;
#pragma unroll
    for (int f = 0; f < kMomFields; ++f) acc[f] += p[f];
  }
  block_sum7(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int f = 0; f < kMomFields; ++f) mom[(size_t)s * kMomFields + f] = acc[f];
  }
}

// ---- covariance (Sec. 4.1) ---------------------------------------------------
// Each density normalised by its mass, mixed with weights 1/m; moment-matched
// Gaussian: mu = mean M1/M0, Sigma_mix = mean M2/M0 - mu mu^T; reported
// Sigma = Sigma_mix(t) - Sigma_mix(0).  One thread per geometry, densities in
// order.  out[g] = {Sxx, Sxy, Syy, mux, muy}.
__global__ void k_covariance(const double *__restrict__ mom, const double *__restrict__ mom0,
                             int m, int G, double *__restrict__ out) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= G) return;
  double r[2][5];
  for (int k = 0; k < 2; ++k) {
    const double *M = (k == 0 ? mom : mom0) + (size_t)gi * m * kMomFields;
    double mx = 0, my = 0, sxx = 0, sxy = 0, syy = 0;
    for (int s = 0; s < m; ++s) {
      const double *q = M + (size_t)s * kMomFields;
      const double inv = 1.0 / q[0];
      mx += q[1] * inv;
      my += q[2] * inv;
      sxx += q[3] * inv;
      sxy += q[4] * inv;
      syy += q[5] * inv;
    }
    const double im = 1.0 / (double)m;
    mx *= im; my *= im; sxx *= im; sxy *= im; syy *= im;
    r[k][0] = sxx - mx * mx;
    r[k][1] = sxy - mx * my;
    r[k][2] = syy - my * my;
    r[k][3] = mx;
    r[k][4] = my;
  }
  double *o = out + (size_t)gi * kCovOut;
  o[0] = r[0][0] - r[1][0];
  o[1] = r[0][1] - r[1][1];
  o[2] = r[0][2] - r[1][2];
  o[3] = r[0][3];
  o[4] = r[0][4];
  o[5] = r[0][0];  // Sigma_mix(t) itself, for the Gaussian fit
  o[6] = r[0][1];
  o[7] = r[0][2];
}

// ---- least-squares residual of the Gaussian fit (Sec. 4.2) -----------------
// Per density (g, s): sum over its nodes of [f(x - x_s - mu) - u / M0]^2 with
// f the bivariate Gaussian of the mixture fit (mu, Sigma_mix) of geometry g.
// grid (B, m, G); partial sums in field 0 of part[((g m + s) B + b)][7].
template <typename T, int P>
__global__ void __launch_bounds__(256)
    k_lsres(const int2 *__restrict__ exy, const int2 *__restrict__ grange,
            const double4 *__restrict__ gpar, long long stride, int m,
            const double *__restrict__ src, const double *__restrict__ cov,
            const double *__restrict__ mom, const NodeGeo g, const T *__restrict__ u,
            double *__restrict__ part) {
  constexpr int n = P + 1, NP = n * n;
  const int s = blockIdx.y, gi = blockIdx.z;
  const int2 rg = grange[gi];
  const double4 gp = gpar[gi];
  const double *cv = cov + (size_t)gi * kCovOut;
  const double mux = cv[3], muy = cv[4], sxx = cv[5], sxy = cv[6], syy = cv[7];
  const double det = sxx * syy - sxy * sxy;
  const double ixx = syy / det, ixy = -sxy / det, iyy = sxx / det;
  const double fnorm = 1.0 / (2.0 * M_PI * sqrt(det));
  const double inv_m0 = 1.0 / mom[((size_t)gi * m + s) * kMomFields];
  const double xs = src[2 * ((size_t)gi * m + s)] + mux, ys = src[2 * ((size_t)gi * m + s) + 1] + muy;
  const double J = 0.5 * gp.z;
  double acc[kMomFields] = {0, 0, 0, 0, 0, 0, 0};
  const T *U = u + (size_t)s * stride * NP;
  for (long long k = (long long)blockIdx.x * 256 + threadIdx.x; k < rg.y;
       k += (long long)gridDim.x * 256) {
    const long long a = rg.x + k;
    const int2 e = exy[a];
    const T *ue = U + (size_t)a * NP;
#pragma unroll
    for (int j = 0; j < n; ++j) {
      const double dy = gp.y + (e.y + 0.5) * gp.z + J * g.xi[j] - ys;
#pragma unroll
      for (int i = 0; i < n; ++i) {
        const double dx = gp.x + (e.x + 0.5) * gp.z + J * g.xi[i] - xs;
        const double q = ixx * dx * dx + 2.0 * ixy * dx * dy + iyy * dy * dy;
        const double d = fnorm * exp(-0.5 * q) - (double)ue[j * n + i] * inv_m0;
        acc[0] += d * d;
      }
    }
  }
  block_sum7(acc);
  if (threadIdx.x == 0) {
    double *o = part + (((size_t)gi * m + s) * gridDim.x + blockIdx.x) * kMomFields;
#pragma unroll
    for (int f = 0; f < kMomFields; ++f) o[f] = acc[f];
  }
}

// out[g] = mean over the densities of geometry g of res[(g m + s)][0]
__global__ void k_ls_mean(const double *__restrict__ res, int m, int G, double *__restrict__ out) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= G) return;
  double t = 0.0;
  for (int s = 0; s < m; ++s) t += res[((size_t)gi * m + s) * kMomFields];
  out[gi] = t / (double)m;
}

// ---- node layout conversion ------------------------------------------------
template <typename T, int NP>
__global__ void k_to_dense(const int2 *__restrict__ exy, long long nA, long long stride,
                           int nx, int ny, const T *__restrict__ u, double *__restrict__ d) {
  const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nA) return;
  const int s = blockIdx.y;
  const int2 e = exy[a];
  const T *src = u + ((size_t)s * stride + a) * NP;
  double *dst = d + (((size_t)s * ny + e.y) * nx + e.x) * NP;
#pragma unroll
  for (int k = 0; k < NP; ++k) dst[k] = (double)src[k];
}

template <typename T, int NP>
__global__ void k_from_dense(const int2 *__restrict__ exy, long long nA, long long stride,
                             int nx, int ny, const double *__restrict__ d, T *__restrict__ u) {
  const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nA) return;
  const int s = blockIdx.y;
  const int2 e = exy[a];
  T *dst = u + ((size_t)s * stride + a) * NP;
  const double *src = d + (((size_t)s * ny + e.y) * nx + e.x) * NP;
#pragma unroll
  for (int k = 0; k < NP; ++k) dst[k] = (T)src[k];
}

// ---- power iteration helpers (FP64, one density) ----------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_random_field(long long nvals, int np, const int2 *__restrict__ chunk_tab,
                               unsigned long long seed, double *__restrict__ v) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nvals) return;
  const long long a = t / np;
  const bool live = (int)(a % kBlock) < chunk_tab[a / kBlock].x;
  v[t] = live ? (double)(splitmix64(seed + (unsigned long long)t) >> 11) * 0x1.0p-53 - 0.5 : 0.0;
}

template <int P>
__global__ void __launch_bounds__(256)
    k_wnorm2(long long n_elems, const int2 *__restrict__ chunk_tab, const double *__restrict__ v,
             const NodeGeo g, double *__restrict__ part) {
  constexpr int n = P + 1, NP = n * n;
  double acc[kMomFields] = {0, 0, 0, 0, 0, 0, 0};
  for (long long a = (long long)blockIdx.x * 256 + threadIdx.x; a < n_elems;
       a += (long long)gridDim.x * 256) {
    if ((int)(a % kBlock) >= chunk_tab[a / kBlock].x) continue;
    const double *ve = v + (size_t)a * NP;
#pragma unroll
    for (int j = 0; j < n; ++j)
#pragma unroll
      for (int i = 0; i < n; ++i) acc[0] += g.w[i] * g.w[j] * ve[j * n + i] * ve[j * n + i];
  }
  block_sum7(acc);
  if (threadIdx.x == 0) {
    double *o = part + (size_t)blockIdx.x * kMomFields;
#pragma unroll
    for (int f = 0; f < kMomFields; ++f) o[f] = acc[f];
  }
}

// res[1] = 1 / sqrt(res[0]), once
__global__ void k_inv_norm(double *__restrict__ res) {
  if (threadIdx.x == 0 && blockIdx.x == 0) res[1] = 1.0 / sqrt(res[0]);
}

__global__ void k_scale_rnorm(long long nvals, const double *__restrict__ in,
                              const double *__restrict__ res, double *__restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nvals) return;
  out[t] = in[t] * res[1];
}

// ---- pixel triangles (Sec. 3.3) ----------------------------------------------------
// Node (r, s) of the reference triangle sits at (x0 + h (ex + r + s), y0 + h (ey + s))
// in triangle A and at (x0 + h (ex + r), y0 + h (ey + r + s)) in triangle B.
struct TriGeo {
  double r[kTriN], s[kTriN];
  double mono[6][kTriN];  // int r^a s^b N_j over the reference triangle
  int N;
};

static TriGeo tri_geo(const Ctx &c) {
  TriGeo g;
  g.N = c.tri.N;
  for (int j = 0; j < c.tri.N; ++j) {
    g.r[j] = c.tri.r[j];
    g.s[j] = c.tri.s[j];
    for (int q = 0; q < 6; ++q) g.mono[q][j] = c.tri.mono[q][j];
  }
  return g;
}

// Gaussian start densities at the triangle nodes (FP64 per node; pixels whose
// nearest point lies beyond 40 sigma0 are set to zero without evaluating).
template <typename T, int NPX>
__global__ void k_init_tri(const int2 *__restrict__ exy, const int2 *__restrict__ chunk_tab,
                           const double4 *__restrict__ gpar, long long stride, int m,
                           const double *__restrict__ src, double cnorm, double inv2s2,
                           double cut2, const TriGeo g, T *__restrict__ u) {
  const long long a = (long long)blockIdx.x * kBlock + threadIdx.x;
  const int s = blockIdx.y;
  const int2 ci = chunk_tab[blockIdx.x];
  T *dst = u + ((size_t)s * stride + a) * NPX;
  if ((int)threadIdx.x >= ci.x) {
#pragma unroll
    for (int k = 0; k < NPX; ++k) dst[k] = (T)0;
    return;
  }
  const double4 gp = gpar[ci.y];
  const double xs = src[2 * ((size_t)ci.y * m + s)], ys = src[2 * ((size_t)ci.y * m + s) + 1];
  const int2 e = exy[a];
  const double px = gp.x + e.x * gp.z, py = gp.y + e.y * gp.z;  // pixel corner
  const double dx = fmax(fmax(px - xs, xs - (px + gp.z)), 0.0);
  const double dy = fmax(fmax(py - ys, ys - (py + gp.z)), 0.0);
  const bool far = dx * dx + dy * dy > cut2;
  constexpr int N = NPX / 2;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const double ra = g.r[k], sa = g.s[k];
    const double xa = px + gp.z * (ra + sa) - xs, ya = py + gp.z * sa - ys;
    const double xb = px + gp.z * ra - xs, yb = py + gp.z * (ra + sa) - ys;
    dst[k] = far ? (T)0 : (T)(cnorm * exp(-(xa * xa + ya * ya) * inv2s2));
    dst[N + k] = far ? (T)0 : (T)(cnorm * exp(-(xb * xb + yb * yb) * inv2s2));
  }
}

// Exact moments of the piecewise polynomial density: per pixel the integrals
// of r^a s^b u over each reference triangle, mapped to the pixel's local
// coordinates (x - x0, y - y0) = h (r + s, s) in A and h (r, r + s) in B and
// shifted to the start point in FP64.  Field 6 is the mass of |u| at the
// nodes weighted by the integrals of the basis functions.
template <typename T, int NPX>
__global__ void __launch_bounds__(256)
    k_moments_tri(const int2 *__restrict__ exy, const int2 *__restrict__ grange,
                  const double4 *__restrict__ gpar, long long stride, int m,
                  const double *__restrict__ src, const TriGeo g, const T *__restrict__ u,
                  double *__restrict__ part) {
  constexpr int N = NPX / 2;
  const int s = blockIdx.y, gi = blockIdx.z;
  const int2 rg = grange[gi];
  const double4 gp = gpar[gi];
  const double h = gp.z, J = h * h;
  const double xs = src[2 * ((size_t)gi * m + s)], ys = src[2 * ((size_t)gi * m + s) + 1];
  double acc[kMomFields] = {0, 0, 0, 0, 0, 0, 0};
  const T *U = u + (size_t)s * stride * NPX;
  for (long long k = (long long)blockIdx.x * 256 + threadIdx.x; k < rg.y;
       k += (long long)gridDim.x * 256) {
    const long long a = rg.x + k;
    const int2 e = exy[a];
    const T *ue = U + (size_t)a * NPX;
    const double cx = gp.x + e.x * h - xs, cy = gp.y + e.y * h - ys;
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      double I[6] = {0, 0, 0, 0, 0, 0}, l1 = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const double v = (double)ue[o * N + j];
#pragma unroll
        for (int q = 0; q < 6; ++q) I[q] += g.mono[q][j] * v;
        l1 += g.mono[0][j] * fabs(v);
      }
      // I: (0,0), (1,0) = r, (0,1) = s, (2,0), (1,1), (0,2)
      double lx, ly, lxx, lxy, lyy;
      if (o == 0) {
        lx = I[1] + I[2]; ly = I[2];
        lxx = I[3] + 2.0 * I[4] + I[5]; lxy = I[4] + I[5]; lyy = I[5];
      } else {
        lx = I[1]; ly = I[1] + I[2];
        lxx = I[3]; lxy = I[3] + I[4]; lyy = I[3] + 2.0 * I[4] + I[5];
      }
      const double m0 = J * I[0], mx = J * h * lx, my = J * h * ly;
      acc[0] += m0;
      acc[1] += cx * m0 + mx;
      acc[2] += cy * m0 + my;
      acc[3] += cx * cx * m0 + 2.0 * cx * mx + J * h * h * lxx;
      acc[4] += cx * cy * m0 + cx * my + cy * mx + J * h * h * lxy;
      acc[5] += cy * cy * m0 + 2.0 * cy * my + J * h * h * lyy;
      acc[6] += J * l1;
    }
  }
  block_sum7(acc);
  if (threadIdx.x == 0) {
    double *o = part + (((size_t)gi * m + s) * gridDim.x + blockIdx.x) * kMomFields;
#pragma unroll
    for (int f = 0; f < kMomFields; ++f) o[f] = acc[f];
  }
}

// Euclidean norm^2 of an FP64 field (power iteration on triangles).
__global__ void __launch_bounds__(256)
    k_norm2(long long nvals, int np, const int2 *__restrict__ chunk_tab,
            const double *__restrict__ v, double *__restrict__ part) {
  double acc[kMomFields] = {0, 0, 0, 0, 0, 0, 0};
  for (long long t = (long long)blockIdx.x * 256 + threadIdx.x; t < nvals;
       t += (long long)gridDim.x * 256) {
    const long long a = t / np;
    if ((int)(a % kBlock) < chunk_tab[a / kBlock].x) acc[0] += v[t] * v[t];
  }
  block_sum7(acc);
  if (threadIdx.x == 0) {
    double *o = part + (size_t)blockIdx.x * kMomFields;
#pragma unroll
    for (int f = 0; f < kMomFields; ++f) o[f] = acc[f];
  }
}

// ---- growing window ---------------------------------------------------------------
// Squared distance from the centre (x0 + (ex + 1/2) h, y0 + (ey + 1/2) h) of
// every mesh element to its geometry's start-point box; each operation is
// rounded on its own (no fused multiply-add) so that the window takes the
// same decisions as a plain FP64 evaluation of the same expression.
// Padding elements get +inf (never advance).
__global__ void k_window_d2(long long n_pad, const int2 *__restrict__ exy,
                            const int2 *__restrict__ chunk_tab, const double4 *__restrict__ gpar,
                            const double *__restrict__ box, double *__restrict__ d2) {
  const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n_pad) return;
  const int2 ci = chunk_tab[a / kBlock];
  if ((int)(a % kBlock) >= ci.x) {
    d2[a] = INFINITY;
    return;
  }
  const double4 gp = gpar[ci.y];
  const double *b = box + 4 * ci.y;
  const int2 e = exy[a];
  const double x = __dadd_rn(gp.x, __dmul_rn((double)e.x + 0.5, gp.z));
  const double y = __dadd_rn(gp.y, __dmul_rn((double)e.y + 0.5, gp.z));
  const double dx = fmax(fmax(__dsub_rn(b[0], x), __dsub_rn(x, b[1])), 0.0);
  const double dy = fmax(fmax(__dsub_rn(b[2], y), __dsub_rn(y, b[3])), 0.0);
  d2[a] = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

__global__ void k_window_flags(long long n_pad, const double *__restrict__ d2, double r2,
                               uint8_t *__restrict__ adv) {
  const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n_pad) adv[a] = d2[a] <= r2 ? 1 : 0;
}

cudaError_t launch_window_d2(const Ctx &c, const double *d_box, double *d2, cudaStream_t s) {
  const long long n = c.geo.n_pad;
  if (n <= 0) return cudaSuccess;
  k_window_d2<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, c.geo.d_exy, c.geo.d_chunk,
                                                          c.geo.d_gpar, d_box, d2);
  return cudaGetLastError();
}

cudaError_t launch_window_flags(const Ctx &c, const double *d2, double r2, uint8_t *adv,
                                cudaStream_t s) {
  const long long n = c.geo.n_pad;
  if (n <= 0) return cudaSuccess;
  k_window_flags<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, d2, r2, adv);
  return cudaGetLastError();
}

// ---- launchers ----------------------------------------------------------------
#define DG_P_SWITCH(p, CALL)          \
  switch (p) {                        \
    case 1: { constexpr int PP = 1; CALL; } break; \
    case 2: { constexpr int PP = 2; CALL; } break; \
    case 3: { constexpr int PP = 3; CALL; } break; \
    case 4: { constexpr int PP = 4; CALL; } break; \
    case 5: { constexpr int PP = 5; CALL; } break; \
    default: return cudaErrorInvalidValue;         \
  }

// nodes per element: (p+1)^2 for squares, 2 (p+1)(p+2)/2 for pixel triangles
#define DG_NP_SWITCH(np, CALL)                                     \
  switch (np) {                                                    \
    case 4: { constexpr int NN = 4; CALL; } break;                 \
    case 9: { constexpr int NN = 9; CALL; } break;                 \
    case 16: { constexpr int NN = 16; CALL; } break;               \
    case 25: { constexpr int NN = 25; CALL; } break;               \
    case 36: { constexpr int NN = 36; CALL; } break;               \
    case 6: { constexpr int NN = 6; CALL; } break;                 \
    case 12: { constexpr int NN = 12; CALL; } break;               \
    case 20: { constexpr int NN = 20; CALL; } break;               \
    default: return cudaErrorInvalidValue;                         \
  }

// nodes per pixel of the triangle elements, p = 1..3
#define DG_TRI_SWITCH(np, CALL)                                    \
  switch (np) {                                                    \
    case 6: { constexpr int NN = 6; CALL; } break;                 \
    case 12: { constexpr int NN = 12; CALL; } break;               \
    case 20: { constexpr int NN = 20; CALL; } break;               \
    default: return cudaErrorInvalidValue;                         \
  }

cudaError_t launch_init_sources(const Ctx &c, void *u, cudaStream_t s) {
  const int G = c.geo.G();
  k_src_rel<<<(G * c.m + 127) / 128, 128, 0, s>>>(c.d_src, c.geo.d_grange, c.geo.d_gpar, c.m, G,
                                                   c.d_srel);
  const dim3 grid((unsigned)c.geo.n_chunks(), (unsigned)c.m);
  if (c.cfg.element == DG_ELEMENT_TRIANGLE) {
    const TriGeo g = tri_geo(c);
    const double s2 = c.cfg.sigma0 * c.cfg.sigma0;
    const double cnorm = 1.0 / (2.0 * M_PI * s2), inv2s2 = 1.0 / (2.0 * s2);
    const double cut2 = 1600.0 * s2;
    if (c.cfg.precision == DG_FP64) {
      DG_TRI_SWITCH(c.np(), (k_init_tri<double, NN><<<grid, kBlock, 0, s>>>(
                               c.geo.d_exy, c.geo.d_chunk, c.geo.d_gpar, c.geo.n_pad, c.m,
                               c.d_src, cnorm, inv2s2, cut2, g, (double *)u)));
    } else {
      DG_TRI_SWITCH(c.np(), (k_init_tri<float, NN><<<grid, kBlock, 0, s>>>(
                               c.geo.d_exy, c.geo.d_chunk, c.geo.d_gpar, c.geo.n_pad, c.m,
                               c.d_src, cnorm, inv2s2, cut2, g, (float *)u)));
    }
    return cudaGetLastError();
  }
  const NodeGeo g = node_geo(c);
  const double s2 = c.cfg.sigma0 * c.cfg.sigma0;
  const double cnorm = 1.0 / (2.0 * M_PI * s2), inv2s2 = 1.0 / (2.0 * s2);
  if (c.cfg.precision == DG_FP64) {
    DG_P_SWITCH(c.cfg.p, (k_init<double, PP><<<grid, kBlock, 0, s>>>(
                             c.geo.d_exy, c.geo.d_chunk, c.geo.d_gpar, c.geo.n_pad, c.m,
                             c.d_src, c.d_srel, cnorm, inv2s2, g, (double *)u)));
  } else {
    DG_P_SWITCH(c.cfg.p, (k_init<float, PP><<<grid, kBlock, 0, s>>>(
                             c.geo.d_exy, c.geo.d_chunk, c.geo.d_gpar, c.geo.n_pad, c.m,
                             c.d_src, c.d_srel, cnorm, inv2s2, g, (float *)u)));
  }
  return cudaGetLastError();
}

int moment_blocks(int G) { return std::max(8, std::min(kMomBlocks, 4864 / std::max(G, 1))); }

cudaError_t launch_moments(const Ctx &c, const void *u, double *d_part, double *d_mom,
                           cudaStream_t s) {
  const int G = c.geo.G();
  const int B = moment_blocks(G);
  const dim3 grid((unsigned)B, (unsigned)c.m, (unsigned)G);
  if (c.cfg.element == DG_ELEMENT_TRIANGLE) {
    const TriGeo tg = tri_geo(c);
    if (c.cfg.precision == DG_FP64) {
      DG_TRI_SWITCH(c.np(), (k_moments_tri<double, NN><<<grid, 256, 0, s>>>(
                               c.geo.d_exy, c.geo.d_grange, c.geo.d_gpar, c.geo.n_pad, c.m,
                               c.d_src, tg, (const double *)u, d_part)));
    } else {
      DG_TRI_SWITCH(c.np(), (k_moments_tri<float, NN><<<grid, 256, 0, s>>>(
                               c.geo.d_exy, c.geo.d_grange, c.geo.d_gpar, c.geo.n_pad, c.m,
                               c.d_src, tg, (const float *)u, d_part)));
    }
    k_moments_final<<<(unsigned)(c.m * G), 256, 0, s>>>(d_part, B, d_mom);
    return cudaGetLastError();
  }
  const NodeGeo g = node_geo(c);
  if (c.cfg.precision == DG_FP64) {
    DG_P_SWITCH(c.cfg.p, (k_moments<double, PP><<<grid, 256, 0, s>>>(
                             c.geo.d_exy, c.geo.d_grange, c.geo.d_gpar, c.geo.n_pad, c.m,
                             c.d_src, c.d_srel, g, (const double *)u, d_part)));
  } else {
    DG_P_SWITCH(c.cfg.p, (k_moments<float, PP><<<grid, 256, 0, s>>>(
                             c.geo.d_exy, c.geo.d_grange, c.geo.d_gpar, c.geo.n_pad, c.m,
                             c.d_src, c.d_srel, g, (const float *)u, d_part)));
  }
  k_moments_final<<<(unsigned)(c.m * G), 256, 0, s>>>(d_part, B, d_mom);
  return cudaGetLastError();
}

cudaError_t launch_covariance(const double *d_mom, const double *d_mom0, int m, int G,
                              double *d_out, cudaStream_t s) {
  k_covariance<<<(G + 127) / 128, 128, 0, s>>>(d_mom, d_mom0, m, G, d_out);
  return cudaGetLastError();
}

cudaError_t launch_ls_residual(const Ctx &c, const void *u, const double *d_cov,
                               double *d_part, double *d_res, double *d_out, cudaStream_t s) {
  const int G = c.geo.G();
  const int B = moment_blocks(G);
  const dim3 grid((unsigned)B, (unsigned)c.m, (unsigned)G);
  const NodeGeo g = node_geo(c);
  if (c.cfg.precision == DG_FP64) {
    DG_P_SWITCH(c.cfg.p, (k_lsres<double, PP><<<grid, 256, 0, s>>>(
                             c.geo.d_exy, c.geo.d_grange, c.geo.d_gpar, c.geo.n_pad, c.m,
                             c.d_src, d_cov, c.d_mom, g, (const double *)u, d_part)));
  } else {
    DG_P_SWITCH(c.cfg.p, (k_lsres<float, PP><<<grid, 256, 0, s>>>(
                             c.geo.d_exy, c.geo.d_grange, c.geo.d_gpar, c.geo.n_pad, c.m,
                             c.d_src, d_cov, c.d_mom, g, (const float *)u, d_part)));
  }
  k_moments_final<<<(unsigned)(c.m * G), 256, 0, s>>>(d_part, B, d_res);
  k_ls_mean<<<(G + 127) / 128, 128, 0, s>>>(d_res, c.m, G, d_out);
  return cudaGetLastError();
}

// Dense node layout of geometry 0 (single-geometry contexts).
cudaError_t launch_nodes_to_dense(const Ctx &c, const void *u, double *d_dense,
                                  cudaStream_t s) {
  const long long nA = c.geo.parts[0].n_active;
  const dim3 grid((unsigned)((nA + 255) / 256), (unsigned)c.m);
  if (c.cfg.precision == DG_FP64) {
    DG_NP_SWITCH(c.np(), (k_to_dense<double, NN><<<grid, 256, 0, s>>>(
                             c.geo.d_exy, nA, c.geo.n_pad, c.geo.nx, c.geo.ny,
                             (const double *)u, d_dense)));
  } else {
    DG_NP_SWITCH(c.np(), (k_to_dense<float, NN><<<grid, 256, 0, s>>>(
                             c.geo.d_exy, nA, c.geo.n_pad, c.geo.nx, c.geo.ny,
                             (const float *)u, d_dense)));
  }
  return cudaGetLastError();
}
cudaError_t launch_dense_to_nodes(const Ctx &c, const double *d_dense, void *u,
                                  cudaStream_t s) {
  const long long nA = c.geo.parts[0].n_active;
  const dim3 grid((unsigned)((nA + 255) / 256), (unsigned)c.m);
  if (c.cfg.precision == DG_FP64) {
    DG_NP_SWITCH(c.np(), (k_from_dense<double, NN><<<grid, 256, 0, s>>>(
                             c.geo.d_exy, nA, c.geo.n_pad, c.geo.nx, c.geo.ny, d_dense,
                             (double *)u)));
  } else {
    DG_NP_SWITCH(c.np(), (k_from_dense<float, NN><<<grid, 256, 0, s>>>(
                             c.geo.d_exy, nA, c.geo.n_pad, c.geo.nx, c.geo.ny, d_dense,
                             (float *)u)));
  }
  return cudaGetLastError();
}
cudaError_t launch_random_field(const Ctx &c, double *v, unsigned long long seed,
                                cudaStream_t s) {
  const long long nv = c.geo.n_pad * c.np();
  k_random_field<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(nv, c.np(), c.geo.d_chunk, seed, v);
  return cudaGetLastError();
}

cudaError_t launch_wnorm2(const Ctx &c, const double *v, double *d_part, double *d_res,
                          cudaStream_t s) {
  if (c.cfg.element == DG_ELEMENT_TRIANGLE) {
    k_norm2<<<kMomBlocks, 256, 0, s>>>(c.geo.n_pad * c.np(), c.np(), c.geo.d_chunk, v, d_part);
    k_moments_final<<<1, 256, 0, s>>>(d_part, kMomBlocks, d_res);
    return cudaGetLastError();
  }
  const NodeGeo g = node_geo(c);
  DG_P_SWITCH(c.cfg.p, (k_wnorm2<PP><<<kMomBlocks, 256, 0, s>>>(c.geo.n_pad, c.geo.d_chunk, v, g,
                                                                 d_part)));
  k_moments_final<<<1, 256, 0, s>>>(d_part, kMomBlocks, d_res);
  return cudaGetLastError();
}

cudaError_t launch_scale_by_rnorm(const Ctx &c, const double *in, const double *d_res,
                                  double *out, cudaStream_t s) {
  const long long nv = c.geo.n_pad * c.np();
  k_inv_norm<<<1, 32, 0, s>>>(const_cast<double *>(d_res));
  k_scale_rnorm<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(nv, in, d_res, out);
  return cudaGetLastError();
}

// ---- moments without allocation ---------------------------------------------
// Some callers cannot allocate device memory: their device memory is held by
// another allocator (a framework's caching pool or a fixed pre-reservation),
// or they run where cudaMalloc is off limits (a latency-critical loop that
// must not risk the implicit synchronisation cudaMalloc can cause, code that
// owns no CUDA context set-up).  dg_moments_dense_static serves them: the
// first-pass partial sums of the two-pass reduction live in this file-scope
// device array, so the call allocates nothing.  Every GPU that loads the
// library holds the array (1.09 MB) until the process exits.

constexpr int kStaticMomBlocks = 152;          // first-pass blocks per density
constexpr int kStaticMomMaxDensities = 128;    // largest m of one call
static __device__ __align__(256) double
    g_static_mom_partials[kStaticMomMaxDensities * kStaticMomBlocks * kMomFields];

// Moments of densities in the dense node layout [m][ny][nx][n][n]; elements
// outside the mesh hold zeros and add nothing.  grid (kStaticMomBlocks, m).
// Per element the weighted node sums are formed in the state precision
// (local_moments, as k_moments does) and combined with the FP64 element
// centre in FP64, so an FP32 density costs no FP64 arithmetic per node.
template <typename T, int P>
__global__ void __launch_bounds__(256)
    k_moments_dense(const T *__restrict__ u, int nx, int ny, const double *__restrict__ xy,
                    const NodeGeo g, double *__restrict__ part) {
  constexpr int n = P + 1, NP = n * n;
  const int s = blockIdx.y;
  const double xs = xy[2 * s], ys = xy[2 * s + 1];
  const double J = 0.5 * g.h;
  T w[n], wx[n], wxx[n];
#pragma unroll
  for (int i = 0; i < n; ++i) {
    w[i] = (T)g.w[i];
    wx[i] = (T)(g.w[i] * g.xi[i]);
    wxx[i] = (T)(g.w[i] * g.xi[i] * g.xi[i]);
  }
  const long long ne = (long long)nx * ny;
  double acc[kMomFields] = {0, 0, 0, 0, 0, 0, 0};
  const T *U = u + (size_t)s * ne * NP;
  for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < ne;
       e += (long long)gridDim.x * 256) {
    const int ex = (int)(e % nx), ey = (int)(e / nx);
    T lmT[7];
    local_moments<T, P>(U + (size_t)e * NP, w, wx, wxx, lmT);
    double lm[7];
#pragma unroll
    for (int q = 0; q < 7; ++q) lm[q] = (double)lmT[q];
    const double X = g.x0 + (ex + 0.5) * g.h - xs;
    const double Y = g.y0 + (ey + 0.5) * g.h - ys;
    add_element_moments(X, Y, J, lm, acc);
  }
  block_sum7(acc);
  if (threadIdx.x == 0) {
    double *o = part + ((size_t)s * gridDim.x + blockIdx.x) * kMomFields;
#pragma unroll
    for (int f = 0; f < kMomFields; ++f) o[f] = acc[f];
  }
}

// Second pass: one block per density, partials summed in a fixed order;
// writes the six moments [m][6].
__global__ void __launch_bounds__(256)
    k_moments_dense_final(const double *__restrict__ part, int nblk, double *__restrict__ mom) {
  const int s = blockIdx.x;
  double acc[kMomFields] = {0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblk; b += 256) {
    const double *p = part + ((size_t)s * nblk + b) * kMomFields;
#pragma unroll
    for (int f = 0; f < kMomFields; ++f) acc[f] += p[f];
  }
  block_sum7(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int f = 0; f < 6; ++f) mom[(size_t)s * 6 + f] = acc[f];
  }
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double *g_static_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
cudaError_t static_scratch(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_static_mom_partials);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}
}  // namespace

}  // namespace dg

extern "C" int dg_moments_dense_static(const void *u, int precision, int m, int nx, int ny,
                                       int p, double h, double x0, double y0,
                                       const double *xy, double *mom, void *stream) {
  using namespace dg;
  if (!u || !xy || !mom) return DG_EINVAL;
  if (m < 1 || m > kStaticMomMaxDensities) return DG_EINVAL;
  if (p < 1 || p > kMaxP || nx < 1 || ny < 1 || !(h > 0.0)) return DG_EINVAL;
  if (!std::isfinite(h) || !std::isfinite(x0) || !std::isfinite(y0)) return DG_EINVAL;
  if (precision != DG_FP64 && precision != DG_FP32) return DG_EINVAL;
  Gll gl;
  if (!gll_tables(p, &gl)) return DG_EINVAL;
  NodeGeo g;
  for (int i = 0; i <= p; ++i) {
    g.xi[i] = gl.xi[i];
    g.w[i] = gl.w[i];
  }
  g.h = h;
  g.x0 = x0;
  g.y0 = y0;
  // an error that earlier work left pending on this thread is not this
  // call's: report it without consuming it, so that its owner still sees it
  if (cudaPeekAtLastError() != cudaSuccess) return DG_ECUDA;
  double *part = nullptr;
  if (static_scratch(&part) != cudaSuccess) return DG_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 grid(kStaticMomBlocks, (unsigned)m);
  auto launch = [&]() -> cudaError_t {
    if (precision == DG_FP64) {
      DG_P_SWITCH(p, (k_moments_dense<double, PP><<<grid, 256, 0, s>>>(
                         (const double *)u, nx, ny, xy, g, part)));
    } else {
      DG_P_SWITCH(p, (k_moments_dense<float, PP><<<grid, 256, 0, s>>>(
                         (const float *)u, nx, ny, xy, g, part)));
    }
    k_moments_dense_final<<<m, 256, 0, s>>>(part, kStaticMomBlocks, mom);
    return cudaGetLastError();  // nothing was pending before: only these launches
  };
  return launch() == cudaSuccess ? DG_OK : DG_ECUDA;
}
