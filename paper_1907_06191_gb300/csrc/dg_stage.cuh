// dg_stage.cuh -- fused SSP-RK3 stage of the DG diffusion operator.
//
// One thread owns one mesh element of one density: the element's (p+1)^2
// nodal values sit in registers, the four face neighbours are read whole
// (through L1/L2; they are other threads' elements) and the stage result
//   out = alpha u0 + beta u + gamma R(u),   L u = (k / J^2) R(u),
// is written once.  q = grad u is never stored: substituting the gradient
// equation into the divergence equation gives, at node (a, b),
//   R_ab = sum_i (D D)_ai u_ib + sum_j (D D)_bj u_aj                  (volume)
//        + sum over faces f: s_f D_{a,i_f} g_f,b / w                  (lifting)
//        + at face nodes:   F_f,b                                      (flux)
// where, for face f with outward sign s_f and own face column i_f,
//   g = u_hat - u^-  is the jump of the central u-flux (Sec. 3.2),
//   d^- / d^+ = outward normal derivative of the own / neighbour element,
//   interior: g = (u^+ - u^-)/2, F = [(d^+ - d^-)/2 - pen (u^- - u^+)] / w
//   removed-wall: g = 0,          F = -d^- / w             (q_hat = 0)
//   paper wall:   g = -u^-/2,     F = -(d^- + g / w) / w   (k^+ = 0)
//   absorbing edge (Eq. 4): g = -u^-, F = -pen u^- / w
// with pen = eta (p+1)^2 / 2.  These follow from Eq. 7 with GLL quadrature
// (summation by parts) and the fluxes h_u, h_q of Sec. 3.2; for interior
// faces the lifting parts of q^- and q^+ cancel in q_hat - k q^-.
#pragma once

#include "dg_internal.h"

namespace dg {

// Whole-element vector loads.  NC = true reads through the non-coherent
// (read-only) path and is used only for arrays no thread writes during the
// launch.
template <typename T, int NP, bool NC = true>
__device__ __forceinline__ void load_elem(const T *p, T (&u)[NP]) {
  constexpr int B = NP * (int)sizeof(T);
  if constexpr (sizeof(T) == 4 && B % 16 == 0) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int k = 0; k < B / 16; ++k) {
      const float4 v = NC ? __ldg(q + k) : q[k];
      u[4 * k] = v.x; u[4 * k + 1] = v.y; u[4 * k + 2] = v.z; u[4 * k + 3] = v.w;
    }
  } else if constexpr (sizeof(T) == 4 && B % 8 == 0) {
    const float2 *q = reinterpret_cast<const float2 *>(p);
#pragma unroll
    for (int k = 0; k < B / 8; ++k) {
      const float2 v = NC ? __ldg(q + k) : q[k];
      u[2 * k] = v.x; u[2 * k + 1] = v.y;
    }
  } else if constexpr (sizeof(T) == 8 && B % 16 == 0) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int k = 0; k < B / 16; ++k) {
      const double2 v = NC ? __ldg(q + k) : q[k];
      u[2 * k] = v.x; u[2 * k + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < NP; ++k) u[k] = NC ? __ldg(p + k) : p[k];
  }
}

template <typename T, int NP>
__device__ __forceinline__ void store_elem(T *p, const T (&u)[NP]) {
  constexpr int B = NP * (int)sizeof(T);
  if constexpr (sizeof(T) == 4 && B % 16 == 0) {
    float4 *q = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int k = 0; k < B / 16; ++k)
      q[k] = make_float4(u[4 * k], u[4 * k + 1], u[4 * k + 2], u[4 * k + 3]);
  } else if constexpr (sizeof(T) == 4 && B % 8 == 0) {
    float2 *q = reinterpret_cast<float2 *>(p);
#pragma unroll
    for (int k = 0; k < B / 8; ++k) q[k] = make_float2(u[2 * k], u[2 * k + 1]);
  } else if constexpr (sizeof(T) == 8 && B % 16 == 0) {
    double2 *q = reinterpret_cast<double2 *>(p);
#pragma unroll
    for (int k = 0; k < B / 16; ++k) q[k] = make_double2(u[2 * k], u[2 * k + 1]);
  } else {
#pragma unroll
    for (int k = 0; k < NP; ++k) p[k] = u[k];
  }
}

// x-faces: S = +1 east (own column i = P, neighbour column 0),
//          S = -1 west (own column 0, neighbour column P).
template <typename T, int P, int S>
__device__ __forceinline__ void face_x(const T (&u)[(P + 1) * (P + 1)],
                                       T (&R)[(P + 1) * (P + 1)], int nbk,
                                       const T *__restrict__ U, const StageTab<T, P> &tb,
                                       const StageCoef<T> &c) {
  constexpr int n = P + 1, NP = n * n;
  constexpr int i_f = S > 0 ? P : 0, i_n = S > 0 ? 0 : P;
  const T sg = (T)S;
  T g[n];
  if (nbk >= 0) {
    T v[NP];
    load_elem<T, NP>(U + (size_t)nbk * NP, v);
#pragma unroll
    for (int b = 0; b < n; ++b) {
      T dm = 0, dp = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        dm += tb.D[i_f * n + m] * u[b * n + m];
        dp += tb.D[i_n * n + m] * v[b * n + m];
      }
      const T um = u[b * n + i_f], up = v[b * n + i_n];
      g[b] = (T)0.5 * (up - um);
      R[b * n + i_f] += tb.inv_w * ((T)0.5 * sg * (dp - dm) - c.pen * (um - up));
    }
  } else if (nbk == kWall && !c.wallA) {
#pragma unroll
    for (int b = 0; b < n; ++b) {
      T dm = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) dm += tb.D[i_f * n + m] * u[b * n + m];
      R[b * n + i_f] -= tb.inv_w * sg * dm;
    }
    return;  // g = 0: no lifting
  } else if (nbk == kWall) {
#pragma unroll
    for (int b = 0; b < n; ++b) {
      T dm = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) dm += tb.D[i_f * n + m] * u[b * n + m];
      g[b] = (T)-0.5 * u[b * n + i_f];
      R[b * n + i_f] -= tb.inv_w * (sg * dm + tb.inv_w * g[b]);
    }
  } else {
#pragma unroll
    for (int b = 0; b < n; ++b) {
      const T um = u[b * n + i_f];
      g[b] = -um;
      R[b * n + i_f] -= tb.inv_w * c.pen * um;
    }
  }
#pragma unroll
  for (int b = 0; b < n; ++b) {
    const T gs = sg * tb.inv_w * g[b];
#pragma unroll
    for (int a = 0; a < n; ++a) R[b * n + a] += tb.D[a * n + i_f] * gs;
  }
}

// y-faces: S = +1 north (own row j = P, neighbour row 0),
//          S = -1 south (own row 0, neighbour row P).
template <typename T, int P, int S>
__device__ __forceinline__ void face_y(const T (&u)[(P + 1) * (P + 1)],
                                       T (&R)[(P + 1) * (P + 1)], int nbk,
                                       const T *__restrict__ U, const StageTab<T, P> &tb,
                                       const StageCoef<T> &c) {
  constexpr int n = P + 1, NP = n * n;
  constexpr int j_f = S > 0 ? P : 0, j_n = S > 0 ? 0 : P;
  const T sg = (T)S;
  T g[n];
  if (nbk >= 0) {
    T v[NP];
    load_elem<T, NP>(U + (size_t)nbk * NP, v);
#pragma unroll
    for (int a = 0; a < n; ++a) {
      T dm = 0, dp = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) {
        dm += tb.D[j_f * n + m] * u[m * n + a];
        dp += tb.D[j_n * n + m] * v[m * n + a];
      }
      const T um = u[j_f * n + a], up = v[j_n * n + a];
      g[a] = (T)0.5 * (up - um);
      R[j_f * n + a] += tb.inv_w * ((T)0.5 * sg * (dp - dm) - c.pen * (um - up));
    }
  } else if (nbk == kWall && !c.wallA) {
#pragma unroll
    for (int a = 0; a < n; ++a) {
      T dm = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) dm += tb.D[j_f * n + m] * u[m * n + a];
      R[j_f * n + a] -= tb.inv_w * sg * dm;
    }
    return;
  } else if (nbk == kWall) {
#pragma unroll
    for (int a = 0; a < n; ++a) {
      T dm = 0;
#pragma unroll
      for (int m = 0; m < n; ++m) dm += tb.D[j_f * n + m] * u[m * n + a];
      g[a] = (T)-0.5 * u[j_f * n + a];
      R[j_f * n + a] -= tb.inv_w * (sg * dm + tb.inv_w * g[a]);
    }
  } else {
#pragma unroll
    for (int a = 0; a < n; ++a) {
      const T um = u[j_f * n + a];
      g[a] = -um;
      R[j_f * n + a] -= tb.inv_w * c.pen * um;
    }
  }
#pragma unroll
  for (int a = 0; a < n; ++a) {
    const T gs = sg * tb.inv_w * g[a];
#pragma unroll
    for (int b = 0; b < n; ++b) R[b * n + a] += tb.D[b * n + j_f] * gs;
  }
}

// grid: (ceil(nA / kBlock), m); density s = blockIdx.y starts at s * stride
// elements.  nb entries are < nA (checked when the table is built).  out may
// alias u0 (the last stage updates u^n in place: each thread reads its own
// element of u0 before writing the same element); it never aliases uin.
template <typename T, int P, bool HAS_U0>
__global__ void __launch_bounds__(kBlock)
    k_stage(const T *__restrict__ uin, const T *u0, T *out,
            const int4 *__restrict__ nb, long long nA, long long stride,
            const StageTab<T, P> tb, const StageCoef<T> c) {
  constexpr int n = P + 1, NP = n * n;
  const long long a = (long long)blockIdx.x * kBlock + threadIdx.x;
  if (a >= nA) return;
  const size_t sbase = (size_t)blockIdx.y * (size_t)stride * NP;
  const T *U = uin + sbase;
  T u[NP], R[NP];
  load_elem<T, NP>(U + (size_t)a * NP, u);
  const int4 f = __ldg(nb + a);
#pragma unroll
  for (int j = 0; j < n; ++j)
#pragma unroll
    for (int i = 0; i < n; ++i) {
      T s = 0;
#pragma unroll
      for (int m = 0; m < n; ++m)
        s += tb.D2[i * n + m] * u[j * n + m] + tb.D2[j * n + m] * u[m * n + i];
      R[j * n + i] = s;
    }
  face_x<T, P, +1>(u, R, f.x, U, tb, c);
  face_x<T, P, -1>(u, R, f.y, U, tb, c);
  face_y<T, P, +1>(u, R, f.z, U, tb, c);
  face_y<T, P, -1>(u, R, f.w, U, tb, c);
  T o[NP];
  if constexpr (HAS_U0) {
    load_elem<T, NP, false>(u0 + sbase + (size_t)a * NP, o);
#pragma unroll
    for (int k = 0; k < NP; ++k) o[k] = c.alpha * o[k] + c.beta * u[k] + c.gamma * R[k];
  } else {
#pragma unroll
    for (int k = 0; k < NP; ++k) o[k] = c.beta * u[k] + c.gamma * R[k];
  }
  store_elem<T, NP>(out + sbase + (size_t)a * NP, o);
}

template <typename T, int P>
StageTab<T, P> make_tab(const Gll &g) {
  StageTab<T, P> t;
  constexpr int n = P + 1;
  for (int k = 0; k < n * n; ++k) {
    t.D[k] = (T)g.D[k];
    t.D2[k] = (T)g.D2[k];
  }
  t.inv_w = (T)(1.0 / g.w[0]);
  return t;
}

template <typename T, int P>
cudaError_t launch_stage_p(const T *u, const T *u0, T *out, const int4 *nb, long long nA,
                           long long stride, int m, const Gll &g, const StageCoef<T> &c,
                           cudaStream_t s) {
  if (nA <= 0 || m <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((nA + kBlock - 1) / kBlock), (unsigned)m);
  const StageTab<T, P> tb = make_tab<T, P>(g);
  if (u0)
    k_stage<T, P, true><<<grid, kBlock, 0, s>>>(u, u0, out, nb, nA, stride, tb, c);
  else
    k_stage<T, P, false><<<grid, kBlock, 0, s>>>(u, u0, out, nb, nA, stride, tb, c);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stage_any(int p, const T *u, const T *u0, T *out, const int4 *nb,
                             long long nA, long long stride, int m, const Gll &g,
                             const StageCoef<T> &c, cudaStream_t s) {
  switch (p) {
    case 1: return launch_stage_p<T, 1>(u, u0, out, nb, nA, stride, m, g, c, s);
    case 2: return launch_stage_p<T, 2>(u, u0, out, nb, nA, stride, m, g, c, s);
    case 3: return launch_stage_p<T, 3>(u, u0, out, nb, nA, stride, m, g, c, s);
    case 4: return launch_stage_p<T, 4>(u, u0, out, nb, nA, stride, m, g, c, s);
    case 5: return launch_stage_p<T, 5>(u, u0, out, nb, nA, stride, m, g, c, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
