// dg_tri.cu -- SSP-RK3 stage on the paper's pixel triangles (Sec. 3.3).
//
// One thread owns one pixel (its two triangles A and B, 2 N nodal values,
// N = (p+1)(p+2)/2) of one density.  With a full (non-diagonal) mass matrix
// the lifted gradient of a neighbour depends on that neighbour's other faces,
// so the stage runs in two passes:
//   pass Q: q = grad u with the central flux u_hat = (u^- + u^+)/2 (Eq. 7,
//           first line), written to a q buffer (4 N values per pixel);
//   pass R: R = div q with the harmonic-mean flux of Sec. 3.2 (second line),
//           then out = u0 + beta (u - u0) + gamma R as for the square elements.
// Both passes use the pixel neighbour tables of the square mesh: a pixel's
// east / west / north / south faces are the edges A e1 / B e2 / B e1 / A e0,
// and the diagonal joins A e2 and B e0 inside the pixel.  Matching edges run
// in opposite directions, so node t of an edge meets node p - t across it.
// Face records in shared memory carry, per pixel face, the trace of u (pass Q)
// or of q . n (pass R) at the p + 1 edge nodes.
#include "dg_internal.h"
#include "dg_stage.cuh"

namespace dg {

template <int P>
struct TriShape {
  static constexpr int N = (P + 1) * (P + 2) / 2, NE = P + 1, NPX = 2 * N;
  __host__ __device__ static constexpr int idx(int i, int j) { return j * (P + 1) - j * (j - 1) / 2 + i; }
  __host__ __device__ static constexpr int en(int e, int t) {
    return e == 0 ? idx(t, 0) : (e == 1 ? idx(P - t, t) : idx(0, P - t));
  }
  // pixel face f -> (triangle, edge)
  __host__ __device__ static constexpr int ftri(int f) { return (f == 0 || f == 3) ? 0 : 1; }
  __host__ __device__ static constexpr int fedge(int f) { return f == 0 ? 1 : (f == 1 ? 2 : (f == 2 ? 1 : 0)); }
};

// FP32 staging of a chunk's q (4 N values per pixel = N 16-byte slots) in
// shared memory, so that the q pass stores and the divergence pass loads it
// with coalesced 16-byte pieces.  A pixel takes SP slots (N rounded up to an
// odd count, so that 16-byte accesses of 8 consecutive threads hit 8 bank
// groups); triangle o's q_x, q_y are its slots o N/2 .. o N/2 + N/2 - 1.
// Needs N even (p = 2, 3).
template <typename T, int P>
struct TriQStage {
  static constexpr int N = TriShape<P>::N;
  static constexpr bool ON = sizeof(T) == 4 && N % 2 == 0;
  static constexpr int S = N, SP = (N % 2 == 0) ? N + 1 : N, HALF = N / 2;
  static constexpr int BYTES = ON ? kBlock * SP * 16 : 0;
  __device__ static __forceinline__ void put(float4 *sq, int el, int o, const T (&qx)[N],
                                             const T (&qy)[N]) {
#pragma unroll
    for (int k = 0; k < HALF; ++k) {
      float v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int w = 4 * k + q;
        v[q] = w < N ? qx[w] : qy[w - N];
      }
      sq[el * SP + o * HALF + k] = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
  __device__ static __forceinline__ void get(const float4 *sq, int el, int o, T (&qx)[N],
                                             T (&qy)[N]) {
#pragma unroll
    for (int k = 0; k < HALF; ++k) {
      const float4 f = sq[el * SP + o * HALF + k];
      const float v[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int w = 4 * k + q;
        if (w < N) qx[w] = v[q];
        else qy[w - N] = v[q];
      }
    }
  }
};

__host__ __device__ constexpr int tri_rec_bytes(int nrec, int ne, int tsize) {
  return (nrec * ne * tsize + 15) / 16 * 16;
}

template <typename T, int P>
struct TriTab {
  static constexpr int N = TriShape<P>::N, NE = TriShape<P>::NE;
  using T2 = typename Vec2<T>::type;
  T G[2][2][N * N];
  T Lf[2][3][N * NE];
  T nrm[2][3][2];
  // rows 2ip and 2ip + 1 of G side by side, for the packed two-lane FP32
  // instructions: Gp[o][c][ip N + j] = (G[o][c][2ip][j], G[o][c][2ip + 1][j])
  T2 Gp[2][2][(N / 2) * N];
  // the liftings likewise: Lfp[o][e][ip NE + t] = (Lf[o][e][2ip][t], Lf[o][e][2ip + 1][t])
  T2 Lfp[2][3][(N / 2) * NE];
};

template <typename T, int P>
TriTab<T, P> make_tri_tab(const TriRef &r) {
  TriTab<T, P> t;
  constexpr int N = TriShape<P>::N, NE = TriShape<P>::NE;
  for (int o = 0; o < 2; ++o) {
    for (int c = 0; c < 2; ++c)
      for (int k = 0; k < N * N; ++k) t.G[o][c][k] = (T)r.G[o][c][k];
    for (int c = 0; c < 2; ++c)
      for (int ip = 0; ip < N / 2; ++ip)
        for (int j = 0; j < N; ++j) {
          t.Gp[o][c][ip * N + j].x = t.G[o][c][2 * ip * N + j];
          t.Gp[o][c][ip * N + j].y = t.G[o][c][(2 * ip + 1) * N + j];
        }
    for (int e = 0; e < 3; ++e) {
      for (int k = 0; k < N * NE; ++k) t.Lf[o][e][k] = (T)r.Lf[o][e][k];
      for (int ip = 0; ip < N / 2; ++ip)
        for (int q = 0; q < NE; ++q) {
          t.Lfp[o][e][ip * NE + q].x = t.Lf[o][e][2 * ip * NE + q];
          t.Lfp[o][e][ip * NE + q].y = t.Lf[o][e][(2 * ip + 1) * NE + q];
        }
      t.nrm[o][e][0] = (T)r.nrm[o][e][0];
      t.nrm[o][e][1] = (T)r.nrm[o][e][1];
    }
  }
  return t;
}

// y[i] += sum_t L[i*NE + t] v[t]
template <typename T, int N, int NE>
__device__ __forceinline__ void lift_add(const T *L, const T (&v)[NE], T s, T (&y)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T a = 0;
#pragma unroll
    for (int t = 0; t < NE; ++t) a += L[i * NE + t] * v[t];
    y[i] += s * a;
  }
}

// Shared set-up of both passes: chunk, element, record slots.
struct TriBlock {
  int chunk, el, cnt, hcnt, geo;
  long long a0;
  bool live;
  int4 l4;
};

__device__ __forceinline__ TriBlock tri_block(const int *chunk_list, const int2 *chunk_tab,
                                              const int4 *loc, const int *halo_cnt) {
  TriBlock b;
  b.chunk = chunk_list ? __ldg(chunk_list + blockIdx.x) : (int)blockIdx.x;
  b.a0 = (long long)b.chunk * kBlock;
  const int2 ci = __ldg(chunk_tab + b.chunk);
  b.cnt = ci.x;
  b.geo = ci.y;
  b.el = threadIdx.x;
  b.live = b.el < b.cnt;
  b.l4 = b.live ? __ldg(loc + b.a0 + b.el) : make_int4(kEdge, kEdge, kEdge, kEdge);
  b.hcnt = __ldg(halo_cnt + b.chunk);
  return b;
}

__device__ __forceinline__ int tri_rec_index(int L, int f, int el, int zero_rec) {
  return L >= kBlock ? 4 * kBlock + (L - kBlock) : (L >= 0 ? (f ^ 1) * kBlock + L : zero_rec);
}

// Register budget per thread: 64 in FP32, 128 in FP64.
template <typename T>
constexpr int tri_min_blocks() { return blocks_for_regs(sizeof(T) == 4 ? 64 : 128); }

// ---- per-triangle pieces shared by the kernels ----------------------------------
// Each is inlined where it is used, so the q pass, the divergence pass and the
// fused stage run the same expressions in the same order (the same bits).

// Face f of a pixel: edge e of triangle o (inverse of ftri / fedge).
__host__ __device__ constexpr int tri_face(int o, int e) {
  return o == 0 ? (e == 1 ? 0 : 3) : (e == 2 ? 1 : 2);
}
__host__ __device__ constexpr bool tri_diag(int o, int e) { return (o == 0 && e == 2) || (o == 1 && e == 0); }

// Packed two-lane FP32 for the element matrices where N is even (p = 2, 3):
// two rows per instruction, each lane rounded like the scalar fused
// multiply-add, in the same order.
template <typename T, int P>
constexpr bool kTriPacked = sizeof(T) == 4 && TriShape<P>::N % 2 == 0;

// q = grad u of triangle o, volume part: q = G u.
template <typename T, int P>
__device__ __forceinline__ void tri_q_volume(const TriTab<T, P> &tb, int o,
                                             const T (&uo)[TriShape<P>::N],
                                             T (&qx)[TriShape<P>::N], T (&qy)[TriShape<P>::N]) {
  constexpr int N = TriShape<P>::N;
  if constexpr (kTriPacked<T, P>) {
#pragma unroll
    for (int ip = 0; ip < N / 2; ++ip) {
      float2 ax = make_float2(0.0f, 0.0f), ay = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float2 uj = make_float2(uo[j], uo[j]);
        ax = __ffma2_rn(tb.Gp[o][0][ip * N + j], uj, ax);
        ay = __ffma2_rn(tb.Gp[o][1][ip * N + j], uj, ay);
      }
      qx[2 * ip] = ax.x;
      qx[2 * ip + 1] = ax.y;
      qy[2 * ip] = ay.x;
      qy[2 * ip + 1] = ay.y;
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T ax = 0, ay = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      ax += tb.G[o][0][i * N + j] * uo[j];
      ay += tb.G[o][1][i * N + j] * uo[j];
    }
    qx[i] = ax;
    qy[i] = ay;
  }
}

// u-flux of edge e at its nodes: the diagonal's mean of both triangles'
// traces (dg[o], dg[1 - o], each in its own edge order), or across a pixel
// face cm u^- + cp u^+ with the neighbour's trace nb in its own edge order.
template <typename T, int P>
__device__ __forceinline__ void tri_uh(int o, int e, const T (&uo)[TriShape<P>::N],
                                       const T (&dg)[2][P + 1], T cm, T cp, const T (&nb)[P + 1],
                                       T (&uh)[P + 1]) {
  using S = TriShape<P>;
  const T half = (T)0.5;
  if (tri_diag(o, e)) {
#pragma unroll
    for (int t = 0; t < P + 1; ++t) uh[t] = half * (dg[o][t] + dg[1 - o][P - t]);
  } else {
#pragma unroll
    for (int t = 0; t < P + 1; ++t) uh[t] = cm * uo[S::en(e, t)] + cp * nb[P - t];
  }
}

// q += n_e (Lf_e uh): the lifting of edge e's u-flux.
template <typename T, int P>
__device__ __forceinline__ void tri_q_edge(const TriTab<T, P> &tb, int o, int e,
                                           const T (&uh)[P + 1], T (&qx)[TriShape<P>::N],
                                           T (&qy)[TriShape<P>::N]) {
  constexpr int N = TriShape<P>::N, NE = P + 1;
  if constexpr (kTriPacked<T, P>) {
    const float2 n0 = make_float2(tb.nrm[o][e][0], tb.nrm[o][e][0]);
    const float2 n1 = make_float2(tb.nrm[o][e][1], tb.nrm[o][e][1]);
#pragma unroll
    for (int ip = 0; ip < N / 2; ++ip) {
      float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int t = 0; t < NE; ++t) a = __ffma2_rn(tb.Lfp[o][e][ip * NE + t], make_float2(uh[t], uh[t]), a);
      const float2 x = __ffma2_rn(n0, a, make_float2(qx[2 * ip], qx[2 * ip + 1]));
      const float2 y = __ffma2_rn(n1, a, make_float2(qy[2 * ip], qy[2 * ip + 1]));
      qx[2 * ip] = x.x;
      qx[2 * ip + 1] = x.y;
      qy[2 * ip] = y.x;
      qy[2 * ip + 1] = y.y;
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T a = 0;
#pragma unroll
    for (int t = 0; t < NE; ++t) a += tb.Lf[o][e][i * NE + t] * uh[t];
    qx[i] += tb.nrm[o][e][0] * a;
    qy[i] += tb.nrm[o][e][1] * a;
  }
}

// Weights of u^- and u^+ across a pixel face with neighbour code L.
template <typename T>
__device__ __forceinline__ void tri_uflux_weights(int L, int wallA, T &cm, T &cp) {
  const T half = (T)0.5;
  cp = L >= 0 ? half : (T)0;                                         // weight of u+
  cm = L >= 0 ? half : (L == kWall ? (wallA ? half : (T)1) : (T)0);  // of u-
}

// q . n (outward normal of triangle o, edge e) at the edge's node t.
template <typename T, int P>
__device__ __forceinline__ T tri_qn(const TriTab<T, P> &tb, const T (&qx)[TriShape<P>::N],
                                    const T (&qy)[TriShape<P>::N], int o, int e, int t) {
  const int k = TriShape<P>::en(e, t);
  return qx[k] * tb.nrm[o][e][0] + qy[k] * tb.nrm[o][e][1];
}

// ---- pass Q -------------------------------------------------------------------
// One triangle at a time: only its N values, its q and the diagonal traces of
// both triangles are live, which keeps the FP32 kernel within 64 registers.
template <typename T, int P>
__global__ void __launch_bounds__(kBlock, tri_min_blocks<T>())
    k_tri_q(const T *__restrict__ uin, T *__restrict__ qout, const int4 *__restrict__ loc,
            const int2 *__restrict__ halo, const int *__restrict__ halo_cnt,
            const int2 *__restrict__ chunk_tab, long long stride, int nrec,
            const int *__restrict__ chunk_list, const TriTab<T, P> tb, int wallA) {
  using S = TriShape<P>;
  constexpr int N = S::N, NE = S::NE, NPX = S::NPX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *rec = reinterpret_cast<T *>(smem_raw);
  const int zero_rec = nrec - 1;
  const TriBlock b = tri_block(chunk_list, chunk_tab, loc, halo_cnt);
  const size_t sbase = (size_t)blockIdx.y * (size_t)stride;
  const T *U = uin + sbase * NPX;
  const T *Ue = U + (size_t)(b.a0 + b.el) * NPX;

  T dg[2][NE];  // diagonal traces: A e2 and B e0, each in its own edge order
  if (b.live) {
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      T uo[N];
      load_elem<T, N>(Ue + o * N, uo);
#pragma unroll
      for (int f = 0; f < 4; ++f)
        if (S::ftri(f) == o)
#pragma unroll
          for (int t = 0; t < NE; ++t) rec[(f * kBlock + b.el) * NE + t] = uo[S::en(S::fedge(f), t)];
#pragma unroll
      for (int t = 0; t < NE; ++t) dg[o][t] = uo[S::en(o == 0 ? 2 : 0, t)];
    }
  }
  if (b.el == 0)
    for (int t = 0; t < NE; ++t) rec[zero_rec * NE + t] = (T)0;
  for (int h = b.el; h < b.hcnt; h += kBlock) {
    const int2 q = __ldg(halo + (size_t)b.chunk * kHaloCap + h);
    const int o = (q.y == 0 || q.y == 3) ? 0 : 1;  // the triangle that owns the face
    T v[N];
    load_elem<T, N>(U + (size_t)q.x * NPX + o * N, v);
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (q.y == f)
#pragma unroll
        for (int t = 0; t < NE; ++t) rec[(4 * kBlock + h) * NE + t] = v[S::en(S::fedge(f), t)];
  }
  __syncthreads();
  using QS = TriQStage<T, P>;
  if (!QS::ON && !b.live) return;
  float4 *sq = reinterpret_cast<float4 *>(smem_raw + tri_rec_bytes(nrec, NE, (int)sizeof(T)));

  const int lq[4] = {b.l4.x, b.l4.y, b.l4.z, b.l4.w};
  T *Q = qout + (sbase + (size_t)(b.a0 + b.el)) * (4 * N);
#pragma unroll 1
  for (int o = 0; o < 2 && b.live; ++o) {
    T uo[N];
    load_elem<T, N>(Ue + o * N, uo);
    T qx[N], qy[N];
    tri_q_volume<T, P>(tb, o, uo, qx, qy);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      T uh[NE], nb[NE];
      T cm = 0, cp = 0;
      if (!tri_diag(o, e)) {
        const int f = tri_face(o, e);
        const int L = lq[f];
        const int rn = tri_rec_index(L, f, b.el, zero_rec);
        tri_uflux_weights<T>(L, wallA, cm, cp);
#pragma unroll
        for (int t = 0; t < NE; ++t) nb[t] = rec[rn * NE + t];
      }
      tri_uh<T, P>(o, e, uo, dg, cm, cp, nb, uh);
      tri_q_edge<T, P>(tb, o, e, uh, qx, qy);
    }
    if constexpr (QS::ON) {
      QS::put(sq, b.el, o, qx, qy);
    } else {
      store_elem<T, N>(Q + (2 * o) * N, qx);
      store_elem<T, N>(Q + (2 * o + 1) * N, qy);
    }
  }
  if constexpr (QS::ON) {  // coalesced 16-byte stores of the chunk's q
    __syncthreads();
    float4 *gq = reinterpret_cast<float4 *>(qout + (sbase + (size_t)b.a0) * (4 * N));
    for (int j = b.el; j < b.cnt * QS::S; j += kBlock)
      gq[j] = sq[(j / QS::S) * QS::SP + j % QS::S];
  }
}

// ---- divergence and stage update of one pixel ------------------------------------
// From its q (load_q(o, qx, qy)), the q . n records of its faces and of its
// neighbours (rec: records f kBlock + el, 4 kBlock + halo slot, the zero
// record) and the diagonal q . n of both triangles (dg): R = div q with the
// harmonic-mean flux of Sec. 3.2, then out = u0 + beta (u - u0) + gamma R.
template <typename T, int P, bool HAS_U0, bool SROUND, typename LoadQ>
__device__ __forceinline__ void tri_finish(const TriBlock &b, LoadQ load_q, const T *rec,
                                           int zero_rec, const T (&dg)[2][P + 1],
                                           const TriTab<T, P> &tb, const StageCoef<T> &c,
                                           const T *__restrict__ uin, const T *u0, T *out,
                                           size_t sbase, const int2 *__restrict__ grange,
                                           const T *__restrict__ gscale,
                                           const uint8_t *__restrict__ adv) {
  using S = TriShape<P>;
  constexpr int N = S::N, NE = S::NE, NPX = S::NPX;
  const int lq[4] = {b.l4.x, b.l4.y, b.l4.z, b.l4.w};
  const T half = (T)0.5;
  // gamma is beta dt D / J^2 with J = h/2 of the square elements: 1/h^2 = gscale / 4
  T gam = c.gamma * (T)0.25 * __ldg(gscale + b.geo);
  if (adv != nullptr && __ldg(adv + b.a0 + b.el) == 0) gam = (T)0;
  const size_t off = (sbase + (size_t)(b.a0 + b.el)) * NPX;
  uint32_t hkey = 0;
#pragma unroll 1
  for (int o = 0; o < 2; ++o) {
    T R[N];
    {
      T qx[N], qy[N];
      load_q(o, qx, qy);
      if constexpr (kTriPacked<T, P>) {
#pragma unroll
        for (int ip = 0; ip < N / 2; ++ip) {
          float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int j = 0; j < N; ++j)
            a = __ffma2_rn(tb.Gp[o][1][ip * N + j], make_float2(qy[j], qy[j]),
                           __ffma2_rn(tb.Gp[o][0][ip * N + j], make_float2(qx[j], qx[j]), a));
          R[2 * ip] = a.x;
          R[2 * ip + 1] = a.y;
        }
      } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          T a = 0;
#pragma unroll
          for (int j = 0; j < N; ++j)
            a = fmaT(tb.G[o][1][i * N + j], qy[j], fmaT(tb.G[o][0][i * N + j], qx[j], a));
          R[i] = a;
        }
      }
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      T hn[NE];  // the normal flux h_q . n / k at the edge nodes
      if (tri_diag(o, e)) {
#pragma unroll
        for (int t = 0; t < NE; ++t) hn[t] = half * (dg[o][t] - dg[1 - o][P - t]);
      } else {
        const int f = tri_face(o, e);
        const int L = lq[f];
        const int rn = tri_rec_index(L, f, b.el, zero_rec);
        // interior: (q- . n - q+ . n+) / 2; wall: 0; absorbing edge: q- . n
        const T cm = L >= 0 ? half : (L == kEdge ? (T)1 : (T)0);
        const T cp = L >= 0 ? -half : (T)0;
#pragma unroll
        for (int t = 0; t < NE; ++t) hn[t] = cm * rec[(f * kBlock + b.el) * NE + t] + cp * rec[rn * NE + (P - t)];
      }
      if constexpr (kTriPacked<T, P>) {
#pragma unroll
        for (int ip = 0; ip < N / 2; ++ip) {
          float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
          for (int t = 0; t < NE; ++t) a = __ffma2_rn(tb.Lfp[o][e][ip * NE + t], make_float2(hn[t], hn[t]), a);
          const float2 r2 = __fadd2_rn(make_float2(R[2 * ip], R[2 * ip + 1]), a);
          R[2 * ip] = r2.x;
          R[2 * ip + 1] = r2.y;
        }
      } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          T a = 0;
#pragma unroll
          for (int t = 0; t < NE; ++t) a += tb.Lf[o][e][i * NE + t] * hn[t];
          R[i] += a;
        }
      }
    }
    T u[N], w[N];
    load_elem<T, N>(uin + off + o * N, u);
    if constexpr (HAS_U0) load_elem<T, N, false>(u0 + off + o * N, w);
    if constexpr (SROUND) {
      if (o == 0)
        hkey = fmix32(((uint32_t)(b.a0 + b.el - __ldg(grange + b.geo).x) * (uint32_t)NPX) ^
                      ((uint32_t)blockIdx.y * 0x632be5abu) ^ __float_as_uint(u[0]) ^
                      (__float_as_uint(u[1]) * 0x85ebca77u));
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T base = HAS_U0 ? w[k] : c.beta * u[k];
        const T inc = HAS_U0 ? fmaf(c.beta, u[k] - w[k], gam * R[k]) : gam * R[k];
        w[k] = add_stochastic(base, inc, hkey + (uint32_t)(o * N + k));
      }
    } else if constexpr (HAS_U0) {
#pragma unroll
      for (int k = 0; k < N; ++k) w[k] = w[k] + c.beta * (u[k] - w[k]) + gam * R[k];
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) w[k] = c.beta * u[k] + gam * R[k];
    }
    store_elem<T, N>(out + off + o * N, w);
  }
}

// q . n records of the pixel's own faces (record f kBlock + el) and its
// diagonal q . n (dg), from its q.
template <typename T, int P, typename LoadQ>
__device__ __forceinline__ void tri_qn_records(const TriBlock &b, LoadQ load_q, T *rec,
                                               const TriTab<T, P> &tb, T (&dg)[2][P + 1]) {
  using S = TriShape<P>;
  constexpr int N = S::N, NE = S::NE;
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    T qx[N], qy[N];
    load_q(o, qx, qy);
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (S::ftri(f) == o)
#pragma unroll
        for (int t = 0; t < NE; ++t)
          rec[(f * kBlock + b.el) * NE + t] = tri_qn<T, P>(tb, qx, qy, o, S::fedge(f), t);
#pragma unroll
    for (int t = 0; t < NE; ++t) dg[o][t] = tri_qn<T, P>(tb, qx, qy, o, o == 0 ? 2 : 0, t);
  }
}

// ---- pass R + stage update ------------------------------------------------------
template <typename T, int P, bool HAS_U0, bool SROUND>
__global__ void __launch_bounds__(kBlock, tri_min_blocks<T>())
    k_tri_r(const T *__restrict__ qin, const T *__restrict__ uin, const T *u0, T *out,
            const int4 *__restrict__ loc, const int2 *__restrict__ halo,
            const int *__restrict__ halo_cnt, const int2 *__restrict__ chunk_tab,
            const int2 *__restrict__ grange, const T *__restrict__ gscale, long long stride,
            int nrec, const int *__restrict__ chunk_list, const uint8_t *__restrict__ adv,
            const TriTab<T, P> tb, const StageCoef<T> c) {
  using S = TriShape<P>;
  constexpr int N = S::N, NE = S::NE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *rec = reinterpret_cast<T *>(smem_raw);
  const int zero_rec = nrec - 1;
  const TriBlock b = tri_block(chunk_list, chunk_tab, loc, halo_cnt);
  const size_t sbase = (size_t)blockIdx.y * (size_t)stride;
  const T *Qb = qin + sbase * (4 * N);
  const T *Qe = Qb + (size_t)(b.a0 + b.el) * (4 * N);
  using QS = TriQStage<T, P>;
  float4 *sq = reinterpret_cast<float4 *>(smem_raw + tri_rec_bytes(nrec, NE, (int)sizeof(T)));
  if constexpr (QS::ON) {  // coalesced 16-byte copies of the chunk's q
    const char *gq = reinterpret_cast<const char *>(Qb + (size_t)b.a0 * (4 * N));
    for (int j = b.el; j < b.cnt * QS::S; j += kBlock)
      cp_async16(sq + (j / QS::S) * QS::SP + j % QS::S, gq + 16 * (size_t)j);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
  }
  auto load_q = [&](int o, T (&qx)[N], T (&qy)[N]) {
    if constexpr (QS::ON) {
      QS::get(sq, b.el, o, qx, qy);
    } else {
      load_elem<T, N>(Qe + (2 * o) * N, qx);
      load_elem<T, N>(Qe + (2 * o + 1) * N, qy);
    }
  };
  T dg[2][NE];  // q . n on the diagonal of A (e2) and of B (e0)
  if (b.live) tri_qn_records<T, P>(b, load_q, rec, tb, dg);
  if (b.el == 0)
    for (int t = 0; t < NE; ++t) rec[zero_rec * NE + t] = (T)0;
  for (int h = b.el; h < b.hcnt; h += kBlock) {
    const int2 hq = __ldg(halo + (size_t)b.chunk * kHaloCap + h);
    const int o = (hq.y == 0 || hq.y == 3) ? 0 : 1;
    T qx[N], qy[N];
    load_elem<T, N>(Qb + (size_t)hq.x * (4 * N) + (2 * o) * N, qx);
    load_elem<T, N>(Qb + (size_t)hq.x * (4 * N) + (2 * o + 1) * N, qy);
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (hq.y == f)
#pragma unroll
        for (int t = 0; t < NE; ++t) rec[(4 * kBlock + h) * NE + t] = tri_qn<T, P>(tb, qx, qy, o, S::fedge(f), t);
  }
  __syncthreads();
  if (!b.live) return;
  tri_finish<T, P, HAS_U0, SROUND>(b, load_q, rec, zero_rec, dg, tb, c, uin, u0, out, sbase,
                                   grange, gscale, adv);
}

// ---- one launch per stage (FP32, p = 2, 3) ------------------------------------------
// Both passes in one block, q never written to global memory.  The chunk's q
// stays in the shared-memory staging; the divergence also needs q . n of each
// halo triangle (the neighbour triangle across a chunk face), so the block
// computes that triangle's q again from its values, the diagonal trace of its
// pixel's other triangle, the chunk pixel's trace and the trace of its third
// neighbour (the per-chunk table d_htri names them) -- by the same inlined
// arithmetic as the q pass, so the stage gives the bits of the two launches.
// A thread computes the q . n of its halo entry first, from device memory
// alone (the chunk pixel's trace included), so that only those P + 1 values
// stay live through the chunk's own work.  Records hold u traces first, then
// (after the barrier behind the last read of a u trace) q . n; a thread's first
// halo q . n waits in registers, the entries past kBlock in a small area
// behind the q staging.
template <typename T, int P>
struct TriHaloIn {
  T uo[TriShape<P>::N];  // the halo triangle's values
  T od[P + 1];           // the diagonal trace of its pixel's other triangle
  T tc[P + 1];           // the chunk pixel's trace across the face toward the chunk
  T t3[P + 1];           // the third neighbour's trace across the triangle's other face (or 0)
};

// Third pixel face of the triangle that owns face fk (A: east, south; B: west, north).
__host__ __device__ constexpr int tri_third_face(int fk) {
  return fk == 0 ? 3 : (fk == 3 ? 0 : (fk == 1 ? 2 : 1));
}

// The halo entry's inputs, face FK of the halo pixel toward the chunk (a
// template argument, so that every register array is indexed by constants).
template <typename T, int P, int FK>
__device__ __forceinline__ void tri_halo_load(const T *U, long long a0, const int4 e,
                                              TriHaloIn<T, P> &hi) {
  using S = TriShape<P>;
  constexpr int N = S::N, NE = S::NE, NPX = S::NPX;
  constexpr int o = S::ftri(FK);
  load_elem<T, N>(U + (size_t)e.x * NPX + o * N, hi.uo);
  T ot[N];
  load_elem<T, N>(U + (size_t)e.x * NPX + (1 - o) * N, ot);
#pragma unroll
  for (int t = 0; t < NE; ++t) hi.od[t] = ot[S::en(o == 0 ? 0 : 2, t)];
  {
    constexpr int fc = FK ^ 1;  // the chunk pixel's face toward the halo pixel
    T vc[N];
    load_elem<T, N>(U + (size_t)(a0 + e.z) * NPX + S::ftri(fc) * N, vc);
#pragma unroll
    for (int t = 0; t < NE; ++t) hi.tc[t] = vc[S::en(S::fedge(fc), t)];
  }
  if (e.w >= 0) {
    constexpr int fb = tri_third_face(FK) ^ 1;  // the third neighbour's face toward the halo pixel
    T v3[N];
    load_elem<T, N>(U + (size_t)e.w * NPX + S::ftri(fb) * N, v3);
#pragma unroll
    for (int t = 0; t < NE; ++t) hi.t3[t] = v3[S::en(S::fedge(fb), t)];
  } else {
#pragma unroll
    for (int t = 0; t < NE; ++t) hi.t3[t] = (T)0;
  }
}

// q . n of the halo triangle at its face FK toward the chunk (in that face's
// edge order), as the q pass computes it in the halo pixel's own block.
template <typename T, int P, int FK>
__device__ __forceinline__ void tri_halo_qn(const int4 e, const TriHaloIn<T, P> &hi,
                                            const TriTab<T, P> &tb, int wallA, T (&qn)[P + 1]) {
  using S = TriShape<P>;
  constexpr int N = S::N, NE = S::NE;
  constexpr int o = S::ftri(FK);
  T dgk[2][NE];
#pragma unroll
  for (int t = 0; t < NE; ++t) {
    dgk[o][t] = hi.uo[S::en(o == 0 ? 2 : 0, t)];
    dgk[1 - o][t] = hi.od[t];
  }
  T qx[N], qy[N];
  tri_q_volume<T, P>(tb, o, hi.uo, qx, qy);
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) {
    T uh[NE], nb[NE];
    T cm = 0, cp = 0;
    if (!tri_diag(o, ed)) {
      // the chunk pixel across FK, else the third neighbour, a wall or the edge
      const bool chunk_side = tri_face(o, ed) == FK;
      const int L = chunk_side ? 0 : e.w;
#pragma unroll
      for (int t = 0; t < NE; ++t) nb[t] = chunk_side ? hi.tc[t] : hi.t3[t];
      tri_uflux_weights<T>(L, wallA, cm, cp);
    }
    tri_uh<T, P>(o, ed, hi.uo, dgk, cm, cp, nb, uh);
    tri_q_edge<T, P>(tb, o, ed, uh, qx, qy);
  }
#pragma unroll
  for (int t = 0; t < NE; ++t) qn[t] = tri_qn<T, P>(tb, qx, qy, o, S::fedge(FK), t);
}

// One halo entry: the halo triangle's u trace at its face toward the chunk
// (ut) and its q . n there (qn).
template <typename T, int P, int FK>
__device__ __forceinline__ void tri_halo_face(const T *U, long long a0, const int4 e,
                                              const TriTab<T, P> &tb, int wallA,
                                              T (&ut)[P + 1], T (&qn)[P + 1]) {
  using S = TriShape<P>;
  TriHaloIn<T, P> hi;
  tri_halo_load<T, P, FK>(U, a0, e, hi);
#pragma unroll
  for (int t = 0; t < P + 1; ++t) ut[t] = hi.uo[S::en(S::fedge(FK), t)];
  tri_halo_qn<T, P, FK>(e, hi, tb, wallA, qn);
}

template <typename T, int P>
__device__ __forceinline__ void tri_halo_entry(const T *U, long long a0, const int4 e,
                                               const TriTab<T, P> &tb, int wallA,
                                               T (&ut)[P + 1], T (&qn)[P + 1]) {
  switch (e.y) {
    case 0: tri_halo_face<T, P, 0>(U, a0, e, tb, wallA, ut, qn); break;
    case 1: tri_halo_face<T, P, 1>(U, a0, e, tb, wallA, ut, qn); break;
    case 2: tri_halo_face<T, P, 2>(U, a0, e, tb, wallA, ut, qn); break;
    default: tri_halo_face<T, P, 3>(U, a0, e, tb, wallA, ut, qn); break;
  }
}

template <typename T, int P, bool HAS_U0, bool SROUND>
__global__ void __launch_bounds__(kBlock, tri_min_blocks<T>())
    k_tri_f(const T *__restrict__ uin, const T *u0, T *out, const int4 *__restrict__ loc,
            const int4 *__restrict__ htri, int hstride, const int *__restrict__ halo_cnt,
            const int2 *__restrict__ chunk_tab, const int2 *__restrict__ grange,
            const T *__restrict__ gscale, long long stride, int nrec,
            const int *__restrict__ chunk_list, const uint8_t *__restrict__ adv,
            const TriTab<T, P> tb, const StageCoef<T> c) {
  using S = TriShape<P>;
  using QS = TriQStage<T, P>;
  static_assert(QS::ON, "the chunk's q is staged in shared memory");
  constexpr int N = S::N, NE = S::NE, NPX = S::NPX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *rec = reinterpret_cast<T *>(smem_raw);
  float4 *sq = reinterpret_cast<float4 *>(smem_raw + tri_rec_bytes(nrec, NE, (int)sizeof(T)));
  T *rx = reinterpret_cast<T *>(smem_raw + tri_rec_bytes(nrec, NE, (int)sizeof(T)) + QS::BYTES);
  const int zero_rec = nrec - 1;
  const TriBlock b = tri_block(chunk_list, chunk_tab, loc, halo_cnt);
  const size_t sbase = (size_t)blockIdx.y * (size_t)stride;
  const T *U = uin + sbase * NPX;
  const T *Ue = U + (size_t)(b.a0 + b.el) * NPX;
  const int4 *H = htri + (size_t)b.chunk * hstride;

  // this thread's first halo entry (entries past the chunk's count hold
  // pixel -1, so the count is not waited for): its u-trace record and its
  // q . n, kept in registers; entries past kBlock: q . n into the small area
  const int4 e0 = b.el < hstride ? __ldg(H + b.el) : make_int4(-1, 0, 0, kEdge);
  T qh[NE];
  if (e0.x >= 0) {
    T ut[NE];
    tri_halo_entry<T, P>(U, b.a0, e0, tb, c.wallA, ut, qh);
#pragma unroll
    for (int t = 0; t < NE; ++t) rec[(4 * kBlock + b.el) * NE + t] = ut[t];
  }
  for (int h = b.el + kBlock; h < b.hcnt; h += kBlock) {  // chunks with > kBlock halo entries
    const int4 e = __ldg(H + h);
    T ut[NE], q2[NE];
    tri_halo_entry<T, P>(U, b.a0, e, tb, c.wallA, ut, q2);
#pragma unroll
    for (int t = 0; t < NE; ++t) {
      rec[(4 * kBlock + h) * NE + t] = ut[t];
      rx[(h - kBlock) * NE + t] = q2[t];
    }
  }

  // u traces of the pixel's faces and diagonals (as the q pass)
  T dg[2][NE];
  if (b.live) {
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      T uo[N];
      load_elem<T, N>(Ue + o * N, uo);
#pragma unroll
      for (int f = 0; f < 4; ++f)
        if (S::ftri(f) == o)
#pragma unroll
          for (int t = 0; t < NE; ++t) rec[(f * kBlock + b.el) * NE + t] = uo[S::en(S::fedge(f), t)];
#pragma unroll
      for (int t = 0; t < NE; ++t) dg[o][t] = uo[S::en(o == 0 ? 2 : 0, t)];
    }
  }
  if (b.el == 0)
    for (int t = 0; t < NE; ++t) rec[zero_rec * NE + t] = (T)0;
  __syncthreads();

  // the chunk's q into the staging (as the q pass)
  const int lq[4] = {b.l4.x, b.l4.y, b.l4.z, b.l4.w};
#pragma unroll 1
  for (int o = 0; o < 2 && b.live; ++o) {
    T uo[N];
    load_elem<T, N>(Ue + o * N, uo);
    T qx[N], qy[N];
    tri_q_volume<T, P>(tb, o, uo, qx, qy);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      T uh[NE], nb[NE];
      T cm = 0, cp = 0;
      if (!tri_diag(o, e)) {
        const int f = tri_face(o, e);
        const int L = lq[f];
        const int rn = tri_rec_index(L, f, b.el, zero_rec);
        tri_uflux_weights<T>(L, c.wallA, cm, cp);
#pragma unroll
        for (int t = 0; t < NE; ++t) nb[t] = rec[rn * NE + t];
      }
      tri_uh<T, P>(o, e, uo, dg, cm, cp, nb, uh);
      tri_q_edge<T, P>(tb, o, e, uh, qx, qy);
    }
    QS::put(sq, b.el, o, qx, qy);
  }
  __syncthreads();  // every u trace read, the staged q complete

  auto load_q = [&](int o, T (&qx)[N], T (&qy)[N]) { QS::get(sq, b.el, o, qx, qy); };
  if (b.live) tri_qn_records<T, P>(b, load_q, rec, tb, dg);
  if (e0.x >= 0) {
#pragma unroll
    for (int t = 0; t < NE; ++t) rec[(4 * kBlock + b.el) * NE + t] = qh[t];
  }
  for (int h = b.el + kBlock; h < b.hcnt; h += kBlock) {
#pragma unroll
    for (int t = 0; t < NE; ++t) rec[(4 * kBlock + h) * NE + t] = rx[(h - kBlock) * NE + t];
  }
  __syncthreads();
  if (!b.live) return;
  tri_finish<T, P, HAS_U0, SROUND>(b, load_q, rec, zero_rec, dg, tb, c, uin, u0, out, sbase,
                                   grange, gscale, adv);
}

template <typename T, int P>
cudaError_t launch_tri_p(const T *u, const T *u0, T *out, T *qbuf, const Geometry &geo,
                         long long stride, int m, const TriRef &ref, const StageCoef<T> &c,
                         cudaStream_t s, const ChunkSel &sel, bool fused) {
  const long long nch = sel.list ? sel.count : geo.n_chunks();
  if (geo.n_pad <= 0 || m <= 0 || nch <= 0) return cudaSuccess;
  if (nch > geo.n_chunks()) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)nch, (unsigned)m);
  const T *gscale;
  if constexpr (sizeof(T) == 8) gscale = geo.d_gscale_d;
  else gscale = geo.d_gscale_f;
  const TriTab<T, P> tb = make_tri_tab<T, P>(ref);
  const int nrec = 4 * kBlock + geo.halo_max + 1;
  constexpr bool kSR = sizeof(T) == 4;
  if constexpr (TriQStage<T, P>::ON) {
    if (fused && geo.d_htri != nullptr) {  // one launch: q stays in shared memory
      const int hstride = geo.halo_max > 0 ? geo.halo_max : 1;
      const int extra = geo.halo_max > kBlock ? (geo.halo_max - kBlock) * TriShape<P>::NE * (int)sizeof(T) : 0;
      const int fsmem = tri_rec_bytes(nrec, TriShape<P>::NE, (int)sizeof(T)) + TriQStage<T, P>::BYTES +
                        (extra + 15) / 16 * 16;
      static int fattr_bytes = 0;
      if (fsmem > fattr_bytes) {
        cudaError_t e = cudaSuccess;
        auto set = [&](auto kern) {
          if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, fsmem);
        };
        set(k_tri_f<T, P, true, false>);
        set(k_tri_f<T, P, false, false>);
        set(k_tri_f<T, P, true, kSR>);
        set(k_tri_f<T, P, false, kSR>);
        if (e != cudaSuccess) return e;
        fattr_bytes = fsmem;
      }
      auto gof = [&](auto kern) {
        kern<<<grid, kBlock, fsmem, s>>>(u, u0, out, geo.d_loc, geo.d_htri, hstride, geo.d_halo_cnt,
                                         geo.d_chunk, geo.d_grange, gscale, stride, nrec, sel.list,
                                         sel.adv, tb, c);
      };
      if (kSR && c.sround) {
        if (u0) gof(k_tri_f<T, P, true, kSR>);
        else gof(k_tri_f<T, P, false, kSR>);
      } else {
        if (u0) gof(k_tri_f<T, P, true, false>);
        else gof(k_tri_f<T, P, false, false>);
      }
      return cudaGetLastError();
    }
  }
  const int smem = tri_rec_bytes(nrec, TriShape<P>::NE, (int)sizeof(T)) + TriQStage<T, P>::BYTES;
  static int attr_bytes = 0;
  if (smem > attr_bytes) {
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kern) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    };
    set(k_tri_q<T, P>);
    set(k_tri_r<T, P, true, false>);
    set(k_tri_r<T, P, false, false>);
    if constexpr (kSR) {
      set(k_tri_r<T, P, true, kSR>);
      set(k_tri_r<T, P, false, kSR>);
    }
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  k_tri_q<T, P><<<grid, kBlock, smem, s>>>(u, qbuf, geo.d_loc, geo.d_halo, geo.d_halo_cnt,
                                           geo.d_chunk, stride, nrec, sel.list, tb, c.wallA);
  auto go = [&](auto kern) {
    kern<<<grid, kBlock, smem, s>>>(qbuf, u, u0, out, geo.d_loc, geo.d_halo, geo.d_halo_cnt,
                                    geo.d_chunk, geo.d_grange, gscale, stride, nrec, sel.list,
                                    sel.adv, tb, c);
  };
  if (kSR && c.sround) {
    if (u0) go(k_tri_r<T, P, true, kSR>);
    else go(k_tri_r<T, P, false, kSR>);
  } else {
    if (u0) go(k_tri_r<T, P, true, false>);
    else go(k_tri_r<T, P, false, false>);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tri_any(int p, const T *u, const T *u0, T *out, T *qbuf, const Geometry &geo,
                           long long stride, int m, const TriRef &ref, const StageCoef<T> &c,
                           cudaStream_t s, const ChunkSel &sel, bool fused) {
  switch (p) {
    case 1: return launch_tri_p<T, 1>(u, u0, out, qbuf, geo, stride, m, ref, c, s, sel, fused);
    case 2: return launch_tri_p<T, 2>(u, u0, out, qbuf, geo, stride, m, ref, c, s, sel, fused);
    case 3: return launch_tri_p<T, 3>(u, u0, out, qbuf, geo, stride, m, ref, c, s, sel, fused);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tri_stage_f64(int p, const double *u, const double *u0, double *out,
                                 double *qbuf, const Geometry &geo, long long stride, int m,
                                 const TriRef &ref, const StageCoef<double> &c, cudaStream_t s,
                                 const ChunkSel &sel, bool fused) {
  return launch_tri_any<double>(p, u, u0, out, qbuf, geo, stride, m, ref, c, s, sel, fused);
}
cudaError_t launch_tri_stage_f32(int p, const float *u, const float *u0, float *out,
                                 float *qbuf, const Geometry &geo, long long stride, int m,
                                 const TriRef &ref, const StageCoef<float> &c, cudaStream_t s,
                                 const ChunkSel &sel, bool fused) {
  return launch_tri_any<float>(p, u, u0, out, qbuf, geo, stride, m, ref, c, s, sel, fused);
}

}  // namespace dg
