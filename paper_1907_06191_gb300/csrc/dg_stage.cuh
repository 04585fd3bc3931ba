// dg_stage.cuh -- fused SSP-RK3 stage of the DG diffusion operator.
//
// One thread owns one mesh element of one density: the element's (p+1)^2
// nodal values sit in registers, the four face neighbours are read whole
// (through L1/L2; they are other threads' elements) and the stage result
//   out = u0 + beta (u - u0) + gamma R(u),   L u = (k / J^2) R(u),
// (gamma = beta dt k / J^2, J = h/2 of the element's geometry),
// is written once (u0 absent: out = beta u + gamma R).  This increment form
// of the Shu-Osher combination (1 - beta) u0 + beta (u + dt L u) keeps the
// weight of u0 exactly 1 - beta in any precision, so FP32 rounding of 1/3
// and 2/3 does not bias the mass.  q = grad u is never stored: substituting the gradient
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

#include <cuda.h>

#include <algorithm>

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

// ---------------------------------------------------------------------------
// Shared-memory staging.  A block owns kBlock consecutive mesh elements (one
// per thread).  Their values are copied into shared memory with 16-byte
// asynchronous copies (coalesced; no registers held while in flight), and the
// result leaves through shared memory with coalesced 16-byte stores.  When an
// element is a whole number S of 16-byte slots, slot k of element e lives at
// slot e*S + (k ^ swz(e)) (S a power of two), which makes the slot reads of 8
// consecutive threads hit 8 different bank groups; other element sizes are
// stored linearly and read word by word (odd word strides are conflict free).
template <typename T, int NP>
struct Stage {
  static constexpr int B = NP * (int)sizeof(T);
  static constexpr bool SLOT = (B % 16) == 0;
  static constexpr int S = SLOT ? B / 16 : 0;
  static constexpr bool POW2 = SLOT && ((S & (S - 1)) == 0);
  static constexpr int WPS = 16 / (int)sizeof(T);
  static constexpr int CHUNK_BYTES = ((kBlock * B + 15) / 16) * 16;

  __device__ static __forceinline__ int swz(int e) {
    if constexpr (!POW2 || S == 1) return 0;
    else if constexpr (S == 2) return (e >> 2) & 1;
    else if constexpr (S == 4) return (e >> 1) & 3;
    else return e & 7;
  }
  __device__ static __forceinline__ int slot(int e, int k) {
    if constexpr (POW2) return e * S + (k ^ swz(e));
    else return e * S + k;
  }
  // index (in T units) of value w of element e
  __device__ static __forceinline__ int word(int e, int w) {
    if constexpr (SLOT) return slot(e, w / WPS) * WPS + (w % WPS);
    else return e * NP + w;
  }
  __device__ static __forceinline__ void read(const T *sm, int e, T (&u)[NP]) {
    if constexpr (SLOT) {
#pragma unroll
      for (int k = 0; k < S; ++k) {
        const float4 v = *reinterpret_cast<const float4 *>(sm + slot(e, k) * WPS);
        const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
        for (int q = 0; q < WPS; ++q) u[k * WPS + q] = pv[q];
      }
    } else {
#pragma unroll
      for (int w = 0; w < NP; ++w) u[w] = sm[e * NP + w];
    }
  }
  __device__ static __forceinline__ void write(T *sm, int e, const T (&u)[NP]) {
    if constexpr (SLOT) {
#pragma unroll
      for (int k = 0; k < S; ++k) {
        float4 v;
        T *pv = reinterpret_cast<T *>(&v);
#pragma unroll
        for (int q = 0; q < WPS; ++q) pv[q] = u[k * WPS + q];
        *reinterpret_cast<float4 *>(sm + slot(e, k) * WPS) = v;
      }
    } else {
#pragma unroll
      for (int w = 0; w < NP; ++w) sm[e * NP + w] = u[w];
    }
  }
  // number of 16-byte pieces covering cnt elements
  __device__ static __forceinline__ int pieces(int cnt) {
    if constexpr (SLOT) return cnt * S;
    else return (cnt * B + 15) / 16;
  }
  __device__ static __forceinline__ int piece_dst(int j) {  // in 16-byte units
    if constexpr (SLOT) return slot(j / S, j % S);
    else return j;
  }
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Tensor-memory-accelerator copies of a whole chunk.  The state array is a 2D
// tensor [rows = densities x padded elements][NP values]; one elected thread
// arms an mbarrier with the expected bytes and issues one tiled copy of
// kBlock rows.  With 32, 64 or 128 bytes per element the copy uses the hardware
// swizzle of that width, which XORs the 16-byte slot index with bits of the
// row exactly as Stage::swz does, so the shared-memory layout is the same as
// with the per-thread cp.async copies.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_rows(uint32_t dst, const CUtensorMap *map, int row,
                                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(bar)
      : "memory");
}
// Tiled store of kBlock rows from shared memory; the issuing thread waits until
// the shared-memory source has been read (the block's other threads may have
// left: shared memory lives until the last thread of the block exits).
__device__ __forceinline__ void tma_store_rows(const CUtensorMap *map, int row, uint32_t src) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(0), "r"(row), "r"(src)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// L2 eviction priorities.  The stage kernels stream three state arrays
// (gigabytes) past the small per-chunk geometry tables that every density's
// blocks read again; marking the streams that no later block of the launch
// reads (u0 chunks, result chunks) evict-first and the tables evict-last
// keeps the tables in L2 from one density to the next.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void tma_load_rows_hint(uint32_t dst, const CUtensorMap *map, int row,
                                                   uint32_t bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1, {%2, %3}], [%4], %5;\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(bar), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void tma_store_rows_hint(const CUtensorMap *map, int row, uint32_t src,
                                                    uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%1, %2}], [%3], "
      "%4;\n" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(0), "r"(row), "r"(src), "l"(pol)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// Read-only loads of table entries with an L2 policy.
__device__ __forceinline__ int4 ldg_hint(const int4 *p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;\n"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int2 ldg_hint(const int2 *p, uint64_t pol) {
  int2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.s32 {%0, %1}, [%2], %3;\n"
               : "=r"(v.x), "=r"(v.y)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int ldg_hint(const int *p, uint64_t pol) {
  int v;
  asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;\n" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}

// Make this thread's shared-memory writes visible to the tensor copies.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Poll phase `parity` of the barrier at most `limit` times (with a short
// sleep in between); false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    __nanosleep(64);
  }
  return false;
}

// Face f of an element: 0 east (x = +1), 1 west, 2 north (y = +1), 3 south.
// Node t runs along the face.  own(f, t): node index on face f; the matching
// node of the neighbour across f is own(opposite(f), t).
template <int P>
struct Faces {
  static constexpr int n = P + 1;
  __host__ __device__ static constexpr int own(int f, int t) {
    return f == 0 ? t * n + P : f == 1 ? t * n : f == 2 ? P * n + t : t;
  }
  __host__ __device__ static constexpr int opp(int f) { return f ^ 1; }
  __host__ __device__ static constexpr int sgn(int f) { return (f & 1) ? -1 : 1; }
  __host__ __device__ static constexpr int row(int f) { return (f & 1) ? 0 : P; }  // D row of the face
};

// murmur3's 32-bit finaliser (Appleby): avalanche mixing of one word.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

// base + inc rounded to FP32 stochastically: s = fl(base + inc) moves one unit
// in the last place toward the exact sum with probability |err| / ulp(s), err
// the rounding error of s (exact by Fast2Sum when |base| >= |inc|), so the
// expected result is base + inc.  The uniform number comes from h, a hash that
// already depends on the element, and the bits of inc (multiplicative hashing
// by the golden ratio; its high bits are used): reproducible, and different
// from step to step because the operands change.  Zero, subnormal and
// non-finite sums are returned as s.
__device__ __forceinline__ float add_stochastic(float base, float inc, uint32_t h) {
  const float s = base + inc;
  const float err = inc - (s - base);
  const float ulp = __uint_as_float(__float_as_uint(s) & 0x7f800000u) * 0x1p-23f;
  const uint32_t hk = (h ^ __float_as_uint(inc)) * 0x9e3779b9u;
  const float r = __uint_as_float(0x3f800000u | (hk >> 9)) - 1.0f;  // uniform in [0, 1)
  return fabsf(err) > r * ulp ? s + copysignf(ulp, err) : s;
}

// Two lanes of add_stochastic with packed FP32 instructions: lane by lane the
// same operations and roundings (s - base and inc - (s - base) as fused
// multiply-adds by -1, which round like the subtractions).
__device__ __forceinline__ float2 add_stochastic2(float2 base, float2 inc, uint32_t h0,
                                                  uint32_t h1) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 s = __fadd2_rn(base, inc);
  const float2 err = __ffma2_rn(__ffma2_rn(base, m1, s), m1, inc);
  const float2 ulp = __fmul2_rn(
      make_float2(__uint_as_float(__float_as_uint(s.x) & 0x7f800000u),
                  __uint_as_float(__float_as_uint(s.y) & 0x7f800000u)),
      make_float2(0x1p-23f, 0x1p-23f));
  const uint32_t k0 = (h0 ^ __float_as_uint(inc.x)) * 0x9e3779b9u;
  const uint32_t k1 = (h1 ^ __float_as_uint(inc.y)) * 0x9e3779b9u;
  const float2 thr = __fmul2_rn(__fadd2_rn(make_float2(__uint_as_float(0x3f800000u | (k0 >> 9)),
                                                       __uint_as_float(0x3f800000u | (k1 >> 9))),
                                           m1),
                                ulp);
  const float2 up = __fadd2_rn(s, make_float2(copysignf(ulp.x, err.x), copysignf(ulp.y, err.y)));
  return make_float2(fabsf(err.x) > thr.x ? up.x : s.x, fabsf(err.y) > thr.y ? up.y : s.y);
}

// Fused multiply-add in the element type: sums of products are written as
// chains of these, one rounding and one FP64 / FP32 pipe instruction per
// product (a * b + c * d left to the compiler becomes a multiply, a fused
// multiply-add and an add).
template <typename T>
__device__ __forceinline__ T fmaT(T a, T b, T c) {
  if constexpr (sizeof(T) == 4) return fmaf(a, b, c);
  else return fma(a, b, c);
}

// FP32: pairs of nodes go through the packed two-lane instructions
// (fma.rn.f32x2 and friends; each lane rounds like the scalar instruction);
// with an odd number of nodes per line the last node of a line (and the last
// node of the element) takes the scalar instruction.
template <typename T, int P>
constexpr bool kPacked = sizeof(T) == 4;

// Outward normal derivative (reference units) at the nodes of face f: the
// face's signed row of D applied along the lines normal to the face.
template <typename T, int P>
__device__ __forceinline__ void outward_derivative(const T (&u)[(P + 1) * (P + 1)], int f,
                                                   const StageTab<T, P> &tb, T (&d)[P + 1]) {
  constexpr int n = P + 1;
  const T *row = tb.Dout + (f & 1) * n;
#pragma unroll
  for (int t = 0; t < n; ++t) {
    T s = 0;
#pragma unroll
    for (int m = 0; m < n; ++m) s += row[m] * (f < 2 ? u[t * n + m] : u[m * n + t]);
    d[t] = s;
  }
}

// Face records in shared memory: for record r, the trace tr[t] and the
// outward normal derivative d[t] (t = 0..n-1) of one element face.  Record
// f*kBlock + e is face f of chunk element e; record 4*kBlock + h is halo entry
// h; the last record is all zeros (read for walls and edges).  When n values
// fill one 16-byte slot, record r is slot r of each array; otherwise the
// arrays are transposed ([t][r]).  Either way threads reading consecutive
// records hit distinct banks.
template <typename T, int P>
struct Records {
  static constexpr int n = P + 1;
  static constexpr bool VEC = n * (int)sizeof(T) == 16;
  T *tr, *d;
  int nrec;
  __device__ __forceinline__ void put(int r, const T (&a)[n], const T (&b)[n]) const {
    if constexpr (VEC) {
      float4 va, vb;
      T *pa = reinterpret_cast<T *>(&va), *pb = reinterpret_cast<T *>(&vb);
#pragma unroll
      for (int t = 0; t < n; ++t) { pa[t] = a[t]; pb[t] = b[t]; }
      reinterpret_cast<float4 *>(tr)[r] = va;
      reinterpret_cast<float4 *>(d)[r] = vb;
    } else {
#pragma unroll
      for (int t = 0; t < n; ++t) {
        tr[t * nrec + r] = a[t];
        d[t * nrec + r] = b[t];
      }
    }
  }
  __device__ __forceinline__ void get_tr(int r, T (&a)[n]) const {
    if constexpr (VEC) {
      const float4 v = reinterpret_cast<const float4 *>(tr)[r];
      const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
      for (int t = 0; t < n; ++t) a[t] = pv[t];
    } else {
#pragma unroll
      for (int t = 0; t < n; ++t) a[t] = tr[t * nrec + r];
    }
  }
  __device__ __forceinline__ void get_d(int r, T (&a)[n]) const {
    if constexpr (VEC) {
      const float4 v = reinterpret_cast<const float4 *>(d)[r];
      const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
      for (int t = 0; t < n; ++t) a[t] = pv[t];
    } else {
#pragma unroll
      for (int t = 0; t < n; ++t) a[t] = d[t * nrec + r];
    }
  }
  __host__ __device__ static constexpr int bytes(int nrec_) {
    return 2 * ((nrec_ * n * (int)sizeof(T) + 15) / 16) * 16;
  }
};

template <typename T, int P>
__device__ __forceinline__ void face_record(const T (&u)[(P + 1) * (P + 1)], int f,
                                            const StageTab<T, P> &tb, T (&tr)[P + 1],
                                            T (&d)[P + 1]) {
  outward_derivative<T, P>(u, f, tb, d);
#pragma unroll
  for (int t = 0; t < P + 1; ++t) tr[t] = u[Faces<P>::own(f, t)];
}

// ---- one stage on one element: the pieces both stage kernels share --------

// The element's face records (trace and outward derivative of each face,
// record f*kBlock + el) and its volume term R = sum_i (DD)_ai u_ib +
// sum_j (DD)_bj u_aj.
template <typename T, int P>
__device__ __forceinline__ void element_records_volume(const T (&u)[(P + 1) * (P + 1)],
                                                       const StageTab<T, P> &tb,
                                                       const Records<T, P> &rec, int el,
                                                       T (&R)[(P + 1) * (P + 1)]) {
  constexpr int n = P + 1;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    T tr[n], d[n];
    face_record<T, P>(u, f, tb, tr, d);
    rec.put(f * kBlock + el, tr, d);
  }
  if constexpr (kPacked<T, P>) {
    // nodes (j, i) and (j, i + 1) together: the x part pairs a column of
    // D2 with u_jm, the y part a value of D2 with u_m,i..i+1
#pragma unroll
    for (int j = 0; j < n; ++j)
#pragma unroll
      for (int ip = 0; ip < n / 2; ++ip) {
        float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int m = 0; m < n; ++m) {
          s = __ffma2_rn(tb.D2x[ip * n + m], make_float2(u[j * n + m], u[j * n + m]), s);
          s = __ffma2_rn(tb.D2y[j * n + m],
                         make_float2(u[m * n + 2 * ip], u[m * n + 2 * ip + 1]), s);
        }
        R[j * n + 2 * ip] = s.x;
        R[j * n + 2 * ip + 1] = s.y;
      }
    if constexpr (n % 2 == 1) {  // the last node of each row
      constexpr int i = n - 1;
#pragma unroll
      for (int j = 0; j < n; ++j) {
        T s = 0;
#pragma unroll
        for (int m = 0; m < n; ++m)
          s = fmaT(tb.D2[j * n + m], u[m * n + i], fmaT(tb.D2[i * n + m], u[j * n + m], s));
        R[j * n + i] = s;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < n; ++j)
#pragma unroll
      for (int i = 0; i < n; ++i) {
        T s = 0;
#pragma unroll
        for (int m = 0; m < n; ++m)
          s = fmaT(tb.D2[j * n + m], u[m * n + i], fmaT(tb.D2[i * n + m], u[j * n + m], s));
        R[j * n + i] = s;
      }
  }
}

// Record of the face `face` of a halo element (values v) in record `r`.
template <typename T, int P>
__device__ __forceinline__ void halo_face_record(const T (&v)[(P + 1) * (P + 1)], int face,
                                                 const StageTab<T, P> &tb,
                                                 const Records<T, P> &rec, int r) {
  constexpr int n = P + 1;
  T tr[n], d[n];
  switch (face) {  // the face of the halo element that touches the chunk
    case 0: face_record<T, P>(v, 0, tb, tr, d); break;
    case 1: face_record<T, P>(v, 1, tb, tr, d); break;
    case 2: face_record<T, P>(v, 2, tb, tr, d); break;
    default: face_record<T, P>(v, 3, tb, tr, d); break;
  }
  rec.put(r, tr, d);
}

// Flux and lifting terms of the four faces added to R (see the file header);
// lq: the element's neighbour codes (chunk slot, kBlock + halo slot, kWall,
// kEdge).
template <typename T, int P, bool FULL>
__device__ __forceinline__ void element_flux(const T (&u)[(P + 1) * (P + 1)],
                                             T (&R)[(P + 1) * (P + 1)], const int (&lq)[4],
                                             int el, int zero_rec, const Records<T, P> &rec,
                                             const StageTab<T, P> &tb, const StageCoef<T> &c) {
  constexpr int n = P + 1;
  using Fc = Faces<P>;
  const T half = (T)0.5, iw = tb.inv_w;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int L = lq[f];
    const int fo = Fc::opp(f);
    // neighbour record: chunk element, halo entry, or the zero record
    const int rn = L >= kBlock ? 4 * kBlock + (L - kBlock) : (L >= 0 ? fo * kBlock + L : zero_rec);
    // face-kind coefficients with 1/w (and, for the lifting, the face sign)
    // folded in: gs = s_f g / w = cg_up u+ + cg_um u-, and the face term
    // F / w = c_od d- + c_odn d+ (+ c_um u- + c_up u+)   (see file header)
    const bool in = L >= 0, wl = L == kWall, wa = wl && c.wallA, ed = L == kEdge;
    const T sw = (f & 1) ? -iw : iw;
    const T cg_up = in ? half * sw : (T)0;
    const T cg_um = in ? -half * sw : (wa ? -half * sw : (ed ? -sw : (T)0));
    const T c_od = in ? half * iw : (ed ? (T)0 : iw);
    const T c_odn = in ? half * iw : (T)0;
    T up[n], odn[n], od[n];
    rec.get_tr(rn, up);
    rec.get_d(rn, odn);
    rec.get_d(f * kBlock + el, od);
    T gs[n];
    if constexpr (FULL) {
      const T c_um = (in ? c.pen : (wa ? -half * iw : (ed ? c.pen : (T)0))) * iw;
      const T c_up = in ? -c.pen * iw : (T)0;
#pragma unroll
      for (int t = 0; t < n; ++t) {
        const T um = u[Fc::own(f, t)];
        gs[t] = cg_up * up[t] + cg_um * um;
        T r = R[Fc::own(f, t)];
        r = fmaT(-c_od, od[t], r);
        r = fmaT(-c_odn, odn[t], r);
        r = fmaT(-c_um, um, r);
        R[Fc::own(f, t)] = fmaT(-c_up, up[t], r);
      }
    } else {
#pragma unroll
      for (int t = 0; t < n; ++t) {
        gs[t] = cg_up * up[t] + cg_um * u[Fc::own(f, t)];
        R[Fc::own(f, t)] = fmaT(-c_odn, odn[t], fmaT(-c_od, od[t], R[Fc::own(f, t)]));
      }
    }
    // lifting of the u-flux jump: column (x-faces) or row (y-faces) of D
    const int r = Fc::row(f);
#pragma unroll
    for (int t = 0; t < n; ++t) {
#pragma unroll
      for (int q = 0; q < n; ++q) {
        if (f < 2) R[t * n + q] += tb.D[q * n + r] * gs[t];
        else R[q * n + t] += tb.D[q * n + r] * gs[t];
      }
    }
  }
}

// Stage update of one element: o = o + beta (u - o) + gam R with o = u0 on
// entry (HAS_U0), else o = beta u + gam R; FP32 with stochastic rounding
// rounds o + increment once per node, keyed by the element hash h.
template <typename T, int P, bool HAS_U0, bool SROUND>
__device__ __forceinline__ void element_update(const T (&u)[(P + 1) * (P + 1)],
                                               const T (&R)[(P + 1) * (P + 1)],
                                               T (&o)[(P + 1) * (P + 1)], T gam, uint32_t h,
                                               const StageCoef<T> &c) {
  constexpr int NP = (P + 1) * (P + 1);
  if constexpr (SROUND) {
    // increment first, then one stochastic rounding onto the state
    if constexpr (kPacked<T, P>) {  // the same arithmetic, two nodes per instruction
      const float2 b2 = make_float2(c.beta, c.beta), g2 = make_float2(gam, gam);
#pragma unroll
      for (int k = 0; k + 1 < NP; k += 2) {
        const float2 u2 = make_float2(u[k], u[k + 1]), gr = __fmul2_rn(g2, make_float2(R[k], R[k + 1]));
        float2 bs, in;
        if constexpr (HAS_U0) {
          bs = make_float2(o[k], o[k + 1]);
          in = __ffma2_rn(b2, __ffma2_rn(bs, make_float2(-1.0f, -1.0f), u2), gr);
        } else {
          bs = __fmul2_rn(b2, u2);
          in = gr;
        }
        const float2 w = add_stochastic2(bs, in, h + (uint32_t)k, h + (uint32_t)(k + 1));
        o[k] = w.x;
        o[k + 1] = w.y;
      }
      if constexpr (NP % 2 == 1) {  // the last node on its own
        constexpr int k = NP - 1;
        const T bs = HAS_U0 ? o[k] : c.beta * u[k];
        const T in = HAS_U0 ? fmaf(c.beta, u[k] - o[k], gam * R[k]) : gam * R[k];
        o[k] = add_stochastic(bs, in, h + (uint32_t)k);
      }
    } else {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const T bs = HAS_U0 ? o[k] : c.beta * u[k];
        const T in = HAS_U0 ? fmaf(c.beta, u[k] - o[k], gam * R[k]) : gam * R[k];
        o[k] = add_stochastic(bs, in, h + (uint32_t)k);
      }
    }
  } else if constexpr (HAS_U0) {
    if constexpr (kPacked<T, P>) {  // o + (beta (u - o) + gam R)
      const float2 b2 = make_float2(c.beta, c.beta), g2 = make_float2(gam, gam);
#pragma unroll
      for (int k = 0; k + 1 < NP; k += 2) {
        const float2 o2 = make_float2(o[k], o[k + 1]);
        const float2 d = __ffma2_rn(o2, make_float2(-1.0f, -1.0f), make_float2(u[k], u[k + 1]));
        const float2 w = __fadd2_rn(
            o2, __ffma2_rn(b2, d, __fmul2_rn(g2, make_float2(R[k], R[k + 1]))));
        o[k] = w.x;
        o[k + 1] = w.y;
      }
      if constexpr (NP % 2 == 1) {
        constexpr int k = NP - 1;
        o[k] = o[k] + fmaf(c.beta, u[k] - o[k], gam * R[k]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < NP; ++k) o[k] = o[k] + c.beta * (u[k] - o[k]) + gam * R[k];
    }
  } else if constexpr (kPacked<T, P>) {
    const float2 b2 = make_float2(c.beta, c.beta), g2 = make_float2(gam, gam);
#pragma unroll
    for (int k = 0; k + 1 < NP; k += 2) {
      const float2 w = __ffma2_rn(b2, make_float2(u[k], u[k + 1]),
                                  __fmul2_rn(g2, make_float2(R[k], R[k + 1])));
      o[k] = w.x;
      o[k + 1] = w.y;
    }
    if constexpr (NP % 2 == 1) {
      constexpr int k = NP - 1;
      o[k] = fmaf(c.beta, u[k], gam * R[k]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NP; ++k) o[k] = c.beta * u[k] + gam * R[k];
  }
}

// Stochastic-rounding key of an element: one avalanche hash of its place in
// its own geometry, its density and the bits of its first two input values
// (they change every stage while the element is advancing), so a geometry
// gives the same bits alone or in a batch, and either stage kernel the same.
template <typename T>
__device__ __forceinline__ uint32_t element_key(long long elem_in_geo, int np, int density,
                                                const T *u) {
  if constexpr (sizeof(T) == 4)
    return fmix32(((uint32_t)elem_in_geo * (uint32_t)np) ^ ((uint32_t)density * 0x632be5abu) ^
                  __float_as_uint(u[0]) ^ (__float_as_uint(u[1]) * 0x85ebca77u));
  else
    return 0u;
}

// grid: (chunks launched, m): block x takes chunk chunk_list[x] (x itself
// without a list); density s = blockIdx.y starts at s * stride
// elements.  loc/halo tables come from the geometry (entries checked when
// built).  out may alias u0 (the last stage updates u^n in place: a block
// reads its whole u0 chunk into shared memory before it writes the same
// chunk); it never aliases uin.  Shared memory: chunk of u, chunk of u0 (then
// of the result), face records.
template <typename T, int P>
constexpr int stage_min_blocks() {
  // registers per thread: 64 (FP32, p <= 3: eight blocks of 128 per SM),
  // 128 (FP32 p >= 4, FP64 p <= 3), 255 (FP64 p >= 4)
  if constexpr (sizeof(T) == 4) return blocks_for_regs(P <= 3 ? 64 : 128);
  else return blocks_for_regs(P <= 3 ? 128 : 255);
}

// FULL = false drops the flux terms in u^- and u^+ that vanish without a
// penalty (eta = 0) and without paper walls (the default configuration).
// Bytes of the front shared-memory buffer (u chunk, then face records),
// rounded to 1024 so that the u0 chunk behind it starts on that boundary.
template <typename T, int P>
__host__ __device__ constexpr int stage_front_bytes(int nrec) {
  return ((Stage<T, (P + 1) * (P + 1)>::CHUNK_BYTES > Records<T, P>::bytes(nrec)
               ? Stage<T, (P + 1) * (P + 1)>::CHUNK_BYTES
               : Records<T, P>::bytes(nrec)) +
          1023) / 1024 * 1024;
}

template <typename T, int P, bool HAS_U0, bool SROUND, bool FULL>
__global__ void __launch_bounds__(kBlock, stage_min_blocks<T, P>())
    k_stage(const T *__restrict__ uin, const T *u0, T *out,
            const int4 *__restrict__ loc, const int2 *__restrict__ halo,
            const int *__restrict__ halo_cnt, const int2 *__restrict__ chunk_tab,
            const int2 *__restrict__ grange, const T *__restrict__ gscale, long long stride,
            int nrec,
            const int *__restrict__ chunk_list, const uint8_t *__restrict__ adv,
            const StageTab<T, P> tb, const StageCoef<T> c,
            const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_u0,
            const __grid_constant__ CUtensorMap tm_out, const CopyArgs ca) {
  constexpr int n = P + 1, NP = n * n;
  using St = Stage<T, NP>;
  // shared memory: [u chunk, later the face records][u0 chunk, later the
  // result][two mbarriers]; the first two start on 1024-byte boundaries so
  // that the swizzled tensor copies land in the Stage layout
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int front = stage_front_bytes<T, P>(nrec);
  const int bar_off = front + ((St::CHUNK_BYTES + 15) / 16) * 16;
  T *su = reinterpret_cast<T *>(smem_raw);
  T *so = reinterpret_cast<T *>(smem_raw + front);
  T *rec_base = reinterpret_cast<T *>(smem_raw);
  Records<T, P> rec{rec_base,
                    rec_base + ((nrec * n * (int)sizeof(T) + 15) / 16) * 16 / (int)sizeof(T), nrec};
  const int zero_rec = nrec - 1;

  const int chunk = chunk_list ? __ldg(chunk_list + blockIdx.x) : (int)blockIdx.x;
  const long long a0 = (long long)chunk * kBlock;
  const int el = threadIdx.x;
  const size_t sbase = (size_t)blockIdx.y * (size_t)stride * NP;
  const T *U = uin + sbase;

  // tensor copies where the element is a whole number of 16-byte slots and the
  // buffers sit on their alignment (the same for every thread of the block);
  // they go out first: nothing they need comes from a table, so no table
  // load's latency delays them
  const bool tma = St::SLOT && ca.use_tma && (smem_u32(smem_raw) & 1023u) == 0;
  const uint32_t bar0 = smem_u32(smem_raw + bar_off), bar1 = bar0 + 8;
  if (tma && el == 0) {
    mbar_init(bar0, 1);
    if constexpr (HAS_U0) mbar_init(bar1, 1);
    mbar_fence_init();
    const uint32_t bytes = (uint32_t)(kBlock * NP * sizeof(T)) + (uint32_t)ca.extra_tx;
    const int row = (int)((long long)blockIdx.y * stride + a0);
    mbar_expect_tx(bar0, bytes);
    tma_load_rows(smem_u32(su), &tm_u, row, bar0);
    if constexpr (HAS_U0) {
      mbar_expect_tx(bar1, bytes);
      tma_load_rows_hint(smem_u32(so), &tm_u0, row, bar1, l2_policy_evict_first());
    }
    if (ca.counter) atomicAdd(ca.counter, 1ull);
  }
  // The table entries, no load waiting for another: this thread's first
  // halo entry (entries past the chunk's count hold element -1, so the count
  // is not waited for), its neighbour codes (slots past the chunk's count
  // hold kEdge), the chunk's element count and geometry, its halo count.
  const uint64_t pol_last = l2_policy_evict_last();
  const int2 hk = ldg_hint(halo + (size_t)chunk * kHaloCap + el, pol_last);
  const int4 l4 = ldg_hint(loc + a0 + el, pol_last);
  const int2 ci = ldg_hint(chunk_tab + chunk, pol_last);
  const int hcnt = ldg_hint(halo_cnt + chunk, pol_last);
  // the halo element's values into registers while the chunk copies are in
  // flight
  T hv[NP];
  if (hk.x >= 0) load_elem<T, NP>(U + (size_t)hk.x * NP, hv);
  const int cnt = ci.x;
  const bool live = el < cnt;
  // beta dt D / J^2 of this geometry; 0 for an element held by the growing
  // window (its value then passes through every stage unchanged)
  T gam = c.gamma * __ldg(gscale + ci.y);
  if (adv != nullptr && live && __ldg(adv + a0 + el) == 0) gam = (T)0;
  if (!tma) {  // async copies of the u chunk (group 0) and the u0 chunk (group 1)
    const char *gu = reinterpret_cast<const char *>(U + (size_t)a0 * NP);
    const int np16 = St::pieces(cnt);
    for (int j = el; j < np16; j += kBlock)
      cp_async16(smem_raw + 16 * St::piece_dst(j), gu + 16 * (size_t)j);
    cp_async_commit();
    if constexpr (HAS_U0) {
      const char *g0 = reinterpret_cast<const char *>(u0 + sbase + (size_t)a0 * NP);
      for (int j = el; j < np16; j += kBlock)
        cp_async16(reinterpret_cast<unsigned char *>(so) + 16 * St::piece_dst(j), g0 + 16 * (size_t)j);
      cp_async_commit();
    }
  }
  // Each thread waits (bounded) for the u chunk itself: completing the
  // barrier phase makes the copied bytes visible to the waiting thread.  A
  // time-out is combined over the block at the barrier that hands the u
  // space over to the face records; the block then leaves as a whole, after
  // a bounded wait for the u0 copy it issued.
  bool ok = true;
  if (tma) {
    __syncthreads();  // the barriers exist before anyone polls them
    ok = mbar_wait(bar0, 0, ca.limit);
  } else {
    if constexpr (HAS_U0) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
  }

  T u[NP], R[NP];
  if (live && ok) St::read(su, el, u);
  // the u chunk is in registers; its space now takes the face records
  if (__syncthreads_or(!ok)) {
    if constexpr (HAS_U0) mbar_wait(bar1, 0, ca.limit);
    if (el == 0) atomicExch(ca.err, 1);
    return;
  }
  if (el == 0) {
    T z[n];
#pragma unroll
    for (int t = 0; t < n; ++t) z[t] = (T)0;
    rec.put(zero_rec, z, z);
  }
  if (live) element_records_volume<T, P>(u, tb, rec, el, R);
  if (hk.x >= 0) halo_face_record<T, P>(hv, hk.y, tb, rec, 4 * kBlock + el);
  for (int h = el + kBlock; h < hcnt; h += kBlock) {  // chunks with > kBlock halo entries
    const int2 q = __ldg(halo + (size_t)chunk * kHaloCap + h);
    T v[NP];
    load_elem<T, NP>(U + (size_t)q.x * NP, v);
    halo_face_record<T, P>(v, q.y, tb, rec, 4 * kBlock + h);
  }
  __syncthreads();

  if (live) {
    const int lq[4] = {l4.x, l4.y, l4.z, l4.w};
    element_flux<T, P, FULL>(u, R, lq, el, zero_rec, rec, tb, c);
  }

  // the u0 chunk: the same per-thread bounded wait.  With stochastic
  // rounding and p <= 3 it is combined over the block at the barrier in front
  // of the result copy (one block-wide barrier less per stage); the other
  // variants keep a barrier of their own, which bounds their live registers
  // (fewer spills; measured faster for p >= 4 and for round-to-nearest)
  if constexpr (HAS_U0) {
    if (tma) {
      ok = mbar_wait(bar1, 0, ca.limit);
      if constexpr (P >= 4 || !SROUND) {
        if (__syncthreads_or(!ok)) {
          if (el == 0) atomicExch(ca.err, 1);
          return;
        }
      }
    } else {
      cp_async_wait<0>();
      __syncthreads();
    }
  }
  if (live && ok) {
    T o[NP];
    if constexpr (HAS_U0) St::read(so, el, o);
    const uint32_t h = SROUND ? element_key<T>(a0 + el - __ldg(grange + ci.y).x, NP,
                                               (int)blockIdx.y, u)
                              : 0u;
    element_update<T, P, HAS_U0, SROUND>(u, R, o, gam, h, c);
    St::write(so, el, o);
  }
  const bool store_tma = tma && ca.store_tma && cnt == kBlock;  // a full chunk: one tiled store
  if (store_tma) fence_proxy_async_smem();
  if (__syncthreads_or(!ok)) {
    if (el == 0) atomicExch(ca.err, 1);
    return;
  }
  if (store_tma) {
    if (el == 0) {
      const int row = (int)((long long)blockIdx.y * stride + a0);
      tma_store_rows_hint(&tm_out, row, smem_u32(so), l2_policy_evict_first());
    }
    return;
  }
  {  // coalesced 16-byte stores of the result chunk
    char *go = reinterpret_cast<char *>(out + sbase + (size_t)a0 * NP);
    const int np16 = St::pieces(cnt);
    for (int j = el; j < np16; j += kBlock)
      *reinterpret_cast<float4 *>(go + 16 * (size_t)j) =
          *reinterpret_cast<const float4 *>(reinterpret_cast<unsigned char *>(so) + 16 * St::piece_dst(j));
  }
}

// ---- persistent variant: each block walks many chunks, one ahead ---------
//
// The kernel above spends a block's life in three phases -- wait for the
// chunk copies and the tables, compute, store -- and with the SM's few blocks
// it often has every block in the same phase.  This variant launches a
// few blocks per SM that stay resident and walk the work items (density,
// chunk) item = blockIdx.x + k gridDim.x, density-major so that the items in
// flight are neighbouring chunks of one density (their halos come from L2).
// Everything the next item needs is fetched behind the current item's work:
// its u chunk (tensor copy) as soon as this item's u is in registers, its
// neighbour codes, halo entry and halo element values (registers) right
// after, and its u0 chunk into the second of two u0 / result buffers, whose
// previous result store has long been read.  Shared memory: [u chunk]
// [u0 / result chunk x 2][face records][two mbarriers]; the chunks start on
// 1024-byte boundaries (hardware swizzle).  Tensor copies only (element rows
// of whole 16-byte slots); every item gives the same bits as the kernel above
// (same arithmetic, same rounding keys).
template <typename T, int P>
__host__ __device__ constexpr int pipe_chunk_bytes() {
  return (Stage<T, (P + 1) * (P + 1)>::CHUNK_BYTES + 1023) / 1024 * 1024;
}

template <typename T, int P>
int pipe_smem_bytes(int halo_max) {
  const int nrec = 4 * kBlock + halo_max + 1;
  return 3 * pipe_chunk_bytes<T, P>() + Records<T, P>::bytes(nrec) + 16;
}

constexpr int kPipeMinBlocks = blocks_for_regs(128);  // 128 registers per thread
// the variants that have a persistent kernel: FP32 with whole-slot rows and
// at least two such blocks per SM in shared memory (p = 1, 3)
template <typename T, int P>
constexpr bool kHasPipe = sizeof(T) == 4 && (P == 1 || P == 3);

// What one thread needs of a work item besides the chunk copies.
template <typename T, int P>
struct PipeItem {
  int sd, chunk;   // density, chunk
  int2 ci;         // {elements in the mesh, geometry}
  T gam;           // beta dt D / J^2, 0 for an element held by the growing window
  int4 l4;         // neighbour codes of this thread's element
  int hcnt;        // halo entries of the chunk
  int2 hk;         // this thread's first halo entry
  T hv[(P + 1) * (P + 1)];  // its element values
};

template <typename T, int P>
__device__ __forceinline__ void pipe_fetch(PipeItem<T, P> &it, long long item, int nch, int el,
                                           const T *__restrict__ uin, long long stride,
                                           const int4 *__restrict__ loc,
                                           const int2 *__restrict__ halo,
                                           const int *__restrict__ halo_cnt,
                                           const int2 *__restrict__ chunk_tab,
                                           const T *__restrict__ gscale,
                                           const int *__restrict__ chunk_list,
                                           const uint8_t *__restrict__ adv, T gamma) {
  constexpr int NP = (P + 1) * (P + 1);
  it.sd = (int)(item / nch);
  const int x = (int)(item - (long long)it.sd * nch);
  it.chunk = chunk_list ? __ldg(chunk_list + x) : x;
  const long long a0 = (long long)it.chunk * kBlock;
  it.ci = __ldg(chunk_tab + it.chunk);
  const bool live = el < it.ci.x;
  it.gam = gamma * __ldg(gscale + it.ci.y);
  if (adv != nullptr && live && __ldg(adv + a0 + el) == 0) it.gam = (T)0;
  it.l4 = live ? __ldg(loc + a0 + el) : make_int4(kEdge, kEdge, kEdge, kEdge);
  it.hcnt = __ldg(halo_cnt + it.chunk);
  it.hk = __ldg(halo + (size_t)it.chunk * kHaloCap + el);
  if (it.hk.x >= 0)
    load_elem<T, NP>(uin + (size_t)it.sd * (size_t)stride * NP + (size_t)it.hk.x * NP, it.hv);
}

template <typename T, int P, bool HAS_U0, bool SROUND, bool FULL>
__global__ void __launch_bounds__(kBlock, kPipeMinBlocks)
    k_stage_pipe(const T *__restrict__ uin, const T *u0, T *out,
                 const int4 *__restrict__ loc, const int2 *__restrict__ halo,
                 const int *__restrict__ halo_cnt, const int2 *__restrict__ chunk_tab,
                 const int2 *__restrict__ grange, const T *__restrict__ gscale, long long stride,
                 int nrec, const int *__restrict__ chunk_list, const uint8_t *__restrict__ adv,
                 const StageTab<T, P> tb, const StageCoef<T> c,
                 const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_u0,
                 const __grid_constant__ CUtensorMap tm_out, const CopyArgs ca, long long n_items,
                 int nch) {
  constexpr int n = P + 1, NP = n * n;
  using St = Stage<T, NP>;
  constexpr int CB = pipe_chunk_bytes<T, P>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  T *su = reinterpret_cast<T *>(smem_raw);
  unsigned char *so_raw = smem_raw + CB;  // two buffers of CB bytes
  T *rec_base = reinterpret_cast<T *>(smem_raw + 3 * CB);
  Records<T, P> rec{rec_base,
                    rec_base + ((nrec * n * (int)sizeof(T) + 15) / 16) * 16 / (int)sizeof(T), nrec};
  const int zero_rec = nrec - 1;
  const uint32_t bar0 = smem_u32(smem_raw + 3 * CB + Records<T, P>::bytes(nrec)), bar1 = bar0 + 8;
  const int el = threadIdx.x;
  if ((smem_u32(smem_raw) & 1023u) != 0) {  // the swizzled copies need this; never expected
    if (el == 0) atomicExch(ca.err, 2);
    return;
  }
  const long long G = gridDim.x;
  long long item = blockIdx.x;
  // first row of an item's chunk in the 2D state tensor [densities x padded elements]
  auto item_row = [&](long long it) -> int {
    const long long sd = it / nch, x = it - sd * nch;
    const long long chunk = chunk_list ? __ldg(chunk_list + x) : x;
    return (int)(sd * stride + chunk * kBlock);
  };
  const uint32_t bytes = (uint32_t)(kBlock * NP * sizeof(T)) + (uint32_t)ca.extra_tx;
  if (el == 0) {
    mbar_init(bar0, 1);
    if constexpr (HAS_U0) mbar_init(bar1, 1);
    mbar_fence_init();
    if (item < n_items) {
      const int row = item_row(item);
      mbar_expect_tx(bar0, bytes);
      tma_load_rows(smem_u32(su), &tm_u, row, bar0);
      if constexpr (HAS_U0) {
        mbar_expect_tx(bar1, bytes);
        tma_load_rows(smem_u32(so_raw), &tm_u0, row, bar1);
      }
      if (ca.counter) atomicAdd(ca.counter, 1ull);
    }
  }
  PipeItem<T, P> cur;
  if (item < n_items)
    pipe_fetch<T, P>(cur, item, nch, el, uin, stride, loc, halo, halo_cnt, chunk_tab, gscale,
                     chunk_list, adv, c.gamma);
  __syncthreads();  // the barriers exist before anyone polls them

  // both barriers complete one phase per item: parity ph for this item;
  // the u0 / result buffer of the k-th item of the block is buffer k & 1
  for (uint32_t ph = 0; item < n_items; item += G, ph ^= 1u) {
    T *so = reinterpret_cast<T *>(so_raw + (ph ? CB : 0));
    const long long a0 = (long long)cur.chunk * kBlock;
    const int cnt = cur.ci.x;
    const bool live = el < cnt;
    bool ok = mbar_wait(bar0, ph, ca.limit);
    T u[NP], R[NP];
    if (live && ok) St::read(su, el, u);
    const long long next = item + G;
    const bool more = next < n_items;
    // order these reads of su before the tensor copy that refills it
    fence_proxy_async_smem();
    if (__syncthreads_or(!ok)) {  // leave as a block, after bounded waits for copies in flight
      if constexpr (HAS_U0) mbar_wait(bar1, ph, ca.limit);
      if (el == 0) {
        asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
        atomicExch(ca.err, 1);
      }
      return;
    }
    // this item's u is in registers: the next item's u chunk and tables come
    // in behind the work
    if (el == 0 && more) {
      mbar_expect_tx(bar0, bytes);
      tma_load_rows(smem_u32(su), &tm_u, item_row(next), bar0);
      if (ca.counter) atomicAdd(ca.counter, 1ull);
    }
    PipeItem<T, P> nxt;
    if (more)
      pipe_fetch<T, P>(nxt, next, nch, el, uin, stride, loc, halo, halo_cnt, chunk_tab, gscale,
                       chunk_list, adv, c.gamma);
    if (el == 0) {
      T z[n];
#pragma unroll
      for (int t = 0; t < n; ++t) z[t] = (T)0;
      rec.put(zero_rec, z, z);
    }
    if (live) element_records_volume<T, P>(u, tb, rec, el, R);
    if (cur.hk.x >= 0) halo_face_record<T, P>(cur.hv, cur.hk.y, tb, rec, 4 * kBlock + el);
    const T *U = uin + (size_t)cur.sd * (size_t)stride * NP;
    for (int h = el + kBlock; h < cur.hcnt; h += kBlock) {  // chunks with > kBlock halo entries
      const int2 q = __ldg(halo + (size_t)cur.chunk * kHaloCap + h);
      T v[NP];
      load_elem<T, NP>(U + (size_t)q.x * NP, v);
      halo_face_record<T, P>(v, q.y, tb, rec, 4 * kBlock + h);
    }
    __syncthreads();
    if (live) {
      const int lq[4] = {cur.l4.x, cur.l4.y, cur.l4.z, cur.l4.w};
      element_flux<T, P, FULL>(u, R, lq, el, zero_rec, rec, tb, c);
    }
    if constexpr (HAS_U0) ok = mbar_wait(bar1, ph, ca.limit);
    if (live && ok) {
      T o[NP];
      if constexpr (HAS_U0) St::read(so, el, o);
      const uint32_t h = SROUND ? element_key<T>(a0 + el - __ldg(grange + cur.ci.y).x, NP,
                                                 cur.sd, u)
                                : 0u;
      element_update<T, P, HAS_U0, SROUND>(u, R, o, cur.gam, h, c);
      St::write(so, el, o);
    }
    const bool store_tma = ca.store_tma && cnt == kBlock;  // a full chunk: one tiled store
    if (store_tma) fence_proxy_async_smem();
    if (__syncthreads_or(!ok)) {  // the u0 wait gave up; the next u copy may be in flight
      if (more) mbar_wait(bar0, ph ^ 1u, ca.limit);
      if (el == 0) {
        asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
        atomicExch(ca.err, 1);
      }
      return;
    }
    if (store_tma) {
      if (el == 0) {
        asm volatile(
            "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                reinterpret_cast<uint64_t>(&tm_out)),
            "r"(0), "r"((int)((long long)cur.sd * stride + a0)), "r"(smem_u32(so))
            : "memory");
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
      }
    } else {  // coalesced 16-byte stores of a partial chunk
      char *go = reinterpret_cast<char *>(out + (size_t)cur.sd * (size_t)stride * NP +
                                          (size_t)a0 * NP);
      const int np16 = St::pieces(cnt);
      for (int j = el; j < np16; j += kBlock)
        *reinterpret_cast<float4 *>(go + 16 * (size_t)j) =
            *reinterpret_cast<const float4 *>(reinterpret_cast<unsigned char *>(so) +
                                              16 * St::piece_dst(j));
    }
    if constexpr (HAS_U0) {
      // the next u0 goes into the other buffer, whose last reader was the
      // previous item's result store: wait until every store but this item's
      // own has been read (all of them after a partial chunk, which committed
      // none); a partial chunk's threads read their buffer one item earlier,
      // ordered by this item's fences and barriers
      if (el == 0 && more) {
        if (store_tma) asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
        else asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
        mbar_expect_tx(bar1, bytes);
        tma_load_rows(smem_u32(so_raw + (ph ? 0 : CB)), &tm_u0, item_row(next), bar1);
      }
    }
    if (more) cur = nxt;
  }
  // shared memory must outlive the reads of the last result stores
  if (el == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}

template <typename T, int P>
int stage_smem_bytes(int halo_max) {
  const int nrec = 4 * kBlock + halo_max + 1;
  const int chunk = Stage<T, (P + 1) * (P + 1)>::CHUNK_BYTES;
  return stage_front_bytes<T, P>(nrec) + ((chunk + 15) / 16) * 16 + 16;
}

template <typename T, int P>
StageTab<T, P> make_tab(const Gll &g) {
  StageTab<T, P> t;
  constexpr int n = P + 1;
  for (int k = 0; k < n * n; ++k) {
    if constexpr (sizeof(T) == 4) {
      t.D[k] = g.Df[k];
      t.D2[k] = g.D2f[k];
    } else {
      t.D[k] = g.D[k];
      t.D2[k] = g.D2[k];
    }
  }
  for (int m = 0; m < n; ++m) {
    t.Dout[m] = t.D[P * n + m];
    t.Dout[n + m] = -t.D[m];
  }
  t.inv_w = (T)(1.0 / g.w[0]);
  for (int ip = 0; ip < n / 2; ++ip)
    for (int m = 0; m < n; ++m) {
      t.D2x[ip * n + m].x = t.D2[2 * ip * n + m];
      t.D2x[ip * n + m].y = t.D2[(2 * ip + 1) * n + m];
    }
  for (int k = 0; k < n * n; ++k) t.D2y[k].x = t.D2y[k].y = t.D2[k];
  return t;
}

template <typename T, int P>
cudaError_t launch_stage_p(const T *u, const T *u0, T *out, const Geometry &geo,
                           long long stride, int m, const Gll &g, const StageCoef<T> &c,
                           cudaStream_t s, const ChunkSel &sel, const StageCopies &cp) {
  const long long nch = sel.list ? sel.count : geo.n_chunks();
  if (geo.n_pad <= 0 || m <= 0 || nch <= 0) return cudaSuccess;
  if (nch > geo.n_chunks()) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)nch, (unsigned)m);
  const T *gscale;
  if constexpr (sizeof(T) == 8) gscale = geo.d_gscale_d;
  else gscale = geo.d_gscale_f;
  const StageTab<T, P> tb = make_tab<T, P>(g);
  const int nrec = 4 * kBlock + geo.halo_max + 1;
  const int smem = stage_smem_bytes<T, P>(geo.halo_max);
  static int attr_bytes = 0;  // per instantiation: largest size configured so far
  constexpr bool kSR = sizeof(T) == 4;  // stochastic-rounding variants exist in FP32 only
  if (smem > attr_bytes) {
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kern) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    };
    set(k_stage<T, P, true, false, false>);
    set(k_stage<T, P, false, false, false>);
    set(k_stage<T, P, true, false, true>);
    set(k_stage<T, P, false, false, true>);
    if constexpr (kSR) {
      set(k_stage<T, P, true, kSR, false>);
      set(k_stage<T, P, false, kSR, false>);
      set(k_stage<T, P, true, kSR, true>);
      set(k_stage<T, P, false, kSR, true>);
    }
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  const bool full = c.pen != (T)0 || c.wallA;
  CopyArgs ca;
  ca.use_tma = cp.map_u != nullptr && (u0 == nullptr || cp.map_u0 != nullptr) ? cp.use_tma : 0;
  ca.extra_tx = cp.extra_tx;
  ca.limit = cp.limit;
  ca.err = cp.err;
  ca.counter = cp.counter;
  if (ca.use_tma && ca.err == nullptr) ca.use_tma = 0;
  ca.store_tma = ca.use_tma && cp.map_out != nullptr ? 1 : 0;
  const CUtensorMap zero_map{};
  const CUtensorMap &mu = ca.use_tma ? *cp.map_u : zero_map;
  const CUtensorMap &mu0 = ca.use_tma && u0 ? *cp.map_u0 : zero_map;
  const CUtensorMap &mo = ca.store_tma ? *cp.map_out : zero_map;
  if constexpr (kHasPipe<T, P>) {
    if (cp.pipe_blocks > 0 && ca.store_tma) {
      const int psmem = pipe_smem_bytes<T, P>(geo.halo_max);
      static int pipe_attr = 0;
      if (psmem > pipe_attr) {
        cudaError_t e = cudaSuccess;
        auto set = [&](auto kern) {
          if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
        };
        set(k_stage_pipe<T, P, true, false, false>);
        set(k_stage_pipe<T, P, false, false, false>);
        set(k_stage_pipe<T, P, true, false, true>);
        set(k_stage_pipe<T, P, false, false, true>);
        set(k_stage_pipe<T, P, true, true, false>);
        set(k_stage_pipe<T, P, false, true, false>);
        set(k_stage_pipe<T, P, true, true, true>);
        set(k_stage_pipe<T, P, false, true, true>);
        if (e != cudaSuccess) return e;
        pipe_attr = psmem;
      }
      int dev = 0, nsm = 0;
      cudaError_t e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      const long long items = nch * (long long)m;
      const long long G = std::min<long long>(items, (long long)nsm * cp.pipe_blocks);
      auto gop = [&](auto kern) {
        kern<<<(unsigned)G, kBlock, psmem, s>>>(u, u0, out, geo.d_loc, geo.d_halo, geo.d_halo_cnt,
                                                geo.d_chunk, geo.d_grange, gscale, stride, nrec,
                                                sel.list, sel.adv, tb, c, mu, mu0, mo, ca, items,
                                                (int)nch);
      };
      if (c.sround) {
        if (u0) full ? gop(k_stage_pipe<T, P, true, true, true>) : gop(k_stage_pipe<T, P, true, true, false>);
        else full ? gop(k_stage_pipe<T, P, false, true, true>) : gop(k_stage_pipe<T, P, false, true, false>);
      } else {
        if (u0) full ? gop(k_stage_pipe<T, P, true, false, true>) : gop(k_stage_pipe<T, P, true, false, false>);
        else full ? gop(k_stage_pipe<T, P, false, false, true>) : gop(k_stage_pipe<T, P, false, false, false>);
      }
      return cudaGetLastError();
    }
  }
  auto go = [&](auto kern) {
    kern<<<grid, kBlock, smem, s>>>(u, u0, out, geo.d_loc, geo.d_halo, geo.d_halo_cnt,
                                    geo.d_chunk, geo.d_grange, gscale, stride, nrec, sel.list,
                                    sel.adv, tb, c, mu, mu0, mo, ca);
  };
  if (kSR && c.sround) {
    if (u0) full ? go(k_stage<T, P, true, kSR, true>) : go(k_stage<T, P, true, kSR, false>);
    else full ? go(k_stage<T, P, false, kSR, true>) : go(k_stage<T, P, false, kSR, false>);
  } else {
    if (u0) full ? go(k_stage<T, P, true, false, true>) : go(k_stage<T, P, true, false, false>);
    else full ? go(k_stage<T, P, false, false, true>) : go(k_stage<T, P, false, false, false>);
  }
  return cudaGetLastError();
}

// Blocks of the persistent kernel that fit on one SM (shared memory and
// registers), 0 where the variant does not exist.
template <typename T, int P>
int stage_pipe_max_blocks_p(const Geometry &geo) {
  if constexpr (!kHasPipe<T, P>) {
    return 0;
  } else {
    const int psmem = pipe_smem_bytes<T, P>(geo.halo_max);
    if (cudaFuncSetAttribute(k_stage_pipe<T, P, true, true, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, psmem) != cudaSuccess)
      return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage_pipe<T, P, true, true, false>,
                                                      kBlock, psmem) != cudaSuccess)
      return 0;
    return nb;
  }
}

template <typename T>
int stage_pipe_max_blocks_any(int p, const Geometry &geo) {
  switch (p) {
    case 1: return stage_pipe_max_blocks_p<T, 1>(geo);
    case 3: return stage_pipe_max_blocks_p<T, 3>(geo);
    default: return 0;
  }
}

template <typename T>
cudaError_t launch_stage_any(int p, const T *u, const T *u0, T *out, const Geometry &geo,
                             long long stride, int m, const Gll &g, const StageCoef<T> &c,
                             cudaStream_t s, const ChunkSel &sel, const StageCopies &cp) {
  switch (p) {
    case 1: return launch_stage_p<T, 1>(u, u0, out, geo, stride, m, g, c, s, sel, cp);
    case 2: return launch_stage_p<T, 2>(u, u0, out, geo, stride, m, g, c, s, sel, cp);
    case 3: return launch_stage_p<T, 3>(u, u0, out, geo, stride, m, g, c, s, sel, cp);
    case 4: return launch_stage_p<T, 4>(u, u0, out, geo, stride, m, g, c, s, sel, cp);
    case 5: return launch_stage_p<T, 5>(u, u0, out, geo, stride, m, g, c, s, sel, cp);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
