// dg_stage_tc.cu -- the FP32 stage at p = 5 with the element contractions on
// the fifth-generation tensor cores.
//
// Each element's update (Sec. 3.1: a small dense system per element, the
// elements independent within a stage) needs, from the element's own 36
// nodal values u, the volume term (DD)u along x and y and the outward
// normal derivative at the nodes of its four faces: a dense [60 x 36]
// operator Op applied to u.  For a chunk of kBlock = 128 elements this is the GEMM
//   [128 x 64] = U [128 x 48] . Op^T [48 x 64]     (K, N padded with zeros)
// run as tcgen05.mma kind::f16 -- FP16 operands from shared memory, FP32
// accumulators in tensor memory -- one M = 128 tile per 128 elements.
// FP16 alone would lose the FP32 state's accuracy, so both operands are
// split (defect correction): per element u is scaled by a power of two
// 2^k so that max |u| lies in [1, 2) (exact), v = 2^k u = v_hi + v_lo with
// v_hi = fp16(v), v_lo = fp16(v - v_hi), and Op = Op_hi + Op_lo likewise;
// the products v_hi Op_hi + v_lo Op_hi + v_hi Op_lo (the dropped v_lo Op_lo
// is ~2^-22 of the element's largest term) accumulate in FP32, and the
// result is scaled back by 2^-k.  Each thread then reads its own element's
// row of the accumulator (tcgen05.ld, lane = element) and finishes the
// stage like the CUDA-core kernel: face records, halo faces, fluxes and
// lifting, the Runge-Kutta update with the same rounding.
#include <cuda_fp16.h>

#include <mutex>

#include "dg_stage.cuh"

namespace dg {
namespace {

constexpr int kTcP = 5, kTcN = kTcP + 1, kTcNP = kTcN * kTcN;
constexpr int kTcK = 48;                         // 36 nodes padded to 3 MMA steps of 16
constexpr int kTcOut = 64;                       // 36 volume + 24 face derivatives + 4 zero
constexpr int kTcTiles = kBlock / 128;           // M = 128 tiles per chunk
static_assert(kBlock % 128 == 0, "whole M = 128 tiles");
constexpr int kTcCols = kTcTiles * kTcOut;       // tensor-memory columns (a power of 2)
constexpr int kTcLBO = 128;                      // bytes between K-adjacent core matrices
constexpr int kTcSBO = (kTcK / 8) * kTcLBO;      // bytes between 8-row groups (768)
constexpr int kTcATile = 16 * kTcSBO;            // one M = 128 tile of U (12 KB)
constexpr int kTcABytes = kTcTiles * kTcATile;   // kBlock rows of U, hi or lo
constexpr int kTcBBytes = (kTcOut / 8) * kTcSBO; // 64 rows of Op, hi or lo (6 KB)

// Byte offset of (row r, column k) in a K-major operand of 48 FP16 columns
// without swizzle: core matrices of 8 rows x 16 bytes, K-adjacent ones
// kTcLBO apart, row groups kTcSBO apart.
__host__ __device__ constexpr int tc_off(int r, int k) {
  return (r / 8) * kTcSBO + (k / 8) * kTcLBO + (r % 8) * 16 + (k % 8) * 2;
}

// The split operator, both halves in the core-matrix layout above.
struct TcOperand {
  uint4 v[2 * kTcBBytes / 16];  // hi, then lo
};

// The split operator in global memory, written once per device by
// k_tc_operand_init; each block fetches it with one bulk copy.
__device__ __align__(128) uint4 g_tc_operand[2 * kTcBBytes / 16];

__global__ void k_tc_operand_init(const __grid_constant__ TcOperand op) {
  for (int j = threadIdx.x; j < 2 * kTcBBytes / 16; j += blockDim.x) g_tc_operand[j] = op.v[j];
}

// Untiled bulk copy of `bytes` (a multiple of 16) from global to shared
// memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kTcLBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((kTcSBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, FP16 A and B, both
// K-major, N = 64, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (0u << 7) | (0u << 10) |
                              ((uint32_t)(kTcOut >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}
// Arrive on the mbarrier once every MMA this thread issued has completed
// (its shared-memory operands read, its accumulators written).
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   bar)
               : "memory");
}
__device__ __forceinline__ void tc_alloc(uint32_t slot) {  // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot),
               "n"(kTcCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr) {  // one whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr),
               "n"(kTcCols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
// 32 consecutive accumulator columns of this thread's lane (warp-wide), and
// the wait for them, in one statement so no use of v can move above the wait.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

__host__ __device__ constexpr int tc_front_bytes(int nrec) {
  return ((Stage<float, kTcNP>::CHUNK_BYTES > Records<float, kTcP>::bytes(nrec)
               ? (Stage<float, kTcNP>::CHUNK_BYTES > 2 * kTcABytes ? Stage<float, kTcNP>::CHUNK_BYTES
                                                                   : 2 * kTcABytes)
               : (Records<float, kTcP>::bytes(nrec) > 2 * kTcABytes ? Records<float, kTcP>::bytes(nrec)
                                                                    : 2 * kTcABytes)) +
          1023) / 1024 * 1024;
}
constexpr int kTcChunkRound = (Stage<float, kTcNP>::CHUNK_BYTES + 1023) / 1024 * 1024;

int tc_smem_bytes(int halo_max) {
  const int nrec = 4 * kBlock + halo_max + 1;
  return tc_front_bytes(nrec) + kTcChunkRound + 2 * kTcBBytes + 32;
}

// Shared memory: [front: u chunk -> U_hi, U_lo operands -> face records]
// [u0 chunk, then the result][Op_hi, Op_lo][3 mbarriers, tensor-memory slot].
// Launched only with tensor copies (rows of 144 bytes are whole 16-byte
// slots) and a full-chunk tensor store.
template <bool HAS_U0, bool SROUND, bool FULL>
__global__ void __launch_bounds__(kBlock, blocks_for_regs(128))
    k_stage_tc(const float *__restrict__ uin, const float *u0, float *out,
               const int4 *__restrict__ loc, const int2 *__restrict__ halo,
               const int *__restrict__ halo_cnt, const int2 *__restrict__ chunk_tab,
               const int2 *__restrict__ grange, const float *__restrict__ gscale, long long stride,
               int nrec, const int *__restrict__ chunk_list, const uint8_t *__restrict__ adv,
               const StageTab<float, kTcP> tb, const StageCoef<float> c,
               const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_u0,
               const __grid_constant__ CUtensorMap tm_out, const CopyArgs ca) {
  constexpr int P = kTcP, n = kTcN, NP = kTcNP;
  using St = Stage<float, NP>;
  using Fc = Faces<P>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int front = tc_front_bytes(nrec);
  float *su = reinterpret_cast<float *>(smem_raw);
  float *so = reinterpret_cast<float *>(smem_raw + front);
  unsigned char *sb = smem_raw + front + kTcChunkRound;
  const uint32_t bar0 = smem_u32(sb + 2 * kTcBBytes), bar1 = bar0 + 8, bar2 = bar0 + 16;
  volatile uint32_t *tslot = reinterpret_cast<volatile uint32_t *>(sb + 2 * kTcBBytes + 24);
  float *rec_base = reinterpret_cast<float *>(smem_raw);
  Records<float, P> rec{rec_base,
                        rec_base + ((nrec * n * (int)sizeof(float) + 15) / 16) * 16 / (int)sizeof(float),
                        nrec};
  const int zero_rec = nrec - 1;
  const int el = threadIdx.x, warp = el >> 5;
  if ((smem_u32(smem_raw) & 1023u) != 0) {  // the swizzle-free copies still want this; never expected
    if (el == 0) atomicExch(ca.err, 2);
    return;
  }

  const int chunk = chunk_list ? __ldg(chunk_list + blockIdx.x) : (int)blockIdx.x;
  const long long a0 = (long long)chunk * kBlock;
  const size_t sbase = (size_t)blockIdx.y * (size_t)stride * NP;
  const float *U = uin + sbase;

  // the copies go out first (nothing they need comes from a table)
  if (el == 0) {
    mbar_init(bar0, 1);
    if constexpr (HAS_U0) mbar_init(bar1, 1);
    mbar_init(bar2, 1);
    mbar_fence_init();
    const uint32_t bytes = (uint32_t)(kBlock * NP * sizeof(float)) + (uint32_t)ca.extra_tx;
    const int row = (int)((long long)blockIdx.y * stride + a0);
    // the u chunk and the split operator complete the same barrier phase
    mbar_expect_tx(bar0, bytes + 2 * kTcBBytes);
    tma_load_rows(smem_u32(su), &tm_u, row, bar0);
    bulk_load(smem_u32(sb), g_tc_operand, 2 * kTcBBytes, bar0);
    if constexpr (HAS_U0) {
      mbar_expect_tx(bar1, bytes);
      tma_load_rows_hint(smem_u32(so), &tm_u0, row, bar1, l2_policy_evict_first());
    }
    if (ca.counter) atomicAdd(ca.counter, 1ull);
  }
  // table entries, no load waiting for another (as in k_stage)
  const uint64_t pol_last = l2_policy_evict_last();
  const int2 hk = ldg_hint(halo + (size_t)chunk * kHaloCap + el, pol_last);
  const int4 l4 = ldg_hint(loc + a0 + el, pol_last);
  const int2 ci = ldg_hint(chunk_tab + chunk, pol_last);
  const int hcnt = ldg_hint(halo_cnt + chunk, pol_last);
  if (warp == 0) tc_alloc(smem_u32((const void *)tslot));
  float hv[NP];
  if (hk.x >= 0) load_elem<float, NP>(U + (size_t)hk.x * NP, hv);
  const int cnt = ci.x;
  const bool live = el < cnt;
  float gam = c.gamma * __ldg(gscale + ci.y);
  if (adv != nullptr && live && __ldg(adv + a0 + el) == 0) gam = 0.0f;
  tc_fence_before();
  __syncthreads();  // barriers initialised, tensor-memory address published
  tc_fence_after();
  const uint32_t tmem = *tslot;
  bool ok = mbar_wait(bar0, 0, ca.limit);
  float u[NP], R[NP];
  if (live && ok) St::read(su, el, u);
  if (__syncthreads_or(!ok)) {  // the front buffer is free after this barrier
    if constexpr (HAS_U0) mbar_wait(bar1, 0, ca.limit);
    if (warp == 0) tc_dealloc(tmem);
    if (el == 0) atomicExch(ca.err, 1);
    return;
  }

  // the halo element's face record, in registers until the front buffer is
  // free for records again
  float htr[n], hd[n];
  if (hk.x >= 0) {
    switch (hk.y) {
      case 0: face_record<float, P>(hv, 0, tb, htr, hd); break;
      case 1: face_record<float, P>(hv, 1, tb, htr, hd); break;
      case 2: face_record<float, P>(hv, 2, tb, htr, hd); break;
      default: face_record<float, P>(hv, 3, tb, htr, hd); break;
    }
  }
  // this element's row of U_hi and U_lo: u scaled by 2^kx, split in FP16,
  // written 8 columns (one core-matrix row, 16 bytes) at a time
  float unscale = 1.0f, scale = 0.0f;
  if (live) {
    float mx = 0.0f;
#pragma unroll
    for (int k = 0; k < NP; ++k) mx = fmaxf(mx, fabsf(u[k]));
    const int e = (int)((__float_as_uint(mx) >> 23) & 0xffu);  // 0: zero or subnormal
    const int kx = e == 0 ? 0 : max(127 - e, -126);
    scale = __uint_as_float((uint32_t)(127 + kx) << 23);
    unscale = __uint_as_float((uint32_t)(127 - kx) << 23);
  }
  {  // two columns per instruction: packed multiply, conversions and subtraction
    const int t = el >> 7, r = el & 127;
    const float2 sc2 = make_float2(scale, scale);
#pragma unroll
    for (int kb = 0; kb < kTcK / 8; ++kb) {
      uint4 hi, lo;
      __half2 *h = reinterpret_cast<__half2 *>(&hi), *l = reinterpret_cast<__half2 *>(&lo);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 8 * kb + 2 * q;
        if (k < NP) {  // NP is even: both columns are nodes
          const float2 v = live ? __fmul2_rn(make_float2(u[k], u[k + 1]), sc2) : make_float2(0.0f, 0.0f);
          const __half2 vh = __float22half2_rn(v);
          h[q] = vh;
          l[q] = __float22half2_rn(__ffma2_rn(__half22float2(vh), make_float2(-1.0f, -1.0f), v));
        } else {
          h[q] = l[q] = __float2half2_rn(0.0f);
        }
      }
      *reinterpret_cast<uint4 *>(smem_raw + t * kTcATile + tc_off(r, 8 * kb)) = hi;
      *reinterpret_cast<uint4 *>(smem_raw + kTcABytes + t * kTcATile + tc_off(r, 8 * kb)) = lo;
    }
  }
  fence_proxy_async_smem();  // the operands are read by the tensor cores
  __syncthreads();
  if (el == 0) {
    tc_fence_after();
    const uint32_t a_base = smem_u32(smem_raw), b_base = smem_u32(sb);
#pragma unroll
    for (int t = 0; t < kTcTiles; ++t) {
      const uint32_t d = tmem + (uint32_t)(t * kTcOut);
#pragma unroll
      for (int ks = 0; ks < kTcK / 16; ++ks) {
        const uint64_t ahi = tc_desc(a_base + t * kTcATile + ks * 2 * kTcLBO);
        const uint64_t alo = tc_desc(a_base + kTcABytes + t * kTcATile + ks * 2 * kTcLBO);
        const uint64_t bhi = tc_desc(b_base + ks * 2 * kTcLBO);
        const uint64_t blo = tc_desc(b_base + kTcBBytes + ks * 2 * kTcLBO);
        tc_mma(d, ahi, bhi, ks > 0);
        tc_mma(d, alo, bhi, 1);
        tc_mma(d, ahi, blo, 1);
      }
    }
    tc_commit(bar2);
  }
  const bool ok2 = mbar_wait(bar2, 0, ca.limit);
  tc_fence_after();
  // the tensor cores have read the operands: the front buffer takes the records
  if (el == 0) {
    float z[n];
#pragma unroll
    for (int t = 0; t < n; ++t) z[t] = 0.0f;
    rec.put(zero_rec, z, z);
  }
  if (hk.x >= 0) rec.put(4 * kBlock + el, htr, hd);
  // lane = element of the tile, columns: 0..35 volume, 36..59 face derivatives
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * kTcOut);
  {
    float v[32];
    tc_ld32(trow + 32, v);
    if (live && ok2) {
#pragma unroll
      for (int k = 32; k < NP; ++k) R[k] = v[k - 32] * unscale;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        float tr[n], d[n];
#pragma unroll
        for (int t = 0; t < n; ++t) {
          tr[t] = u[Fc::own(f, t)];
          d[t] = v[NP - 32 + f * n + t] * unscale;
        }
        rec.put(f * kBlock + el, tr, d);
      }
    }
    tc_ld32(trow, v);
    if (live && ok2) {
      const float2 us2 = make_float2(unscale, unscale);
#pragma unroll
      for (int k = 0; k < 32; k += 2) {
        const float2 w = __fmul2_rn(make_float2(v[k], v[k + 1]), us2);
        R[k] = w.x;
        R[k + 1] = w.y;
      }
    }
  }
  for (int hh = el + kBlock; hh < hcnt; hh += kBlock) {  // chunks with > kBlock halo entries
    const int2 q = __ldg(halo + (size_t)chunk * kHaloCap + hh);
    float w[NP];
    load_elem<float, NP>(U + (size_t)q.x * NP, w);
    halo_face_record<float, P>(w, q.y, tb, rec, 4 * kBlock + hh);
  }
  tc_fence_before();
  const bool bad = __syncthreads_or(!ok2);
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem);  // every read of the accumulators is complete
  if (bad) {
    if constexpr (HAS_U0) mbar_wait(bar1, 0, ca.limit);
    if (el == 0) atomicExch(ca.err, 1);
    return;
  }

  if (live) {
    const int lq[4] = {l4.x, l4.y, l4.z, l4.w};
    element_flux<float, P, FULL>(u, R, lq, el, zero_rec, rec, tb, c);
  }
  if constexpr (HAS_U0) {
    ok = mbar_wait(bar1, 0, ca.limit);
    if (__syncthreads_or(!ok)) {
      if (el == 0) atomicExch(ca.err, 1);
      return;
    }
  }
  if (live) {
    float o[NP];
    if constexpr (HAS_U0) St::read(so, el, o);
    const uint32_t hsh = SROUND ? element_key<float>(a0 + el - __ldg(grange + ci.y).x, NP,
                                                     (int)blockIdx.y, u)
                                : 0u;
    element_update<float, P, HAS_U0, SROUND>(u, R, o, gam, hsh, c);
    St::write(so, el, o);
  }
  const bool store_tma = ca.store_tma && cnt == kBlock;
  if (store_tma) fence_proxy_async_smem();
  __syncthreads();
  if (store_tma) {
    if (el == 0) {
      const int row = (int)((long long)blockIdx.y * stride + a0);
      tma_store_rows_hint(&tm_out, row, smem_u32(so), l2_policy_evict_first());
    }
    return;
  }
  {  // coalesced 16-byte stores of a partial chunk
    char *go = reinterpret_cast<char *>(out + sbase + (size_t)a0 * NP);
    const int np16 = St::pieces(cnt);
    for (int j = el; j < np16; j += kBlock)
      *reinterpret_cast<float4 *>(go + 16 * (size_t)j) =
          *reinterpret_cast<const float4 *>(reinterpret_cast<unsigned char *>(so) + 16 * St::piece_dst(j));
  }
}

// Op of order 5 from the FP64 tables, rows 0..35 the volume term of node
// (j, i) (index j*6 + i), rows 36 + 6f + t the outward derivative at node t
// of face f, split into FP16 hi + lo and laid out for the MMA.
void build_tc_operand(const Gll &g, TcOperand *out) {
  constexpr int n = kTcN;
  double Op[kTcOut][kTcK] = {};
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i)
      for (int m = 0; m < n; ++m) {
        Op[j * n + i][j * n + m] += g.D2[i * n + m];
        Op[j * n + i][m * n + i] += g.D2[j * n + m];
      }
  for (int f = 0; f < 4; ++f)
    for (int t = 0; t < n; ++t)
      for (int m = 0; m < n; ++m) {
        const double row = (f & 1) ? -g.D[m] : g.D[kTcP * n + m];
        Op[kTcNP + f * n + t][f < 2 ? t * n + m : m * n + t] = row;
      }
  unsigned char *hi = reinterpret_cast<unsigned char *>(out->v);
  unsigned char *lo = hi + kTcBBytes;
  for (int r = 0; r < kTcOut; ++r)
    for (int k = 0; k < kTcK; ++k) {
      const __half h = __double2half(Op[r][k]);
      const __half l = __double2half(Op[r][k] - (double)__half2float(h));
      *reinterpret_cast<__half *>(hi + tc_off(r, k)) = h;
      *reinterpret_cast<__half *>(lo + tc_off(r, k)) = l;
    }
}

}  // namespace

// The device copy of the split operator, written once per device ahead on
// stream s.  Not from inside a stream capture (a captured copy would run
// only with the graph): cudaErrorNotSupported then, and the CUDA-core kernel
// serves until a launch outside a capture has made the copy.
cudaError_t stage_tc_prepare(const Gll &g, cudaStream_t s) {
  if (g.p != kTcP) return cudaErrorNotSupported;
  static TcOperand op;
  static std::once_flag once;
  std::call_once(once, [&] { build_tc_operand(g, &op); });
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return e;
  if (cap != cudaStreamCaptureStatusNone) return cudaErrorNotSupported;
  k_tc_operand_init<<<1, 256, 0, s>>>(op);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  done[dev] = true;
  return cudaSuccess;
}

cudaError_t launch_stage_tc_f32(const float *u, const float *u0, float *out, const Geometry &geo,
                                long long stride, int m, const Gll &g,
                                const StageCoef<float> &c, cudaStream_t s, const ChunkSel &sel,
                                const StageCopies &cp) {
  if (g.p != kTcP) return cudaErrorNotSupported;
  const long long nch = sel.list ? sel.count : geo.n_chunks();
  if (geo.n_pad <= 0 || m <= 0 || nch <= 0) return cudaSuccess;
  if (nch > geo.n_chunks()) return cudaErrorInvalidValue;
  CopyArgs ca;
  ca.use_tma = cp.map_u != nullptr && (u0 == nullptr || cp.map_u0 != nullptr) ? cp.use_tma : 0;
  if (!ca.use_tma || cp.err == nullptr || cp.map_out == nullptr) return cudaErrorNotSupported;
  ca.store_tma = 1;
  ca.extra_tx = cp.extra_tx;
  ca.limit = cp.limit;
  ca.err = cp.err;
  ca.counter = cp.counter;
  if (const cudaError_t e = stage_tc_prepare(g, s); e != cudaSuccess) return e;
  const StageTab<float, kTcP> tb = make_tab<float, kTcP>(g);
  const int nrec = 4 * kBlock + geo.halo_max + 1;
  const int smem = tc_smem_bytes(geo.halo_max);
  static int attr_bytes = 0;
  if (smem > attr_bytes) {
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kern) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    };
    set(k_stage_tc<true, false, false>);
    set(k_stage_tc<false, false, false>);
    set(k_stage_tc<true, false, true>);
    set(k_stage_tc<false, false, true>);
    set(k_stage_tc<true, true, false>);
    set(k_stage_tc<false, true, false>);
    set(k_stage_tc<true, true, true>);
    set(k_stage_tc<false, true, true>);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  const bool full = c.pen != 0.0f || c.wallA;
  const CUtensorMap zero_map{};
  const CUtensorMap &mu0 = u0 ? *cp.map_u0 : zero_map;
  const dim3 grid((unsigned)nch, (unsigned)m);
  auto go = [&](auto kern) {
    kern<<<grid, kBlock, smem, s>>>(u, u0, out, geo.d_loc, geo.d_halo, geo.d_halo_cnt, geo.d_chunk,
                                    geo.d_grange, geo.d_gscale_f, stride, nrec, sel.list, sel.adv,
                                    tb, c, *cp.map_u, mu0, *cp.map_out, ca);
  };
  if (c.sround) {
    if (u0) full ? go(k_stage_tc<true, true, true>) : go(k_stage_tc<true, true, false>);
    else full ? go(k_stage_tc<false, true, true>) : go(k_stage_tc<false, true, false>);
  } else {
    if (u0) full ? go(k_stage_tc<true, false, true>) : go(k_stage_tc<true, false, false>);
    else full ? go(k_stage_tc<false, false, true>) : go(k_stage_tc<false, false, false>);
  }
  return cudaGetLastError();
}

// Blocks of the tensor-core kernel that fit on one SM with this geometry.
int stage_tc_max_blocks(const Geometry &geo) {
  const int smem = tc_smem_bytes(geo.halo_max);
  if (cudaFuncSetAttribute(k_stage_tc<true, true, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage_tc<true, true, false>, kBlock,
                                                    smem) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace dg
