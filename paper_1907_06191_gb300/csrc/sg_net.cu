// sg_net.cu -- learned surrogate of the covariance: a CNN that maps the
// occupancy raster of an axon substrate plus (D, Delta) to Sigma / (2 D Delta).
//
// Network (channels-last NHWC, batch B, raster 128 x 128):
//   x0 = occupancy (1 inside a disk, 0 outside), BF16
//   for l = 1..4: z_l = conv3x3(x_{l-1}; W_l) + b_l (zero padding),
//                 a_l = relu(z_l), x_l = avgpool2x2(a_l)      channels 48, 96, 192, 384
//   g = mean over pixels of x_4                                 [B][384]
//   h = relu(F1 [g, c] + b1), c = (log(D Delta / 1 um^2), D)    [B][256]
//   y = F2 h + b2                                               [B][3]
// Weights and activations are stored in BF16; every sum accumulates in FP32;
// gradients and the Adam state are FP32, with FP32 master weights.  The
// convolutions -- forward, and the input and weight gradients -- are
// implicit GEMMs on the fifth-generation tensor cores (tcgen05.mma kind::f16,
// BF16 operands gathered into shared memory, FP32 accumulators in tensor
// memory); the dense layers and the pooling glue run on the CUDA cores.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "../../include/dgsigma.h"
#include "../../include/dgsurrogate.h"

namespace dg {
cudaError_t dev_alloc(void **p, size_t bytes);  // the library's allocator (dg_api.cu)
}

namespace sg {

constexpr int kRes = 128;
constexpr int kLayers = 4;
constexpr int kCh[kLayers + 1] = {1, 48, 96, 192, 384};
constexpr int kCond = 2, kHidden = 256, kOut = 3;
constexpr int kFeat = 384 + kCond;

struct Param {
  size_t off, n;  // offset into the flat FP32 parameter vector
};

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// ---------------------------------------------------------------------------
// implicit-GEMM convolution on the tensor cores
// ---------------------------------------------------------------------------
//
// One CTA of 128 threads computes a 128 x 64 tile of D = A B^T over a range of
// K, in chunks of 32: every thread gathers one row of the A chunk (and two
// 16-byte pieces of the B chunk) into shared memory in the core-matrix layout
// of the MMA (K-major, no swizzle: 8 rows x 16 bytes per core matrix), one
// thread issues two tcgen05.mma (K = 16 each) per chunk, and two buffers let
// the next chunk's gather run while the tensor cores work on this one.  The
// accumulator tile lives in 64 tensor-memory columns; thread r reads row r
// (lane r) for the epilogue.
//   FWD  : D[pixel][co] = sum_(tap, ci) x[pixel + tap][ci] W[co][tap][ci]
//          (pixels in quad order, so that 4 consecutive rows are a 2x2 block:
//          the epilogue adds the bias, applies ReLU, keeps a = relu(z) in BF16
//          and writes the 2x2 average x = pool(a))
//   DGRAD: D[pixel][ci] = sum_(tap, co) dz[pixel - tap][co] W[co][tap][ci]
//   WGRAD: D[co][(tap, ci)] = sum_pixel dz[pixel][co] x[pixel + tap][ci],
//          and column 9 Cin the bias gradient sum_pixel dz[pixel][co]; split
//          over pixel ranges, partial tiles summed in a fixed order after.
constexpr int kMmaThreads = 128;
constexpr int kTileN = 64;
constexpr int kChunk = 32;                        // K per chunk
constexpr int kLBO = 128;                         // bytes between K-adjacent core matrices
constexpr int kSBO = (kChunk / 8) * kLBO;         // bytes between 8-row groups (512)
constexpr int kABytes = 16 * kSBO;                // 128 rows x 32 K of BF16 (8 KB)
constexpr int kBBytes = (kTileN / 8) * kSBO;      // 64 rows x 32 K (4 KB)
constexpr int kStageBytes = kABytes + kBBytes;
// 26 KB of dynamic shared memory caps a SM at 8 CTAs: 8 x 64 tensor-memory
// columns fit the 512 a SM has, so no CTA waits for tensor memory
constexpr int kMmaSmem = 26 * 1024;
constexpr int kPixSplit = 4096;                   // pixels per CTA of the weight gradient
enum ConvMode { kFwd = 0, kDgrad = 1, kWgrad = 2 };

__host__ __device__ constexpr int core_off(int r, int k) {  // bytes, k in [0, kChunk)
  return (r / 8) * kSBO + (k / 8) * kLBO + (r % 8) * 16 + (k % 8) * 2;
}

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t mma_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((kSBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// kind::f16, FP32 accumulator, BF16 A and B (both K-major), N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    __nanosleep(32);
  }
  return false;
}

struct ConvArgs {
  const __nv_bfloat16 *x;    // FWD / WGRAD: the layer input [B][H][W][Cin]
  const __nv_bfloat16 *dz;   // DGRAD / WGRAD: gradient of z [B][H][W][Cout]
  const __nv_bfloat16 *w;    // FWD: Wk [Cout][kpad]; DGRAD: Wt [Cin][kpad]
  const float *bias;         // FWD
  __nv_bfloat16 *a;          // FWD: relu(z) [B][H][W][Cout] (may be null)
  __nv_bfloat16 *xo;         // FWD: pooled [B][H/2][W/2][Cout]
  float *dx;                 // DGRAD: [B][H][W][Cin]
  float *part;               // WGRAD: partial tiles [splits][Cout rows][ncol]
  int B, H, W, Cin, Cout;
  int kpad;                  // row stride of the weight tables (K padded to kChunk)
  int ncol;                  // WGRAD: 9 Cin + 1 columns (the last: bias)
  int *err;                  // set to 1 when a bounded wait gives up
  int limit;
};

template <int MODE>
__global__ void __launch_bounds__(kMmaThreads)
    k_conv_mma(const ConvArgs p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int t = threadIdx.x, warp = t >> 5;
  unsigned char *stage[2] = {sm, sm + kStageBytes};
  const uint32_t bars = su32(sm + 2 * kStageBytes);  // two MMA barriers
  volatile uint32_t *tslot = reinterpret_cast<volatile uint32_t *>(sm + 2 * kStageBytes + 16);
  const int HW = p.H * p.W;
  const long long npix = (long long)p.B * HW;
  // tile origin: rows (pixels, or output channels for WGRAD), columns
  const long long row0 = (long long)blockIdx.x * 128;
  const int col0 = blockIdx.y * kTileN;
  // K range of this CTA
  long long k_begin = 0, k_end = 0;
  if (MODE == kFwd) k_end = 9 * p.Cin;
  else if (MODE == kDgrad) k_end = 9 * p.Cout;
  else {
    k_begin = (long long)blockIdx.z * kPixSplit;
    k_end = npix < k_begin + kPixSplit ? npix : k_begin + kPixSplit;
  }
  const int nchunks = (int)((k_end - k_begin + kChunk - 1) / kChunk);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bars) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bars + 8) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;\n" ::"r"(
                     su32((const void *)tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tslot;

  // this thread's A row: a pixel (FWD: quad order; DGRAD: plain order) or an
  // output channel (WGRAD)
  const long long arow = row0 + t;
  int pb = 0, py = 0, px = 0;
  bool row_ok = false;
  if (MODE == kWgrad) {
    row_ok = arow < p.Cout;
  } else if (arow < npix) {
    row_ok = true;
    if (MODE == kFwd) {  // quad order: 4 consecutive rows are one 2x2 block
      const long long q = arow >> 2;
      const int d = (int)(arow & 3), w2 = p.W / 2, hw4 = HW / 4;
      pb = (int)(q / hw4);
      const int r = (int)(q % hw4);
      py = 2 * (r / w2) + (d >> 1);
      px = 2 * (r % w2) + (d & 1);
    } else {
      pb = (int)(arow / HW);
      const int r = (int)(arow % HW);
      py = r / p.W;
      px = r % p.W;
    }
  }
  // Gather state, computed once per thread.  FWD / DGRAD with C >= 8
  // channels (a multiple of 8) in the gathered tensor: the pixel index of
  // each of the 9 tap pixels (-1 outside the map), and per 8-wide K group its
  // (tap, channel), advanced by 32 channels per chunk.  WGRAD: this
  // thread's B column (tap, channel) and its 16 pixels per chunk, decoded
  // once per chunk and stepped.
  constexpr int kGroups = kChunk / 8;
  const int C = MODE == kFwd ? p.Cin : p.Cout;  // channels of the gathered tensor (FWD / DGRAD)
  int toff[9];
  int gtap[kGroups], gch[kGroups];
  if (MODE != kWgrad) {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3 - 1, dx = tap % 3 - 1;
      const int yy = MODE == kFwd ? py + dy : py - dy, xx = MODE == kFwd ? px + dx : px - dx;
      toff[tap] = (row_ok && yy >= 0 && yy < p.H && xx >= 0 && xx < p.W)
                      ? (pb * p.H + yy) * p.W + xx  // pixel index (< 2^31 for B <= 65535)
                      : -1;
    }
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
      gtap[g] = C >= 8 ? (8 * g) / C : 0;
      gch[g] = C >= 8 ? (8 * g) % C : 0;
    }
  }
  const int wn = col0 + (t >> 1);            // WGRAD: this thread's B column
  const int wtap = MODE == kWgrad ? wn / p.Cin : 0, wci = MODE == kWgrad ? wn % p.Cin : 0;
  const int wdy = wtap / 3 - 1, wdx = wtap % 3 - 1;
  const __nv_bfloat16 *src = MODE == kFwd ? p.x : p.dz;
  bool ok = true;
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    unsigned char *sa = stage[buf], *sbm = stage[buf] + kABytes;
    if (c >= 2) {  // the MMAs of chunk c - 2 have read this buffer
      if (!wait_bar(bars + 8 * buf, (uint32_t)(((c - 2) >> 1) & 1), p.limit)) ok = false;
    }
    const long long kc = k_begin + (long long)c * kChunk;
    // ---- A chunk: row t, 32 K values as 4 pieces of 8 ----
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
      alignas(16) __nv_bfloat16 v[8];
      if (MODE != kWgrad && C >= 8) {  // 8 channels of one tap: one 16-byte load
        uint4 q = make_uint4(0, 0, 0, 0);
        const int off = gtap[g] < 9 ? toff[gtap[g]] : -1;
        if (off >= 0) q = *reinterpret_cast<const uint4 *>(src + (size_t)off * C + gch[g]);
        *reinterpret_cast<uint4 *>(v) = q;
        gch[g] += kChunk;  // the same group of the next chunk
        while (gch[g] >= C) {
          gch[g] -= C;
          ++gtap[g];
        }
      } else if (MODE == kFwd) {  // Cin = 1: K = the 9 taps
        const int k0 = (int)kc + g * 8;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int tap = k0 + e;
          const int off = tap < 9 ? toff[tap] : -1;
          v[e] = off >= 0 ? p.x[off] : __float2bfloat16(0.0f);
        }
      } else {  // WGRAD: dz[pixel][co] for 8 consecutive pixels
        const long long k0 = kc + g * 8;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const long long m = k0 + e;
          v[e] = (row_ok && m < k_end) ? p.dz[(size_t)m * p.Cout + arow] : __float2bfloat16(0.0f);
        }
      }
      *reinterpret_cast<uint4 *>(sa + core_off(t, g * 8)) = *reinterpret_cast<const uint4 *>(v);
    }
    // ---- B chunk: 64 rows x 32 K, two pieces of 8 per thread ----
    if (MODE == kFwd || MODE == kDgrad) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int piece = t * 2 + h;  // 0..255
        const int r = piece >> 2, g = piece & 3;
        const int n = col0 + r;
        const int nrows = MODE == kFwd ? p.Cout : p.Cin;
        uint4 q = make_uint4(0, 0, 0, 0);
        if (n < nrows) q = *reinterpret_cast<const uint4 *>(p.w + (size_t)n * p.kpad + kc + g * 8);
        *reinterpret_cast<uint4 *>(sbm + core_off(r, g * 8)) = q;
      }
    } else {  // WGRAD: column wn of im2col(x) (or ones for the bias), 16 pixels
      const long long m0 = kc + 16 * (t & 1);
      int b = (int)(m0 / HW);
      int rr = (int)(m0 % HW);
      int yy = rr / p.W, xx = rr % p.W;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        alignas(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const long long m = m0 + 8 * h + e;
          float val = 0.0f;
          if (m < k_end && wn < p.ncol) {
            if (wn == p.ncol - 1) {
              val = 1.0f;
            } else {
              const int y2 = yy + wdy, x2 = xx + wdx;
              if (y2 >= 0 && y2 < p.H && x2 >= 0 && x2 < p.W)
                val = bf(p.x[(((size_t)b * p.H + y2) * p.W + x2) * p.Cin + wci]);
            }
          }
          v[e] = __float2bfloat16(val);
          if (++xx == p.W) {  // the next pixel
            xx = 0;
            if (++yy == p.H) {
              yy = 0;
              ++b;
            }
          }
        }
        *reinterpret_cast<uint4 *>(sbm + core_off(t >> 1, (2 * (t & 1) + h) * 8)) =
            *reinterpret_cast<const uint4 *>(v);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < kChunk / 16; ++ks) {
        const uint64_t ad = mma_desc(su32(sa) + ks * 2 * kLBO);
        const uint64_t bd = mma_desc(su32(sbm) + ks * 2 * kLBO);
        const int acc = (c > 0 || ks > 0) ? 1 : 0;
        asm volatile(
            "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              bars + 8 * buf)
          : "memory");
    }
  }
  // the last commit arrives when every MMA of the CTA has completed
  if (nchunks > 0 &&
      !wait_bar(bars + 8 * ((nchunks - 1) & 1), (uint32_t)(((nchunks - 1) >> 1) & 1), p.limit))
    ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  // ---- epilogue: row t of the tile, 64 columns ----
  float acc[kTileN];
  {
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
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
          : "r"(taddr + (uint32_t)(half * 32))
          : "memory");
#pragma unroll
      for (int k = 0; k < 32; ++k) acc[half * 32 + k] = __uint_as_float(r[k]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;\n" ::"r"(tmem) : "memory");
  if (!ok) {
    if (t == 0) atomicExch(p.err, 1);
    return;
  }
  if (MODE == kFwd) {
    // bias, ReLU (kept in BF16), then the 2x2 average over the quad of rows
    // 4q..4q+3 (consecutive lanes of this warp)
    const int h2 = p.H / 2, w2 = p.W / 2;
    const size_t prow = (((size_t)pb * p.H + py) * p.W + px) * p.Cout;
    const size_t qrow = (((size_t)pb * h2 + (py >> 1)) * w2 + (px >> 1)) * p.Cout;
#pragma unroll
    for (int c8 = 0; c8 < kTileN; c8 += 8) {
      alignas(16) __nv_bfloat16 av[8], pv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int n = col0 + c8 + e;
        const float z = n < p.Cout ? acc[c8 + e] + p.bias[n] : 0.0f;
        av[e] = __float2bfloat16(fmaxf(z, 0.0f));
        float s = bf(av[e]);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        pv[e] = __float2bfloat16(0.25f * s);
      }
      if (row_ok && col0 + c8 < p.Cout) {
        if (p.a) *reinterpret_cast<uint4 *>(p.a + prow + col0 + c8) = *reinterpret_cast<const uint4 *>(av);
        if ((t & 3) == 0)
          *reinterpret_cast<uint4 *>(p.xo + qrow + col0 + c8) = *reinterpret_cast<const uint4 *>(pv);
      }
    }
  } else if (MODE == kDgrad) {
    if (row_ok) {
      float *o = p.dx + (size_t)arow * p.Cin;
#pragma unroll
      for (int c = 0; c < kTileN; ++c)
        if (col0 + c < p.Cin) o[col0 + c] = acc[c];
    }
  } else {
    if (row_ok) {
      float *o = p.part + ((size_t)blockIdx.z * p.Cout + arow) * p.ncol;
#pragma unroll
      for (int c = 0; c < kTileN; ++c)
        if (col0 + c < p.ncol) o[col0 + c] = acc[c];
    }
  }
}

// Sum of the weight-gradient partial tiles over the pixel splits (fixed
// order), scattered into the gradient vector: weights [Cout][Cin][3][3] and
// the bias [Cout].
__global__ void k_wgrad_reduce(const float *__restrict__ part, int splits, int Cout, int Cin,
                               float *__restrict__ gw, float *__restrict__ gb) {
  const int ncol = 9 * Cin + 1;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)Cout * ncol) return;
  const int co = (int)(i / ncol), j = (int)(i % ncol);
  float s = 0.0f;
  for (int k = 0; k < splits; ++k) s += part[((size_t)k * Cout + co) * ncol + j];
  if (j == ncol - 1) gb[co] = s;
  else gw[((size_t)co * Cin + j % Cin) * 9 + j / Cin] = s;
}

// BF16 weight tables of a convolution from the FP32 master weights [Cout][Cin][3][3]:
// Wk[co][tap Cin + ci] (forward) and Wt[ci][tap Cout + co] (input gradient),
// rows padded with zeros to kpad.
__global__ void k_conv_tables(const float *__restrict__ w, int Cout, int Cin, int kpad_k,
                              int kpad_t, __nv_bfloat16 *__restrict__ wk,
                              __nv_bfloat16 *__restrict__ wt) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nk = (long long)Cout * kpad_k, nt = (long long)Cin * kpad_t;
  if (i < nk) {
    const int co = (int)(i / kpad_k), k = (int)(i % kpad_k);
    const int tap = k / Cin, ci = k % Cin;
    wk[i] = __float2bfloat16(tap < 9 ? w[((size_t)co * Cin + ci) * 9 + tap] : 0.0f);
  } else if (wt != nullptr && i < nk + nt) {
    const long long j = i - nk;
    const int ci = (int)(j / kpad_t), k = (int)(j % kpad_t);
    const int tap = k / Cout, co = k % Cout;
    wt[j] = __float2bfloat16(tap < 9 ? w[((size_t)co * Cin + ci) * 9 + tap] : 0.0f);
  }
}

// occupancy bytes -> BF16 input (one channel: NCHW and NHWC coincide)
__global__ void k_occ_to_bf16(const uint8_t *__restrict__ occ, long long n,
                              __nv_bfloat16 *__restrict__ x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = __float2bfloat16(occ[i] ? 1.0f : 0.0f);
}

// feature vector [B][kFeat]: channel means of x4 (NHWC), then the
// conditioning; one block per sample, one thread per channel
__global__ void k_gap_fwd(const __nv_bfloat16 *__restrict__ x, int C, int HW,
                          const float *__restrict__ cond, float *__restrict__ f) {
  const int b = blockIdx.x;
  for (int c = threadIdx.x; c < C + kCond; c += blockDim.x) {
    if (c < C) {
      const __nv_bfloat16 *s = x + (size_t)b * HW * C + c;
      float t = 0.0f;
      for (int k = 0; k < HW; ++k) t += bf(s[(size_t)k * C]);
      f[(size_t)b * kFeat + c] = t / (float)HW;
    } else {
      f[(size_t)b * kFeat + c] = cond[(size_t)b * kCond + (c - C)];
    }
  }
}

// out[b][n] = act(sum_k in[b][k] W[n][k] + bias[n]), W in BF16; in rounded to
// BF16 before the product (BF16 activations).  grid (B), block >= N.
__global__ void k_dense_fwd(const float *__restrict__ in, int K, const __nv_bfloat16 *__restrict__ w,
                            const float *__restrict__ bias, int N, int relu,
                            float *__restrict__ out) {
  const int b = blockIdx.x, nn = threadIdx.x;
  if (nn >= N) return;
  float s = bias[nn];
  for (int k = 0; k < K; ++k)
    s += bf(w[(size_t)nn * K + k]) * __bfloat162float(__float2bfloat16(in[(size_t)b * K + k]));
  out[(size_t)b * N + nn] = relu ? fmaxf(s, 0.0f) : s;
}

// loss = mean_b sum_o (y - t)^2 / kOut; dy = 2 (y - t) / (B kOut)
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, int B,
                      float *__restrict__ dy, float *__restrict__ loss) {
  __shared__ float sh[256];
  float acc = 0.0f;
  for (int i = threadIdx.x; i < B * kOut; i += 256) {
    const float d = y[i] - t[i];
    dy[i] = 2.0f * d / (float)(B * kOut);
    acc += d * d;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / (float)(B * kOut);
}

// dense backward: din[b][k] = sum_n dout'[b][n] W[n][k] with dout' = dout *
// [out > 0] for a ReLU layer; grid (B), block K
__global__ void k_dense_bwd_in(const float *__restrict__ dout, const float *__restrict__ out,
                               int N, int relu, const __nv_bfloat16 *__restrict__ w, int K,
                               float *__restrict__ din) {
  const int b = blockIdx.x, k = threadIdx.x;
  if (k >= K) return;
  float s = 0.0f;
  for (int nn = 0; nn < N; ++nn) {
    float g = dout[(size_t)b * N + nn];
    if (relu && out[(size_t)b * N + nn] <= 0.0f) g = 0.0f;
    s += g * bf(w[(size_t)nn * K + k]);
  }
  din[(size_t)b * K + k] = s;
}

// dW[n][k] = sum_b dout'[b][n] bf16(in[b][k]), db[n] = sum_b dout'[b][n];
// grid (N), block 256 over k (k = K is the bias)
__global__ void k_dense_bwd_w(const float *__restrict__ dout, const float *__restrict__ out,
                              int N, int relu, const float *__restrict__ in, int K, int B,
                              float *__restrict__ dw, float *__restrict__ db) {
  const int nn = blockIdx.x;
  for (int k = threadIdx.x; k <= K; k += blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < B; ++b) {
      float g = dout[(size_t)b * N + nn];
      if (relu && out[(size_t)b * N + nn] <= 0.0f) g = 0.0f;
      s += g * (k < K ? __bfloat162float(__float2bfloat16(in[(size_t)b * K + k])) : 1.0f);
    }
    if (k < K) dw[(size_t)nn * K + k] = s;
    else db[nn] = s;
  }
}

// global-average-pool backward into the pooled map of layer 4 (NHWC, FP32)
__global__ void k_gap_bwd(const float *__restrict__ df, int C, int HW, long long total,
                          float *__restrict__ dx) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int c = (int)(i % C);
  const long long b = i / ((long long)HW * C);
  dx[i] = df[(size_t)b * kFeat + c] / (float)HW;
}

// pool backward and ReLU mask (NHWC): dz[b][y][x][c] =
// bf16(dx[b][y/2][x/2][c] / 4 * [a > 0]); dz feeds the tensor-core gradients
__global__ void k_pool_relu_bwd(const float *__restrict__ dx, const __nv_bfloat16 *__restrict__ a,
                                int B, int H, int W, int C, __nv_bfloat16 *__restrict__ dz) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)B * H * W * C;
  if (i >= tot) return;
  const int c = (int)(i % C);
  const long long pix = i / C;
  const int xx = (int)(pix % W), yy = (int)((pix / W) % H);
  const long long b = pix / ((long long)H * W);
  const float g = 0.25f * dx[((b * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C + c];
  dz[i] = __float2bfloat16(bf(a[i]) > 0.0f ? g : 0.0f);
}

// Adam on the FP32 master weights; refresh the BF16 copies of the weights
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2, const int *__restrict__ is_w,
                       __nv_bfloat16 *__restrict__ pbf) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  pbf[i] = __float2bfloat16(pi);
  (void)is_w;
}

__global__ void k_to_bf16(const float *__restrict__ p, long long n, __nv_bfloat16 *__restrict__ o) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = __float2bfloat16(p[i]);
}

// ---------------------------------------------------------------------------
// network object
// ---------------------------------------------------------------------------

struct Net {
  int device = 0, max_batch = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  Param conv_w[kLayers], conv_b[kLayers], f1_w, f1_b, f2_w, f2_b;
  size_t n_params = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master, grad, Adam
  __nv_bfloat16 *pbf = nullptr;                                  // BF16 copies (dense layers)
  __nv_bfloat16 *wk[kLayers] = {}, *wt[kLayers] = {};           // conv tables for the MMA
  int kpad_k[kLayers] = {}, kpad_t[kLayers] = {};
  long long step = 0;
  // activations (NHWC)
  __nv_bfloat16 *x[kLayers + 1] = {};  // pooled maps (x0 = input)
  __nv_bfloat16 *a[kLayers] = {};      // post-ReLU conv outputs (pre-pool)
  float *feat = nullptr, *hid = nullptr, *y = nullptr, *loss = nullptr;
  float *dy = nullptr, *dhid = nullptr, *dfeat = nullptr;
  float *dx = nullptr;                 // FP32 gradient of a pooled map
  __nv_bfloat16 *dz = nullptr;         // BF16 gradient of a conv output
  float *part = nullptr;               // weight-gradient partial tiles
  int *d_err = nullptr;                // a bounded wait of a tensor-core kernel gave up
};

int res_of(int l) { return kRes >> l; }  // spatial size of x_l
int round_up(int v, int q) { return (v + q - 1) / q * q; }

void free_net(Net &n) {
  void *ptrs[] = {n.p, n.g, n.m, n.v, n.pbf, n.feat, n.hid, n.y, n.loss, n.dy, n.dhid, n.dfeat,
                  n.dx, n.dz, n.part, n.d_err};
  for (void *q : ptrs) cudaFree(q);
  for (int l = 0; l <= kLayers; ++l) cudaFree(n.x[l]);
  for (int l = 0; l < kLayers; ++l) {
    cudaFree(n.a[l]);
    cudaFree(n.wk[l]);
    cudaFree(n.wt[l]);
  }
}

// splitmix64 -> uniform in [-1, 1)
uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// pixel splits of the weight gradient of layer l at batch B
long long wgrad_splits(int l, int B) {
  const long long npix = (long long)B * res_of(l) * res_of(l);
  return (npix + kPixSplit - 1) / kPixSplit;
}

}  // namespace sg

using namespace sg;

struct sg_net {
  Net n;
};

namespace {

#define SGK(expr)                                                   \
  do {                                                              \
    cudaError_t _e = (expr);                                        \
    if (_e != cudaSuccess) {                                        \
      net->n.err = cudaGetErrorString(_e);                          \
      return DG_ECUDA;                                              \
    }                                                               \
  } while (0)

unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

const __nv_bfloat16 *wbf(const Net &n, const Param &q) { return n.pbf + q.off; }
const float *pf(const Net &n, const Param &q) { return n.p + q.off; }
float *gf(const Net &n, const Param &q) { return n.g + q.off; }

// BF16 copies of the dense weights and the MMA tables of the convolutions,
// after every change of the master weights
cudaError_t refresh_weights(Net &n) {
  k_to_bf16<<<blocks((long long)n.n_params), 256, 0, n.stream>>>(n.p, (long long)n.n_params, n.pbf);
  for (int l = 0; l < kLayers; ++l) {
    const long long tot = (long long)kCh[l + 1] * n.kpad_k[l] + (n.wt[l] ? (long long)kCh[l] * n.kpad_t[l] : 0);
    k_conv_tables<<<blocks(tot), 256, 0, n.stream>>>(pf(n, n.conv_w[l]), kCh[l + 1], kCh[l], n.kpad_k[l],
                                                     n.kpad_t[l], n.wk[l], n.wt[l]);
  }
  return cudaGetLastError();
}

bool set_mma_smem() {
  static bool done = false;
  if (done) return true;
  if (cudaFuncSetAttribute(k_conv_mma<kFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_conv_mma<kDgrad>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_conv_mma<kWgrad>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem) !=
          cudaSuccess)
    return false;
  done = true;
  return true;
}

ConvArgs conv_args(const Net &n, int l, int B) {
  ConvArgs a{};
  a.B = B;
  a.H = a.W = res_of(l);
  a.Cin = kCh[l];
  a.Cout = kCh[l + 1];
  a.err = n.d_err;
  a.limit = 1 << 22;
  return a;
}

int forward(sg_net *net, const uint8_t *occ, const float *cond, int B, bool keep) {
  Net &n = net->n;
  cudaStream_t s = n.stream;
  k_occ_to_bf16<<<blocks((long long)B * kRes * kRes), 256, 0, s>>>(occ, (long long)B * kRes * kRes, n.x[0]);
  for (int l = 0; l < kLayers; ++l) {
    ConvArgs a = conv_args(n, l, B);
    a.x = n.x[l];
    a.w = n.wk[l];
    a.kpad = n.kpad_k[l];
    a.bias = pf(n, n.conv_b[l]);
    a.a = keep ? n.a[l] : nullptr;
    a.xo = n.x[l + 1];
    const long long npix = (long long)B * a.H * a.W;
    const dim3 grid((unsigned)((npix + 127) / 128), (unsigned)((a.Cout + kTileN - 1) / kTileN));
    k_conv_mma<kFwd><<<grid, kMmaThreads, kMmaSmem, s>>>(a);
  }
  const int H4 = res_of(kLayers);
  k_gap_fwd<<<B, 128, 0, s>>>(n.x[kLayers], kCh[kLayers], H4 * H4, cond, n.feat);
  k_dense_fwd<<<B, kHidden, 0, s>>>(n.feat, kFeat, wbf(n, n.f1_w), pf(n, n.f1_b), kHidden, 1, n.hid);
  k_dense_fwd<<<B, 32, 0, s>>>(n.hid, kHidden, wbf(n, n.f2_w), pf(n, n.f2_b), kOut, 0, n.y);
  SGK(cudaGetLastError());
  return DG_OK;
}

int backward(sg_net *net, const float *target, int B) {
  Net &n = net->n;
  cudaStream_t s = n.stream;
  k_mse<<<1, 256, 0, s>>>(n.y, target, B, n.dy, n.loss);
  k_dense_bwd_w<<<kOut, 256, 0, s>>>(n.dy, n.y, kOut, 0, n.hid, kHidden, B, gf(n, n.f2_w), gf(n, n.f2_b));
  k_dense_bwd_in<<<B, kHidden, 0, s>>>(n.dy, n.y, kOut, 0, wbf(n, n.f2_w), kHidden, n.dhid);
  k_dense_bwd_w<<<kHidden, 256, 0, s>>>(n.dhid, n.hid, kHidden, 1, n.feat, kFeat, B, gf(n, n.f1_w),
                                        gf(n, n.f1_b));
  k_dense_bwd_in<<<B, kFeat, 0, s>>>(n.dhid, n.hid, kHidden, 1, wbf(n, n.f1_w), kFeat, n.dfeat);
  const int H4 = res_of(kLayers);
  const long long tot4 = (long long)B * kCh[kLayers] * H4 * H4;
  k_gap_bwd<<<blocks(tot4), 256, 0, s>>>(n.dfeat, kCh[kLayers], H4 * H4, tot4, n.dx);
  for (int l = kLayers - 1; l >= 0; --l) {
    ConvArgs a = conv_args(n, l, B);
    const long long npix = (long long)B * a.H * a.W;
    k_pool_relu_bwd<<<blocks(npix * a.Cout), 256, 0, s>>>(n.dx, n.a[l], B, a.H, a.W, a.Cout, n.dz);
    // weight and bias gradients: tiles over (output channel, weight column), split over pixels
    a.x = n.x[l];
    a.dz = n.dz;
    a.part = n.part;
    a.ncol = 9 * a.Cin + 1;
    const long long splits = wgrad_splits(l, B);
    const dim3 gw((unsigned)((a.Cout + 127) / 128), (unsigned)((a.ncol + kTileN - 1) / kTileN),
                  (unsigned)splits);
    k_conv_mma<kWgrad><<<gw, kMmaThreads, kMmaSmem, s>>>(a);
    k_wgrad_reduce<<<blocks((long long)a.Cout * a.ncol), 256, 0, s>>>(n.part, (int)splits, a.Cout, a.Cin,
                                                                      gf(n, n.conv_w[l]), gf(n, n.conv_b[l]));
    if (l > 0) {  // gradient of the pooled map x_l: the next (lower) layer's input
      ConvArgs d = conv_args(n, l, B);
      d.dz = n.dz;
      d.w = n.wt[l];
      d.kpad = n.kpad_t[l];
      d.dx = n.dx;
      const dim3 gd((unsigned)((npix + 127) / 128), (unsigned)((d.Cin + kTileN - 1) / kTileN));
      k_conv_mma<kDgrad><<<gd, kMmaThreads, kMmaSmem, s>>>(d);
    }
  }
  SGK(cudaGetLastError());
  return DG_OK;
}

// DG_ETIMEOUT if a tensor-core kernel gave up waiting (the flag is cleared)
int take_error(sg_net *net) {
  Net &n = net->n;
  int flag = 0;
  SGK(cudaMemcpyAsync(&flag, n.d_err, sizeof(int), cudaMemcpyDeviceToHost, n.stream));
  SGK(cudaStreamSynchronize(n.stream));
  if (flag) {
    SGK(cudaMemsetAsync(n.d_err, 0, sizeof(int), n.stream));
    n.err = "a tensor-core kernel gave up waiting for its MMAs";
    return DG_ETIMEOUT;
  }
  return DG_OK;
}

int check_io(sg_net *net, const void *occ, const float *cond, int B) {
  if (!net) return DG_EINVAL;
  if (!occ || !cond || B < 1 || B > net->n.max_batch) {
    net->n.err = "bad batch arguments (1 <= B <= max_batch, device pointers)";
    return DG_EINVAL;
  }
  return DG_OK;
}

}  // namespace

extern "C" {

int sg_create(int max_batch, unsigned long long seed, int device, sg_net **out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  if (max_batch < 1 || max_batch > 65535) return DG_EINVAL;
  sg_net *net = new (std::nothrow) sg_net();
  if (!net) return DG_ENOMEM;
  Net &n = net->n;
  int dev = device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) { delete net; return DG_ECUDA; }
  if (cudaSetDevice(dev) != cudaSuccess) { delete net; return DG_ECUDA; }
  if (!set_mma_smem()) { delete net; return DG_ECUDA; }
  n.device = dev;
  n.max_batch = max_batch;
  if (cudaStreamCreateWithFlags(&n.stream, cudaStreamNonBlocking) != cudaSuccess) { delete net; return DG_ECUDA; }
  size_t off = 0;
  auto add = [&](size_t cnt) { Param q{off, cnt}; off += cnt; return q; };
  for (int l = 0; l < kLayers; ++l) {
    n.conv_w[l] = add((size_t)kCh[l + 1] * kCh[l] * 9);
    n.conv_b[l] = add((size_t)kCh[l + 1]);
  }
  n.f1_w = add((size_t)kHidden * kFeat);
  n.f1_b = add(kHidden);
  n.f2_w = add((size_t)kOut * kHidden);
  n.f2_b = add(kOut);
  n.n_params = off;
  // He-uniform initial weights from a counter-based generator, zero biases
  std::vector<float> h(off, 0.0f);
  auto fill = [&](const Param &q, int fan_in) {
    const double a = std::sqrt(6.0 / fan_in);
    for (size_t k = 0; k < q.n; ++k) {
      const double uni = (double)(mix64(seed * 0x100000001B3ull + q.off + k) >> 11) * 0x1.0p-53;
      h[q.off + k] = (float)(a * (2.0 * uni - 1.0));
    }
  };
  for (int l = 0; l < kLayers; ++l) fill(n.conv_w[l], kCh[l] * 9);
  fill(n.f1_w, kFeat);
  fill(n.f2_w, kHidden);
  bool ok = true;
  auto al = [&](auto **ptr, size_t bytes) {
    if (ok && dg::dev_alloc(reinterpret_cast<void **>(ptr), bytes) != cudaSuccess) ok = false;
  };
  al(&n.p, off * 4); al(&n.g, off * 4); al(&n.m, off * 4); al(&n.v, off * 4); al(&n.pbf, off * 2);
  size_t big_dx = 0, big_dz = 0, big_part = 0;
  for (int l = 0; l < kLayers; ++l) {
    n.kpad_k[l] = round_up(9 * kCh[l], kChunk);
    n.kpad_t[l] = round_up(9 * kCh[l + 1], kChunk);
    al(&n.wk[l], (size_t)kCh[l + 1] * n.kpad_k[l] * 2);
    if (l > 0) al(&n.wt[l], (size_t)kCh[l] * n.kpad_t[l] * 2);  // no input gradient of layer 1
    const size_t pix = (size_t)max_batch * res_of(l) * res_of(l);
    big_dz = std::max(big_dz, pix * kCh[l + 1]);
    big_dx = std::max(big_dx, pix / 4 * kCh[l + 1]);  // gradient of the pooled output
    if (l > 0) big_dx = std::max(big_dx, pix * kCh[l]);  // gradient of the layer input
    big_part = std::max(big_part, (size_t)wgrad_splits(l, max_batch) * kCh[l + 1] * (9 * kCh[l] + 1));
  }
  for (int l = 0; l <= kLayers; ++l) al(&n.x[l], (size_t)max_batch * kCh[l] * res_of(l) * res_of(l) * 2);
  for (int l = 0; l < kLayers; ++l) al(&n.a[l], (size_t)max_batch * kCh[l + 1] * res_of(l) * res_of(l) * 2);
  al(&n.dx, big_dx * 4); al(&n.dz, big_dz * 2); al(&n.part, big_part * 4);
  al(&n.feat, (size_t)max_batch * kFeat * 4); al(&n.dfeat, (size_t)max_batch * kFeat * 4);
  al(&n.hid, (size_t)max_batch * kHidden * 4); al(&n.dhid, (size_t)max_batch * kHidden * 4);
  al(&n.y, (size_t)max_batch * kOut * 4); al(&n.dy, (size_t)max_batch * kOut * 4);
  al(&n.loss, 4);
  al(&n.d_err, 16);
  if (!ok) { free_net(n); cudaStreamDestroy(n.stream); delete net; return DG_ENOMEM; }
  cudaError_t e = cudaMemcpyAsync(n.p, h.data(), off * 4, cudaMemcpyHostToDevice, n.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n.m, 0, off * 4, n.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n.v, 0, off * 4, n.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n.g, 0, off * 4, n.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n.d_err, 0, 16, n.stream);
  if (e == cudaSuccess) e = refresh_weights(n);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n.stream);
  if (e != cudaSuccess) {
    free_net(n);
    cudaStreamDestroy(n.stream);
    delete net;
    return DG_ECUDA;
  }
  *out = net;
  return DG_OK;
}

void sg_destroy(sg_net *net) {
  if (!net) return;
  cudaSetDevice(net->n.device);
  cudaStreamSynchronize(net->n.stream);
  free_net(net->n);
  cudaStreamDestroy(net->n.stream);
  delete net;
}

const char *sg_last_error(const sg_net *net) { return net ? net->n.err.c_str() : ""; }

int sg_param_count(sg_net *net, size_t *count) {
  if (!net || !count) return DG_EINVAL;
  *count = net->n.n_params;
  return DG_OK;
}

int sg_get_params(sg_net *net, float *host) {
  if (!net || !host) return DG_EINVAL;
  SGK(cudaSetDevice(net->n.device));
  SGK(cudaMemcpyAsync(host, net->n.p, net->n.n_params * 4, cudaMemcpyDeviceToHost, net->n.stream));
  SGK(cudaStreamSynchronize(net->n.stream));
  return DG_OK;
}

int sg_set_params(sg_net *net, const float *host) {
  if (!net || !host) return DG_EINVAL;
  Net &n = net->n;
  SGK(cudaSetDevice(n.device));
  SGK(cudaMemcpyAsync(n.p, host, n.n_params * 4, cudaMemcpyHostToDevice, n.stream));
  SGK(refresh_weights(n));
  SGK(cudaStreamSynchronize(n.stream));
  return DG_OK;
}

int sg_predict(sg_net *net, const uint8_t *occ, const float *cond, int B, float *out) {
  int r = check_io(net, occ, cond, B);
  if (r != DG_OK) return r;
  if (!out) return DG_EINVAL;
  Net &n = net->n;
  SGK(cudaSetDevice(n.device));
  r = forward(net, occ, cond, B, false);
  if (r != DG_OK) return r;
  SGK(cudaMemcpyAsync(out, n.y, (size_t)B * kOut * 4, cudaMemcpyDeviceToDevice, n.stream));
  return take_error(net);
}

int sg_gradients(sg_net *net, const uint8_t *occ, const float *cond, const float *target, int B,
                 float *loss_host, float *grad_host) {
  int r = check_io(net, occ, cond, B);
  if (r != DG_OK) return r;
  if (!target) return DG_EINVAL;
  Net &n = net->n;
  SGK(cudaSetDevice(n.device));
  if ((r = forward(net, occ, cond, B, true)) != DG_OK) return r;
  if ((r = backward(net, target, B)) != DG_OK) return r;
  if (loss_host) SGK(cudaMemcpyAsync(loss_host, n.loss, 4, cudaMemcpyDeviceToHost, n.stream));
  if (grad_host) SGK(cudaMemcpyAsync(grad_host, n.g, n.n_params * 4, cudaMemcpyDeviceToHost, n.stream));
  return take_error(net);
}

int sg_train_step(sg_net *net, const uint8_t *occ, const float *cond, const float *target, int B,
                  float lr, float *loss_host) {
  int r = check_io(net, occ, cond, B);
  if (r != DG_OK) return r;
  if (!target || !(lr > 0.0f) || !std::isfinite(lr)) return DG_EINVAL;
  Net &n = net->n;
  SGK(cudaSetDevice(n.device));
  if ((r = forward(net, occ, cond, B, true)) != DG_OK) return r;
  if ((r = backward(net, target, B)) != DG_OK) return r;
  n.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)n.step), c2 = 1.0f - std::pow(b2, (float)n.step);
  k_adam<<<blocks((long long)n.n_params), 256, 0, n.stream>>>(n.p, n.g, n.m, n.v, (long long)n.n_params, lr,
                                                              b1, b2, 1e-8f, c1, c2, nullptr, n.pbf);
  SGK(cudaGetLastError());
  SGK(refresh_weights(n));
  if (loss_host) SGK(cudaMemcpyAsync(loss_host, n.loss, 4, cudaMemcpyDeviceToHost, n.stream));
  return take_error(net);
}

}  // extern "C"
