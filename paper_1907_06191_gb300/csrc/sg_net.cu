// sg_net.cu -- learned surrogate of the covariance: a small CNN that maps the
// occupancy raster of an axon substrate plus (D, Delta) to Sigma / (2 D Delta).
//
// Network (NCHW, batch B, raster 128 x 128):
//   x0 = occupancy (1 inside a disk, 0 outside), BF16
//   for l = 1..4: z_l = conv3x3(x_{l-1}; W_l) + b_l (zero padding),
//                 a_l = relu(z_l), x_l = avgpool2x2(a_l)      channels 16, 32, 64, 64
//   g = mean over pixels of x_4                                 [B][64]
//   h = relu(F1 [g, c] + b1), c = (log(D Delta / 1 um^2), D)    [B][128]
//   y = F2 h + b2                                               [B][3]
// Weights and activations are stored in BF16; every sum accumulates in FP32;
// gradients and the Adam state are FP32, with FP32 master weights.
#include <cuda_bf16.h>

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
constexpr int kCh[kLayers + 1] = {1, 16, 32, 64, 64};
constexpr int kCond = 2, kHidden = 128, kOut = 3;
constexpr int kFeat = 64 + kCond;

struct Param {
  size_t off, n;  // offset into the flat FP32 parameter vector
};

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// occupancy bytes -> BF16 input
__global__ void k_occ_to_bf16(const uint8_t *__restrict__ occ, long long n,
                              __nv_bfloat16 *__restrict__ x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = __float2bfloat16(occ[i] ? 1.0f : 0.0f);
}

// z = conv3x3(x) + b, a = relu(z) stored in BF16.  One thread per output
// (b, co, y, x); grid (ceil(H W / 256), Cout, B).
__global__ void k_conv_fwd(const __nv_bfloat16 *__restrict__ x, int Cin, int H, int W,
                           const __nv_bfloat16 *__restrict__ w, const float *__restrict__ bias,
                           int Cout, __nv_bfloat16 *__restrict__ a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= H * W) return;
  const int co = blockIdx.y, b = blockIdx.z;
  const int yy = p / W, xx = p % W;
  float s = bias[co];
  const __nv_bfloat16 *xb = x + (size_t)b * Cin * H * W;
  const __nv_bfloat16 *wc = w + (size_t)co * Cin * 9;
  for (int ci = 0; ci < Cin; ++ci) {
    const __nv_bfloat16 *xc = xb + (size_t)ci * H * W;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int y2 = yy + ky - 1;
      if (y2 < 0 || y2 >= H) continue;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int x2 = xx + kx - 1;
        if (x2 < 0 || x2 >= W) continue;
        s += bf(wc[ci * 9 + ky * 3 + kx]) * bf(xc[y2 * W + x2]);
      }
    }
  }
  a[((size_t)b * Cout + co) * H * W + p] = __float2bfloat16(fmaxf(s, 0.0f));
}

// 2x2 average pool, BF16 in and out; grid over B*C*(H/2)*(W/2)
__global__ void k_pool_fwd(const __nv_bfloat16 *__restrict__ a, long long BC, int H, int W,
                           __nv_bfloat16 *__restrict__ x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int h2 = H / 2, w2 = W / 2;
  if (i >= BC * h2 * w2) return;
  const long long bc = i / (h2 * w2);
  const int q = (int)(i % (h2 * w2)), yy = q / w2, xx = q % w2;
  const __nv_bfloat16 *s = a + bc * H * W + (2 * yy) * W + 2 * xx;
  x[i] = __float2bfloat16(0.25f * (bf(s[0]) + bf(s[1]) + bf(s[W]) + bf(s[W + 1])));
}

// feature vector [B][kFeat]: channel means of x4, then the conditioning
__global__ void k_gap_fwd(const __nv_bfloat16 *__restrict__ x, int C, int HW,
                          const float *__restrict__ cond, float *__restrict__ f) {
  const int b = blockIdx.x, c = threadIdx.x;
  if (c < C) {
    const __nv_bfloat16 *s = x + ((size_t)b * C + c) * HW;
    float t = 0.0f;
    for (int k = 0; k < HW; ++k) t += bf(s[k]);
    f[(size_t)b * kFeat + c] = t / (float)HW;
  } else if (c < C + kCond) {
    f[(size_t)b * kFeat + c] = cond[(size_t)b * kCond + (c - C)];
  }
}

// out[b][n] = act(sum_k in[b][k] W[n][k] + bias[n]), W in BF16; in rounded to
// BF16 before the product (BF16 activations).  grid (B), block N.
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

// global-average-pool backward into the pooled map of layer 4 (FP32 grads)
__global__ void k_gap_bwd(const float *__restrict__ df, int C, int HW, long long total,
                          float *__restrict__ dx) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const long long bc = i / HW;
  const int b = (int)(bc / C), c = (int)(bc % C);
  dx[i] = df[(size_t)b * kFeat + c] / (float)HW;
}

// pool backward and ReLU mask: dz[b][c][y][x] = dx[b][c][y/2][x/2] / 4 * [a > 0]
__global__ void k_pool_relu_bwd(const float *__restrict__ dx, const __nv_bfloat16 *__restrict__ a,
                                long long BC, int H, int W, float *__restrict__ dz) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= BC * H * W) return;
  const long long bc = i / (H * W);
  const int q = (int)(i % (H * W)), yy = q / W, xx = q % W;
  const float g = 0.25f * dx[bc * (H / 2) * (W / 2) + (yy / 2) * (W / 2) + (xx / 2)];
  dz[i] = bf(a[i]) > 0.0f ? g : 0.0f;
}

// conv backward to the input: dx[b][ci][y][x] = sum_co sum_taps W[co][ci][k]
// dz[b][co][y - ky + 1][x - kx + 1]; grid (ceil(HW/256), Cin, B)
__global__ void k_conv_bwd_in(const float *__restrict__ dz, int Cout, int H, int W,
                              const __nv_bfloat16 *__restrict__ w, int Cin,
                              float *__restrict__ dx) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= H * W) return;
  const int ci = blockIdx.y, b = blockIdx.z;
  const int yy = p / W, xx = p % W;
  float s = 0.0f;
  for (int co = 0; co < Cout; ++co) {
    const float *g = dz + ((size_t)b * Cout + co) * H * W;
    const __nv_bfloat16 *wk = w + ((size_t)co * Cin + ci) * 9;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int y2 = yy - ky + 1;
      if (y2 < 0 || y2 >= H) continue;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int x2 = xx - kx + 1;
        if (x2 < 0 || x2 >= W) continue;
        s += bf(wk[ky * 3 + kx]) * g[y2 * W + x2];
      }
    }
  }
  dx[((size_t)b * Cin + ci) * H * W + p] = s;
}

// conv weight gradient: dW[co][ci][k] = sum_{b,y,x} dz[b][co][y][x] x[b][ci][y+ky-1][x+kx-1],
// db[co] = sum dz[b][co]; one block per (co, ci), fixed-order block reduction
__global__ void k_conv_bwd_w(const float *__restrict__ dz, int Cout, int H, int W, int B,
                             const __nv_bfloat16 *__restrict__ x, int Cin,
                             float *__restrict__ dw, float *__restrict__ db) {
  __shared__ float sh[10][256];
  const int co = blockIdx.x / Cin, ci = blockIdx.x % Cin;
  float acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const long long tot = (long long)B * H * W;
  for (long long i = threadIdx.x; i < tot; i += blockDim.x) {
    const int b = (int)(i / (H * W));
    const int q = (int)(i % (H * W)), yy = q / W, xx = q % W;
    const float g = dz[((size_t)b * Cout + co) * H * W + q];
    if (g == 0.0f) continue;
    const __nv_bfloat16 *xc = x + ((size_t)b * Cin + ci) * H * W;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int y2 = yy + ky - 1;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int x2 = xx + kx - 1;
        if (y2 >= 0 && y2 < H && x2 >= 0 && x2 < W) acc[ky * 3 + kx] += g * bf(xc[y2 * W + x2]);
      }
    }
    acc[9] += g;
  }
  for (int k = 0; k < 10; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < 10; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < 9; ++k) dw[((size_t)co * Cin + ci) * 9 + k] = sh[k][0];
  }
  if (threadIdx.x == 0 && ci == 0) {
    // bias gradient once per output channel: the tenth accumulator of ci = 0
    db[co] = sh[9][0];
  }
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
  __nv_bfloat16 *pbf = nullptr;                                  // BF16 copies
  long long step = 0;
  // activations
  __nv_bfloat16 *x[kLayers + 1] = {};  // pooled maps (x0 = input)
  __nv_bfloat16 *a[kLayers] = {};      // post-ReLU conv outputs (pre-pool)
  float *feat = nullptr, *hid = nullptr, *y = nullptr, *loss = nullptr;
  float *dy = nullptr, *dhid = nullptr, *dfeat = nullptr;
  float *dx = nullptr, *dz = nullptr;  // largest FP32 grad maps (ping-pong)
  size_t big = 0;
};

int res_of(int l) { return kRes >> l; }  // spatial size of x_l

void free_net(Net &n) {
  void *ptrs[] = {n.p, n.g, n.m, n.v, n.pbf, n.feat, n.hid, n.y, n.loss, n.dy, n.dhid, n.dfeat, n.dx, n.dz};
  for (void *q : ptrs) cudaFree(q);
  for (int l = 0; l <= kLayers; ++l) cudaFree(n.x[l]);
  for (int l = 0; l < kLayers; ++l) cudaFree(n.a[l]);
}

// splitmix64 -> uniform in [-1, 1)
uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
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

int forward(sg_net *net, const uint8_t *occ, const float *cond, int B) {
  Net &n = net->n;
  cudaStream_t s = n.stream;
  k_occ_to_bf16<<<blocks((long long)B * kRes * kRes), 256, 0, s>>>(occ, (long long)B * kRes * kRes, n.x[0]);
  for (int l = 0; l < kLayers; ++l) {
    const int H = res_of(l);
    dim3 grid(blocks((long long)H * H), kCh[l + 1], B);
    k_conv_fwd<<<grid, 256, 0, s>>>(n.x[l], kCh[l], H, H, wbf(n, n.conv_w[l]), pf(n, n.conv_b[l]), kCh[l + 1],
                                    n.a[l]);
    const long long BC = (long long)B * kCh[l + 1];
    k_pool_fwd<<<blocks(BC * (H / 2) * (H / 2)), 256, 0, s>>>(n.a[l], BC, H, H, n.x[l + 1]);
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
  k_dense_bwd_in<<<B, 128, 0, s>>>(n.dhid, n.hid, kHidden, 1, wbf(n, n.f1_w), kFeat, n.dfeat);
  const int H4 = res_of(kLayers);
  const long long tot4 = (long long)B * kCh[kLayers] * H4 * H4;
  k_gap_bwd<<<blocks(tot4), 256, 0, s>>>(n.dfeat, kCh[kLayers], H4 * H4, tot4, n.dx);
  for (int l = kLayers - 1; l >= 0; --l) {
    const int H = res_of(l);
    const long long BC = (long long)B * kCh[l + 1];
    k_pool_relu_bwd<<<blocks(BC * H * H), 256, 0, s>>>(n.dx, n.a[l], BC, H, H, n.dz);
    k_conv_bwd_w<<<kCh[l + 1] * kCh[l], 256, 0, s>>>(n.dz, kCh[l + 1], H, H, B, n.x[l], kCh[l],
                                                    gf(n, n.conv_w[l]), gf(n, n.conv_b[l]));
    if (l > 0) {
      dim3 grid(blocks((long long)H * H), kCh[l], B);
      k_conv_bwd_in<<<grid, 256, 0, s>>>(n.dz, kCh[l + 1], H, H, wbf(n, n.conv_w[l]), kCh[l], n.dx);
      // dx now holds d(pooled map x_l) at resolution H: the next (lower) layer
      // pools from 2H, so its pool/relu backward reads this map.
    }
  }
  SGK(cudaGetLastError());
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
  for (int l = 0; l <= kLayers; ++l) al(&n.x[l], (size_t)max_batch * kCh[l] * res_of(l) * res_of(l) * 2);
  for (int l = 0; l < kLayers; ++l) al(&n.a[l], (size_t)max_batch * kCh[l + 1] * res_of(l) * res_of(l) * 2);
  size_t big = 0;
  for (int l = 0; l < kLayers; ++l) big = std::max(big, (size_t)max_batch * kCh[l + 1] * res_of(l) * res_of(l));
  n.big = big;
  al(&n.dx, big * 4); al(&n.dz, big * 4);
  al(&n.feat, (size_t)max_batch * kFeat * 4); al(&n.dfeat, (size_t)max_batch * kFeat * 4);
  al(&n.hid, (size_t)max_batch * kHidden * 4); al(&n.dhid, (size_t)max_batch * kHidden * 4);
  al(&n.y, (size_t)max_batch * kOut * 4); al(&n.dy, (size_t)max_batch * kOut * 4);
  al(&n.loss, 4);
  if (!ok) { free_net(n); cudaStreamDestroy(n.stream); delete net; return DG_ENOMEM; }
  cudaError_t e = cudaMemcpyAsync(n.p, h.data(), off * 4, cudaMemcpyHostToDevice, n.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n.m, 0, off * 4, n.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n.v, 0, off * 4, n.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n.g, 0, off * 4, n.stream);
  if (e == cudaSuccess) {
    k_to_bf16<<<blocks((long long)off), 256, 0, n.stream>>>(n.p, (long long)off, n.pbf);
    e = cudaGetLastError();
  }
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
  k_to_bf16<<<blocks((long long)n.n_params), 256, 0, n.stream>>>(n.p, (long long)n.n_params, n.pbf);
  SGK(cudaStreamSynchronize(n.stream));
  return DG_OK;
}

int sg_predict(sg_net *net, const uint8_t *occ, const float *cond, int B, float *out) {
  int r = check_io(net, occ, cond, B);
  if (r != DG_OK) return r;
  if (!out) return DG_EINVAL;
  Net &n = net->n;
  SGK(cudaSetDevice(n.device));
  r = forward(net, occ, cond, B);
  if (r != DG_OK) return r;
  SGK(cudaMemcpyAsync(out, n.y, (size_t)B * kOut * 4, cudaMemcpyDeviceToDevice, n.stream));
  SGK(cudaStreamSynchronize(n.stream));
  return DG_OK;
}

int sg_gradients(sg_net *net, const uint8_t *occ, const float *cond, const float *target, int B,
                 float *loss_host, float *grad_host) {
  int r = check_io(net, occ, cond, B);
  if (r != DG_OK) return r;
  if (!target) return DG_EINVAL;
  Net &n = net->n;
  SGK(cudaSetDevice(n.device));
  if ((r = forward(net, occ, cond, B)) != DG_OK) return r;
  if ((r = backward(net, target, B)) != DG_OK) return r;
  if (loss_host) SGK(cudaMemcpyAsync(loss_host, n.loss, 4, cudaMemcpyDeviceToHost, n.stream));
  if (grad_host) SGK(cudaMemcpyAsync(grad_host, n.g, n.n_params * 4, cudaMemcpyDeviceToHost, n.stream));
  SGK(cudaStreamSynchronize(n.stream));
  return DG_OK;
}

int sg_train_step(sg_net *net, const uint8_t *occ, const float *cond, const float *target, int B,
                  float lr, float *loss_host) {
  int r = check_io(net, occ, cond, B);
  if (r != DG_OK) return r;
  if (!target || !(lr > 0.0f) || !std::isfinite(lr)) return DG_EINVAL;
  Net &n = net->n;
  SGK(cudaSetDevice(n.device));
  if ((r = forward(net, occ, cond, B)) != DG_OK) return r;
  if ((r = backward(net, target, B)) != DG_OK) return r;
  n.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)n.step), c2 = 1.0f - std::pow(b2, (float)n.step);
  k_adam<<<blocks((long long)n.n_params), 256, 0, n.stream>>>(n.p, n.g, n.m, n.v, (long long)n.n_params, lr,
                                                              b1, b2, 1e-8f, c1, c2, nullptr, n.pbf);
  SGK(cudaGetLastError());
  if (loss_host) SGK(cudaMemcpyAsync(loss_host, n.loss, 4, cudaMemcpyDeviceToHost, n.stream));
  SGK(cudaStreamSynchronize(n.stream));
  return DG_OK;
}

}  // extern "C"
