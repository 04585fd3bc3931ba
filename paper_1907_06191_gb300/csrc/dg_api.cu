// dg_api.cu -- the C ABI of include/dgsigma.h.
//
// Host code here validates arguments, owns device memory and sequences the
// kernels; every arithmetic step of the path runs in the kernels of
// dg_stage.cuh, dg_geometry.cu and dg_reduce.cu.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

#include "dg_internal.h"

using namespace dg;

namespace dg {

// countdown to an injected allocation failure; -1 = none armed
static std::atomic<long long> g_fail_alloc{-1};

cudaError_t dev_alloc(void **p, size_t bytes) {
  long long n = g_fail_alloc.load();
  while (n >= 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  // the failure is returned here; clear it from the thread's last-error state
  // so that a later launch check does not report it as a launch failure
  if (e != cudaSuccess) (void)cudaGetLastError();
  return e;
}

}  // namespace dg

struct dg_ctx {
  Ctx c;
};

namespace {

constexpr int kGraphChunk = 64;             // RK steps per captured graph
constexpr int kCheckChunk = 4096;           // steps between stability checks
constexpr uint64_t kStateMagic = 0x31474453474432ull;  // "2DGSDG1"

int fail(dg_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->c.last_error = msg;
  return code;
}

int cuda_fail(dg_ctx *ctx, cudaError_t e, const char *what) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr, what)                                   \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, what); \
  } while (0)

void drop_graph(Ctx &c) {
  if (c.graph) cudaGraphExecDestroy(c.graph);
  c.graph = nullptr;
  c.graph_steps = 0;
}

void free_window(Ctx &c) {
  cudaFree(c.d_gw_d2);
  cudaFree(c.d_gw_adv);
  cudaFree(c.d_gw_order);
  c.d_gw_d2 = nullptr;
  c.d_gw_adv = nullptr;
  c.d_gw_order = nullptr;
  c.gw_cmin.clear();
  c.gw_ready = false;
  c.gw_synced = false;
}

void free_state(Ctx &c) {
  drop_graph(c);
  if (c.state_owned && c.d_state) cudaFree(c.d_state);
  c.d_state = nullptr;
  cudaFree(c.d_src);
  cudaFree(c.d_srel);
  c.d_srel = nullptr;
  cudaFree(c.d_mom);
  cudaFree(c.d_mom0);
  cudaFree(c.d_part);
  cudaFree(c.d_out);
  cudaFree(c.d_q);
  c.d_q = nullptr;
  c.tmap_ok = false;
  c.d_src = c.d_mom = c.d_mom0 = c.d_part = c.d_out = nullptr;
  free_window(c);
  c.m = 0;
  c.t = 0;
  c.steps = 0;
  c.state_bytes = 0;
  c.src.clear();
}

void *state_array(Ctx &c, int k) {
  return (char *)c.d_state + (size_t)k * c.m * c.field_elems() * c.esize();
}

size_t state_bytes_for(const Ctx &c, int m) {
  size_t b = 3 * (size_t)m * c.field_elems() * c.esize();
  return (b + 255) / 256 * 256;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor maps of the three state arrays: rows of np values, boxes of kBlock
// rows, the hardware swizzle that matches Stage's layout (32, 64 or 128 bytes
// per row; none otherwise).  Left unset (cp.async copies) when the rows are
// not whole 16-byte slots, when the row count m * n_pad does not fit the
// tensor copies' 32-bit row coordinate (possible at p = 1, whose rows are
// 16 or 32 bytes), or when the encoder is unavailable.
void make_tensor_maps(Ctx &c) {
  c.tmap_ok = false;
  if (c.triangles() || !c.d_state) return;
  const size_t row_bytes = (size_t)c.np() * c.esize();
  if (row_bytes % 16 != 0) return;
  if ((long long)c.m * c.geo.n_pad > (long long)INT_MAX) return;
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return;
  const CUtensorMapSwizzle sw = row_bytes == 32    ? CU_TENSOR_MAP_SWIZZLE_32B
                                : row_bytes == 64  ? CU_TENSOR_MAP_SWIZZLE_64B
                                : row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                                   : CU_TENSOR_MAP_SWIZZLE_NONE;
  const cuuint64_t dims[2] = {(cuuint64_t)c.np(), (cuuint64_t)c.m * (cuuint64_t)c.geo.n_pad};
  const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)c.np(), (cuuint32_t)kBlock};
  const cuuint32_t estr[2] = {1, 1};
  for (int k = 0; k < 3; ++k) {
    const CUresult r = enc(&c.tmap[k],
                           c.cfg.precision == DG_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                           2, state_array(c, k), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return;
  }
  c.tmap_ok = true;
}

// DG_ETIMEOUT if a bounded wait of a stage kernel gave up since the last
// check (the flag is cleared); synchronises the stream.
int take_device_error(dg_ctx *ctx) {
  Ctx &c = ctx->c;
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c.d_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "error flag");
  CK(cudaStreamSynchronize(c.stream), "error flag");
  if (flag) {
    CK(cudaMemsetAsync(c.d_err, 0, sizeof(int), c.stream), "error flag");
    if (flag == 2)
      return fail(ctx, DG_ECUDA, "a stage kernel found its shared memory misaligned for tensor copies");
    return fail(ctx, DG_ETIMEOUT,
                "a stage kernel gave up waiting for its shared-memory copies or a grid barrier");
  }
  return DG_OK;
}

// Copy settings of RK stage k (input array k; u0 = array 0; output array
// k + 1 mod 3: U1, U2, then U in place).
StageCopies stage_copies(Ctx &c, int in_array, bool with_u0) {
  StageCopies cp;
  if (!c.tmap_ok || c.copy_mode == 1) return cp;
  cp.map_u = &c.tmap[in_array];
  cp.map_u0 = with_u0 ? &c.tmap[0] : nullptr;
  cp.map_out = &c.tmap[(in_array + 1) % 3];
  cp.use_tma = 1;
  cp.extra_tx = c.copy_mode == 2 ? 16 : 0;
  cp.limit = c.copy_mode == 2 ? (1 << 12) : (1 << 22);
  cp.err = c.d_err;
  cp.counter = c.d_tma;
  cp.pipe_blocks = c.launch_blocks;
  cp.tensor_core = c.contraction_tc;
  return cp;
}

// Launch shape of the FP32 stage kernel (one block per chunk, or persistent
// with k blocks per SM) and, at p = 5, where its element contractions run
// (CUDA cores or tensor cores).  Tuned: each candidate runs RK stage 1 with
// dt = 0 (U1 = U, bit for bit, so the probe changes nothing the next step
// reads) once untimed and three times timed with CUDA events on the
// context's stream; the fastest is kept for this number of densities and
// elements.  Under stream capture nothing can be timed: the one-block-per-
// chunk launch on the CUDA cores is taken.
int resolve_launch(dg_ctx *ctx) {
  Ctx &c = ctx->c;
  const bool fp32 = c.cfg.precision == DG_FP32 && !c.triangles() && c.tmap_ok && c.copy_mode != 1;
  const int maxb = fp32 ? stage_pipe_max_blocks(c.cfg.precision, c.cfg.p, c.geo) : 0;
  const bool tc_ok = fp32 && c.cfg.p == 5 && stage_tc_max_blocks(c.geo) >= 1;
  // the launch shapes this context has; one launch per step is opt-in only:
  // it removes launch gaps, which a timing probe under a profiler (that
  // serialises and slows every launch) would overrate
  std::vector<int> shapes{0};
  const bool step_ok = fp32 && (c.cfg.p == 1 || c.cfg.p == 3 || c.cfg.p == 5);
  if (step_ok && c.launch_req == kLaunchStep) shapes.push_back(kLaunchStep);
  for (int k = 1; k <= maxb; ++k) shapes.push_back(k);
  int want = 0, want_tc = 0;
  const bool fixed = c.launch_req != -1 || shapes.size() == 1;
  const bool fixed_tc = c.contraction_req >= 0 || !tc_ok;
  if (fixed) {
    if (c.launch_req == kLaunchStep) want = step_ok ? kLaunchStep : 0;
    else if (c.launch_req >= 1) want = std::min(c.launch_req, maxb);  // 0 without a persistent kernel
    else want = 0;
  }
  if (fixed_tc) want_tc = tc_ok && c.contraction_req == 1 ? 1 : 0;
  if (!(fixed && fixed_tc)) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(c.stream, &cap), "capture status");
    if (c.copy_mode != 0 || cap != cudaStreamCaptureStatusNone) {
      // a test hook is active or nothing can be timed: the plain launch
      if (!fixed) want = 0;
      if (!fixed_tc) want_tc = 0;
    } else if (c.tuned_key[0] == c.m && c.tuned_key[1] == c.geo.n_pad && c.tuned_blocks != -1) {
      if (!fixed) want = c.tuned_blocks;
      if (!fixed_tc) want_tc = c.tuned_tc;
    } else {
      TraceRange trace("launch tuning");
      std::vector<std::pair<int, int>> cand;  // (launch shape, tensor cores)
      for (const int k : shapes) {
        if (fixed && k != want) continue;
        for (int t = fixed_tc ? want_tc : 0; t <= (fixed_tc ? want_tc : 1); ++t)
          if (t == 0 || k == 0) cand.push_back({k, t});  // tensor cores: one block per chunk
      }
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      CK(cudaEventCreate(&e0), "tuning event");
      cudaError_t e = cudaEventCreate(&e1);
      const double pen = c.cfg.eta * (c.cfg.p + 1.0) * (c.cfg.p + 1.0) * 0.5;
      const StageCoef<float> sc{0.0f, 1.0f, 0.0f, (float)pen, c.cfg.wall_mode == DG_WALL_PAPER,
                                c.cfg.rounding == DG_ROUND_STOCHASTIC};
      float best = 0.0f;
      std::pair<int, int> best_c = cand[0];
      for (size_t q = 0; q < cand.size() && e == cudaSuccess; ++q) {
        StageCopies cp = stage_copies(c, 0, false);
        cp.pipe_blocks = cand[q].first;
        cp.tensor_core = cand[q].second;
        // one step with dt = 0 leaves the state unchanged as well (every
        // stage adds an exact zero); it counts as three stage launches
        const StageCoef<float> sc3[3] = {sc, {0.75f, 0.25f, 0.0f, sc.pen, sc.wallA, sc.sround},
                                         {1.0f / 3.0f, 2.0f / 3.0f, 0.0f, sc.pen, sc.wallA, sc.sround}};
        const bool whole_step = cand[q].first == kLaunchStep;
        auto probe = [&]() {
          if (whole_step)
            return launch_rk3_grid_f32(c.cfg.p, (float *)state_array(c, 0), (float *)state_array(c, 1),
                                       (float *)state_array(c, 2), c.geo, c.geo.n_pad, c.m, c.gll,
                                       sc3, c.stream, ChunkSel{}, c.tmap, c.d_err, c.d_tma, c.d_grid,
                                       0, 1 << 22, 0, 1 << 22);
          return launch_stage_f32(c.cfg.p, (const float *)state_array(c, 0), nullptr,
                                  (float *)state_array(c, 1), c.geo, c.geo.n_pad, c.m, c.gll, sc,
                                  c.stream, ChunkSel{}, cp);
        };
        e = probe();
        if (e == cudaSuccess) e = cudaEventRecord(e0, c.stream);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = probe();
        if (e == cudaSuccess) e = cudaEventRecord(e1, c.stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (whole_step) ms /= 3.0f;
        if (e == cudaErrorNotSupported) {  // the variant cannot take this shape: skip it
          e = cudaSuccess;
          continue;
        }
        if (e == cudaSuccess && (q == 0 || ms < best)) {
          best = ms;
          best_c = cand[q];
        }
      }
      cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "launch tuning");
      if (const int r = take_device_error(ctx); r != DG_OK) return r;
      c.tuned_blocks = best_c.first;
      c.tuned_tc = best_c.second;
      c.tuned_key[0] = c.m;
      c.tuned_key[1] = c.geo.n_pad;
      if (!fixed) want = best_c.first;
      if (!fixed_tc) want_tc = best_c.second;
    }
  }
  if (want_tc) {  // the tensor-core kernel's operator table, before any capture
    const cudaError_t e = stage_tc_prepare(c.gll, c.stream);
    if (e == cudaErrorNotSupported) want_tc = 0;
    else if (e != cudaSuccess) return cuda_fail(ctx, e, "tensor-core operator");
  }
  if (want != c.launch_blocks || want_tc != c.contraction_tc) {
    c.launch_blocks = want;
    c.contraction_tc = want_tc;
    drop_graph(c);  // captured launches carry the old shape
  }
  return DG_OK;
}

// One SSP-RK3 step: U1 = U + dt L U; U2 = 3/4 U + 1/4 (U1 + dt L U1);
// U <- 1/3 U + 2/3 (U2 + dt L U2).  L = (k/J^2) R.
cudaError_t rk3_step(Ctx &c, double dt, cudaStream_t s, const ChunkSel &sel = ChunkSel{}) {
  const double kc = c.cfg.D;  // the kernel applies 1/J^2 of each element's geometry
  const double pen = c.cfg.eta * (c.cfg.p + 1.0) * (c.cfg.p + 1.0) * 0.5;
  const int wallA = c.cfg.wall_mode == DG_WALL_PAPER;
  const long long st = c.geo.n_pad;
  const double co[3][3] = {{0.0, 1.0, dt * kc},
                           {0.75, 0.25, 0.25 * dt * kc},
                           {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0 * dt * kc}};
  void *U0 = state_array(c, 0), *U1 = state_array(c, 1), *U2 = state_array(c, 2);
  if (c.launch_blocks == kLaunchStep && c.cfg.precision == DG_FP32 && !c.triangles() && c.tmap_ok) {
    const int rnd = c.cfg.rounding == DG_ROUND_STOCHASTIC;
    const StageCoef<float> sc[3] = {
        {(float)co[0][0], (float)co[0][1], (float)co[0][2], (float)pen, wallA, rnd},
        {(float)co[1][0], (float)co[1][1], (float)co[1][2], (float)pen, wallA, rnd},
        {(float)co[2][0], (float)co[2][1], (float)co[2][2], (float)pen, wallA, rnd}};
    const cudaError_t e = launch_rk3_grid_f32(
        c.cfg.p, (float *)U0, (float *)U1, (float *)U2, c.geo, st, c.m, c.gll, sc, s, sel, c.tmap,
        c.d_err, c.d_tma, c.d_grid, c.copy_mode == 2 ? 16 : 0, c.copy_mode == 2 ? (1 << 12) : (1 << 22),
        c.copy_mode == 3 ? 1 : 0, c.copy_mode == 3 ? (1 << 12) : (1 << 22));
    if (e != cudaErrorNotSupported) return e;
  }
  void *in[3] = {U0, U1, U2};
  void *outp[3] = {U1, U2, U0};
  void *base[3] = {nullptr, U0, U0};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    if (c.cfg.precision == DG_FP64) {
      StageCoef<double> sc{co[k][0], co[k][1], co[k][2], pen, wallA};
      if (c.triangles())
        e = launch_tri_stage_f64(c.cfg.p, (const double *)in[k], (const double *)base[k],
                                 (double *)outp[k], (double *)c.d_q, c.geo, st, c.m, c.tri, sc,
                                 s, sel);
      else
        e = launch_stage_f64(c.cfg.p, (const double *)in[k], (const double *)base[k],
                             (double *)outp[k], c.geo, st, c.m, c.gll, sc, s, sel,
                             stage_copies(c, k, base[k] != nullptr));
    } else {
      StageCoef<float> sc{(float)co[k][0], (float)co[k][1], (float)co[k][2], (float)pen,
                          wallA, c.cfg.rounding == DG_ROUND_STOCHASTIC};
      if (c.triangles())
        e = launch_tri_stage_f32(c.cfg.p, (const float *)in[k], (const float *)base[k],
                                 (float *)outp[k], (float *)c.d_q, c.geo, st, c.m, c.tri, sc,
                                 s, sel, c.tri_fused != 0);
      else
        e = launch_stage_f32(c.cfg.p, (const float *)in[k], (const float *)base[k],
                             (float *)outp[k], c.geo, st, c.m, c.gll, sc, s, sel,
                             stage_copies(c, k, base[k] != nullptr));
    }
  }
  return e;
}

int run_steps_fixed(dg_ctx *ctx, int nsteps, double dt) {
  Ctx &c = ctx->c;
  TraceRange trace("RK3 steps");
  c.gw_synced = false;  // arrays 1 and 2 now hold stage values everywhere
  int left = nsteps;
  if (left >= kGraphChunk) {
    if (!c.graph || c.graph_dt != dt || c.graph_stream != c.stream) {
      drop_graph(c);
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      cudaError_t e = cudaSuccess;
      for (int k = 0; k < kGraphChunk && e == cudaSuccess; ++k) e = rk3_step(c, dt, c.stream);
      cudaError_t e2 = cudaStreamEndCapture(c.stream, &g);
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "stage launch during capture");
      }
      CK(e2, "end capture");
      e = cudaGraphInstantiate(&c.graph, g, 0);
      cudaGraphDestroy(g);
      CK(e, "graph instantiate");
      c.graph_dt = dt;
      c.graph_steps = kGraphChunk;
      c.graph_stream = c.stream;
    }
    while (left >= kGraphChunk) {
      CK(cudaGraphLaunch(c.graph, c.stream), "graph launch");
      left -= kGraphChunk;
    }
  }
  for (int k = 0; k < left; ++k) CK(rk3_step(c, dt, c.stream), "stage launch");
  c.steps += nsteps;
  return DG_OK;
}

// Window tables for the current sources: per element the squared distance to
// its geometry's start-point box, chunks ordered by their nearest element.
int prepare_window(dg_ctx *ctx) {
  Ctx &c = ctx->c;
  TraceRange trace("growing window tables");
  const int G = c.geo.G();
  const long long n = c.geo.n_pad, nch = c.geo.n_chunks();
  std::vector<double> box((size_t)4 * G);
  for (int g = 0; g < G; ++g) {
    double *b = &box[(size_t)4 * g];
    b[0] = b[2] = INFINITY;
    b[1] = b[3] = -INFINITY;
    for (int s = 0; s < c.m; ++s) {
      const double x = c.src[2 * ((size_t)g * c.m + s)], y = c.src[2 * ((size_t)g * c.m + s) + 1];
      b[0] = std::min(b[0], x); b[1] = std::max(b[1], x);
      b[2] = std::min(b[2], y); b[3] = std::max(b[3], y);
    }
  }
  double *d_box = nullptr;
  {
    cudaError_t e = cudaSuccess;
    if (!c.d_gw_d2) {
      e = dev_alloc(&c.d_gw_d2, sizeof(double) * (size_t)n);
      if (e == cudaSuccess) e = dev_alloc(&c.d_gw_adv, (size_t)n);
      if (e == cudaSuccess) e = dev_alloc(&c.d_gw_order, sizeof(int) * (size_t)nch);
    }
    if (e == cudaSuccess) e = dev_alloc(&d_box, sizeof(double) * box.size());
    if (e != cudaSuccess) {
      free_window(c);
      return cuda_fail(ctx, e, "window allocation");
    }
  }
  std::vector<double> d2((size_t)n);
  cudaError_t e = cudaMemcpyAsync(d_box, box.data(), sizeof(double) * box.size(),
                                  cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = launch_window_d2(c, d_box, c.d_gw_d2, c.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d2.data(), c.d_gw_d2, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost,
                        c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  cudaFree(d_box);
  CK(e, "window distances");
  std::vector<double> cmin((size_t)nch, INFINITY);
  c.gw_dmax = 0.0;
  for (long long a = 0; a < n; ++a) {
    const double v = d2[(size_t)a];
    if (std::isinf(v)) continue;  // padding
    cmin[(size_t)(a / kBlock)] = std::min(cmin[(size_t)(a / kBlock)], v);
    c.gw_dmax = std::max(c.gw_dmax, v);
  }
  std::vector<int> order((size_t)nch);
  for (long long k = 0; k < nch; ++k) order[(size_t)k] = (int)k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return cmin[(size_t)a] < cmin[(size_t)b]; });
  c.gw_cmin.resize((size_t)nch);
  for (long long k = 0; k < nch; ++k) c.gw_cmin[(size_t)k] = cmin[(size_t)order[(size_t)k]];
  CK(cudaMemcpyAsync(c.d_gw_order, order.data(), sizeof(int) * (size_t)nch, cudaMemcpyHostToDevice,
                     c.stream), "window order");
  CK(cudaStreamSynchronize(c.stream), "window order");
  c.gw_ready = true;
  return DG_OK;
}

// Steps on the growing window, starting at time t0.  Chunks that have not
// been launched since the stage arrays were synchronised hold array 0's
// values in arrays 1 and 2, so launched chunks read their halos correctly.
int run_steps_window(dg_ctx *ctx, int nsteps, double dt, double t0) {
  Ctx &c = ctx->c;
  TraceRange trace("RK3 steps (growing window)");
  if (!c.gw_ready) {
    const int r = prepare_window(ctx);
    if (r != DG_OK) return r;
  }
  if (!c.gw_synced) {
    const size_t bytes = (size_t)c.m * c.field_elems() * c.esize();
    CK(cudaMemcpyAsync(state_array(c, 1), state_array(c, 0), bytes, cudaMemcpyDeviceToDevice,
                       c.stream), "window sync");
    CK(cudaMemcpyAsync(state_array(c, 2), state_array(c, 0), bytes, cudaMemcpyDeviceToDevice,
                       c.stream), "window sync");
    c.gw_synced = true;
  }
  const double s0 = c.cfg.sigma0, D = c.cfg.D;
  int done = 0;
  while (done < nsteps) {
    const int k = std::min(kGraphChunk, nsteps - done);
    const double t_end = t0 + (double)(done + k) * dt;
    const double r2 = c.gw_r * c.gw_r * (s0 * s0 + 2.0 * D * t_end);
    if (r2 >= c.gw_dmax) {
      // every mesh element advances from here on: the fixed-window path
      c.steps += done;
      return run_steps_fixed(ctx, nsteps - done, dt);
    }
    const long long nact =
        std::upper_bound(c.gw_cmin.begin(), c.gw_cmin.end(), r2) - c.gw_cmin.begin();
    CK(launch_window_flags(c, c.d_gw_d2, r2, c.d_gw_adv, c.stream), "window flags");
    ChunkSel sel;
    sel.list = c.d_gw_order;
    sel.count = nact;
    sel.adv = c.d_gw_adv;
    for (int j = 0; j < k; ++j) CK(rk3_step(c, dt, c.stream, sel), "stage launch");
    done += k;
  }
  c.steps += nsteps;
  return DG_OK;
}

int run_steps(dg_ctx *ctx, int nsteps, double dt, double t0) {
  if (nsteps > 0) {
    if (const int r = resolve_launch(ctx); r != DG_OK) return r;
  }
  if (ctx->c.gw_r > 0.0) return run_steps_window(ctx, nsteps, dt, t0);
  return run_steps_fixed(ctx, nsteps, dt);
}

int compute_moments(dg_ctx *ctx, double *d_dst) {
  Ctx &c = ctx->c;
  TraceRange trace("moments");
  CK(launch_moments(c, state_array(c, 0), c.d_part, d_dst, c.stream), "moments");
  return DG_OK;
}

int ensure_rho(dg_ctx *ctx) {
  Ctx &c = ctx->c;
  TraceRange trace("spectral radius (power iteration)");
  if (c.have_rho) return DG_OK;
  if (!c.have_geo) return fail(ctx, DG_ESTATE, "no geometry");
  const size_t nv = (size_t)c.geo.n_pad * c.np();
  double *v = nullptr, *w = nullptr, *res = nullptr, *part = nullptr, *qb = nullptr;
  auto cleanup = [&]() { cudaFree(v); cudaFree(w); cudaFree(res); cudaFree(part); cudaFree(qb); };
  cudaError_t e;
  if ((e = dev_alloc(&v, nv * 8)) != cudaSuccess || (e = dev_alloc(&w, nv * 8)) != cudaSuccess ||
      (e = dev_alloc(&res, 8 * kMomFields)) != cudaSuccess ||
      (e = dev_alloc(&part, 8 * kMomFields * (size_t)kMomBlocks)) != cudaSuccess ||
      (c.triangles() && (e = dev_alloc(&qb, nv * 2 * 8)) != cudaSuccess)) {
    cleanup();
    return fail(ctx, DG_ENOMEM, std::string("power iteration buffers: ") + cudaGetErrorString(e));
  }
  const double kc = c.cfg.D;
  const double pen = c.cfg.eta * (c.cfg.p + 1.0) * (c.cfg.p + 1.0) * 0.5;
  StageCoef<double> sc{0.0, 0.0, kc, pen, c.cfg.wall_mode == DG_WALL_PAPER};
  const int iters = c.cfg.power_iters > 0 ? c.cfg.power_iters : 200;
  e = launch_random_field(c, v, 12345ull, c.stream);
  if (e == cudaSuccess) e = launch_wnorm2(c, v, part, res, c.stream);
  if (e == cudaSuccess) e = launch_scale_by_rnorm(c, v, res, v, c.stream);
  for (int it = 0; it < iters && e == cudaSuccess; ++it) {
    if (c.triangles())
      e = launch_tri_stage_f64(c.cfg.p, v, nullptr, w, qb, c.geo, c.geo.n_pad, 1, c.tri, sc,
                               c.stream);
    else
      e = launch_stage_f64(c.cfg.p, v, nullptr, w, c.geo, c.geo.n_pad, 1, c.gll, sc, c.stream);
    if (e == cudaSuccess) e = launch_wnorm2(c, w, part, res, c.stream);
    if (e == cudaSuccess && it + 1 < iters) e = launch_scale_by_rnorm(c, w, res, v, c.stream);
  }
  double r2 = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r2, res, 8, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "power iteration");
  if (!(r2 > 0.0) || !std::isfinite(r2)) return fail(ctx, DG_ENONFINITE, "power iteration gave no finite spectral radius");
  c.rho = std::sqrt(r2);
  c.dt_max = c.cfg.cfl_safety * rk3_real_axis_limit() / c.rho;
  c.have_rho = true;
  return DG_OK;
}

int check_config(const dg_config *cfg, std::string &why) {
  if (cfg->p < 1 || cfg->p > kMaxP) { why = "p must be in 1..5"; return DG_EINVAL; }
  if (cfg->precision != DG_FP64 && cfg->precision != DG_FP32) { why = "bad precision"; return DG_EINVAL; }
  if (!(cfg->D > 0.0) || !std::isfinite(cfg->D)) { why = "D must be > 0"; return DG_EINVAL; }
  if (!(cfg->sigma0 > 0.0)) { why = "sigma0 must be > 0"; return DG_EINVAL; }
  if (!(cfg->eta >= 0.0)) { why = "eta must be >= 0"; return DG_EINVAL; }
  if (!(cfg->cfl_safety > 0.0 && cfg->cfl_safety <= 1.0)) { why = "cfl_safety must be in (0, 1]"; return DG_EINVAL; }
  if (cfg->wall_mode != DG_WALL_REMOVED && cfg->wall_mode != DG_WALL_PAPER) { why = "bad wall_mode"; return DG_EINVAL; }
  if (cfg->boundary != DG_BC_ABSORBING && cfg->boundary != DG_BC_PERIODIC) { why = "bad boundary"; return DG_EINVAL; }
  if (cfg->power_iters < 0) { why = "power_iters must be >= 0"; return DG_EINVAL; }
  if (cfg->rounding != DG_ROUND_NEAREST && cfg->rounding != DG_ROUND_STOCHASTIC) { why = "bad rounding"; return DG_EINVAL; }
  if (cfg->element != DG_ELEMENT_SQUARE && cfg->element != DG_ELEMENT_TRIANGLE) { why = "bad element"; return DG_EINVAL; }
  if (cfg->element == DG_ELEMENT_TRIANGLE && (cfg->p > kTriMaxP || cfg->eta != 0.0)) {
    why = "triangles take p = 1..3 and eta = 0";
    return DG_EINVAL;
  }
  return DG_OK;
}

int set_parts(dg_ctx *ctx, const std::vector<PartSpec> &parts) {
  Ctx &c = ctx->c;
  TraceRange trace("geometry upload");
  free_state(c);
  c.have_geo = false;
  c.have_rho = false;
  std::string err;
  const int code = build_geometry(c.geo, parts, c.cfg.boundary == DG_BC_PERIODIC, c.triangles(),
                                  c.stream, err);
  if (code != DG_OK) return fail(ctx, code, err);
  c.have_geo = true;
  return DG_OK;
}

bool check_disk_args(const double *cx, const double *cy, const double *r, int nd, double L,
                     int n_cell, int tiles, std::string &why) {
  if (nd < 0 || (nd > 0 && (!cx || !cy || !r)) || !(L > 0.0) || !std::isfinite(L) || n_cell < 1 ||
      tiles < 1 || tiles % 2 == 0) {
    why = "bad disk geometry arguments (tiles must be odd)";
    return false;
  }
  const long long nwin = (long long)n_cell * tiles;
  if (nwin * nwin > (1ll << 31) - 1) {
    why = "domain too large";
    return false;
  }
  for (int d = 0; d < nd; ++d)
    if (!(r[d] >= 0.0) || !std::isfinite(r[d]) || !std::isfinite(cx[d]) || !std::isfinite(cy[d])) {
      why = "bad disk " + std::to_string(d);
      return false;
    }
  return true;
}

PartSpec disk_part(const double *cx, const double *cy, const double *r, int nd, double L,
                   int n_cell, int tiles) {
  PartSpec q;
  q.nx = q.ny = n_cell * tiles;
  q.h = L / n_cell;
  q.x0 = q.y0 = -(double)(tiles / 2) * L;
  q.cx = cx; q.cy = cy; q.r = r; q.nd = nd;
  q.L = L; q.n_cell = n_cell; q.tiles = tiles;
  return q;
}

// xy holds m start points for each geometry: [G][m][2].
int set_sources_impl(dg_ctx *ctx, const double *xy, int m) {
  Ctx &c = ctx->c;
  TraceRange trace("start densities");
  if (!c.have_geo) return fail(ctx, DG_ESTATE, "dg_set_sources before a geometry");
  if (!xy || m < 1 || m > 65535) return fail(ctx, DG_EINVAL, "need 1 <= m <= 65535 start points");
  const int G = c.geo.G();
  // validate: inside the domain and in a mesh element of its geometry
  for (int g = 0; g < G; ++g) {
    const GeoPart &p = c.geo.parts[g];
    const uint8_t *mask = c.geo.h_mask.data() + p.dense_off;
    for (int s = 0; s < m; ++s) {
      const double x = xy[2 * ((size_t)g * m + s)], y = xy[2 * ((size_t)g * m + s) + 1];
      const double fx = (x - p.x0) / p.h, fy = (y - p.y0) / p.h;
      const std::string who = "start point " + std::to_string(s) +
                              (G > 1 ? " of geometry " + std::to_string(g) : std::string());
      if (!(fx >= 0.0 && fy >= 0.0 && fx < p.nx && fy < p.ny))
        return fail(ctx, DG_EINVAL, who + " outside the domain");
      const int ex = (int)fx, ey = (int)fy;
      if (!mask[(size_t)ey * p.nx + ex]) return fail(ctx, DG_EINVAL, who + " lies in an axon element");
    }
  }
  // Same number of start points on the same geometry: keep the buffers (and
  // any captured graph, whose pointers stay valid).
  const bool reuse = c.m == m && c.d_state != nullptr;
  const size_t nd = (size_t)G * m;
  if (!reuse) {
    free_state(c);
    const size_t need = state_bytes_for(c, m);
    // a failed allocation leaves the context without sources, as before the call
#define SK(expr, what)                            \
  do {                                            \
    const cudaError_t _e = (expr);                \
    if (_e != cudaSuccess) {                      \
      free_state(c);                              \
      return cuda_fail(ctx, _e, what);            \
    }                                             \
  } while (0)
    if (c.bound_ptr) {
      if (c.bound_bytes < need) return fail(ctx, DG_EINVAL, "bound state buffer too small");
      c.d_state = c.bound_ptr;
      c.state_owned = false;
    } else {
      c.state_owned = true;
      SK(dev_alloc(&c.d_state, need), "state allocation");
    }
    c.state_bytes = need;
    c.m = m;
    SK(dev_alloc(&c.d_src, sizeof(double) * 2 * nd), "source allocation");
    SK(dev_alloc(&c.d_srel, sizeof(float4) * nd), "source allocation");
    SK(dev_alloc(&c.d_mom, sizeof(double) * kMomFields * nd), "moment allocation");
    SK(dev_alloc(&c.d_mom0, sizeof(double) * kMomFields * nd), "moment allocation");
    SK(dev_alloc(&c.d_part, sizeof(double) * kMomFields * moment_blocks(G) * nd), "partial allocation");
    SK(dev_alloc(&c.d_out, sizeof(double) * (kCovOut + 1) * G), "output allocation");
    if (c.triangles())
      SK(dev_alloc(&c.d_q, (size_t)m * c.field_elems() * 2 * c.esize()), "q allocation");
#undef SK
  }
  c.src.assign(xy, xy + 2 * nd);
  c.gw_ready = false;
  c.gw_synced = false;
  make_tensor_maps(c);
  CK(cudaMemcpyAsync(c.d_src, c.src.data(), sizeof(double) * 2 * nd, cudaMemcpyHostToDevice, c.stream), "source copy");
  CK(launch_init_sources(c, state_array(c, 0), c.stream), "init sources");
  int r = compute_moments(ctx, c.d_mom0);
  if (r != DG_OK) return r;
  CK(cudaMemcpyAsync(c.d_mom, c.d_mom0, sizeof(double) * kMomFields * nd, cudaMemcpyDeviceToDevice, c.stream), "moment copy");
  c.t = 0.0;
  c.steps = 0;
  return DG_OK;
}

int check_growth(dg_ctx *ctx) {
  Ctx &c = ctx->c;
  TraceRange trace("stability check");
  if (const int r = take_device_error(ctx); r != DG_OK) return r;
  const int nd = c.m * c.geo.G();
  std::vector<double> mom((size_t)nd * kMomFields), mom0((size_t)nd * kMomFields);
  int r = compute_moments(ctx, c.d_mom);
  if (r != DG_OK) return r;
  CK(cudaMemcpyAsync(mom.data(), c.d_mom, mom.size() * 8, cudaMemcpyDeviceToHost, c.stream), "moment copy");
  CK(cudaMemcpyAsync(mom0.data(), c.d_mom0, mom0.size() * 8, cudaMemcpyDeviceToHost, c.stream), "moment copy");
  CK(cudaStreamSynchronize(c.stream), "moments");
  for (int s = 0; s < nd; ++s) {
    const double *q = &mom[(size_t)s * kMomFields];
    for (int f = 0; f < kMomFields; ++f)
      if (!std::isfinite(q[f]))
        return fail(ctx, DG_EUNSTABLE, "density " + std::to_string(s) + " became non-finite: time step above the stability bound");
    if (q[6] > 2.0 * mom0[(size_t)s * kMomFields + 6])
      return fail(ctx, DG_EUNSTABLE, "density " + std::to_string(s) + " grew: time step above the stability bound");
  }
  return DG_OK;
}

}  // namespace

extern "C" {

void dg_config_default(dg_config *cfg) {
  if (!cfg) return;
  cfg->p = 3;
  cfg->precision = DG_FP64;
  cfg->D = 2.0;
  cfg->sigma0 = 0.2;
  cfg->eta = 0.0;
  cfg->cfl_safety = 0.9;
  cfg->wall_mode = DG_WALL_REMOVED;
  cfg->boundary = DG_BC_ABSORBING;
  cfg->power_iters = 200;
  cfg->device = -1;
  cfg->rounding = DG_ROUND_STOCHASTIC;
  cfg->element = DG_ELEMENT_SQUARE;
}

const char *dg_strerror(int code) {
  switch (code) {
    case DG_OK: return "ok";
    case DG_EINVAL: return "invalid argument";
    case DG_ENOMEM: return "out of memory";
    case DG_ECUDA: return "CUDA error";
    case DG_EUNSTABLE: return "unstable time step";
    case DG_ENONFINITE: return "non-finite values";
    case DG_ETIMEOUT: return "device wait timed out";
    case DG_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

const char *dg_last_error(const dg_ctx *ctx) { return ctx ? ctx->c.last_error.c_str() : ""; }

int dg_create(const dg_config *cfg, dg_ctx **out) {
  if (!out) return DG_EINVAL;
  *out = nullptr;
  if (!cfg) return DG_EINVAL;
  std::string why;
  if (check_config(cfg, why) != DG_OK) return DG_EINVAL;
  dg_ctx *ctx = new (std::nothrow) dg_ctx();
  if (!ctx) return DG_ENOMEM;
  Ctx &c = ctx->c;
  c.cfg = *cfg;
  if (c.cfg.power_iters == 0) c.cfg.power_iters = 200;
  int dev = cfg->device;
  cudaError_t e;
  if (dev < 0) {
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) { delete ctx; return DG_ECUDA; }
  }
  if ((e = cudaSetDevice(dev)) != cudaSuccess) { delete ctx; return DG_ECUDA; }
  c.device = dev;
  if ((e = cudaStreamCreateWithFlags(&c.own_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    delete ctx;
    return DG_ECUDA;
  }
  c.stream = c.own_stream;
  if (!gll_tables(c.cfg.p, &c.gll) || (c.triangles() && !tri_tables(c.cfg.p, &c.tri))) {
    cudaStreamDestroy(c.own_stream);
    delete ctx;
    return DG_EINVAL;
  }
  void *flags = nullptr;
  if (dev_alloc(&flags, 32) != cudaSuccess || cudaMemset(flags, 0, 32) != cudaSuccess) {
    cudaFree(flags);
    cudaStreamDestroy(c.own_stream);
    delete ctx;
    return DG_ENOMEM;
  }
  c.d_err = static_cast<int *>(flags);
  c.d_tma = reinterpret_cast<unsigned long long *>(static_cast<char *>(flags) + 8);
  c.d_grid = reinterpret_cast<unsigned *>(static_cast<char *>(flags) + 16);
  *out = ctx;
  return DG_OK;
}

void dg_destroy(dg_ctx *ctx) {
  if (!ctx) return;
  Ctx &c = ctx->c;
  cudaSetDevice(c.device);
  if (c.stream) cudaStreamSynchronize(c.stream);
  free_state(c);
  free_geometry(c.geo);
  cudaFree(c.d_err);
  if (c.own_stream) cudaStreamDestroy(c.own_stream);
  delete ctx;
}

int dg_set_stream(dg_ctx *ctx, void *stream) {
  if (!ctx) return DG_EINVAL;
  Ctx &c = ctx->c;
  c.stream = stream ? (cudaStream_t)stream : c.own_stream;
  drop_graph(c);
  return DG_OK;
}

int dg_set_geometry_mask(dg_ctx *ctx, const uint8_t *active, int nx, int ny, double h,
                         double x0, double y0) {
  if (!ctx) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (!active || nx < 1 || ny < 1 || !(h > 0.0) || !std::isfinite(h) || !std::isfinite(x0) ||
      !std::isfinite(y0))
    return fail(ctx, DG_EINVAL, "bad mask geometry arguments");
  if ((long long)nx * ny > (1ll << 31) - 1) return fail(ctx, DG_EINVAL, "domain too large");
  CK(cudaSetDevice(c.device), "set device");
  PartSpec q;
  q.nx = nx; q.ny = ny; q.h = h; q.x0 = x0; q.y0 = y0; q.host_mask = active;
  try {
    return set_parts(ctx, {q});
  } catch (const std::bad_alloc &) {
    return fail(ctx, DG_ENOMEM, "host allocation");
  }
}

int dg_set_geometry_disks(dg_ctx *ctx, const double *cx, const double *cy, const double *r,
                          int ndisks, double L, int n_cell, int tiles) {
  if (!ctx) return DG_EINVAL;
  Ctx &c = ctx->c;
  std::string why;
  if (!check_disk_args(cx, cy, r, ndisks, L, n_cell, tiles, why)) return fail(ctx, DG_EINVAL, why);
  CK(cudaSetDevice(c.device), "set device");
  try {
    return set_parts(ctx, {disk_part(cx, cy, r, ndisks, L, n_cell, tiles)});
  } catch (const std::bad_alloc &) {
    return fail(ctx, DG_ENOMEM, "host allocation");
  }
}

int dg_set_geometry_batch(dg_ctx *ctx, int G, const int *ndisks, const double *cx,
                          const double *cy, const double *r, const double *L,
                          const int *n_cell, const int *tiles) {
  if (!ctx) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (G < 1 || !ndisks || !L || !n_cell || !tiles) return fail(ctx, DG_EINVAL, "bad batch arguments");
  CK(cudaSetDevice(c.device), "set device");
  try {
    std::vector<PartSpec> parts;
    long long off = 0;
    for (int g = 0; g < G; ++g) {
      std::string why;
      const int nd = ndisks[g];
      if (nd < 0) return fail(ctx, DG_EINVAL, "bad disk count of geometry " + std::to_string(g));
      const double *gx = cx ? cx + off : nullptr, *gy = cy ? cy + off : nullptr, *gr = r ? r + off : nullptr;
      if (!check_disk_args(gx, gy, gr, nd, L[g], n_cell[g], tiles[g], why))
        return fail(ctx, DG_EINVAL, "geometry " + std::to_string(g) + ": " + why);
      parts.push_back(disk_part(gx, gy, gr, nd, L[g], n_cell[g], tiles[g]));
      off += nd;
    }
    return set_parts(ctx, parts);
  } catch (const std::bad_alloc &) {
    return fail(ctx, DG_ENOMEM, "host allocation");
  }
}

int dg_rasterize_disks(const double *cx, const double *cy, const double *r, int ndisks,
                       double L, int npix, uint8_t *out) {
  if (!out || ndisks < 0 || (ndisks > 0 && (!cx || !cy || !r)) || !(L > 0.0) || !std::isfinite(L) ||
      npix < 1 || npix > 16384)
    return DG_EINVAL;
  const int nd = ndisks > 0 ? ndisks : 1;
  double *d = nullptr;
  uint8_t *m = nullptr;
  if (dev_alloc(&d, sizeof(double) * 3 * nd) != cudaSuccess) return DG_ENOMEM;
  if (dev_alloc(&m, (size_t)npix * npix) != cudaSuccess) {
    cudaFree(d);
    return DG_ENOMEM;
  }
  cudaError_t e = cudaSuccess;
  if (ndisks > 0) {
    e = cudaMemcpy(d, cx, 8 * (size_t)ndisks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + nd, cy, 8 * (size_t)ndisks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + 2 * nd, r, 8 * (size_t)ndisks, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = build_mask_disks(d, d + nd, d + 2 * nd, ndisks, L, npix, 1, m, 0);
  std::vector<uint8_t> h((size_t)npix * npix);
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), m, h.size(), cudaMemcpyDeviceToHost);
  cudaFree(d);
  cudaFree(m);
  if (e != cudaSuccess) return DG_ECUDA;
  for (size_t k = 0; k < h.size(); ++k) out[k] = h[k] ? 0 : 1;
  return DG_OK;
}

int dg_basis_tables(int p, int precision, double *xi, double *w, double *D, double *D2) {
  if (precision != DG_FP32 && precision != DG_FP64) return DG_EINVAL;
  Gll g;
  if (!gll_tables(p, &g)) return DG_EINVAL;
  const int n = p + 1;
  for (int i = 0; i < n; ++i) {
    if (xi) xi[i] = g.xi[i];
    if (w) w[i] = g.w[i];
  }
  for (int k = 0; k < n * n; ++k) {
    if (D) D[k] = precision == DG_FP32 ? (double)g.Df[k] : g.D[k];
    if (D2) D2[k] = precision == DG_FP32 ? (double)g.D2f[k] : g.D2[k];
  }
  return DG_OK;
}

int dg_triangle_tables(int p, double *r, double *s, double *G, double *Lf, double *mono) {
  TriRef t;
  if (!tri_tables(p, &t)) return DG_EINVAL;
  const int N = t.N, NE = p + 1;
  for (int k = 0; k < N; ++k) {
    if (r) r[k] = t.r[k];
    if (s) s[k] = t.s[k];
  }
  for (int o = 0; o < 2; ++o) {
    for (int c = 0; c < 2; ++c)
      for (int k = 0; k < N * N; ++k)
        if (G) G[((size_t)o * 2 + c) * N * N + k] = t.G[o][c][k];
    for (int e = 0; e < 3; ++e)
      for (int k = 0; k < N * NE; ++k)
        if (Lf) Lf[((size_t)o * 3 + e) * N * NE + k] = t.Lf[o][e][k];
  }
  for (int q = 0; q < 6; ++q)
    for (int k = 0; k < N; ++k)
      if (mono) mono[q * N + k] = t.mono[q][k];
  return DG_OK;
}

int dg_get_mask(dg_ctx *ctx, uint8_t *active) {
  if (!ctx || !active) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (!c.have_geo) return fail(ctx, DG_ESTATE, "no geometry");
  std::memcpy(active, c.geo.h_mask.data(), (size_t)c.geo.nx * c.geo.ny);
  return DG_OK;
}

int dg_get_info(dg_ctx *ctx, dg_info *info) {
  if (!ctx || !info) return DG_EINVAL;
  const Ctx &c = ctx->c;
  std::memset(info, 0, sizeof(*info));
  info->p = c.cfg.p;
  info->n_nodes = c.np();
  info->precision = c.cfg.precision;
  info->nx = c.geo.nx;
  info->ny = c.geo.ny;
  info->n_active = c.geo.n_active;
  info->dof_per_source = c.geo.n_active * c.np();
  info->m = c.m;
  info->h = c.geo.h;
  info->x0 = c.geo.x0;
  info->y0 = c.geo.y0;
  info->t = c.t;
  info->steps = c.steps;
  info->state_bytes = c.state_bytes;
  info->halo_max = c.geo.halo_max;
  info->n_geometries = c.geo.G();
  info->n_elements_padded = c.geo.n_pad;
  return DG_OK;
}

int dg_set_sources(dg_ctx *ctx, const double *xy, int m) {
  if (!ctx) return DG_EINVAL;
  CK(cudaSetDevice(ctx->c.device), "set device");
  try {
    return set_sources_impl(ctx, xy, m);
  } catch (const std::bad_alloc &) {
    return fail(ctx, DG_ENOMEM, "host allocation");
  }
}

int dg_debug_copies(dg_ctx *ctx, int mode, unsigned long long *tensor_copies) {
  if (!ctx || mode < 0 || mode > 3) return DG_EINVAL;
  Ctx &c = ctx->c;
  CK(cudaSetDevice(c.device), "set device");
  unsigned long long n = 0;
  CK(cudaMemcpyAsync(&n, c.d_tma, sizeof(n), cudaMemcpyDeviceToHost, c.stream), "copy counter");
  CK(cudaMemsetAsync(c.d_tma, 0, sizeof(n), c.stream), "copy counter");
  CK(cudaStreamSynchronize(c.stream), "copy counter");
  if (tensor_copies) *tensor_copies = n;
  if (mode != c.copy_mode) {
    c.copy_mode = mode;
    drop_graph(c);  // captured launches carry the old settings
  }
  return DG_OK;
}

int dg_set_launch(dg_ctx *ctx, int blocks_per_sm) {
  if (!ctx || blocks_per_sm < kLaunchStep || blocks_per_sm > 64) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (blocks_per_sm != c.launch_req) {
    c.launch_req = blocks_per_sm;
    c.tuned_blocks = -1;
    c.tuned_key[0] = c.tuned_key[1] = -1;
  }
  return DG_OK;
}

int dg_set_contraction(dg_ctx *ctx, int mode) {
  if (!ctx || mode < -1 || mode > 1) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (mode != c.contraction_req) {
    c.contraction_req = mode;
    c.tuned_blocks = -1;
    c.tuned_key[0] = c.tuned_key[1] = -1;
  }
  return DG_OK;
}

int dg_set_triangle_fusion(dg_ctx *ctx, int fused) {
  if (!ctx || fused < 0 || fused > 1) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (fused != c.tri_fused) {
    c.tri_fused = fused;
    drop_graph(c);  // captured launches carry the old kernels
  }
  return DG_OK;
}

int dg_get_triangle_fusion(dg_ctx *ctx, int *fused) {
  if (!ctx || !fused) return DG_EINVAL;
  const Ctx &c = ctx->c;
  *fused = (c.tri_fused && c.triangles() && c.cfg.precision == DG_FP32 &&
            (c.cfg.p == 2 || c.cfg.p == 3))
               ? 1
               : 0;
  return DG_OK;
}

int dg_get_contraction(dg_ctx *ctx, int *mode) {
  if (!ctx || !mode) return DG_EINVAL;
  *mode = ctx->c.contraction_tc;
  return DG_OK;
}

int dg_get_launch(dg_ctx *ctx, int *blocks_per_sm) {
  if (!ctx || !blocks_per_sm) return DG_EINVAL;
  *blocks_per_sm = ctx->c.launch_blocks;
  return DG_OK;
}

int dg_debug_fail_alloc(int n) {
  if (n < -1) return DG_EINVAL;
  g_fail_alloc.store(n);
  return DG_OK;
}

int dg_set_growing_window(dg_ctx *ctx, double r_factor) {
  if (!ctx) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (!(r_factor >= 0.0) || !std::isfinite(r_factor))
    return fail(ctx, DG_EINVAL, "r_factor must be finite and >= 0");
  c.gw_r = r_factor;
  return DG_OK;
}

int dg_query_dt(dg_ctx *ctx, double *dt_max, double *rho) {
  if (!ctx) return DG_EINVAL;
  CK(cudaSetDevice(ctx->c.device), "set device");
  const int r = ensure_rho(ctx);
  if (r != DG_OK) return r;
  if (dt_max) *dt_max = ctx->c.dt_max;
  if (rho) *rho = ctx->c.rho;
  return DG_OK;
}

int dg_step(dg_ctx *ctx, int nsteps, double dt) {
  if (!ctx) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (c.m < 1) return fail(ctx, DG_ESTATE, "dg_step before dg_set_sources");
  if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, DG_EINVAL, "need nsteps >= 0 and dt > 0");
  CK(cudaSetDevice(c.device), "set device");
  const int r = run_steps(ctx, nsteps, dt, c.t);
  if (r == DG_OK) c.t += nsteps * dt;
  return r;
}

int dg_propagate_to(dg_ctx *ctx, double Delta) {
  if (!ctx) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (c.m < 1) return fail(ctx, DG_ESTATE, "dg_propagate_to before dg_set_sources");
  if (!std::isfinite(Delta) || Delta < c.t) return fail(ctx, DG_EINVAL, "Delta must be >= the current time");
  CK(cudaSetDevice(c.device), "set device");
  int r = ensure_rho(ctx);
  if (r != DG_OK) return r;
  if (Delta == c.t) return DG_OK;
  const double span = Delta - c.t;
  const double q = span / c.dt_max;
  long long N = (long long)std::ceil(q - 1e-12);
  if (N < 1) N = 1;
  if (N > (1ll << 40)) return fail(ctx, DG_EINVAL, "too many steps");
  const double dt = span / (double)N;
  long long done = 0;
  while (done < N) {
    const int chunk = (int)std::min<long long>(kCheckChunk, N - done);
    r = run_steps(ctx, chunk, dt, c.t + (double)done * dt);
    if (r != DG_OK) return r;
    done += chunk;
    r = check_growth(ctx);
    if (r != DG_OK) return r;
  }
  c.t = Delta;
  return DG_OK;
}

int dg_moments(dg_ctx *ctx, double *out) {
  if (!ctx || !out) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (c.m < 1) return fail(ctx, DG_ESTATE, "no sources");
  CK(cudaSetDevice(c.device), "set device");
  int r = compute_moments(ctx, c.d_mom);
  if (r != DG_OK) return r;
  const int nd = c.m * c.geo.G();
  std::vector<double> tmp((size_t)nd * kMomFields);
  CK(cudaMemcpyAsync(tmp.data(), c.d_mom, tmp.size() * 8, cudaMemcpyDeviceToHost, c.stream), "moment copy");
  CK(cudaStreamSynchronize(c.stream), "moments");
  if (const int e = take_device_error(ctx); e != DG_OK) return e;
  for (int s = 0; s < nd; ++s)
    for (int f = 0; f < 6; ++f) out[(size_t)s * 6 + f] = tmp[(size_t)s * kMomFields + f];
  return DG_OK;
}

int dg_covariance_batch(dg_ctx *ctx, double *sigma3, double *mu2, double *mass) {
  if (!ctx || !sigma3 || !mu2) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (c.m < 1) return fail(ctx, DG_ESTATE, "no sources");
  CK(cudaSetDevice(c.device), "set device");
  int r = compute_moments(ctx, c.d_mom);
  if (r != DG_OK) return r;
  const int G = c.geo.G();
  CK(launch_covariance(c.d_mom, c.d_mom0, c.m, G, c.d_out, c.stream), "covariance");
  std::vector<double> out((size_t)kCovOut * G);
  CK(cudaMemcpyAsync(out.data(), c.d_out, sizeof(double) * out.size(), cudaMemcpyDeviceToHost, c.stream),
     "covariance copy");
  if (mass)
    CK(cudaMemcpy2DAsync(mass, sizeof(double), c.d_mom, sizeof(double) * kMomFields, sizeof(double),
                         (size_t)c.m * G, cudaMemcpyDeviceToHost, c.stream), "mass copy");
  CK(cudaStreamSynchronize(c.stream), "covariance");
  if (const int e = take_device_error(ctx); e != DG_OK) return e;
  for (int g = 0; g < G; ++g) {
    const double *o = &out[(size_t)kCovOut * g];
    sigma3[3 * g] = o[0]; sigma3[3 * g + 1] = o[1]; sigma3[3 * g + 2] = o[2];
    mu2[2 * g] = o[3]; mu2[2 * g + 1] = o[4];
  }
  return DG_OK;
}

int dg_ls_residual(dg_ctx *ctx, double *out) {
  if (!ctx || !out) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (c.m < 1) return fail(ctx, DG_ESTATE, "no sources");
  if (c.triangles()) return fail(ctx, DG_EINVAL, "the least-squares residual is defined on the square elements");
  CK(cudaSetDevice(c.device), "set device");
  int r = compute_moments(ctx, c.d_mom);
  if (r != DG_OK) return r;
  const int G = c.geo.G();
  CK(launch_covariance(c.d_mom, c.d_mom0, c.m, G, c.d_out, c.stream), "covariance");
  double *d_res = nullptr;
  CK(dev_alloc(&d_res, sizeof(double) * kMomFields * (size_t)c.m * G), "residual buffer");
  double *d_ls = c.d_out + (size_t)kCovOut * G;  // G slots after the covariance outputs
  cudaError_t e = launch_ls_residual(c, state_array(c, 0), c.d_out, c.d_part, d_res, d_ls, c.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_ls, sizeof(double) * G, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  cudaFree(d_res);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "least-squares residual");
  return DG_OK;
}

int dg_covariance(dg_ctx *ctx, double *sigma3, double *mu2, double *mass) {
  if (!ctx || !sigma3 || !mu2) return DG_EINVAL;
  if (ctx->c.geo.G() > 1) return fail(ctx, DG_EINVAL, "several geometries: use dg_covariance_batch");
  return dg_covariance_batch(ctx, sigma3, mu2, mass);
}

int dg_mixture_covariance(dg_ctx *ctx, const double *mom, const double *mom0, int m,
                          double *sigma3, double *mu2) {
  if (!ctx || !mom || !mom0 || !sigma3 || !mu2 || m < 1) return DG_EINVAL;
  Ctx &c = ctx->c;
  CK(cudaSetDevice(c.device), "set device");
  std::vector<double> h(2 * (size_t)m * kMomFields, 0.0);
  for (int s = 0; s < m; ++s)
    for (int f = 0; f < 6; ++f) {
      h[(size_t)s * kMomFields + f] = mom[(size_t)s * 6 + f];
      h[((size_t)m + s) * kMomFields + f] = mom0[(size_t)s * 6 + f];
    }
  double *d = nullptr;
  CK(dev_alloc(&d, sizeof(double) * (h.size() + kCovOut)), "moment buffer");
  double out[5];
  cudaError_t e = cudaMemcpyAsync(d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, c.stream);
  double *dout = d + h.size();
  if (e == cudaSuccess) e = launch_covariance(d, d + (size_t)m * kMomFields, m, 1, dout, c.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(out), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mixture covariance");
  sigma3[0] = out[0]; sigma3[1] = out[1]; sigma3[2] = out[2];
  mu2[0] = out[3]; mu2[1] = out[4];
  return DG_OK;
}

int dg_apply_operator(dg_ctx *ctx) {
  if (!ctx) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (c.m < 1) return fail(ctx, DG_ESTATE, "no sources");
  CK(cudaSetDevice(c.device), "set device");
  const double kc = c.cfg.D;
  const double pen = c.cfg.eta * (c.cfg.p + 1.0) * (c.cfg.p + 1.0) * 0.5;
  const int wallA = c.cfg.wall_mode == DG_WALL_PAPER;
  void *U0 = state_array(c, 0), *U1 = state_array(c, 1);
  c.gw_synced = false;
  cudaError_t e;
  if (c.triangles()) {
    if (c.cfg.precision == DG_FP64) {
      StageCoef<double> sc{0.0, 0.0, kc, pen, wallA};
      e = launch_tri_stage_f64(c.cfg.p, (const double *)U0, nullptr, (double *)U1, (double *)c.d_q,
                               c.geo, c.geo.n_pad, c.m, c.tri, sc, c.stream);
    } else {
      StageCoef<float> sc{0.0f, 0.0f, (float)kc, (float)pen, wallA};
      e = launch_tri_stage_f32(c.cfg.p, (const float *)U0, nullptr, (float *)U1, (float *)c.d_q,
                               c.geo, c.geo.n_pad, c.m, c.tri, sc, c.stream, ChunkSel{},
                               c.tri_fused != 0);
    }
  } else if (c.cfg.precision == DG_FP64) {
    StageCoef<double> sc{0.0, 0.0, kc, pen, wallA};
    e = launch_stage_f64(c.cfg.p, (const double *)U0, nullptr, (double *)U1, c.geo, c.geo.n_pad, c.m,
                         c.gll, sc, c.stream);
  } else {
    StageCoef<float> sc{0.0f, 0.0f, (float)kc, (float)pen, wallA};
    e = launch_stage_f32(c.cfg.p, (const float *)U0, nullptr, (float *)U1, c.geo, c.geo.n_pad, c.m,
                         c.gll, sc, c.stream);
  }
  CK(e, "operator launch");
  CK(cudaMemcpyAsync(U0, U1, (size_t)c.m * c.field_elems() * c.esize(), cudaMemcpyDeviceToDevice, c.stream), "copy");
  CK(cudaStreamSynchronize(c.stream), "operator");
  return DG_OK;
}

int dg_get_nodes(dg_ctx *ctx, double *host) {
  if (!ctx || !host) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (c.m < 1) return fail(ctx, DG_ESTATE, "no sources");
  if (c.geo.G() > 1) return fail(ctx, DG_EINVAL, "several geometries: use dg_get_elements_batch");
  CK(cudaSetDevice(c.device), "set device");
  const size_t nd = (size_t)c.m * c.geo.nx * c.geo.ny * c.np();
  double *d = nullptr;
  CK(dev_alloc(&d, nd * 8), "dense buffer");
  cudaError_t e = cudaMemsetAsync(d, 0, nd * 8, c.stream);
  if (e == cudaSuccess) e = launch_nodes_to_dense(c, state_array(c, 0), d, c.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, d, nd * 8, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "get nodes");
  return DG_OK;
}

int dg_set_nodes(dg_ctx *ctx, const double *host) {
  if (!ctx || !host) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (c.m < 1) return fail(ctx, DG_ESTATE, "no sources");
  if (c.geo.G() > 1) return fail(ctx, DG_EINVAL, "several geometries: not supported");
  CK(cudaSetDevice(c.device), "set device");
  c.gw_synced = false;
  const size_t nd = (size_t)c.m * c.geo.nx * c.geo.ny * c.np();
  double *d = nullptr;
  CK(dev_alloc(&d, nd * 8), "dense buffer");
  cudaError_t e = cudaMemcpyAsync(d, host, nd * 8, cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = launch_dense_to_nodes(c, d, state_array(c, 0), c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "set nodes");
  return DG_OK;
}

int dg_get_elements_batch(dg_ctx *ctx, const int *idx, int k, double *out) {
  if (!ctx || k < 0 || (k > 0 && (!idx || !out))) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (c.m < 1) return fail(ctx, DG_ESTATE, "no sources");
  CK(cudaSetDevice(c.device), "set device");
  const int np = c.np();
  std::vector<char> tmp((size_t)np * c.esize());
  for (int q = 0; q < k; ++q) {
    const int g = idx[4 * q], s = idx[4 * q + 1], ex = idx[4 * q + 2], ey = idx[4 * q + 3];
    if (g < 0 || g >= c.geo.G()) return fail(ctx, DG_EINVAL, "geometry index out of range");
    const GeoPart &p = c.geo.parts[g];
    if (s < 0 || s >= c.m || ex < 0 || ex >= p.nx || ey < 0 || ey >= p.ny)
      return fail(ctx, DG_EINVAL, "element index out of range");
    int a = -1;
    CK(cudaMemcpyAsync(&a, c.geo.d_cidx + p.dense_off + (size_t)ey * p.nx + ex, sizeof(int),
                       cudaMemcpyDeviceToHost, c.stream), "index copy");
    CK(cudaStreamSynchronize(c.stream), "index copy");
    double *o = out + (size_t)q * np;
    if (a < 0) {
      for (int t = 0; t < np; ++t) o[t] = 0.0;
      continue;
    }
    const char *src = (const char *)state_array(c, 0) + ((size_t)s * c.field_elems() + (size_t)a * np) * c.esize();
    CK(cudaMemcpyAsync(tmp.data(), src, tmp.size(), cudaMemcpyDeviceToHost, c.stream), "element copy");
    CK(cudaStreamSynchronize(c.stream), "element copy");
    for (int t = 0; t < np; ++t)
      o[t] = c.cfg.precision == DG_FP64 ? ((const double *)tmp.data())[t] : (double)((const float *)tmp.data())[t];
  }
  return DG_OK;
}

int dg_get_elements(dg_ctx *ctx, const int *idx, int k, double *out) {
  if (!ctx || k < 0 || (k > 0 && (!idx || !out))) return DG_EINVAL;
  std::vector<int> q4((size_t)4 * k);
  for (int q = 0; q < k; ++q) {
    q4[4 * q] = 0;
    q4[4 * q + 1] = idx[3 * q];
    q4[4 * q + 2] = idx[3 * q + 1];
    q4[4 * q + 3] = idx[3 * q + 2];
  }
  return dg_get_elements_batch(ctx, q4.data(), k, out);
}

// Snapshot layout: 8 x uint64 header {magic, precision, p, m, padded element
// count, steps, bits of t, payload bytes}, G x m x 2 start points, G x m x 7
// start moments, then m x n_pad x Np values of U (state precision,
// concatenated element order).
int dg_state_size(dg_ctx *ctx, size_t *bytes) {
  if (!ctx || !bytes) return DG_EINVAL;
  const Ctx &c = ctx->c;
  if (c.m < 1) return fail(ctx, DG_ESTATE, "no sources");
  const size_t nd = (size_t)c.m * c.geo.G();
  *bytes = 64 + nd * 16 + nd * kMomFields * 8 + (size_t)c.m * c.field_elems() * c.esize();
  return DG_OK;
}

int dg_get_state(dg_ctx *ctx, void *host, size_t bytes) {
  size_t need = 0;
  int r = dg_state_size(ctx, &need);
  if (r != DG_OK) return r;
  if (!host || bytes < need) return fail(ctx, DG_EINVAL, "snapshot buffer too small");
  Ctx &c = ctx->c;
  CK(cudaSetDevice(c.device), "set device");
  const size_t nd = (size_t)c.m * c.geo.G();
  uint64_t hdr[8];
  double tt = c.t;
  std::memcpy(&hdr[6], &tt, 8);
  hdr[0] = kStateMagic; hdr[1] = (uint64_t)c.cfg.precision; hdr[2] = (uint64_t)c.cfg.p;
  hdr[3] = (uint64_t)c.m; hdr[4] = (uint64_t)c.geo.n_pad; hdr[5] = (uint64_t)c.steps;
  hdr[7] = need;
  char *p = (char *)host;
  std::memcpy(p, hdr, 64);
  std::memcpy(p + 64, c.src.data(), nd * 16);
  char *pm = p + 64 + nd * 16;
  CK(cudaMemcpyAsync(pm, c.d_mom0, nd * kMomFields * 8, cudaMemcpyDeviceToHost, c.stream), "snapshot");
  char *pu = pm + nd * kMomFields * 8;
  CK(cudaMemcpyAsync(pu, state_array(c, 0), (size_t)c.m * c.field_elems() * c.esize(), cudaMemcpyDeviceToHost,
                     c.stream), "snapshot");
  CK(cudaStreamSynchronize(c.stream), "snapshot");
  return DG_OK;
}

int dg_set_state(dg_ctx *ctx, const void *host, size_t bytes) {
  if (!ctx || !host || bytes < 64) return DG_EINVAL;
  Ctx &c = ctx->c;
  if (!c.have_geo) return fail(ctx, DG_ESTATE, "dg_set_state before a geometry");
  uint64_t hdr[8];
  std::memcpy(hdr, host, 64);
  if (hdr[0] != kStateMagic) return fail(ctx, DG_EINVAL, "not a snapshot");
  if (hdr[1] != (uint64_t)c.cfg.precision || hdr[2] != (uint64_t)c.cfg.p || hdr[4] != (uint64_t)c.geo.n_pad)
    return fail(ctx, DG_EINVAL, "snapshot does not match the context (precision, order or mesh)");
  if (hdr[3] < 1 || hdr[3] > 65535) return fail(ctx, DG_EINVAL, "snapshot with a bad number of densities");
  const int m = (int)hdr[3];
  const size_t nd = (size_t)m * c.geo.G();
  // the size the header's m implies for this context must be the stated one
  // and fit the caller's buffer: a corrupt header must not make the copies
  // below read past it
  const size_t need = 64 + nd * 16 + nd * kMomFields * 8 + (size_t)m * c.field_elems() * c.esize();
  if (hdr[7] != need) return fail(ctx, DG_EINVAL, "snapshot does not match the context (size)");
  if (need > bytes) return fail(ctx, DG_EINVAL, "truncated snapshot");
  double t_snap = 0.0;
  std::memcpy(&t_snap, &hdr[6], 8);
  if (!std::isfinite(t_snap) || t_snap < 0.0 || (long long)hdr[5] < 0)
    return fail(ctx, DG_EINVAL, "snapshot with a bad time or step count");
  const char *p = (const char *)host;
  std::vector<double> xy(2 * nd);
  std::memcpy(xy.data(), p + 64, nd * 16);
  int r = dg_set_sources(ctx, xy.data(), m);
  if (r != DG_OK) return r;
  const char *pm = p + 64 + nd * 16;
  CK(cudaMemcpyAsync(c.d_mom0, pm, nd * kMomFields * 8, cudaMemcpyHostToDevice, c.stream), "restore");
  const char *pu = pm + nd * kMomFields * 8;
  CK(cudaMemcpyAsync(state_array(c, 0), pu, (size_t)m * c.field_elems() * c.esize(), cudaMemcpyHostToDevice,
                     c.stream), "restore");
  CK(cudaStreamSynchronize(c.stream), "restore");
  std::memcpy(&c.t, &hdr[6], 8);
  c.steps = (long long)hdr[5];
  return DG_OK;
}

int dg_state_bytes(dg_ctx *ctx, int m, size_t *bytes) {
  if (!ctx || !bytes || m < 1) return DG_EINVAL;
  if (!ctx->c.have_geo) return fail(ctx, DG_ESTATE, "no geometry");
  *bytes = state_bytes_for(ctx->c, m);
  return DG_OK;
}

int dg_bind_state(dg_ctx *ctx, void *device_ptr, size_t bytes) {
  if (!ctx) return DG_EINVAL;
  if (device_ptr && ((uintptr_t)device_ptr % 256) != 0) return fail(ctx, DG_EINVAL, "state buffer must be 256-byte aligned");
  Ctx &c = ctx->c;
  CK(cudaSetDevice(c.device), "set device");
  free_state(c);
  c.bound_ptr = device_ptr;
  c.bound_bytes = device_ptr ? bytes : 0;
  return DG_OK;
}

}  // extern "C"
