// dg_internal.h -- internal types of the dgsigma library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dgsigma.h"

namespace dg {

// NVTX range in the "dgsigma" domain for the lifetime of the object (a no-op
// unless a profiler is attached): geometry upload, start densities, stepping,
// moments.
inline nvtxDomainHandle_t trace_domain() {
  static const nvtxDomainHandle_t d = nvtxDomainCreateA("dgsigma");
  return d;
}
struct TraceRange {
  explicit TraceRange(const char *what) {
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = what;
    nvtxDomainRangePushEx(trace_domain(), &a);
  }
  ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

// Every device allocation of the library goes through dev_alloc.  A test can
// make the n-th call from now fail as if the device were out of memory
// (dg_debug_fail_alloc), to exercise the error paths without a GPU fault.
cudaError_t dev_alloc(void **p, size_t bytes);
template <typename X>
cudaError_t dev_alloc(X **p, size_t bytes) {
  return dev_alloc(reinterpret_cast<void **>(p), bytes);
}

constexpr int kMaxP = 5;
constexpr int kMaxN = kMaxP + 1;
constexpr int kBlock = 128;         // threads per block of the element kernels = elements per chunk
constexpr int kTile = 16;           // element ordering: 16 x 16 tiles, row-major inside
constexpr int kMomBlocks = 608;     // fixed grid of the moment reduction (4 x 152 SMs)
constexpr int kMomFields = 7;       // M0, Mx, My, Mxx, Mxy, Myy, |u| mass
constexpr int kHaloCap = 4 * kBlock;  // halo entries a chunk can have (4 faces x kBlock)
// Blocks of kBlock threads per SM that fit the SM's 64K registers at `regs`
// registers per thread: the __launch_bounds__ minimum that holds a kernel to
// that register budget.
constexpr int blocks_for_regs(int regs) { return 65536 / (regs * kBlock); }
constexpr int kCovOut = 8;          // per geometry: Sigma(t)-Sigma(0) [3], mu [2], Sigma_mix(t) [3]

// Face codes in the neighbour table (>= 0: neighbour element index).
constexpr int kWall = -1;
constexpr int kEdge = -2;

// GLL tables of order p, computed on the host in FP64.
struct Gll {
  int p = 0;
  double xi[kMaxN], w[kMaxN];
  double D[kMaxN * kMaxN];   // D[a*n + i] = l_i'(xi_a)
  double D2[kMaxN * kMaxN];  // (D D)[a*n + i]
  // FP32 copies of D and D D whose rows sum to exactly zero (a constant has
  // exactly zero derivative, so the volume term adds no mass) and that keep
  // the centro-(anti)symmetry of the FP64 tables; each entry within a few
  // FP32 ulps of the FP64 value
  float Df[kMaxN * kMaxN], D2f[kMaxN * kMaxN];
};
bool gll_tables(int p, Gll *g);

// Triangles of the pixel split (Sec. 3.3): each pixel of side h is cut by its
// lower-left to upper-right diagonal into A (vertices (x0,y0), (x1,y0),
// (x1,y1)) and B ((x0,y0), (x1,y1), (x0,y1)), both affine images of the
// reference triangle (0,0), (1,0), (0,1) with Jacobian determinant h^2.  The
// basis is the Lagrange P_p basis on the equispaced nodes (i/p, j/p), node
// index k running over j = 0..p, then i = 0..p - j; edges e0 (0,0)->(1,0),
// e1 (1,0)->(0,1), e2 (0,1)->(0,0).  A pixel's four faces are A e1 (east),
// B e2 (west), B e1 (north) and A e0 (south); A e2 and B e0 are the diagonal.
constexpr int kTriMaxP = 3;
constexpr int kTriN = (kTriMaxP + 1) * (kTriMaxP + 2) / 2;
struct TriRef {
  int p = 0, N = 0;
  double r[kTriN], s[kTriN];                  // reference nodes
  // q = (1/h) [G_t u + sum_e n_te Lf_te uhat_e] on triangle t (0 = A, 1 = B):
  // G_t,x = -M^-1 (rx Sr^T + sx Ss^T), (rx, ry, sx, sy) the inverse Jacobian
  // times h; Lf_te = (|e|/h) M^-1 E_e, E_e the edge mass matrix placed on the
  // edge's nodes.  The divergence uses the same matrices.
  double G[2][2][kTriN * kTriN];
  double Lf[2][3][kTriN * (kTriMaxP + 1)];
  double nrm[2][3][2];                         // outward unit normals
  // int over the reference triangle of r^a s^b N_j for
  // (a, b) = (0,0), (1,0), (0,1), (2,0), (1,1), (0,2)
  double mono[6][kTriN];
};
bool tri_tables(int p, TriRef *t);
double rk3_real_axis_limit();

// Operator scalars of one stage launch: out = u0 + beta (u - u0) + gamma s_g R
// (or beta u + gamma s_g R without u0), where L u = k s_g R and s_g = 1/J^2
// of the element's geometry (J = h/2): gamma = beta dt k.
template <typename T>
struct StageCoef {
  T alpha, beta, gamma;  // alpha = 1 - beta, kept for reference only
  T pen;     // eta (p+1)^2 / 2
  int wallA; // paper wall mode
  int sround = 0;  // FP32: stochastic rounding of the stage result
};

template <typename T> struct Vec2;  // two lanes of T
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// Tables by value in the kernel parameter space (constant bank).  The paired
// forms of D2 feed the packed two-lane FP32 instructions of the volume term
// (two nodes per instruction; n = P + 1 even):
//   D2x[ip n + m] = (D2[2ip][m], D2[2ip+1][m]),  D2y[j n + m] = (D2[j][m], D2[j][m]).
template <typename T, int P>
struct StageTab {
  using T2 = typename Vec2<T>::type;
  T D[(P + 1) * (P + 1)];
  T D2[(P + 1) * (P + 1)];
  T Dout[2 * (P + 1)];  // outward derivative rows: D[p][:] (east, north), -D[0][:] (west, south)
  T inv_w;  // 1 / w_0 = 1 / w_p
  T2 D2x[((P + 1) / 2) * (P + 1)];
  T2 D2y[(P + 1) * (P + 1)];
};

// One geometry (domain) of a context.  A context holds G >= 1 of them; their
// mesh elements are concatenated, each geometry padded to a multiple of
// kBlock elements so that every block of kBlock consecutive elements (a
// "chunk") belongs to one geometry.
struct GeoPart {
  int nx = 0, ny = 0;
  double h = 0, x0 = 0, y0 = 0;
  long long n_active = 0;     // elements in the mesh
  long long off = 0;          // first element in the concatenated numbering
  long long dense_off = 0;    // offset of its [ny][nx] mask / index map
  int periodic = 0;
};

// Host description of a geometry to build: a mask, or disks in a periodic
// cell tiled into a window.
struct PartSpec {
  int nx = 0, ny = 0;
  double h = 0, x0 = 0, y0 = 0;
  const uint8_t *host_mask = nullptr;  // [ny][nx] or null
  const double *cx = nullptr, *cy = nullptr, *r = nullptr;
  int nd = 0;
  double L = 0;
  int n_cell = 0, tiles = 0;
};

struct Geometry {
  std::vector<GeoPart> parts;
  // geometry 0, for the single-geometry calls
  int nx = 0, ny = 0;
  double h = 0, x0 = 0, y0 = 0;
  long long n_active = 0;       // all geometries
  long long n_pad = 0;          // concatenated, padded element count = per-density stride
  uint8_t *d_mask = nullptr;    // dense masks, geometry after geometry
  int *d_cidx = nullptr;        // dense maps to the concatenated element index, or -1
  int4 *d_nb = nullptr;         // [n_pad] E, W, N, S (concatenated indices, kWall, kEdge)
  int2 *d_exy = nullptr;        // [n_pad] element coordinates inside its geometry
  int2 *d_chunk = nullptr;      // [n_pad / kBlock] {live elements, geometry}
  double4 *d_gpar = nullptr;    // [G] {x0, y0, h, 1/J^2}
  float *d_gscale_f = nullptr;  // [G] 1/J^2
  double *d_gscale_d = nullptr; // [G] 1/J^2
  int2 *d_grange = nullptr;     // [G] {first element, elements in the mesh}
  std::vector<uint8_t> h_mask;  // host copy of d_mask
  // Per chunk: face neighbours outside the chunk are halo entries
  // {element, its face toward the chunk}.  d_loc gives, per element and face,
  // the chunk-local index (0..kBlock-1), kBlock + halo slot, kWall or kEdge.
  int4 *d_loc = nullptr;        // [n_pad]
  int2 *d_halo = nullptr;       // [n_chunks][kHaloCap]
  int *d_halo_cnt = nullptr;    // [n_chunks + 1]
  int halo_max = 0;             // largest halo of any chunk
  // Pixel triangles, one launch per stage: per chunk and halo entry (stride
  // halo_max) {pixel k, its face toward the chunk, the chunk element across
  // that face, k's neighbour across the other face of the same triangle
  // (index, kWall or kEdge)}; entries past the chunk's count hold pixel -1.
  int4 *d_htri = nullptr;       // [n_chunks][halo_max], built for triangle contexts
  int G() const { return (int)parts.size(); }
  long long n_chunks() const { return n_pad / kBlock; }
};

struct Ctx {
  dg_config cfg{};
  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  std::string last_error;
  Gll gll;
  TriRef tri;                     // element == DG_ELEMENT_TRIANGLE
  Geometry geo;
  bool have_geo = false;

  // time-step bound
  bool have_rho = false;
  double rho = 0, dt_max = 0;

  // sources and state
  int m = 0;
  double t = 0;
  long long steps = 0;
  std::vector<double> src;        // [m][2]
  double *d_src = nullptr;        // [G][m][2]
  float4 *d_srel = nullptr;       // [G][m] start points in element units (hi, lo pairs)
  void *d_state = nullptr;        // 3 arrays of m * n_pad * Np elements
  size_t state_bytes = 0;
  bool state_owned = true;
  void *bound_ptr = nullptr;
  size_t bound_bytes = 0;
  double *d_mom = nullptr;        // [m][7] current moments
  double *d_mom0 = nullptr;       // [m][7] start moments
  double *d_part = nullptr;       // [m][kMomBlocks][7] partial sums
  double *d_out = nullptr;        // [G][kCovOut] covariance results
  void *d_q = nullptr;            // triangles: q of one stage, [m][n_pad][4 N]
  // state arrays 0..2 as 2D tensors [m n_pad rows][np values] for the tensor
  // copies of the stage kernel (square elements whose rows are whole 16-byte
  // slots)
  CUtensorMap tmap[3];
  bool tmap_ok = false;
  int copy_mode = 0;              // 0 tensor copies where possible, 1 cp.async only,
                                  // 2 test hook: barriers that never complete,
                                  // 3 test hook: grid barriers that never complete
  // Launch shape of the FP32 stage kernel: launch_req -1 = tuned (the
  // candidates are timed before the first steps of a set of densities),
  // 0 = one block per chunk, k >= 1 = persistent with k blocks per SM.
  // launch_blocks is the shape in use; the tuned value is kept per
  // (densities, padded elements).
  int launch_req = -1;
  int launch_blocks = 0;
  int tuned_blocks = -1;
  // Element contractions of the FP32 p = 5 stage: contraction_req 0 = CUDA
  // cores (the default), 1 = tensor cores, -1 = tuned with the launch shape;
  // contraction_tc is the choice in use.
  int contraction_req = 0;
  int contraction_tc = 0;
  // Pixel triangles in FP32 at p = 2, 3: one launch per stage (1, the
  // default) or the q pass and the divergence pass (0).
  int tri_fused = 1;
  int tuned_tc = 0;
  long long tuned_key[2] = {-1, -1};
  int *d_err = nullptr;           // a bounded device wait gave up (and the copy counter)
  unsigned *d_grid = nullptr;     // arrival counter of the one-launch-per-step grid barriers
  unsigned long long *d_tma = nullptr;
  size_t part_elems = 0;

  // Growing window (off while gw_r <= 0): in each group of up to 64 steps an
  // element advances only if its centre lies within
  // R = gw_r sqrt(sigma0^2 + 2 D t_end) of its geometry's start-point box;
  // chunks with no such element are not launched.
  double gw_r = 0;
  bool gw_ready = false;          // tables below match the current sources
  bool gw_synced = false;         // arrays 1 and 2 equal array 0 (held chunks)
  double *d_gw_d2 = nullptr;      // [n_pad] squared centre-to-box distance (inf: padding)
  uint8_t *d_gw_adv = nullptr;    // [n_pad] 1 = advances in the current group
  int *d_gw_order = nullptr;      // [n_chunks] chunks by increasing nearest distance
  std::vector<double> gw_cmin;    // nearest squared distance of each chunk, same order
  double gw_dmax = 0;             // largest squared distance of a mesh element

  // graph of a chunk of steps
  cudaGraphExec_t graph = nullptr;
  double graph_dt = 0;
  int graph_steps = 0;
  cudaStream_t graph_stream = nullptr;

  bool triangles() const { return cfg.element == DG_ELEMENT_TRIANGLE; }
  // nodes per pixel element
  int np() const {
    return triangles() ? (cfg.p + 1) * (cfg.p + 2) : (cfg.p + 1) * (cfg.p + 1);
  }
  size_t esize() const { return cfg.precision == DG_FP64 ? 8 : 4; }
  size_t field_elems() const { return (size_t)geo.n_pad * np(); }  // one density slot
};

// ---- launchers (defined in the .cu files) ----
// Which chunks a stage launch covers.  Default: every chunk, every element
// advances.  list: the first count entries are the chunks to launch (the
// others are not touched); adv (per element, may be null): 0 holds the
// element's value (gamma = 0), 1 advances it.
struct ChunkSel {
  const int *list = nullptr;
  long long count = -1;
  const uint8_t *adv = nullptr;
};
// How a stage launch moves its chunks into shared memory.  Device side:
struct CopyArgs {
  int use_tma = 0;                         // tensor copies (else per-thread cp.async)
  int store_tma = 0;                       // tensor stores of full result chunks
  int extra_tx = 0;                        // test hook: bytes awaited beyond the copy
  int limit = 1 << 22;                     // polls of a barrier before giving up
  int *err = nullptr;                      // set to 1 when a wait gave up
  unsigned long long *counter = nullptr;   // chunk copies made by the tensor path
};
// Host side: the tensor maps of the input and u0 arrays and the settings above.
struct StageCopies {
  const CUtensorMap *map_u = nullptr, *map_u0 = nullptr, *map_out = nullptr;
  int use_tma = 0, extra_tx = 0, limit = 1 << 22;
  int *err = nullptr;
  unsigned long long *counter = nullptr;
  // launch shape: 0 one block per chunk, one thread per element (k_stage);
  // k >= 1 persistent (k_stage_pipe, FP32 p = 1, 3 with tensor copies) with
  // k blocks per SM
  int pipe_blocks = 0;
  // FP32 p = 5: element contractions on the tensor cores (k_stage_tc)
  int tensor_core = 0;
};
// Blocks per SM the persistent stage kernel of (precision, p) can keep
// resident with this geometry's shared memory; 0 if it has no such variant.
int stage_pipe_max_blocks(int precision, int p, const Geometry &geo);
// The FP32 stage at p = 5 with the element contractions on the tensor cores;
// cudaErrorNotSupported where it does not apply (other p, no tensor copies).
cudaError_t launch_stage_tc_f32(const float *u, const float *u0, float *out, const Geometry &geo,
                                long long stride, int m, const Gll &g,
                                const StageCoef<float> &c, cudaStream_t s, const ChunkSel &sel,
                                const StageCopies &cp);
int stage_tc_max_blocks(const Geometry &geo);
cudaError_t stage_tc_prepare(const Gll &g, cudaStream_t s);
// One SSP-RK3 step in one cooperative launch with bounded grid barriers
// between the stages (FP32, p = 1, 3, 5, tensor copies); c[k] the stage
// coefficients; grid_extra > 0 (test hook) makes every barrier wait for
// arrivals no block makes.  cudaErrorNotSupported where it does not apply.
cudaError_t launch_rk3_grid_f32(int p, float *U0, float *U1, float *U2, const Geometry &geo,
                                long long stride, int m, const Gll &g,
                                const StageCoef<float> (&c)[3], cudaStream_t s,
                                const ChunkSel &sel, const CUtensorMap *maps, int *err,
                                unsigned long long *counter, unsigned *grid_count,
                                int extra_tx, int limit, int grid_extra, int grid_limit);
constexpr int kLaunchStep = -2;  // one cooperative launch per RK step (DG_LAUNCH_STEP)
// One stage over all m densities: out = u0 + beta (u - u0) + gamma R(u).
cudaError_t launch_stage_f64(int p, const double *u, const double *u0, double *out,
                             const Geometry &geo, long long stride, int m,
                             const Gll &g, const StageCoef<double> &c, cudaStream_t s,
                             const ChunkSel &sel = ChunkSel{},
                             const StageCopies &cp = StageCopies{});
cudaError_t launch_stage_f32(int p, const float *u, const float *u0, float *out,
                             const Geometry &geo, long long stride, int m,
                             const Gll &g, const StageCoef<float> &c, cudaStream_t s,
                             const ChunkSel &sel = ChunkSel{},
                             const StageCopies &cp = StageCopies{});

// One stage on the pixel triangles: two passes through qbuf ([m][n_pad][4 N]),
// or with `fused` (FP32, p = 2, 3, a geometry built with its triangle halo
// table) one launch that keeps q in shared memory.
cudaError_t launch_tri_stage_f64(int p, const double *u, const double *u0, double *out,
                                 double *qbuf, const Geometry &geo, long long stride, int m,
                                 const TriRef &ref, const StageCoef<double> &c, cudaStream_t s,
                                 const ChunkSel &sel = ChunkSel{}, bool fused = false);
cudaError_t launch_tri_stage_f32(int p, const float *u, const float *u0, float *out,
                                 float *qbuf, const Geometry &geo, long long stride, int m,
                                 const TriRef &ref, const StageCoef<float> &c, cudaStream_t s,
                                 const ChunkSel &sel = ChunkSel{}, bool fused = false);

cudaError_t build_mask_disks(const double *d_cx, const double *d_cy, const double *d_r,
                             int nd, double L, int n_cell, int tiles, uint8_t *d_mask,
                             cudaStream_t s);
// Geometry construction: masks, compaction in tile order, neighbour and halo
// tables for every part; fills geo (allocates).  Returns a DG_* code.
int build_geometry(Geometry &geo, const std::vector<PartSpec> &parts, int periodic,
                   bool tri_halo, cudaStream_t s, std::string &err);
void free_geometry(Geometry &geo);

// Densities, moments, covariance.
cudaError_t launch_init_sources(const Ctx &c, void *u, cudaStream_t s);
cudaError_t launch_moments(const Ctx &c, const void *u, double *d_part, double *d_mom,
                           cudaStream_t s);
cudaError_t launch_covariance(const double *d_mom, const double *d_mom0, int m, int G,
                              double *d_out, cudaStream_t s);
int moment_blocks(int G);  // first-pass blocks per density of the moment reduction
// Least-squares residual of the Gaussian fit per geometry (needs d_mom and the
// covariance output d_cov of the same t); d_res is [G m][7] scratch.
cudaError_t launch_ls_residual(const Ctx &c, const void *u, const double *d_cov,
                               double *d_part, double *d_res, double *d_out, cudaStream_t s);
// Growing window: squared distance of every element centre to its
// geometry's box d_box [G][4] = {x_lo, x_hi, y_lo, y_hi} (FP64, rounded
// operation by operation), and the advance flags d2 <= r2.
cudaError_t launch_window_d2(const Ctx &c, const double *d_box, double *d2, cudaStream_t s);
cudaError_t launch_window_flags(const Ctx &c, const double *d2, double r2, uint8_t *adv,
                                cudaStream_t s);
cudaError_t launch_nodes_to_dense(const Ctx &c, const void *u, double *d_dense,
                                  cudaStream_t s);
cudaError_t launch_dense_to_nodes(const Ctx &c, const double *d_dense, void *u,
                                  cudaStream_t s);
// Power iteration helpers (FP64, one density).
cudaError_t launch_random_field(const Ctx &c, double *v, unsigned long long seed,
                                cudaStream_t s);
cudaError_t launch_wnorm2(const Ctx &c, const double *v, double *d_part, double *d_res,
                          cudaStream_t s);
cudaError_t launch_scale_by_rnorm(const Ctx &c, const double *in, const double *d_res,
                                  double *out, cudaStream_t s);

}  // namespace dg
