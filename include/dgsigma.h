/*
 * dgsigma.h -- C ABI of the GB300 (sm_103a) DG diffusion / covariance library.
 *
 * Method: Cervantes, Moreles, Pena, Ramirez-Manzanares, "A GPU implementation
 * of the Discontinuous Galerkin method for simulation of diffusion in brain
 * tissue" (arXiv 1907.06191).  Diffusion u_t = div(k grad u) in the
 * extracellular space around disk-shaped axons (Sec. 2.1, Eqs. 1-5),
 * discontinuous Galerkin in space (Sec. 3.1, Eqs. 6-8) with the central u-flux
 * and the harmonic-mean q-flux (Sec. 3.2), explicit Runge-Kutta in time
 * (SSP-RK3), then the covariance Sigma of the mixture of normalised densities
 * (Sec. 4.1).
 *
 * Discretisation fixed by this library where the paper is silent: square
 * elements on a uniform grid, tensor-product Gauss-Lobatto-Legendre (GLL)
 * nodal basis of order p with the nodes as quadrature points (diagonal mass),
 * SSP-RK3 (Shu-Osher form), moments by GLL nodal quadrature.
 *
 * Conventions for every call:
 *   - Return value: DG_OK (0) or a positive DG_E* code; dg_last_error() gives
 *     the message.  No call aborts, throws or exits.
 *   - Host pointers are read or written only during the call; the library
 *     copies inputs.  Outputs go to caller-owned host buffers of the stated
 *     size.  Device memory belongs to the context unless bound with
 *     dg_bind_state().
 *   - Units: micrometres (um), milliseconds (ms), um^2/ms.
 *   - Node values are exchanged in the dense layout [m][ny][nx][n][n]
 *     (source, element row, element column, node row j along y, node column
 *     i along x), n = p+1, FP64; elements outside the mesh read as 0.
 *   - A context is used by one host thread at a time.  All device work goes
 *     to the context's stream (dg_set_stream); calls that return host data
 *     synchronise that stream.
 */
#ifndef DGSIGMA_H
#define DGSIGMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define DG_OK 0
#define DG_EINVAL 1     /* bad argument (range, size, NULL, point outside mesh) */
#define DG_ENOMEM 2     /* device or host allocation failed */
#define DG_ECUDA 3      /* CUDA runtime error (no device, launch failure, ...) */
#define DG_EUNSTABLE 4  /* the solution grew: time step above the stability bound */
#define DG_ENONFINITE 5 /* NaN or Inf in the moments */
#define DG_ETIMEOUT 6   /* a bounded device wait ran out */
#define DG_ESTATE 7     /* call out of order (e.g. step before sources) */

/* Arithmetic of the state and of the element operator.  Moments and the
 * covariance are always accumulated in FP64. */
#define DG_FP64 0
#define DG_FP32 1

/* Axon (inactive) elements.  DG_WALL_REMOVED: the elements are not in the
 * mesh; their faces are reflecting walls with u_hat = u^- and q_hat = 0
 * (Eq. 3).  DG_WALL_PAPER: the paper's Sec. 3.3 treatment, elements kept with
 * k = 0 and frozen at u = 0, so u_hat = u^-/2 and the harmonic mean of
 * Sec. 3.2 gives q_hat = 0. */
#define DG_WALL_REMOVED 0
#define DG_WALL_PAPER 1

/* Outer edge of the domain: DG_BC_ABSORBING is Eq. 4 (u = 0, u_hat = 0,
 * normal flux k q^- . n); DG_BC_PERIODIC wraps both axes. */
#define DG_BC_ABSORBING 0
#define DG_BC_PERIODIC 1

/* Rounding of the FP32 state at every RK stage (FP64 always rounds to
 * nearest).  DG_ROUND_NEAREST: u_new = fl(u0 + beta (u - u0) + gamma R).
 * DG_ROUND_STOCHASTIC (default): the increment inc = beta (u - u0) + gamma R
 * is formed first and u0 + inc is rounded up or down with probabilities that
 * make the result unbiased (E[u_new] = u0 + inc); the uniform number comes
 * from a hash of the two operands' bits and the node's position, so runs are
 * reproducible bit for bit.  Round-to-nearest biases long FP32 runs: with
 * p = 3 Sigma falls behind the FP64 path by 1.3e-6 at 6,000 steps and 2.2e-5
 * at 48,000; stochastic rounding keeps the gap at the 1e-7 level. */
#define DG_ROUND_NEAREST 0
#define DG_ROUND_STOCHASTIC 1

/* Element of the mesh of pixels.  DG_ELEMENT_SQUARE: one square element per
 * pixel with the tensor-product GLL basis of order p (collocated, diagonal
 * mass; p = 1..5).  DG_ELEMENT_TRIANGLE: the paper's own element (Sec. 3.3),
 * each pixel split by its lower-left to upper-right diagonal into two
 * triangles with the Lagrange basis of order p on equispaced nodes and
 * exactly integrated (full) mass matrices (p = 1..3, eta = 0); node k of a
 * triangle is the reference point (i/p, j/p) with k running over j = 0..p,
 * then i = 0..p-j; a pixel holds the lower-right triangle's nodes, then the
 * upper-left one's.  Both use the fluxes of Sec. 3.2 and the same walls,
 * edges, stepping and moments (integrated exactly on the triangles). */
#define DG_ELEMENT_SQUARE 0
#define DG_ELEMENT_TRIANGLE 1

typedef struct dg_config {
  int p;             /* polynomial order of the GLL basis, 1..5 (Eq. 8) */
  int precision;     /* DG_FP64 or DG_FP32 */
  double D;          /* diffusivity k0 of the extracellular region (Eq. 5), > 0 */
  double sigma0;     /* width of the Gaussian start density (um), > 0; it
                        stands in for the Dirac data of Sec. 4.1 */
  double eta;        /* interior-penalty factor >= 0; 0 = the paper's fluxes */
  double cfl_safety; /* dt_max = cfl_safety * 2.5127.../rho(L); (0, 1] */
  int wall_mode;     /* DG_WALL_REMOVED or DG_WALL_PAPER */
  int boundary;      /* DG_BC_ABSORBING or DG_BC_PERIODIC */
  int power_iters;   /* power iterations for rho(L); 0 selects 200 */
  int device;        /* CUDA device ordinal; -1 = the calling thread's current */
  int rounding;      /* DG_ROUND_STOCHASTIC or DG_ROUND_NEAREST (FP32 state) */
  int element;       /* DG_ELEMENT_SQUARE or DG_ELEMENT_TRIANGLE */
} dg_config;

typedef struct dg_ctx dg_ctx;

typedef struct dg_info {
  int p, n_nodes;         /* order and nodes per element (p+1)^2 */
  int nx, ny;             /* elements of the domain grid */
  long long n_active;     /* elements in the mesh (extracellular) */
  long long dof_per_source; /* n_active * n_nodes */
  int m;                  /* number of start points (0 before dg_set_sources) */
  int precision;
  double h, x0, y0;       /* element side and lower-left corner */
  double t;               /* current time (ms) */
  long long steps;        /* RK steps taken since dg_set_sources */
  size_t state_bytes;     /* device bytes of the three RK state arrays */
  int halo_max;           /* largest number of out-of-block face neighbours of
                             a block of 128 consecutive elements */
  int n_geometries;       /* G: geometries held by the context */
  long long n_elements_padded; /* element slots of all geometries, each padded to
                             a multiple of 128 (the state stride per density) */
} dg_info;

/* Fill *cfg with defaults: p=3, FP64, D=2, sigma0=0.2, eta=0, cfl 0.9,
 * removed walls, absorbing edge, 200 power iterations, device -1. */
void dg_config_default(dg_config *cfg);

/* Create a context on cfg->device.  *out receives the handle (NULL on
 * failure).  Errors: DG_EINVAL (cfg out of range), DG_ECUDA (no device),
 * DG_ENOMEM. */
int dg_create(const dg_config *cfg, dg_ctx **out);

/* Release the context and all device memory it owns.  NULL is ignored. */
void dg_destroy(dg_ctx *ctx);

/* Static message of a status code. */
const char *dg_strerror(int code);

/* Message of the last failing call on ctx ("" if none); valid until the next
 * call on ctx. */
const char *dg_last_error(const dg_ctx *ctx);

/* Use the given cudaStream_t (as void*) for all later device work; NULL
 * returns to the context's own stream.  The caller keeps ownership. */
int dg_set_stream(dg_ctx *ctx, void *stream);

/* Domain from an explicit element mask (Sec. 3.3 pixel mesh): active is
 * [ny][nx] bytes, nonzero = extracellular element; element (ex, ey) covers
 * [x0 + ex h, x0 + (ex+1) h] x [y0 + ey h, y0 + (ey+1) h].  Clears sources.
 * Errors: DG_EINVAL (nx, ny < 1, h <= 0, no active element), DG_ENOMEM. */
int dg_set_geometry_mask(dg_ctx *ctx, const uint8_t *active, int nx, int ny,
                         double h, double x0, double y0);

/* Domain from disks in a periodic square cell (substrate of Sec. 2.2; axons
 * of Eq. 5).  cx, cy, r: ndisks centres and radii in [0, L)^2.  The cell is
 * meshed with n_cell x n_cell elements of side h = L/n_cell; an element is
 * removed when its centre lies strictly inside a disk (squared periodic
 * minimum-image distance < r^2).  The domain is a tiles x tiles window of
 * copies of the cell (tiles odd, >= 1) with the central copy at [0, L)^2,
 * i.e. x0 = y0 = -(tiles/2) L; its outer edge follows cfg->boundary.  The
 * mask is built on the device.  Clears sources.  Errors: DG_EINVAL. */
int dg_set_geometry_disks(dg_ctx *ctx, const double *cx, const double *cy,
                          const double *r, int ndisks, double L, int n_cell,
                          int tiles);

/* Batch of G geometries advanced together (one launch per RK stage covers
 * all of them).  Geometry g is given like dg_set_geometry_disks: ndisks[g]
 * disks whose centres and radii are consecutive in cx, cy, r (geometry after
 * geometry), a periodic cell of side L[g] meshed with n_cell[g] elements per
 * side, tiled into a tiles[g] x tiles[g] window centred on the cell (window
 * origin -(tiles[g]/2) L[g]).  Geometries may differ in size and element
 * side; the context's p, precision, D and wall treatment apply to all.
 * Start points then come as [G][m][2] (dg_set_sources), moments as
 * [G][m][6] (dg_moments), and Sigma per geometry (dg_covariance_batch); the
 * time step bound covers every geometry.  Clears sources.  Errors:
 * DG_EINVAL (bad counts or cells), DG_ENOMEM. */
int dg_set_geometry_batch(dg_ctx *ctx, int G, const int *ndisks, const double *cx,
                          const double *cy, const double *r, const double *L,
                          const int *n_cell, const int *tiles);

/* Occupancy raster of disks in a periodic cell (the substrate of Sec. 2.2):
 * out[npix][npix] bytes, 1 where the pixel centre ((i + 1/2) L/npix,
 * (j + 1/2) L/npix) lies strictly inside a disk (the complement of the mesh
 * rule of dg_set_geometry_disks), computed on the calling thread's current
 * device.  Errors: DG_EINVAL, DG_ENOMEM, DG_ECUDA. */
int dg_rasterize_disks(const double *cx, const double *cy, const double *r, int ndisks,
                       double L, int npix, uint8_t *out);

/* The nodal tables the stage kernels use for order p (Eq. 8: Lagrange basis
 * on the p+1 Gauss-Lobatto-Legendre nodes of [-1, 1], quadrature at the
 * nodes, Sec. 3.2).  Host only, no device call.  xi[p+1], w[p+1],
 * D[(p+1)^2] with D[a*(p+1) + i] = l_i'(xi_a), D2[(p+1)^2] = D D.  With
 * precision DG_FP32 the matrices are the FP32 values the FP32 kernels use,
 * widened to double: within a few FP32 ulps of the FP64 ones, every row
 * summing to exactly zero.  Any output pointer may be NULL.  Errors:
 * DG_EINVAL (p outside 1..5 or an unknown precision). */
int dg_basis_tables(int p, int precision, double *xi, double *w, double *D, double *D2);

/* The tables of the triangle elements (DG_ELEMENT_TRIANGLE, Sec. 3.3, Eq. 7
 * integrated exactly) for order p = 1..3, N = (p+1)(p+2)/2.  Host only.
 * r[N], s[N]: reference nodes.  G[2][2][N][N]: for triangle t (0 = lower
 * right, 1 = upper left) and component c (x, y), h q_c = G[t][c] u +
 * sum_e n_ec Lf[t][e] uhat_e, i.e. G = -M^-1 (d(r,s)/dx Sr^T + ...) with M,
 * Sr, Ss the reference mass and derivative matrices.  Lf[2][3][N][p+1]: the
 * lifting of edge values (edge length / h times M^-1 times the edge mass
 * matrix on the edge's nodes).  mono[6][N]: integrals of r^a s^b N_j for
 * (a, b) = (0,0), (1,0), (0,1), (2,0), (1,1), (0,2).  Any pointer may be
 * NULL.  Errors: DG_EINVAL (p outside 1..3). */
int dg_triangle_tables(int p, double *r, double *s, double *G, double *Lf, double *mono);

/* Copy the element mask as built, [ny][nx] bytes (1 = in the mesh); the
 * first geometry of a batch. */
int dg_get_mask(dg_ctx *ctx, uint8_t *active);

/* Sizes and state of the context. */
int dg_get_info(dg_ctx *ctx, dg_info *info);

/* Start points of the Sigma scheme (Sec. 4.1): xy is [m][2] (um); for a
 * batch of G geometries [G][m][2], m points in each geometry.  Each
 * density starts as the normalised Gaussian of width sigma0 about its point,
 * interpolated at the GLL nodes of mesh elements (Dirac data of Sec. 4.1
 * regularised).  Sets t = 0 and records the start moments for
 * Sigma(0).  Errors: DG_EINVAL (m < 1, a point outside the domain or in an
 * element outside the mesh), DG_ENOMEM, DG_ESTATE (no geometry). */
int dg_set_sources(dg_ctx *ctx, const double *xy, int m);

/* Stability bound of the explicit step: rho = spectral radius of L from
 * cfg->power_iters FP64 power iterations (seeded, deterministic), and
 * dt_max = cfl_safety * x3 / rho with x3 = 2.5127... the real-axis limit of
 * SSP-RK3.  Computed once per geometry.  Either pointer may be NULL. */
int dg_query_dt(dg_ctx *ctx, double *dt_max, double *rho);

/* Advance every density by nsteps SSP-RK3 steps of size dt (ms):
 * u1 = u + dt L u, u2 = 3/4 u + 1/4 (u1 + dt L u1),
 * u <- 1/3 u + 2/3 (u2 + dt L u2) (Sec. 3.1, explicit Runge-Kutta).
 * No host synchronisation.  Errors: DG_EINVAL (nsteps < 0, dt <= 0),
 * DG_ESTATE (no sources). */
int dg_step(dg_ctx *ctx, int nsteps, double dt);

/* Growing window (the Sec. 4.1 window sized to the density instead of to
 * the largest Delta).  r_factor > 0 turns it on, 0 off (the default).  While
 * on, dg_step and dg_propagate_to advance steps in groups of at most 64; in
 * each group an element advances only if the squared distance from its
 * centre (x0 + (ex + 1/2) h, y0 + (ey + 1/2) h) to the box spanned by its
 * geometry's start points is <= r_factor^2 (sigma0^2 + 2 D t_end), t_end the
 * time at the group's end (FP64, each operation rounded on its own).  Other
 * elements keep their values and act as frozen neighbours; chunks of the
 * element order with no advancing element are not launched.  For a
 * Gaussian tail the density beyond the radius is of relative size
 * exp(-r_factor^2 / 2) and Sigma moves by about 70 times that (r_factor = 7:
 * 2e-9); odd p with the central fluxes and start densities narrower than
 * about 2h have heavier tails (p = 3, sigma0 = 1.2 h: 4e-6 at r_factor = 7,
 * 1e-8 at 10).  Once the radius covers every mesh element, stepping is the
 * fixed-window path.  Errors: DG_EINVAL (negative or non-finite r_factor). */
int dg_set_growing_window(dg_ctx *ctx, double r_factor);

/* Test hook (no counterpart in the paper) for the shared-memory copies of the
 * stage kernel.  By default a chunk of square elements whose node values fill
 * whole 16-byte slots (p = 1, 3, 5) arrives by one tensor copy (TMA) per
 * chunk, waited for on an mbarrier at most ~4M polls; a wait that runs out
 * makes the block give up and the next dg_moments, dg_covariance or
 * dg_propagate_to return DG_ETIMEOUT (the state is then undefined and the
 * context usable again after dg_set_sources).  mode 0: that default; 1:
 * per-thread cp.async copies only; 2: the barriers also wait for 16 bytes no
 * copy delivers, so every wait runs out (after ~4k polls); 3: every grid
 * barrier of the DG_LAUNCH_STEP launch waits for one more block than the
 * launch has, so its wait runs out (after ~4k polls).  Returns in
 * *tensor_copies (may be NULL) the chunk copies made by the tensor path since
 * the last call.  Errors: DG_EINVAL (mode outside 0..3). */
int dg_debug_copies(dg_ctx *ctx, int mode, unsigned long long *tensor_copies);

/* Launch shape of the FP32 stage kernel (no counterpart in the paper: how the
 * element updates of Sec. 3.3, one independent update per element, are
 * mapped onto the GPU).  DG_LAUNCH_CHUNK (0): one block of 128 threads per
 * chunk of 128 elements and density, one thread per element (all chunks in
 * one launch per RK stage); k >= 1: a persistent launch of k blocks per SM
 * that walk the (density, chunk) work items of every geometry of the
 * context and copy the next item's chunks into shared memory behind the
 * current item's work (clamped to the blocks that fit; FP32 at p = 1 and 3
 * with tensor copies; every other variant keeps DG_LAUNCH_CHUNK);
 * DG_LAUNCH_STEP (-2): all three stages of an SSP-RK3 step in one
 * cooperative launch, the blocks meeting at a grid-wide barrier between
 * stages (FP32 at p = 1, 3, 5 with tensor copies; pays where launches are
 * short); every barrier wait is bounded and one that runs out ends the
 * launch with DG_ETIMEOUT at the next synchronising call;
 * DG_LAUNCH_TUNED (-1, the default): before the first steps after a change
 * of the densities or geometry, DG_LAUNCH_CHUNK and each persistent shape
 * (and, at p = 5 when asked for, the tensor-core contraction, see
 * dg_set_contraction) run
 * stage 1 with dt = 0, which leaves the state's values unchanged, four times
 * on the context's stream and the fastest is kept (under stream capture,
 * where nothing can be timed, DG_LAUNCH_CHUNK); DG_LAUNCH_STEP is taken only
 * when asked for.  Every shape gives the same bits.  Errors: DG_EINVAL
 * (blocks_per_sm < -2 or > 64). */
#define DG_LAUNCH_TUNED (-1)
#define DG_LAUNCH_CHUNK 0
#define DG_LAUNCH_STEP (-2)
int dg_set_launch(dg_ctx *ctx, int blocks_per_sm);

/* The launch shape the last steps used (DG_LAUNCH_CHUNK or blocks per SM,
 * see dg_set_launch). */
int dg_get_launch(dg_ctx *ctx, int *blocks_per_sm);

/* Where the element contractions of the FP32 stage at p = 5 run.  Sec. 3.1
 * (Remark) notes that each element's update is a small dense local system;
 * the element's volume term and the normal derivatives at its faces are one
 * dense [60 x 36] operator applied to its 36 nodal values, for 128 elements
 * at a time a GEMM.  mode 0: sum-factorised on the CUDA cores (FP32); 1: on
 * the tensor cores (tcgen05.mma, FP16 operands, FP32 accumulation) with
 * both operands split into FP16 high and low parts after a per-element
 * power-of-two scaling (three products, ~2^-21 of each element's largest
 * term; a reduced-precision path: the split operator's rows do not sum to
 * exactly zero, which lets the mass drift by ~3e-9 per step); -1: tuned
 * together with the launch shape (see dg_set_launch).  The default is 0.
 * Other orders and FP64 always use the CUDA cores.  Errors: DG_EINVAL
 * (mode outside -1..1). */
int dg_set_contraction(dg_ctx *ctx, int mode);

/* The contraction the last steps used (0 CUDA cores, 1 tensor cores). */
int dg_get_contraction(dg_ctx *ctx, int *mode);

/* How a stage on the pixel triangles (DG_ELEMENT_TRIANGLE, Sec. 3.3, Eq. 7)
 * runs.  With a full mass matrix a triangle's lifted gradient q needs its
 * neighbours' traces, and the divergence needs the neighbours' q.  fused 0:
 * two launches per stage, the first writing q of every pixel to device
 * memory, the second reading it; 1 (the default): one launch per stage that
 * keeps a chunk's q in shared memory and computes the q of each neighbouring
 * triangle across the chunk boundary again from the values around it, with
 * the same arithmetic, so both give the same bits.  One launch per stage runs
 * in FP32 at p = 2 and 3; other triangle contexts keep two launches.
 * Errors: DG_EINVAL (fused outside 0..1). */
int dg_set_triangle_fusion(dg_ctx *ctx, int fused);

/* 1 when the context's triangle stages run as one launch, else 0. */
int dg_get_triangle_fusion(dg_ctx *ctx, int *fused);

/* Test hook (no counterpart in the paper): the n-th device allocation of the
 * library from now on (0 = the next one, in any context) fails as if the
 * device were out of memory; -1 disarms.  Calls that hit it return
 * DG_ENOMEM and leave their context as it was before the call (no geometry
 * or no sources), so it can be used again or destroyed.  Errors: DG_EINVAL
 * (n < -1). */
int dg_debug_fail_alloc(int n);

/* Advance from the current t to Delta in N = ceil((Delta - t)/dt_max) equal
 * steps, then check the moments: DG_ENONFINITE on NaN/Inf, DG_EUNSTABLE when
 * the L1 norm of any density grew above twice its start value.  Delta >= t. */
int dg_propagate_to(dg_ctx *ctx, double Delta);

/* Raw FP64 moments at the current t, out[m][6] ([G][m][6] for a batch)
 * = {M0, Mx, My, Mxx, Mxy, Myy}
 * with M_f = sum over nodes of J^2 w_i w_j f(x - xs, y - ys) u, about each
 * start point (xs, ys) (Sec. 4.1, nodal quadrature). */
int dg_moments(dg_ctx *ctx, double *out);

/* Covariance by the Sigma scheme of Sec. 4.1: each density normalised by its
 * mass and centred at its start point, mixed with weights 1/m, moment-matched
 * Gaussian: mu = mean_s M1/M0, Sigma_mix = mean_s M2/M0 - mu mu^T.  sigma3
 * receives {Sxx, Sxy, Syy} of Sigma(t) = Sigma_mix(t) - Sigma_mix(0) (the
 * start width removed), mu2 the mixture mean displacement, mass (m values,
 * may be NULL) each M0(t).  Computed on the device in FP64. */
int dg_covariance(dg_ctx *ctx, double *sigma3, double *mu2, double *mass);

/* dg_covariance of every geometry of a batch: sigma3 [G][3], mu2 [G][2],
 * mass [G][m] (or NULL); the mixture of geometry g is its own m densities. */
int dg_covariance_batch(dg_ctx *ctx, double *sigma3, double *mu2, double *mass);

/* Least-squares residual of the Gaussian fit (Sec. 4.2, the sum over nodes of
 * [f(x; Sigma) - u_ij]^2 by which the paper assesses the fit).  For each
 * density, normalised by its mass and centred at its start point, the sum
 * runs over its own nodes against the bivariate Gaussian f of the mixture
 * fit (mean mu and covariance Sigma_mix(t), the start width not removed);
 * out[g] (one value per geometry) is the mean over the densities, in um^-4.
 * Computed on the device in FP64. */
int dg_ls_residual(dg_ctx *ctx, double *out);

/* Mixture covariance (Sec. 4.1) of raw moments supplied by the caller, e.g.
 * moments of densities propagated on several GPUs and gathered: mom and mom0
 * are host arrays [m][6] = {M0, Mx, My, Mxx, Mxy, Myy} at t and at t = 0.
 * Same formula as dg_covariance, computed on ctx's device in FP64; needs no
 * geometry.  Errors: DG_EINVAL (m < 1, NULL pointers). */
int dg_mixture_covariance(dg_ctx *ctx, const double *mom, const double *mom0, int m,
                          double *sigma3, double *mu2);

/* Replace every density u by L u (the DG operator alone, Eq. 7 with the
 * fluxes of Sec. 3.2); for operator tests.  Leaves t unchanged. */
int dg_apply_operator(dg_ctx *ctx);

/* Node values in the dense FP64 layout (see above), host buffer of
 * m * ny * nx * n * n doubles; single-geometry contexts only. */
int dg_get_nodes(dg_ctx *ctx, double *host);
int dg_set_nodes(dg_ctx *ctx, const double *host);

/* Node values of selected elements: idx is [k][3] = {source, ex, ey};
 * out receives [k][n][n] doubles (node row j along y, column i along x); an
 * element outside the mesh reads as 0.  Errors: DG_EINVAL (index out of
 * range). */
int dg_get_elements(dg_ctx *ctx, const int *idx, int k, double *out);

/* dg_get_elements for a batch: idx is [k][4] = {geometry, source, ex, ey}. */
int dg_get_elements_batch(dg_ctx *ctx, const int *idx, int k, double *out);

/* Checkpoint: dg_state_size gives the bytes of a snapshot (header, start
 * points, start moments, t, step count and the densities in the state
 * precision); dg_get_state writes it to host memory, dg_set_state restores it
 * into a context with the same geometry, order and precision.  Restored runs
 * continue bit for bit. */
int dg_state_size(dg_ctx *ctx, size_t *bytes);
int dg_get_state(dg_ctx *ctx, void *host, size_t bytes);
int dg_set_state(dg_ctx *ctx, const void *host, size_t bytes);

/* Bytes of device memory the three RK state arrays need for m start points
 * (after a geometry is set). */
int dg_state_bytes(dg_ctx *ctx, int m, size_t *bytes);

/* Use caller-owned device memory (e.g. a torch tensor's data_ptr) of at least
 * dg_state_bytes(m) bytes, 256-byte aligned, for the state arrays of the
 * next dg_set_sources with m points.  The caller keeps it alive until the
 * context is destroyed or rebound; NULL returns to library-owned memory. */
int dg_bind_state(dg_ctx *ctx, void *device_ptr, size_t bytes);

/* Moments of densities without allocating anything.  No counterpart in the
 * paper: it is a service to callers that cannot allocate device memory --
 * their memory is owned by another allocator (a framework's caching pool, a
 * fixed pre-reservation) or they run where cudaMalloc is off limits (a loop
 * that must not risk the implicit synchronisation of an allocation).  The
 * caller passes device pointers: u holds m densities in the dense layout
 * [m][ny][nx][n][n] (n = p+1; FP64 or FP32 per precision; elements outside
 * the mesh hold 0) on the grid of dg_set_geometry_mask (side h, lower-left
 * corner x0, y0), xy the start points [m][2] (FP64), and mom receives the
 * raw moments [m][6] = {M0, Mx, My, Mxx, Mxy, Myy} (FP64) as dg_moments
 * defines them.  Work is queued on stream (a cudaStream_t, NULL = legacy
 * default stream) of the calling thread's current device; the call does not
 * synchronise.
 * Scratch: the reduction's partial sums live in one fixed device array of
 * 1.09 MB inside the library (room for m <= 128), which every GPU that loads
 * the library holds until the process exits.  The first call on a device
 * looks up that array's address with the device current; make that first
 * call before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset (or any other end of the device's primary
 * context) it is stale, and this entry point must not be called again in
 * that process.  All calls share the array: calls whose work overlaps on the
 * GPU (different streams, or threads) race and give wrong moments; serialise
 * them.  The array needs no clearing (each call overwrites every partial it
 * reads).
 * Errors: DG_EINVAL (NULL pointer, m < 1 or m > 128, p outside 1..5, nx or
 * ny < 1, h <= 0, h, x0 or y0 not finite, bad precision), DG_ECUDA (a CUDA
 * error already pending on the calling thread from earlier work -- reported,
 * not consumed, and nothing is launched -- or a launch failure of this
 * call).  No cudaMalloc, cudaFree or other allocating call is made. */
int dg_moments_dense_static(const void *u, int precision, int m, int nx, int ny, int p,
                            double h, double x0, double y0, const double *xy, double *mom,
                            void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DGSIGMA_H */
