// dg_geometry.cu -- element mask from disks, compaction of the mesh elements
// in tile order, and the face-neighbour table.
//
// Substrate (Sec. 2.2): disks in a periodic square cell; the pixel mesh of
// Sec. 3.3 keeps an element when its centre lies outside every disk.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "dg_internal.h"

namespace dg {

// One thread per window element.  Element (ex, ey) of the window is element
// (ex mod n_cell, ey mod n_cell) of the cell, centre ((i + 1/2) h, (j + 1/2) h),
// h = L / n_cell.  The squared minimum-image distance is formed with
// separately rounded products and sum (no fused multiply-add), so the
// decision d^2 < r^2 rounds like plain C.
__global__ void k_mask_disks(const double *__restrict__ cx, const double *__restrict__ cy,
                             const double *__restrict__ r, int nd, double L, int n_cell,
                             int nwin, uint8_t *__restrict__ mask) {
  extern __shared__ double sd[];  // 3 * chunk
  const int chunk = blockDim.x;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = t < (long long)nwin * nwin;
  const int ex = live ? (int)(t % nwin) : 0, ey = live ? (int)(t / nwin) : 0;
  const double h = L / n_cell;
  const double x = ((double)(ex % n_cell) + 0.5) * h;
  const double y = ((double)(ey % n_cell) + 0.5) * h;
  const double half = 0.5 * L;
  uint8_t act = 1;
  for (int base = 0; base < nd; base += chunk) {
    const int k = base + threadIdx.x;
    __syncthreads();
    if (k < nd) {
      sd[threadIdx.x] = cx[k];
      sd[chunk + threadIdx.x] = cy[k];
      sd[2 * chunk + threadIdx.x] = r[k];
    }
    __syncthreads();
    const int cnt = min(chunk, nd - base);
    for (int d = 0; d < cnt; ++d) {
      double dx = x - sd[d], dy = y - sd[chunk + d];
      if (dx > half) dx -= L;
      if (dx < -half) dx += L;
      if (dy > half) dy -= L;
      if (dy < -half) dy += L;
      const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      const double rr = sd[2 * chunk + d];
      if (d2 < __dmul_rn(rr, rr)) act = 0;
    }
  }
  if (live) mask[t] = act;
}

cudaError_t build_mask_disks(const double *d_cx, const double *d_cy, const double *d_r,
                             int nd, double L, int n_cell, int tiles, uint8_t *d_mask,
                             cudaStream_t s) {
  const int nwin = n_cell * tiles;
  const long long tot = (long long)nwin * nwin;
  const int blk = 256;
  const unsigned grid = (unsigned)((tot + blk - 1) / blk);
  k_mask_disks<<<grid, blk, 3 * blk * sizeof(double), s>>>(d_cx, d_cy, d_r, nd, L, n_cell,
                                                           nwin, d_mask);
  return cudaGetLastError();
}

// ---- compaction in tile order --------------------------------------------
// Elements are numbered tile by tile (kTile x kTile tiles, tiles row-major),
// row-major inside a tile, skipping elements outside the mesh, so that
// consecutive threads own neighbouring elements.

__device__ __forceinline__ bool tile_elem(int tile, int t, int nx, int ny, int *ex, int *ey) {
  const int tx = (nx + kTile - 1) / kTile;
  const int bx = tile % tx, by = tile / tx;
  *ex = bx * kTile + (t % kTile);
  *ey = by * kTile + (t / kTile);
  return *ex < nx && *ey < ny;
}

// block = kTile*kTile threads, one block per tile
__global__ void k_tile_count(const uint8_t *__restrict__ mask, int nx, int ny,
                             int *__restrict__ count) {
  int ex, ey;
  const bool in = tile_elem(blockIdx.x, threadIdx.x, nx, ny, &ex, &ey);
  const int f = in ? (mask[(size_t)ey * nx + ex] != 0) : 0;
  const int c = __syncthreads_count(f);
  if (threadIdx.x == 0) count[blockIdx.x] = c;
}

// single block of 1024 threads: exclusive scan of n counts into off[0..n]
__global__ void k_scan_counts(const int *__restrict__ count, int n, int *__restrict__ off) {
  __shared__ int warp_sum[32];
  __shared__ int carry_s;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < n ? count[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int w = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_sum[lane] = w;
    }
    __syncthreads();
    const int carry = carry_s;
    const int incl = x + (wid > 0 ? warp_sum[wid - 1] : 0) + carry;
    if (i < n) off[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry_s = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n] = carry_s;
}

// block = kTile*kTile threads, one block per tile; element numbers start at
// elem0 (the geometry's place in the concatenated numbering)
__global__ void k_assign(const uint8_t *__restrict__ mask, int nx, int ny,
                         const int *__restrict__ off, int elem0, int *__restrict__ cidx,
                         int2 *__restrict__ exy) {
  __shared__ int wsum[kTile * kTile / 32];
  int ex, ey;
  const bool in = tile_elem(blockIdx.x, threadIdx.x, nx, ny, &ex, &ey);
  const bool f = in && mask[(size_t)ey * nx + ex] != 0;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wsum[wid] = __popc(bal);
  __syncthreads();
  int pre = 0;
  for (int w = 0; w < wid; ++w) pre += wsum[w];
  pre += __popc(bal & ((1u << lane) - 1u));
  if (in) {
    const int idx = f ? elem0 + off[blockIdx.x] + pre : -1;
    cidx[(size_t)ey * nx + ex] = idx;
    if (f) exy[idx] = make_int2(ex, ey);
  }
}

// one thread per mesh element of one geometry (elements elem0 .. elem0+nA-1):
// E, W, N, S neighbours as concatenated indices, kWall or kEdge
__global__ void k_neighbours(const int2 *__restrict__ exy, const int *__restrict__ cidx,
                             int elem0, int nA, int nx, int ny, int periodic, int lo, int hi,
                             int4 *__restrict__ nb, int *__restrict__ bad) {
  const int a = elem0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= elem0 + nA) return;
  const int2 e = exy[a];
  int res[4];
  const int dx[4] = {1, -1, 0, 0}, dy[4] = {0, 0, 1, -1};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    int qx = e.x + dx[d], qy = e.y + dy[d];
    if (qx < 0 || qx >= nx || qy < 0 || qy >= ny) {
      if (!periodic) { res[d] = kEdge; continue; }
      qx = (qx + nx) % nx;
      qy = (qy + ny) % ny;
    }
    const int c = cidx[(size_t)qy * nx + qx];
    res[d] = c >= 0 ? c : kWall;
    if (c >= 0 && (c < lo || c >= hi)) atomicExch(bad, 1);
  }
  nb[a] = make_int4(res[0], res[1], res[2], res[3]);
}

// ---- halo lists ----------------------------------------------------------
// One block per chunk of kBlock consecutive elements.  For each face f (in
// order), the elements whose neighbour across f lies outside the chunk get
// consecutive halo slots (block-wide prefix of a ballot), so the table does
// not depend on scheduling.  A halo entry is {neighbour, neighbour's face
// toward the chunk element} = {k, f ^ 1}.
__global__ void k_halo(const int4 *__restrict__ nb, const int2 *__restrict__ chunk_tab,
                       int4 *__restrict__ loc, int2 *__restrict__ halo,
                       int *__restrict__ halo_cnt) {
  __shared__ int wsum[kBlock / 32];
  __shared__ int base_s;
  const int c = blockIdx.x;
  const int a0 = c * kBlock;
  const int el = threadIdx.x;
  const int a = a0 + el;
  const int cnt = chunk_tab[c].x;
  const bool live = el < cnt;
  const int4 q = live ? nb[a] : make_int4(kEdge, kEdge, kEdge, kEdge);
  int qn[4] = {q.x, q.y, q.z, q.w};
  int out[4];
  const int lane = el & 31, wid = el >> 5;
  if (el == 0) base_s = 0;
  __syncthreads();
  for (int f = 0; f < 4; ++f) {
    const int k = qn[f];
    const bool inside = k >= a0 && k < a0 + cnt;
    const bool need = live && k >= 0 && !inside;
    const unsigned bal = __ballot_sync(0xffffffffu, need);
    if (lane == 0) wsum[wid] = __popc(bal);
    __syncthreads();
    int pre = 0, tot = 0;
    for (int w = 0; w < kBlock / 32; ++w) {
      if (w < wid) pre += wsum[w];
      tot += wsum[w];
    }
    pre += __popc(bal & ((1u << lane) - 1u));
    const int base = base_s;
    if (k < 0) out[f] = k;
    else if (inside) out[f] = k - a0;
    else {
      const int slot = base + pre;  // < kHaloCap by construction
      out[f] = kBlock + slot;
      halo[(size_t)c * kHaloCap + slot] = make_int2(k, f ^ 1);
    }
    __syncthreads();
    if (el == 0) base_s = base + tot;
    __syncthreads();
  }
  loc[a] = live ? make_int4(out[0], out[1], out[2], out[3]) : make_int4(kEdge, kEdge, kEdge, kEdge);
  if (el == 0) halo_cnt[c] = base_s;
  // every slot after the last entry holds element -1 (and the neighbour codes
  // of the slots past the chunk's count kEdge): the stage kernels read their
  // threads' slots without waiting for the counts
  for (int h = base_s + el; h < kHaloCap; h += kBlock)
    halo[(size_t)c * kHaloCap + h] = make_int2(-1, 0);
}

// Triangle halo entries: one block per chunk, one thread per entry slot below
// the stride.  The halo pixel k meets the chunk across its face fk; the
// triangle of k on that face has one more pixel face, f3 (A: east and south,
// B: west and north), whose neighbour the fused triangle stage needs too.
__global__ void k_halo_tri(const int4 *__restrict__ nb, const int2 *__restrict__ halo,
                           const int *__restrict__ halo_cnt, int stride,
                           int4 *__restrict__ htri) {
  const int c = blockIdx.x;
  const long long a0 = (long long)c * kBlock;
  const int cnt = halo_cnt[c];
  for (int h = threadIdx.x; h < stride; h += blockDim.x) {
    int4 out = make_int4(-1, 0, 0, kEdge);
    if (h < cnt) {
      const int2 q = halo[(size_t)c * kHaloCap + h];
      const int4 n4 = nb[q.x];
      const int fn[4] = {n4.x, n4.y, n4.z, n4.w};
      const int fk = q.y;
      const int f3 = fk == 0 ? 3 : (fk == 3 ? 0 : (fk == 1 ? 2 : 1));
      out = make_int4(q.x, fk, (int)(fn[fk] - a0), fn[f3]);
    }
    htri[(size_t)c * stride + h] = out;
  }
}

__global__ void k_max_int(const int *__restrict__ v, int n, int *__restrict__ out) {
  __shared__ int sm[256];
  int m = 0;
  for (int i = threadIdx.x; i < n; i += 256) m = max(m, v[i]);
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = max(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

void free_geometry(Geometry &geo) {
  void *ptrs[] = {geo.d_mask, geo.d_cidx, geo.d_nb, geo.d_exy, geo.d_chunk, geo.d_gpar,
                  geo.d_gscale_f, geo.d_gscale_d, geo.d_grange, geo.d_loc, geo.d_halo,
                  geo.d_halo_cnt, geo.d_htri};
  for (void *p : ptrs) cudaFree(p);
  geo = Geometry();
}

__global__ void k_fill_int4(int4 *__restrict__ p, long long n, int4 v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

namespace {
struct Tmp {
  std::vector<void *> ptrs;
  ~Tmp() {
    for (void *p : ptrs) cudaFree(p);
  }
  template <typename X>
  cudaError_t alloc(X **p, size_t n) {
    cudaError_t e = dev_alloc(p, sizeof(X) * (n ? n : 1));
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};
}  // namespace

int build_geometry(Geometry &geo, const std::vector<PartSpec> &specs, int periodic,
                   bool tri_halo, cudaStream_t s, std::string &err) {
  free_geometry(geo);
  const int G = (int)specs.size();
  if (G < 1) {
    err = "no geometry";
    return DG_EINVAL;
  }
  cudaError_t e = cudaSuccess;
  Tmp tmp;
#define GK(expr, what, code)                                            \
  do {                                                                  \
    if ((e = (expr)) != cudaSuccess) {                                  \
      err = std::string(what) + ": " + cudaGetErrorString(e);           \
      free_geometry(geo);                                               \
      return code;                                                      \
    }                                                                   \
  } while (0)
  // dense masks, geometry after geometry
  geo.parts.resize(G);
  long long dense = 0;
  for (int g = 0; g < G; ++g) {
    GeoPart &p = geo.parts[g];
    const PartSpec &q = specs[g];
    p.nx = q.nx; p.ny = q.ny; p.h = q.h; p.x0 = q.x0; p.y0 = q.y0;
    p.periodic = periodic;
    p.dense_off = dense;
    dense += (long long)q.nx * q.ny;
  }
  if (dense > (1ll << 31) - 1) {
    err = "domains too large";
    free_geometry(geo);
    return DG_EINVAL;
  }
  GK(dev_alloc(&geo.d_mask, (size_t)dense), "mask allocation", DG_ENOMEM);
  GK(dev_alloc(&geo.d_cidx, sizeof(int) * (size_t)dense), "index map allocation", DG_ENOMEM);
  int max_nd = 1;
  for (const PartSpec &q : specs) max_nd = std::max(max_nd, q.nd);
  double *d_disk = nullptr;
  GK(tmp.alloc(&d_disk, 3 * (size_t)max_nd), "disk allocation", DG_ENOMEM);
  for (int g = 0; g < G; ++g) {
    const PartSpec &q = specs[g];
    uint8_t *m = geo.d_mask + geo.parts[g].dense_off;
    const size_t cells = (size_t)q.nx * q.ny;
    if (q.host_mask) {
      std::vector<uint8_t> m01(cells);
      for (size_t k = 0; k < cells; ++k) m01[k] = q.host_mask[k] ? 1 : 0;
      GK(cudaMemcpyAsync(m, m01.data(), cells, cudaMemcpyHostToDevice, s), "mask copy", DG_ECUDA);
      GK(cudaStreamSynchronize(s), "mask copy", DG_ECUDA);
    } else {
      if (q.nd > 0) {
        GK(cudaMemcpyAsync(d_disk, q.cx, 8 * (size_t)q.nd, cudaMemcpyHostToDevice, s), "disk copy", DG_ECUDA);
        GK(cudaMemcpyAsync(d_disk + max_nd, q.cy, 8 * (size_t)q.nd, cudaMemcpyHostToDevice, s), "disk copy", DG_ECUDA);
        GK(cudaMemcpyAsync(d_disk + 2 * max_nd, q.r, 8 * (size_t)q.nd, cudaMemcpyHostToDevice, s), "disk copy", DG_ECUDA);
      }
      GK(build_mask_disks(d_disk, d_disk + max_nd, d_disk + 2 * max_nd, q.nd, q.L, q.n_cell, q.tiles, m, s),
         "disk mask", DG_ECUDA);
      GK(cudaStreamSynchronize(s), "disk mask", DG_ECUDA);
    }
  }
  // per geometry: tile counts and their scan -> elements in the mesh
  std::vector<int *> offs(G, nullptr);
  long long elems = 0;
  for (int g = 0; g < G; ++g) {
    GeoPart &p = geo.parts[g];
    const int tx = (p.nx + kTile - 1) / kTile, ty = (p.ny + kTile - 1) / kTile;
    const int nt = tx * ty;
    int *d_count = nullptr;
    GK(tmp.alloc(&d_count, (size_t)nt), "tile count allocation", DG_ENOMEM);
    GK(tmp.alloc(&offs[g], (size_t)nt + 1), "tile offset allocation", DG_ENOMEM);
    const uint8_t *m = geo.d_mask + p.dense_off;
    k_tile_count<<<nt, kTile * kTile, 0, s>>>(m, p.nx, p.ny, d_count);
    k_scan_counts<<<1, 1024, 0, s>>>(d_count, nt, offs[g]);
    GK(cudaGetLastError(), "tile scan", DG_ECUDA);
    int total = 0;
    GK(cudaMemcpyAsync(&total, offs[g] + nt, sizeof(int), cudaMemcpyDeviceToHost, s), "tile scan", DG_ECUDA);
    GK(cudaStreamSynchronize(s), "tile scan", DG_ECUDA);
    if (total <= 0) {
      err = "geometry " + std::to_string(g) + " has no element in the mesh";
      free_geometry(geo);
      return DG_EINVAL;
    }
    p.n_active = total;
    p.off = elems;
    elems += ((long long)total + kBlock - 1) / kBlock * kBlock;
  }
  if (elems > (1ll << 31) - 1) {
    err = "too many elements";
    free_geometry(geo);
    return DG_EINVAL;
  }
  geo.n_pad = elems;
  long long active = 0;
  for (const GeoPart &p : geo.parts) active += p.n_active;
  geo.n_active = active;
  GK(dev_alloc(&geo.d_nb, sizeof(int4) * (size_t)elems), "neighbour table allocation", DG_ENOMEM);
  GK(dev_alloc(&geo.d_exy, sizeof(int2) * (size_t)elems), "coordinate allocation", DG_ENOMEM);
  const int4 pad = make_int4(kEdge, kEdge, kEdge, kEdge);
  k_fill_int4<<<(unsigned)((elems + 255) / 256), 256, 0, s>>>(geo.d_nb, elems, pad);
  GK(cudaGetLastError(), "neighbour table", DG_ECUDA);
  GK(cudaMemsetAsync(geo.d_exy, 0, sizeof(int2) * (size_t)elems, s), "coordinate table", DG_ECUDA);
  int *d_bad = nullptr;
  GK(tmp.alloc(&d_bad, 1), "flag allocation", DG_ENOMEM);
  GK(cudaMemsetAsync(d_bad, 0, sizeof(int), s), "flag", DG_ECUDA);
  for (int g = 0; g < G; ++g) {
    const GeoPart &p = geo.parts[g];
    const int tx = (p.nx + kTile - 1) / kTile, ty = (p.ny + kTile - 1) / kTile;
    const uint8_t *m = geo.d_mask + p.dense_off;
    int *ci = geo.d_cidx + p.dense_off;
    k_assign<<<tx * ty, kTile * kTile, 0, s>>>(m, p.nx, p.ny, offs[g], (int)p.off, ci, geo.d_exy);
    k_neighbours<<<(unsigned)((p.n_active + 255) / 256), 256, 0, s>>>(
        geo.d_exy, ci, (int)p.off, (int)p.n_active, p.nx, p.ny, p.periodic, (int)p.off,
        (int)(p.off + p.n_active), geo.d_nb, d_bad);
    GK(cudaGetLastError(), "neighbour table", DG_ECUDA);
  }
  int bad = 0;
  GK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s), "neighbour table", DG_ECUDA);
  GK(cudaStreamSynchronize(s), "neighbour table", DG_ECUDA);
  if (bad) {
    err = "neighbour table out of range";
    free_geometry(geo);
    return DG_ECUDA;
  }
  // chunk table and per-geometry parameters
  const long long nch = elems / kBlock;
  std::vector<int2> chunk((size_t)nch);
  std::vector<double4> gpar(G);
  std::vector<float> gsf(G);
  std::vector<double> gsd(G);
  std::vector<int2> grange(G);
  for (int g = 0; g < G; ++g) {
    const GeoPart &p = geo.parts[g];
    const long long c0 = p.off / kBlock;
    const long long nc = (p.n_active + kBlock - 1) / kBlock;
    for (long long c = 0; c < nc; ++c)
      chunk[(size_t)(c0 + c)] = make_int2((int)std::min<long long>(kBlock, p.n_active - c * kBlock), g);
    const double J = 0.5 * p.h;
    gpar[g] = make_double4(p.x0, p.y0, p.h, 1.0 / (J * J));
    gsf[g] = (float)(1.0 / (J * J));
    gsd[g] = 1.0 / (J * J);
    grange[g] = make_int2((int)p.off, (int)p.n_active);
  }
  GK(dev_alloc(&geo.d_chunk, sizeof(int2) * (size_t)nch), "chunk table allocation", DG_ENOMEM);
  GK(dev_alloc(&geo.d_gpar, sizeof(double4) * G), "parameter allocation", DG_ENOMEM);
  GK(dev_alloc(&geo.d_gscale_f, sizeof(float) * G), "parameter allocation", DG_ENOMEM);
  GK(dev_alloc(&geo.d_gscale_d, sizeof(double) * G), "parameter allocation", DG_ENOMEM);
  GK(dev_alloc(&geo.d_grange, sizeof(int2) * G), "parameter allocation", DG_ENOMEM);
  GK(cudaMemcpyAsync(geo.d_chunk, chunk.data(), sizeof(int2) * chunk.size(), cudaMemcpyHostToDevice, s), "copy", DG_ECUDA);
  GK(cudaMemcpyAsync(geo.d_gpar, gpar.data(), sizeof(double4) * G, cudaMemcpyHostToDevice, s), "copy", DG_ECUDA);
  GK(cudaMemcpyAsync(geo.d_gscale_f, gsf.data(), sizeof(float) * G, cudaMemcpyHostToDevice, s), "copy", DG_ECUDA);
  GK(cudaMemcpyAsync(geo.d_gscale_d, gsd.data(), sizeof(double) * G, cudaMemcpyHostToDevice, s), "copy", DG_ECUDA);
  GK(cudaMemcpyAsync(geo.d_grange, grange.data(), sizeof(int2) * G, cudaMemcpyHostToDevice, s), "copy", DG_ECUDA);
  // halo lists of every chunk
  int hmax = 0;
  GK(dev_alloc(&geo.d_loc, sizeof(int4) * (size_t)elems), "halo table allocation", DG_ENOMEM);
  GK(dev_alloc(&geo.d_halo, sizeof(int2) * (size_t)nch * kHaloCap), "halo table allocation", DG_ENOMEM);
  GK(dev_alloc(&geo.d_halo_cnt, sizeof(int) * ((size_t)nch + 1)), "halo table allocation", DG_ENOMEM);
  k_halo<<<(unsigned)nch, kBlock, 0, s>>>(geo.d_nb, geo.d_chunk, geo.d_loc, geo.d_halo, geo.d_halo_cnt);
  k_max_int<<<1, 256, 0, s>>>(geo.d_halo_cnt, (int)nch, geo.d_halo_cnt + nch);
  GK(cudaGetLastError(), "halo table", DG_ECUDA);
  GK(cudaMemcpyAsync(&hmax, geo.d_halo_cnt + nch, sizeof(int), cudaMemcpyDeviceToHost, s), "halo table", DG_ECUDA);
  geo.h_mask.resize((size_t)dense);
  GK(cudaMemcpyAsync(geo.h_mask.data(), geo.d_mask, (size_t)dense, cudaMemcpyDeviceToHost, s), "mask copy", DG_ECUDA);
  GK(cudaStreamSynchronize(s), "halo table", DG_ECUDA);
  if (hmax < 0 || hmax > kHaloCap) {
    err = "halo table out of range";
    free_geometry(geo);
    return DG_ECUDA;
  }
  geo.halo_max = hmax;
  if (tri_halo) {
    const int stride = hmax > 0 ? hmax : 1;
    GK(dev_alloc(&geo.d_htri, sizeof(int4) * (size_t)nch * stride), "halo table allocation", DG_ENOMEM);
    k_halo_tri<<<(unsigned)nch, kBlock, 0, s>>>(geo.d_nb, geo.d_halo, geo.d_halo_cnt, stride, geo.d_htri);
    GK(cudaGetLastError(), "triangle halo table", DG_ECUDA);
  }
  const GeoPart &p0 = geo.parts[0];
  geo.nx = p0.nx; geo.ny = p0.ny; geo.h = p0.h; geo.x0 = p0.x0; geo.y0 = p0.y0;
#undef GK
  return DG_OK;
}

}  // namespace dg
