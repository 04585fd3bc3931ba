// dg_geometry.cu -- element mask from disks, compaction of the mesh elements
// in tile order, and the face-neighbour table.
//
// Substrate (Sec. 2.2): disks in a periodic square cell; the pixel mesh of
// Sec. 3.3 keeps an element when its centre lies outside every disk.
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

// block = kTile*kTile threads, one block per tile
__global__ void k_assign(const uint8_t *__restrict__ mask, int nx, int ny,
                         const int *__restrict__ off, int *__restrict__ cidx,
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
    const int idx = f ? off[blockIdx.x] + pre : -1;
    cidx[(size_t)ey * nx + ex] = idx;
    if (f) exy[idx] = make_int2(ex, ey);
  }
}

// one thread per mesh element: E, W, N, S neighbours
__global__ void k_neighbours(const int2 *__restrict__ exy, const int *__restrict__ cidx,
                             int nA, int nx, int ny, int periodic, int4 *__restrict__ nb,
                             int *__restrict__ bad) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nA) return;
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
    if (c >= nA) atomicExch(bad, 1);
  }
  nb[a] = make_int4(res[0], res[1], res[2], res[3]);
}

// ---- halo lists ----------------------------------------------------------
// One block per chunk of kBlock consecutive elements.  For each face f (in
// order), the elements whose neighbour across f lies outside the chunk get
// consecutive halo slots (block-wide prefix of a ballot), so the table does
// not depend on scheduling.  A halo entry is {neighbour, neighbour's face
// toward the chunk element} = {k, f ^ 1}.
__global__ void k_halo(const int4 *__restrict__ nb, int nA, int4 *__restrict__ loc,
                       int2 *__restrict__ halo, int *__restrict__ halo_cnt) {
  __shared__ int wsum[kBlock / 32];
  __shared__ int base_s;
  const int c = blockIdx.x;
  const int a0 = c * kBlock;
  const int el = threadIdx.x;
  const int a = a0 + el;
  const bool live = a < nA;
  const int4 q = live ? nb[a] : make_int4(kEdge, kEdge, kEdge, kEdge);
  int qn[4] = {q.x, q.y, q.z, q.w};
  int out[4];
  const int lane = el & 31, wid = el >> 5;
  if (el == 0) base_s = 0;
  __syncthreads();
  for (int f = 0; f < 4; ++f) {
    const int k = qn[f];
    const bool inside = k >= a0 && k < a0 + kBlock && k < nA;
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
  if (live) loc[a] = make_int4(out[0], out[1], out[2], out[3]);
  if (el == 0) halo_cnt[c] = base_s;
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
  cudaFree(geo.d_mask);
  cudaFree(geo.d_cidx);
  cudaFree(geo.d_nb);
  cudaFree(geo.d_exy);
  cudaFree(geo.d_loc);
  cudaFree(geo.d_halo);
  cudaFree(geo.d_halo_cnt);
  geo.d_mask = nullptr;
  geo.d_cidx = nullptr;
  geo.d_nb = nullptr;
  geo.d_exy = nullptr;
  geo.d_loc = nullptr;
  geo.d_halo = nullptr;
  geo.d_halo_cnt = nullptr;
  geo.n_active = 0;
  geo.halo_max = 0;
}

// geo.d_mask, nx, ny must be set.  Returns a DG_* code.
int build_connectivity(Geometry &geo, int periodic, cudaStream_t s, std::string &err) {
  const int nx = geo.nx, ny = geo.ny;
  const int tx = (nx + kTile - 1) / kTile, ty = (ny + kTile - 1) / kTile;
  const int nt = tx * ty;
  int *d_count = nullptr, *d_off = nullptr, *d_bad = nullptr;
  cudaError_t e;
  int code = DG_OK;
  int total = 0, bad = 0;
  if ((e = cudaMalloc(&d_count, sizeof(int) * (size_t)nt)) != cudaSuccess ||
      (e = cudaMalloc(&d_off, sizeof(int) * ((size_t)nt + 1))) != cudaSuccess ||
      (e = cudaMalloc(&d_bad, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&geo.d_cidx, sizeof(int) * (size_t)nx * ny)) != cudaSuccess) {
    err = std::string("connectivity allocation: ") + cudaGetErrorString(e);
    code = DG_ENOMEM;
    goto done;
  }
  k_tile_count<<<nt, kTile * kTile, 0, s>>>(geo.d_mask, nx, ny, d_count);
  k_scan_counts<<<1, 1024, 0, s>>>(d_count, nt, d_off);
  if ((e = cudaMemcpyAsync(&total, d_off + nt, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    err = std::string("connectivity scan: ") + cudaGetErrorString(e);
    code = DG_ECUDA;
    goto done;
  }
  if (total <= 0) {
    err = "the mask has no element in the mesh";
    code = DG_EINVAL;
    goto done;
  }
  geo.n_active = total;
  geo.n_pad = ((long long)total + 31) / 32 * 32;
  if ((e = cudaMalloc(&geo.d_nb, sizeof(int4) * (size_t)total)) != cudaSuccess ||
      (e = cudaMalloc(&geo.d_exy, sizeof(int2) * (size_t)total)) != cudaSuccess) {
    err = std::string("neighbour table allocation: ") + cudaGetErrorString(e);
    code = DG_ENOMEM;
    goto done;
  }
  k_assign<<<nt, kTile * kTile, 0, s>>>(geo.d_mask, nx, ny, d_off, geo.d_cidx, geo.d_exy);
  cudaMemsetAsync(d_bad, 0, sizeof(int), s);
  k_neighbours<<<(total + 255) / 256, 256, 0, s>>>(geo.d_exy, geo.d_cidx, total, nx, ny,
                                                   periodic, geo.d_nb, d_bad);
  if ((e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    err = std::string("neighbour table: ") + cudaGetErrorString(e);
    code = DG_ECUDA;
    goto done;
  }
  if (bad) {
    err = "neighbour table out of range";
    code = DG_ECUDA;
    goto done;
  }
  {
    const int nch = (int)((total + kBlock - 1) / kBlock);
    int hmax = 0;
    if ((e = cudaMalloc(&geo.d_loc, sizeof(int4) * (size_t)total)) != cudaSuccess ||
        (e = cudaMalloc(&geo.d_halo, sizeof(int2) * (size_t)nch * kHaloCap)) != cudaSuccess ||
        (e = cudaMalloc(&geo.d_halo_cnt, sizeof(int) * ((size_t)nch + 1))) != cudaSuccess) {
      err = std::string("halo table allocation: ") + cudaGetErrorString(e);
      code = DG_ENOMEM;
      goto done;
    }
    k_halo<<<nch, kBlock, 0, s>>>(geo.d_nb, total, geo.d_loc, geo.d_halo, geo.d_halo_cnt);
    k_max_int<<<1, 256, 0, s>>>(geo.d_halo_cnt, nch, geo.d_halo_cnt + nch);
    if ((e = cudaMemcpyAsync(&hmax, geo.d_halo_cnt + nch, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      err = std::string("halo table: ") + cudaGetErrorString(e);
      code = DG_ECUDA;
      goto done;
    }
    if (hmax < 0 || hmax > kHaloCap) {
      err = "halo table out of range";
      code = DG_ECUDA;
      goto done;
    }
    geo.halo_max = hmax;
  }
done:
  cudaFree(d_count);
  cudaFree(d_off);
  cudaFree(d_bad);
  return code;
}

}  // namespace dg
