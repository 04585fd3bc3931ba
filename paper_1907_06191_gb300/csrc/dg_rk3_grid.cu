// dg_rk3_grid.cu -- one SSP-RK3 step in one cooperative launch.
//
// The three stages of a step depend on each other only through the face
// neighbours of every element (Sec. 3.1: within a stage the element updates
// are independent), so one launch can run all three if every block has
// finished stage k before any block reads stage k's results.  The blocks
// (all resident: a cooperative launch) walk the (density, chunk) work
// items of the stage, then meet at a grid-wide barrier: an arrival counter
// in global memory, polled by one thread per block at most `limit` times;
// a wait that runs out sets the error flag (DG_ETIMEOUT on the host) and the
// block leaves, so the launch always ends.  Per item the arithmetic is that
// of the one-block-per-chunk kernel (same helpers, same rounding keys), so
// the results are the same bits.  Results leave by tensor store and are
// complete (not only read out of shared memory) before the arrival; halo
// values of arrays written earlier in the launch are read through L2
// (ld.global.cg), never through the read-only cache.  It pays where
// launches are short (small windows): one launch per RK step instead of
// three.
#include "dg_stage.cuh"

namespace dg {
namespace {

template <typename T, int NP>
__device__ __forceinline__ void load_elem_cg(const T *p, T (&u)[NP]) {
  static_assert(NP * sizeof(T) % 16 == 0, "whole 16-byte slots");
  const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
  for (int k = 0; k < NP * (int)sizeof(T) / 16; ++k) {
    float4 v;
    asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(q + k));
    const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
    for (int w = 0; w < 16 / (int)sizeof(T); ++w) u[k * (16 / (int)sizeof(T)) + w] = pv[w];
  }
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Every block arrives once; the barrier is passed when `target` arrivals
// are counted (targets grow from stage to stage: the counter is zeroed
// before the launch).  false if the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned target, int limit) {
  __syncthreads();  // the block's own work (and its tensor stores) done
  bool ok = true;
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
    __threadfence();
    atomicAdd(count, 1u);
    int i = 0;
    while (ld_acquire_gpu(count) < target) {
      if (++i > limit) {
        ok = false;
        break;
      }
      __nanosleep(128);
    }
    __threadfence();
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
  }
  return __syncthreads_or(!ok) == 0;
}

struct GridArgs {
  unsigned *count = nullptr;   // arrival counter, zero at launch
  int expect_extra = 0;        // test hook: arrivals no block makes
  int limit = 1 << 20;         // polls of the counter before giving up
};

template <typename T, int P, bool SROUND, bool FULL>
__global__ void __launch_bounds__(kBlock, blocks_for_regs(128))
    k_rk3_grid(T *U0, T *U1, T *U2, const int4 *__restrict__ loc,
               const int2 *__restrict__ halo, const int *__restrict__ halo_cnt,
               const int2 *__restrict__ chunk_tab, const int2 *__restrict__ grange,
               const T *__restrict__ gscale, long long stride, int nrec,
               const int *__restrict__ chunk_list, const uint8_t *__restrict__ adv,
               const StageTab<T, P> tb, const StageCoef<T> c0, const StageCoef<T> c1,
               const StageCoef<T> c2, const __grid_constant__ CUtensorMap tm0,
               const __grid_constant__ CUtensorMap tm1, const __grid_constant__ CUtensorMap tm2,
               const CopyArgs ca, const GridArgs ga, long long n_items, int nch) {
  constexpr int n = P + 1, NP = n * n;
  using St = Stage<T, NP>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int front = stage_front_bytes<T, P>(nrec);
  const int bar_off = front + ((St::CHUNK_BYTES + 15) / 16) * 16;
  T *su = reinterpret_cast<T *>(smem_raw);
  T *so = reinterpret_cast<T *>(smem_raw + front);
  T *rec_base = reinterpret_cast<T *>(smem_raw);
  Records<T, P> rec{rec_base,
                    rec_base + ((nrec * n * (int)sizeof(T) + 15) / 16) * 16 / (int)sizeof(T), nrec};
  const int zero_rec = nrec - 1;
  const int el = threadIdx.x;
  const uint32_t bar0 = smem_u32(smem_raw + bar_off), bar1 = bar0 + 8;
  const bool aligned = (smem_u32(smem_raw) & 1023u) == 0;  // the swizzled copies need it
  if (el == 0) {
    if (!aligned) atomicExch(ca.err, 2);
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    mbar_fence_init();
  }
  __syncthreads();
  bool ok = aligned;
  uint32_t ph0 = 0, ph1 = 0;
  const uint32_t bytes = (uint32_t)(kBlock * NP * sizeof(T)) + (uint32_t)ca.extra_tx;
  const unsigned G = gridDim.x + (unsigned)ga.expect_extra;
#pragma unroll 1
  for (int stage = 0; stage < 3; ++stage) {
    const T *uin = stage == 0 ? U0 : (stage == 1 ? U1 : U2);
    T *out = stage == 0 ? U1 : (stage == 1 ? U2 : U0);
    const CUtensorMap *tin = stage == 0 ? &tm0 : (stage == 1 ? &tm1 : &tm2);
    const CUtensorMap *tout = stage == 0 ? &tm1 : (stage == 1 ? &tm2 : &tm0);
    const StageCoef<T> &c = stage == 0 ? c0 : (stage == 1 ? c1 : c2);
    const bool has_u0 = stage > 0;
    for (long long item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
      const int sd = (int)(item / nch);
      const int x = (int)(item - (long long)sd * nch);
      const int chunk = chunk_list ? __ldg(chunk_list + x) : x;
      const long long a0 = (long long)chunk * kBlock;
      const int2 ci = __ldg(chunk_tab + chunk);
      const int cnt = ci.x;
      const bool live = el < cnt;
      T gam = c.gamma * __ldg(gscale + ci.y);
      if (adv != nullptr && live && __ldg(adv + a0 + el) == 0) gam = (T)0;
      const size_t sbase = (size_t)sd * (size_t)stride * NP;
      const T *U = uin + sbase;
      const int row = (int)((long long)sd * stride + a0);
      if (el == 0) {
        // the stores of the previous item and stage are complete: the async
        // proxy reads what they wrote
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
        mbar_expect_tx(bar0, bytes);
        tma_load_rows(smem_u32(su), tin, row, bar0);
        if (has_u0) {
          mbar_expect_tx(bar1, bytes);
          tma_load_rows(smem_u32(so), &tm0, row, bar1);
        }
        if (ca.counter) atomicAdd(ca.counter, 1ull);
      }
      const int4 l4 = live ? __ldg(loc + a0 + el) : make_int4(kEdge, kEdge, kEdge, kEdge);
      const int hcnt = __ldg(halo_cnt + chunk);
      const int2 hk = __ldg(halo + (size_t)chunk * kHaloCap + el);
      T hv[NP];
      if (hk.x >= 0) load_elem_cg<T, NP>(U + (size_t)hk.x * NP, hv);
      bool okw = mbar_wait(bar0, ph0, ca.limit);
      ph0 ^= 1u;
      T u[NP], R[NP];
      if (live && okw) St::read(su, el, u);
      if (__syncthreads_or(!okw)) {  // leave the item loop after a bounded wait for u0
        if (has_u0) mbar_wait(bar1, ph1, ca.limit);
        if (el == 0) atomicExch(ca.err, 1);
        ok = false;
        break;
      }
      if (el == 0) {
        T z[n];
#pragma unroll
        for (int t = 0; t < n; ++t) z[t] = (T)0;
        rec.put(zero_rec, z, z);
      }
      if (live) element_records_volume<T, P>(u, tb, rec, el, R);
      if (hk.x >= 0) halo_face_record<T, P>(hv, hk.y, tb, rec, 4 * kBlock + el);
      for (int h = el + kBlock; h < hcnt; h += kBlock) {
        const int2 q = __ldg(halo + (size_t)chunk * kHaloCap + h);
        T v[NP];
        load_elem_cg<T, NP>(U + (size_t)q.x * NP, v);
        halo_face_record<T, P>(v, q.y, tb, rec, 4 * kBlock + h);
      }
      __syncthreads();
      if (live) {
        const int lq[4] = {l4.x, l4.y, l4.z, l4.w};
        element_flux<T, P, FULL>(u, R, lq, el, zero_rec, rec, tb, c);
      }
      if (has_u0) {
        okw = mbar_wait(bar1, ph1, ca.limit);
        ph1 ^= 1u;
      }
      if (live && okw) {
        T o[NP];
        const uint32_t hsh = SROUND ? element_key<T>(a0 + el - __ldg(grange + ci.y).x, NP, sd, u) : 0u;
        if (has_u0) {
          St::read(so, el, o);
          element_update<T, P, true, SROUND>(u, R, o, gam, hsh, c);
        } else {
          element_update<T, P, false, SROUND>(u, R, o, gam, hsh, c);
        }
        St::write(so, el, o);
      }
      const bool store_tma = cnt == kBlock;
      if (store_tma) fence_proxy_async_smem();
      if (__syncthreads_or(!okw)) {
        if (el == 0) atomicExch(ca.err, 1);
        ok = false;
        break;
      }
      if (store_tma) {
        if (el == 0) {
          asm volatile(
              "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                  reinterpret_cast<uint64_t>(tout)),
              "r"(0), "r"(row), "r"(smem_u32(so))
              : "memory");
          asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
          // complete, not only read: other blocks read it after the barrier
          asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
        }
      } else {  // coalesced 16-byte stores of a partial chunk
        char *go = reinterpret_cast<char *>(out + sbase + (size_t)a0 * NP);
        const int np16 = St::pieces(cnt);
        for (int j = el; j < np16; j += kBlock)
          *reinterpret_cast<float4 *>(go + 16 * (size_t)j) =
              *reinterpret_cast<const float4 *>(reinterpret_cast<unsigned char *>(so) +
                                                16 * St::piece_dst(j));
        fence_proxy_async_smem();  // so is rewritten by the next item's u0 copy
      }
      __syncthreads();  // so and the records are free for the next item
    }
    // blocks that gave up still arrive, so the others are not kept waiting
    const bool passed = grid_barrier(ga.count, (unsigned)(stage + 1) * G, ga.limit);
    if (!passed) {
      if (el == 0) atomicExch(ca.err, 1);
      return;
    }
    if (!ok) return;
  }
}

template <typename T, int P>
cudaError_t launch_grid_p(T *U0, T *U1, T *U2, const Geometry &geo, long long stride, int m,
                          const Gll &g, const StageCoef<T> (&c)[3], cudaStream_t s,
                          const ChunkSel &sel, const CUtensorMap *maps, const CopyArgs &ca,
                          const GridArgs &ga) {
  const long long nch = sel.list ? sel.count : geo.n_chunks();
  if (geo.n_pad <= 0 || m <= 0 || nch <= 0) return cudaSuccess;
  const T *gscale;
  if constexpr (sizeof(T) == 8) gscale = geo.d_gscale_d;
  else gscale = geo.d_gscale_f;
  const StageTab<T, P> tb = make_tab<T, P>(g);
  const int nrec = 4 * kBlock + geo.halo_max + 1;
  const int smem = stage_smem_bytes<T, P>(geo.halo_max);
  const bool full = c[0].pen != (T)0 || c[0].wallA;
  const bool sr = sizeof(T) == 4 && c[0].sround;
  void (*kern)(T *, T *, T *, const int4 *, const int2 *, const int *, const int2 *,
               const int2 *, const T *, long long, int, const int *, const uint8_t *,
               const StageTab<T, P>, const StageCoef<T>, const StageCoef<T>, const StageCoef<T>,
               const CUtensorMap, const CUtensorMap, const CUtensorMap, const CopyArgs,
               const GridArgs, long long, int);
  if (sr) kern = full ? k_rk3_grid<T, P, true, true> : k_rk3_grid<T, P, true, false>;
  else kern = full ? k_rk3_grid<T, P, false, true> : k_rk3_grid<T, P, false, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  const long long items = nch * (long long)m;
  const unsigned G = (unsigned)std::min<long long>(items, (long long)nsm * per_sm);
  if ((e = cudaMemsetAsync(ga.count, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int nch_i = (int)nch;
  return cudaLaunchKernelEx(&cfg, kern, U0, U1, U2, geo.d_loc, geo.d_halo, geo.d_halo_cnt,
                            geo.d_chunk, geo.d_grange, gscale, stride, nrec, sel.list, sel.adv,
                            tb, c[0], c[1], c[2], maps[0], maps[1], maps[2], ca, ga, items, nch_i);
}

}  // namespace

// One SSP-RK3 step of every density in one cooperative launch (FP32, p = 1,
// 3, 5 with tensor copies); cudaErrorNotSupported otherwise.
cudaError_t launch_rk3_grid_f32(int p, float *U0, float *U1, float *U2, const Geometry &geo,
                                long long stride, int m, const Gll &g,
                                const StageCoef<float> (&c)[3], cudaStream_t s,
                                const ChunkSel &sel, const CUtensorMap *maps, int *err,
                                unsigned long long *counter, unsigned *grid_count,
                                int extra_tx, int limit, int grid_extra, int grid_limit) {
  if (maps == nullptr || err == nullptr || grid_count == nullptr) return cudaErrorNotSupported;
  CopyArgs ca;
  ca.use_tma = 1;
  ca.store_tma = 1;
  ca.extra_tx = extra_tx;
  ca.limit = limit;
  ca.err = err;
  ca.counter = counter;
  GridArgs ga;
  ga.count = grid_count;
  ga.expect_extra = grid_extra;
  ga.limit = grid_limit;
  switch (p) {
    case 1: return launch_grid_p<float, 1>(U0, U1, U2, geo, stride, m, g, c, s, sel, maps, ca, ga);
    case 3: return launch_grid_p<float, 3>(U0, U1, U2, geo, stride, m, g, c, s, sel, maps, ca, ga);
    case 5: return launch_grid_p<float, 5>(U0, U1, U2, geo, stride, m, g, c, s, sel, maps, ca, ga);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace dg
