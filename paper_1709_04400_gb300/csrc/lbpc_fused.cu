// Fused step of one domain: one kernel per time step, one CTA per tile (tile body in lbpc_tile.cuh),
// with the interior tiles' populations staged in shared memory by TMA where the row stride allows.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>

#include "lbpc_tile.cuh"

namespace lbpc {

template <class S, class R, int TX, int TY, int NPT>
__global__ void __launch_bounds__(TX* TY / NPT, fused_min_blocks<S, TX * TY / NPT, NPT>()) k_fused(PopBuf<S> fsrc, PopBuf<S> gsrc, PopBuf<S> fdst, PopBuf<S> gdst,
                                                   R* __restrict__ phi_prev, DevParams P, long long step, int first,
                                                   const double* __restrict__ rho_ave, double* __restrict__ partials,
                                                   long long* __restrict__ status) {
  __shared__ FusedSmem<R, TX, TY> sm;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const bool interior = x0 >= 3 && x0 + TX + 3 <= P.nx && y0 >= 3 && y0 + TY + 3 <= P.ny;
  const int pslot = blockIdx.y * gridDim.x + blockIdx.x;
  if (interior)
    fused_body<1, S, R, TX, TY, NPT>(fsrc, gsrc, fdst, gdst, phi_prev, P, step, first, rho_ave, partials, status, sm,
                                     x0, y0, pslot);
  else
    fused_body<0, S, R, TX, TY, NPT>(fsrc, gsrc, fdst, gdst, phi_prev, P, step, first, rho_ave, partials, status, sm,
                                     x0, y0, pslot);
}

// Same step with the interior tiles' populations staged in shared memory by TMA (dynamic shared
// memory of TmaBox<S, TX, TY>::BYTES). Tiles that touch an edge take the general path.
template <class S, class R, int TX, int TY, int NPT>
__global__ void __launch_bounds__(TX* TY / NPT, fused_min_blocks<S, TX * TY / NPT, NPT>()) k_fused_tma(PopBuf<S> fsrc, PopBuf<S> gsrc, PopBuf<S> fdst, PopBuf<S> gdst,
                                                       R* __restrict__ phi_prev, DevParams P, long long step, int first,
                                                       const double* __restrict__ rho_ave,
                                                       double* __restrict__ partials, long long* __restrict__ status,
                                                       const __grid_constant__ TmaMaps maps) {
  using B = TmaBox<S, TX, TY>;
  __shared__ FusedSmem<R, TX, TY> sm;
  extern __shared__ __align__(128) unsigned char dyn[];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const bool interior = x0 >= 3 && x0 + TX + 3 <= P.nx && y0 >= 3 && y0 + TY + 3 <= P.ny;
  const int pslot = blockIdx.y * gridDim.x + blockIdx.x;
  if (!interior) {
    fused_body<0, S, R, TX, TY, NPT>(fsrc, gsrc, fdst, gdst, phi_prev, P, step, first, rho_ave, partials, status, sm,
                                     x0, y0, pslot);
    return;
  }
  uint64_t* bar = (uint64_t*)(dyn + B::BYTES - 128);
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (unsigned)(18 * B::BX * B::BY * sizeof(S) + (B::HALF ? 2 * B::REFX * B::BY * 4 : 0)));
    for (int a = 0; a < 9; ++a) {
      tma_load_3d(dyn + a * B::PLANE, &maps.f, x0 - B::XOFF, y0 - 3, a, bar);
      tma_load_3d(dyn + (9 + a) * B::PLANE, &maps.g, x0 - B::XOFF, y0 - 3, a, bar);
    }
    if (B::HALF) {
      tma_load_2d(dyn + 18 * B::PLANE, &maps.rf, x0 - B::XOFF, y0 - 3, bar);
      tma_load_2d(dyn + 18 * B::PLANE + B::RPLANE, &maps.rg, x0 - B::XOFF, y0 - 3, bar);
    }
  }
  // Every thread polls the barrier. Measured against one polling thread with the others parked at a block
  // barrier (820 instead of 888 instructions per node, but 1 % slower in FP32, also with two kernels
  // sharing the GPU) and against waits that sleep in the barrier with a suspend-time hint (slower, more
  // instructions): polling wakes the warps soonest.
  if (!mbar_wait_bounded(bar, 0)) {
    if (threadIdx.x == 0) report(status, step, x0, y0, ST_TIMEOUT);
    mbar_wait_bounded(bar, 0);  // let the copies in flight land before the block's shared memory goes away
    return;
  }
  fused_body<2, S, R, TX, TY, NPT>(fsrc, gsrc, fdst, gdst, phi_prev, P, step, first, rho_ave, partials, status, sm,
                                   x0, y0, pslot, TmaTile<S>{dyn});
}

// Persistent form of the TMA-staged step: resident CTAs take tiles in order from a ticket counter (so
// the tiles in flight stay one compact band of the grid, as with one CTA per tile, and the rings they
// re-read meet in L2), and each starts its next interior tile's copy as soon as the current tile has
// finished reading its staged populations (after stage 1). The copy then runs under stages 2 and 3
// instead of in front of the next tile. An edge tile reads nothing staged, so the next copy starts
// before it. One mbarrier serves every copy; the waits alternate its phase parity. tickets is zeroed
// before the launch.
template <class S, int TX, int TY>
__device__ __forceinline__ void tma_issue_tile(unsigned char* dyn, uint64_t* bar, const TmaMaps& maps, int x0, int y0) {
  using B = TmaBox<S, TX, TY>;
  // the box was last read through the generic proxy (stage 1, before a block barrier); order those
  // reads before the copy engine's writes
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, (unsigned)(18 * B::BX * B::BY * sizeof(S) + (B::HALF ? 2 * B::REFX * B::BY * 4 : 0)));
  for (int a = 0; a < 9; ++a) {
    tma_load_3d(dyn + a * B::PLANE, &maps.f, x0 - B::XOFF, y0 - 3, a, bar);
    tma_load_3d(dyn + (9 + a) * B::PLANE, &maps.g, x0 - B::XOFF, y0 - 3, a, bar);
  }
  if (B::HALF) {
    tma_load_2d(dyn + 18 * B::PLANE, &maps.rf, x0 - B::XOFF, y0 - 3, bar);
    tma_load_2d(dyn + 18 * B::PLANE + B::RPLANE, &maps.rg, x0 - B::XOFF, y0 - 3, bar);
  }
}

template <class S, class R, int TX, int TY, int NPT>
__global__ void __launch_bounds__(TX* TY / NPT, fused_min_blocks<S, TX * TY / NPT, NPT>())
    k_fused_tma_loop(PopBuf<S> fsrc, PopBuf<S> gsrc, PopBuf<S> fdst, PopBuf<S> gdst, R* __restrict__ phi_prev,
                     DevParams P, long long step, int first, const double* __restrict__ rho_ave,
                     double* __restrict__ partials, long long* __restrict__ status,
                     unsigned long long* __restrict__ tickets, const __grid_constant__ TmaMaps maps) {
  using B = TmaBox<S, TX, TY>;
  __shared__ FusedSmem<R, TX, TY> sm;
  // walk state, double-buffered by iteration parity: this tile and the next one (being staged); thread 0
  // fills the other slot during the tile, so one block barrier per tile orders both
  __shared__ int s_tile[2], s_next[2];
  extern __shared__ __align__(128) unsigned char dyn[];
  uint64_t* bar = (uint64_t*)(dyn + B::BYTES - 128);
  const int ntx = (P.nx + TX - 1) / TX, ntiles = ntx * ((P.ny + TY - 1) / TY);
  // tile origin, and whether the tile, its 2-ring and their pull sources stay inside the domain
  auto origin = [&](int tile, int& x0, int& y0) {
    x0 = (tile % ntx) * TX;
    y0 = (tile / ntx) * TY;
    return x0 >= 3 && x0 + TX + 3 <= P.nx && y0 >= 3 && y0 + TY + 3 <= P.ny;
  };
  auto take = [&]() {  // thread 0: the next tile in order, or ntiles when none is left
    const unsigned long long k = atomicAdd(tickets, 1ull);
    return k < (unsigned long long)ntiles ? (int)k : ntiles;
  };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    const int t0 = take();
    int x0, y0;
    if (t0 < ntiles && origin(t0, x0, y0)) tma_issue_tile<S, TX, TY>(dyn, bar, maps, x0, y0);
    s_tile[0] = t0;
    s_next[0] = t0 < ntiles ? take() : ntiles;
  }
  __syncthreads();
  unsigned parity = 0;  // of the mbarrier phase awaited next
  for (int it = 0;; it ^= 1) {
    const int tile = s_tile[it];
    if (tile >= ntiles) break;
    // thread 0 starts the copy of the next tile, if interior, and records it and the tile after it as
    // the next iteration's walk state
    auto start_next = [&]() {
      if (threadIdx.x != 0) return;
      const int next = s_next[it];
      int nx0, ny0;
      if (next < ntiles && origin(next, nx0, ny0)) tma_issue_tile<S, TX, TY>(dyn, bar, maps, nx0, ny0);
      s_tile[it ^ 1] = next;
      s_next[it ^ 1] = next < ntiles ? take() : ntiles;
    };
    int x0, y0;
    if (origin(tile, x0, y0)) {
      if (!mbar_wait_bounded(bar, parity)) {
        if (threadIdx.x == 0) report(status, step, x0, y0, ST_TIMEOUT);
        mbar_wait_bounded(bar, parity);  // let the copy in flight land before the block's shared memory goes away
        return;
      }
      parity ^= 1u;
      fused_body<2, S, R, TX, TY, NPT>(fsrc, gsrc, fdst, gdst, phi_prev, P, step, first, rho_ave, partials, status, sm,
                                       x0, y0, tile, TmaTile<S>{dyn}, nullptr, start_next);
    } else {
      start_next();
      fused_body<0, S, R, TX, TY, NPT>(fsrc, gsrc, fdst, gdst, phi_prev, P, step, first, rho_ave, partials, status, sm,
                                       x0, y0, tile);
    }
    __syncthreads();  // the tile body is done with the shared arrays; the next walk state has landed
  }
}

// Resident CTAs of the persistent kernel on the current device (SMs x CTAs per SM), queried once per
// device: the value cannot change while the process runs, so two first calls racing only store the
// same number twice. The dynamic shared-memory attribute is set before the query.
template <class S, class R, int TX, int TY, int NPT>
static cudaError_t loop_residency(int smem, int* out) {
  static std::atomic<int> cache[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && (*out = cache[dev].load(std::memory_order_relaxed)) > 0) return cudaSuccess;
  int sms = 0, occ = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused_tma_loop<S, R, TX, TY, NPT>, TX * TY / NPT,
                                                         (size_t)smem)) != cudaSuccess)
    return e;
  *out = std::max(occ, 1) * sms;
  if (dev >= 0 && dev < 64) cache[dev].store(*out, std::memory_order_relaxed);
  return cudaSuccess;
}

// ------------------------------------------------------------------------------------------------
template <class S, class R, int TX, int TY, int NPT = 1, bool LOOP = false>
static cudaError_t fused_impl(const SplitBuffers& b, const DevParams& P, int cur, long long step, cudaStream_t st,
                              cudaEvent_t* ev) {
  dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
  const PopBuf<S> fs{(S*)b.f[cur], b.ref_f[cur], b.wall[cur]}, gs{(S*)b.g[cur], b.ref_g[cur]};
  const PopBuf<S> fd{(S*)b.f[cur ^ 1], b.ref_f[cur ^ 1], b.wall[cur ^ 1]}, gd{(S*)b.g[cur ^ 1], b.ref_g[cur ^ 1]};
  if (ev) cudaEventRecord(ev[0], st);
  bool staged = false;
  if constexpr (sizeof(S) <= 4) {  // the TMA-staged kernel exists for FP32 and FP16 storage
    if (b.tma[cur]) {
      using B = TmaBox<S, TX, TY>;
      // The dynamic shared-memory limit is held per device context, so it is set before every launch:
      // the call is cheap, thread-safe, and right after a device reset or on a second device.
      bool persistent = false;
      if constexpr (LOOP) {
        cudaError_t e = cudaFuncSetAttribute(k_fused_tma_loop<S, R, TX, TY, NPT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, B::BYTES);
        if (e != cudaSuccess) return e;
        int resident = 0;  // CTAs of the persistent kernel that fit on the device at once
        if ((e = loop_residency<S, R, TX, TY, NPT>(B::BYTES, &resident)) != cudaSuccess) return e;
        // persistent CTAs pay off where each walks many tiles (measured: +5 % to +12 % in FP32 from
        // 2048^2, 27 or more per CTA; 1-8 % slower at 1024^2, 7 per CTA); smaller grids take one CTA per tile
        if ((long long)grid.x * grid.y > 8LL * resident) {
          unsigned long long* tickets = (unsigned long long*)(b.status + 6);
          if ((e = cudaMemsetAsync(tickets, 0, sizeof *tickets, st)) != cudaSuccess) return e;
          k_fused_tma_loop<S, R, TX, TY, NPT><<<resident, TX * TY / NPT, B::BYTES, st>>>(
              fs, gs, fd, gd, (R*)b.phi_prev, P, step, step == 0, b.scalars, b.partials, b.status, tickets,
              *b.tma[cur]);
          persistent = true;
        }
      }
      if (!persistent) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_fused_tma<S, R, TX, TY, NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, B::BYTES);
        if (e != cudaSuccess) return e;
        k_fused_tma<S, R, TX, TY, NPT><<<grid, TX * TY / NPT, B::BYTES, st>>>(
            fs, gs, fd, gd, (R*)b.phi_prev, P, step, step == 0, b.scalars, b.partials, b.status, *b.tma[cur]);
      }
      staged = true;
    }
  }
  if (!staged)
    k_fused<S, R, TX, TY, NPT><<<grid, TX * TY / NPT, 0, st>>>(fs, gs, fd, gd, (R*)b.phi_prev, P, step, step == 0,
                                                               b.scalars, b.partials, b.status);
  if (ev) cudaEventRecord(ev[1], st);
  if (P.buoyancy == 1) {
    fused_finish(b, P, (int)(grid.x * grid.y), st);
    if (ev) cudaEventRecord(ev[2], st);
  }
  return cudaGetLastError();
}

// ---- tensor maps of the TMA-staged path ----
static PFN_cuTensorMapEncodeTiled_v12000 query_encode_fn() {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    return (PFN_cuTensorMapEncodeTiled_v12000)p;
  return nullptr;
}

// The driver's entry point is the same for every device and context; the function-local static is
// initialised once, thread-safely.
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = query_encode_fn();
  return fn;
}

template <class S, int TX, int TY>
static bool encode_t(TmaMaps* m, void* f, void* g, float* rf, float* rg, const DevParams& P) {
  using B = TmaBox<S, TX, TY>;
  auto fn = encode_fn();
  if (!fn) return false;
  if (((size_t)P.nx * sizeof(S)) % 16 != 0) return false;  // row stride must be a multiple of 16 bytes
  const CUtensorMapDataType dt = sizeof(S) == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                : (sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64);
  const cuuint64_t dims[3] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, 9};
  const cuuint64_t strides[2] = {(cuuint64_t)P.nx * sizeof(S), (cuuint64_t)P.N * sizeof(S)};
  const cuuint32_t box[3] = {(cuuint32_t)B::BX, (cuuint32_t)B::BY, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  auto enc3 = [&](CUtensorMap* t, void* base) {
    return fn(t, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  if (!enc3(&m->f, f) || !enc3(&m->g, g)) return false;
  if (B::HALF) {
    const cuuint64_t d2[2] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny};
    const cuuint64_t s2[1] = {(cuuint64_t)P.nx * 4};
    const cuuint32_t b2[2] = {(cuuint32_t)B::REFX, (cuuint32_t)B::BY};
    auto enc2 = [&](CUtensorMap* t, void* base) {
      return fn(t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, d2, s2, b2, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
             CUDA_SUCCESS;
    };
    if (!enc2(&m->rf, rf) || !enc2(&m->rg, rg)) return false;
  }
  return true;
}

template <class S>
static bool encode_tile(TmaMaps* m, int tile, void* f, void* g, float* rf, float* rg, const DevParams& P) {
  if (tile == 1 || tile == 4) return encode_t<S, 32, 8>(m, f, g, rf, rg, P);
  if (tile == 3) return encode_t<S, 32, 32>(m, f, g, rf, rg, P);
  return encode_t<S, 32, 16>(m, f, g, rf, rg, P);  // tiles 0 and 2
}

bool fused_tma_encode(TmaMaps* m, int prec, int tile, void* f, void* g, float* rf, float* rg, const DevParams& P) {
  if (prec == 1) return encode_tile<float>(m, tile, f, g, rf, rg, P);
  if (prec == 2) return encode_tile<__half>(m, tile, f, g, rf, rg, P);
  return false;  // FP64 runs the split step by default; its fused form keeps per-thread loads
}

// Tile configurations of the FP32 / FP16 fused step: 0 = 32x16, 1 = 32x8, 2 = 32x16 with 2 nodes per
// thread, 3 = 32x32 with 2 nodes per thread, 4 = 32x8 in persistent CTAs that start each next tile's copy
// early.
template <class S, class R>
static cudaError_t fused_tiles(const SplitBuffers& b, const DevParams& P, int cur, long long step, cudaStream_t st,
                               cudaEvent_t* ev) {
  switch (b.fused_tile) {
    case 1: return fused_impl<S, R, 32, 8, 1>(b, P, cur, step, st, ev);
    case 2: return fused_impl<S, R, 32, 16, 2>(b, P, cur, step, st, ev);
    case 3: return fused_impl<S, R, 32, 32, 2>(b, P, cur, step, st, ev);
    case 4: return fused_impl<S, R, 32, 8, 1, true>(b, P, cur, step, st, ev);
    default: return fused_impl<S, R, 32, 16, 1>(b, P, cur, step, st, ev);
  }
}

cudaError_t fused_step(const SplitBuffers& b, const DevParams& P, int prec, int cur, long long step, cudaStream_t st,
                       cudaEvent_t* ev) {
  if (prec == 0) {
    SplitBuffers nb = b;
    nb.tma[0] = nb.tma[1] = nullptr;
    return fused_impl<double, double, 32, 8>(nb, P, cur, step, st, ev);
  }
  if (prec == 3) {
    SplitBuffers nb = b;
    nb.tma[0] = nb.tma[1] = nullptr;
    return fused_impl<dw, dw, 32, 8>(nb, P, cur, step, st, ev);
  }
  if (prec == 1) return fused_tiles<float, float>(b, P, cur, step, st, ev);
  return fused_tiles<__half, float>(b, P, cur, step, st, ev);
}

}  // namespace lbpc
