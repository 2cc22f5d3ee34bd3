// Batched step as per-tile launches (the configuration with 0 CTAs per SM): one CTA per tile, the
// instances of a launch in its kernel parameters (tile body in lbpc_tile.cuh).
#include "lbpc_tile.cuh"

namespace lbpc {

// Per-tile launch of a batched step: CTA b finds its instance by the launch's first-tile offsets (a
// uniform search over the kernel parameters) and runs the tile body on that instance's tile
// b - first_tile. Every value of the instance is then a parameter-space operand, as in the single-instance
// kernel, so the body has none of the work-list kernel's per-use shared-memory loads.
//
// The launches of one step cover disjoint instances, so each lets the next one start while its own
// last CTAs run (programmatic dependent launch). The last CTA of a launch waits, before it exits, for
// the launch before it to complete: a launch then completes only after every earlier launch of the step
// has, and the advance kernel that follows in stream order sees the whole step. The earlier launch's
// CTAs have all started when this one starts, so the wait always ends.
template <class S, class R, int TX, int TY, int NPT, int CAP>
__global__ void __launch_bounds__(TX* TY / NPT, fused_min_blocks<S, TX * TY / NPT, NPT>())
    k_batch_tiles(const __grid_constant__ SegLaunch<S, CAP> L) {
  // The next launch of the step covers other instances: let it start as this one's last CTAs run.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ FusedSmem<R, TX, TY> sm;
  const int b = blockIdx.x;
  int k = 0, hi = L.n - 1;  // the last instance whose first CTA is at most b (a uniform binary search)
#pragma unroll 1
  while (k < hi) {
    const int mid = (k + hi + 1) >> 1;
    if (L.first_tile[mid] <= b) k = mid;
    else hi = mid - 1;
  }
  const SegInst<S>& I = L.in[k];
  const auto& P = I.P;
  const int t = b - L.first_tile[k];
  const int x0 = (t % I.tiles_x) * TX, y0 = (t / I.tiles_x) * TY;
  const bool interior = x0 >= 3 && x0 + TX + 3 <= P.nx && y0 >= 3 && y0 + TY + 3 <= P.ny;
  if (interior)
    fused_body<1, S, R, TX, TY, NPT>(I.fs, I.gs, I.fd, I.gd, (R*)I.phi_prev, P, 0, I.first, I.scalars, I.partials,
                                     I.status, sm, x0, y0, t, TmaTile<S>{nullptr}, I.step);
  else  // edge tiles wrap and clamp their indices: cheaper in 32 bits
    fused_body<0, S, R, TX, TY, NPT, true>(I.fs, I.gs, I.fd, I.gd, (R*)I.phi_prev, P, 0, I.first, I.scalars,
                                           I.partials, I.status, sm, x0, y0, t, TmaTile<S>{nullptr}, I.step);
  if (b == (int)gridDim.x - 1) asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <class S, class R, int TX, int TY, int NPT, int CAP>
static cudaError_t seg_launch_t(const void* Lh, bool pdl, cudaStream_t st) {
  const SegLaunch<S, CAP>& L = *(const SegLaunch<S, CAP>*)Lh;
  if (L.n <= 0 || L.tiles <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)L.tiles);
  cfg.blockDim = dim3(TX * TY / NPT);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_batch_tiles<S, R, TX, TY, NPT, CAP>, L);
}

template <class S, class R, int CAP>
static cudaError_t seg_launch_c(int variant, const void* L, bool pdl, cudaStream_t st) {
  switch (variant) {
    case 1: return seg_launch_t<S, R, 32, 16, 1, CAP>(L, pdl, st);
    case 2: return seg_launch_t<S, R, 64, 8, 1, CAP>(L, pdl, st);
    case 3: return seg_launch_t<S, R, 32, 16, 2, CAP>(L, pdl, st);
    case 4: return seg_launch_t<S, R, 64, 16, 2, CAP>(L, pdl, st);
    case 5: return seg_launch_t<S, R, 32, 32, 2, CAP>(L, pdl, st);
    default: return seg_launch_t<S, R, 32, 8, 1, CAP>(L, pdl, st);
  }
}

template <class S, class R>
static cudaError_t seg_launch_p(int variant, bool small, const void* L, bool pdl, cudaStream_t st) {
  return small ? seg_launch_c<S, R, kSegSmall>(variant, L, pdl, st)
               : seg_launch_c<S, R, seg_capacity<S>()>(variant, L, pdl, st);
}

cudaError_t batch_seg_launch(int prec, int variant, bool small, const void* L, bool pdl, cudaStream_t st) {
  if (prec == 0) return seg_launch_p<double, double>(variant, small, L, pdl, st);
  if (prec == 1) return seg_launch_p<float, float>(variant, small, L, pdl, st);
  return seg_launch_p<__half, float>(variant, small, L, pdl, st);
}

}  // namespace lbpc
