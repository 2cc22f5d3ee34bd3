// Batched step: the persistent work-list kernel over many domains (tile body in lbpc_tile.cuh),
// the per-instance advance kernel, and their launchers.
#include <stddef.h>

#include "lbpc_tile.cuh"

namespace lbpc {

// ------------------------------------------------------------------------------------------------
// Batched step: many independent instances of uneven size in one persistent launch. CTAs walk a work
// list of (instance, tile) entries round-robin (the tiles in flight at any moment form one compact
// band of the list, so neighbouring tiles' halos meet in L2); each tile runs the same body as the
// single-instance kernel with that instance's parameters and buffers, so an instance's result does
// not depend on what else is in the batch. The tile count and every per-instance value live in
// device memory, so a captured CUDA graph of these launches stays valid when instances join or leave.
//
// The walk is software-pipelined: while a tile computes, the CTA already holds the next tile's list
// entry and copies the next instance's descriptor (integer header, the coefficient set of the
// arithmetic type, buffer pointers and step state) into the second of two shared-memory slots with
// 16-byte asynchronous copies, so a change of instance costs no exposed global-memory latency.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class R> struct CoefSpan;  // byte range of the coefficient set a kernel of arithmetic R reads
template <> struct CoefSpan<double> { static constexpr size_t off = offsetof(DevParams, cd), len = sizeof(Coefs<double>); };
template <> struct CoefSpan<float> { static constexpr size_t off = offsetof(DevParams, cf), len = sizeof(Coefs<float>); };
template <> struct CoefSpan<dw> { static constexpr size_t off = offsetof(DevParams, cw), len = sizeof(Coefs<dw>); };

// Copy the parts of an instance descriptor a kernel of arithmetic R reads, in 16-byte chunks issued by
// the first threads of the block; completes at the issuing threads' next cp_async_wait_all.
template <class S, class R>
__device__ __forceinline__ void desc_copy_async(BatchInst<S>* dst, const BatchInst<S>* src) {
  constexpr size_t HEAD = offsetof(DevParams, cd) / 16;                 // nx .. heat_unit_rates
  constexpr size_t COEF = (CoefSpan<R>::len + 15) / 16;                  // the coefficient set
  constexpr size_t TAIL_OFF = offsetof(BatchInst<S>, f);                 // pointers and step state
  constexpr size_t TAIL = (sizeof(BatchInst<S>) - TAIL_OFF) / 16;
  static_assert(offsetof(DevParams, cd) % 16 == 0 && CoefSpan<R>::off % 16 == 0 && TAIL_OFF % 16 == 0 &&
                    sizeof(BatchInst<S>) % 16 == 0,
                "descriptor parts must be 16-byte aligned");
  static_assert(CoefSpan<R>::off + 16 * COEF <= sizeof(DevParams), "coefficient span inside the parameters");
  static_assert(HEAD + COEF + TAIL <= 128, "one copy per thread of the (at least 128) threads");
  const unsigned char* s = (const unsigned char*)src;
  unsigned char* d = (unsigned char*)dst;
  const int k = threadIdx.x;
  if (k < (int)HEAD) {
    cp_async16(d + 16 * k, s + 16 * k);
  } else if (k < (int)(HEAD + COEF)) {
    const size_t o = CoefSpan<R>::off + 16 * (k - HEAD);
    cp_async16(d + o, s + o);
  } else if (k < (int)(HEAD + COEF + TAIL)) {
    const size_t o = TAIL_OFF + 16 * (k - HEAD - COEF);
    cp_async16(d + o, s + o);
  }
}

template <class S, class R, int TX, int TY, int NPT>
__global__ void __launch_bounds__(TX* TY / NPT, fused_min_blocks<S, TX * TY / NPT, NPT>())
    k_batch_step(const BatchMeta* __restrict__ meta, const BatchInst<S>* __restrict__ insts) {
  constexpr int NTH = TX * TY / NPT;
  static_assert(NTH >= 128, "the descriptor copy needs at least 128 threads");
  static_assert(sizeof(BatchTile) == 16, "a work-list entry is one 16-byte copy");
  __shared__ FusedSmem<R, TX, TY> sm;
  __shared__ BatchInst<S> sI[2];
  __shared__ BatchTile st[3];  // this tile's entry, the next one's, and the one after (filled while computing)
  // walk state (work-list position, descriptor slot, ring position) and the list length, kept in shared
  // memory so that no register holds them across the tile body
  __shared__ int s_t, s_slot, s_r, s_n;
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    const int t0 = blockIdx.x, n = meta->ntiles;
    s_n = n;
    if (t0 < n) st[0] = meta->tiles[t0];
    if (t0 + G < n) st[1] = meta->tiles[t0 + G];
    s_t = t0;
    s_slot = 0;
    s_r = 0;
  }
  __syncthreads();
  if ((int)blockIdx.x >= s_n) return;
  desc_copy_async<S, R>(&sI[0], &insts[st[0].inst]);
  cp_async_wait_all();
  __syncthreads();
  for (;;) {
    {
      const int t = s_t, slot = s_slot, r = s_r, ntiles = s_n;
      const BatchTile tile = st[r];
      const int rn = r == 2 ? 0 : r + 1, ra = rn == 2 ? 0 : rn + 1;
      const bool more = t + G < ntiles;
      if (more && st[rn].inst != tile.inst) desc_copy_async<S, R>(&sI[slot ^ 1], &insts[st[rn].inst]);
      if (threadIdx.x == NTH - 1 && t + 2 * G < ntiles) cp_async16(&st[ra], &meta->tiles[t + 2 * G]);
      const BatchInst<S>& I = sI[slot];
      const DevParams& P = I.P;
      const int cur = I.cur;
      const long long step = I.step;
      const bool interior = tile.x0 >= 3 && tile.x0 + TX + 3 <= P.nx && tile.y0 >= 3 && tile.y0 + TY + 3 <= P.ny;
      if (interior)
        fused_body<1, S, R, TX, TY, NPT, true>(I.f[cur], I.g[cur], I.f[cur ^ 1], I.g[cur ^ 1], (R*)I.phi_prev, P, step,
                                         step == 0, I.scalars, I.partials, I.status, sm, tile.x0, tile.y0, tile.pslot);
      else
        fused_body<0, S, R, TX, TY, NPT, true>(I.f[cur], I.g[cur], I.f[cur ^ 1], I.g[cur ^ 1], (R*)I.phi_prev, P, step,
                                         step == 0, I.scalars, I.partials, I.status, sm, tile.x0, tile.y0, tile.pslot);
    }
    // The CTA's last tile: it issued no copy, so its threads leave without waiting for one another.
    if (s_t + G >= s_n) return;
    cp_async_wait_all();
    __syncthreads();  // the tile is done with the shared memory; the next descriptor and entry have landed
    const int t = s_t, r = s_r, rn = r == 2 ? 0 : r + 1;
    const bool change = st[rn].inst != st[r].inst;
    __syncthreads();  // every thread has read the walk state
    if (threadIdx.x == 0) {
      s_t = t + G;
      s_r = rn;
      if (change) s_slot ^= 1;
    }
    __syncthreads();
  }
}

// One block per instance slot: rho_ave from the tile partials (fixed order), then flip the buffers
// and count the step.
template <class S>
__global__ void __launch_bounds__(128) k_batch_advance(BatchInst<S>* __restrict__ insts) {
  __shared__ double red[4];
  BatchInst<S>& I = insts[blockIdx.x];
  if (!I.active) return;
  if (I.P.buoyancy == 1) {  // rho_ave for the next step
    double acc = 0.0;
    for (int j = threadIdx.x; j < I.ntiles; j += 128) acc += I.partials[j];
    acc = block_sum<128>(acc, red);
    if (threadIdx.x == 0) I.scalars[0] = acc / (double)I.P.N;
  }
  if (threadIdx.x == 0) {
    I.cur ^= 1;
    I.step += 1;
  }
}

template <class S, class R, int TX, int TY, int NPT>
static cudaError_t batch_launch_t(int ctas, const BatchMeta* d_meta, void* d_insts, int ninst, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_batch_step<S, R, TX, TY, NPT><<<sms * ctas, TX * TY / NPT, 0, st>>>(d_meta, (const BatchInst<S>*)d_insts);
  if (ninst > 0) k_batch_advance<S><<<ninst, 128, 0, st>>>((BatchInst<S>*)d_insts);
  return cudaGetLastError();
}

template <class S, class R>
static cudaError_t batch_launch_p(int variant, int ctas, const BatchMeta* d_meta, void* d_insts, int ninst,
                                  cudaStream_t st) {
  switch (variant) {
    case 1: return batch_launch_t<S, R, 32, 16, 1>(ctas, d_meta, d_insts, ninst, st);
    case 2: return batch_launch_t<S, R, 64, 8, 1>(ctas, d_meta, d_insts, ninst, st);
    case 3: return batch_launch_t<S, R, 32, 16, 2>(ctas, d_meta, d_insts, ninst, st);
    case 4: return batch_launch_t<S, R, 64, 16, 2>(ctas, d_meta, d_insts, ninst, st);
    case 5: return batch_launch_t<S, R, 32, 32, 2>(ctas, d_meta, d_insts, ninst, st);
    default: return batch_launch_t<S, R, 32, 8, 1>(ctas, d_meta, d_insts, ninst, st);
  }
}

cudaError_t batch_advance_launch(int prec, void* d_insts, int ninst, cudaStream_t st) {
  if (ninst <= 0) return cudaSuccess;
  if (prec == 0) k_batch_advance<double><<<ninst, 128, 0, st>>>((BatchInst<double>*)d_insts);
  else if (prec == 1) k_batch_advance<float><<<ninst, 128, 0, st>>>((BatchInst<float>*)d_insts);
  else k_batch_advance<__half><<<ninst, 128, 0, st>>>((BatchInst<__half>*)d_insts);
  return cudaGetLastError();
}

cudaError_t batch_step_launch(int prec, int variant, int ctas, const BatchMeta* d_meta, void* d_insts, int ninst,
                              cudaStream_t st) {
  if (prec == 0) return batch_launch_p<double, double>(variant, ctas, d_meta, d_insts, ninst, st);
  if (prec == 1) return batch_launch_p<float, float>(variant, ctas, d_meta, d_insts, ninst, st);
  return batch_launch_p<__half, float>(variant, ctas, d_meta, d_insts, ninst, st);
}

template <class S, class R, int TX, int TY, int NPT> static int occ_t() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step<S, R, TX, TY, NPT>, TX * TY / NPT, 0);
  return n;
}

template <class S, class R> static int occ_p(int variant) {
  switch (variant) {
    case 1: return occ_t<S, R, 32, 16, 1>();
    case 2: return occ_t<S, R, 64, 8, 1>();
    case 3: return occ_t<S, R, 32, 16, 2>();
    case 4: return occ_t<S, R, 64, 16, 2>();
    case 5: return occ_t<S, R, 32, 32, 2>();
    default: return occ_t<S, R, 32, 8, 1>();
  }
}

int batch_max_ctas_per_sm(int prec, int variant) {
  if (prec == 0) return occ_p<double, double>(variant);
  if (prec == 1) return occ_p<float, float>(variant);
  return occ_p<__half, float>(variant);
}

}  // namespace lbpc
