// Internal interfaces between the C-ABI layer (lbpc_api.cu) and the kernel files.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include "lbpc_device.cuh"

namespace lbpc {

// NVTX range over a host call of the library (NVTX v3 is header-only: without an attached profiler a
// range costs a check of a null function pointer). Profilers show and filter by these names.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

template <class S, int TX, int TY> struct TmaBox {
  static constexpr int XOFF = 16 / (int)sizeof(S) > 4 ? 16 / (int)sizeof(S) : 4;
  static constexpr int EPR = 16 / (int)sizeof(S);                // elements per 16 bytes
  static constexpr int BX = ((TX + XOFF + 3 + EPR - 1) / EPR) * EPR;
  static constexpr int BY = TY + 6;
  static constexpr int PLANE = ((BX * BY * (int)sizeof(S) + 127) / 128) * 128;  // bytes, 128-aligned
  static constexpr int REFX = ((TX + XOFF + 3 + 3) / 4) * 4;                    // float reference planes
  static constexpr int RPLANE = ((REFX * BY * 4 + 127) / 128) * 128;
  static constexpr bool HALF = is_half_t<S>::value;
  static constexpr int BYTES = 18 * PLANE + (HALF ? 2 * RPLANE : 0) + 128;       // + the mbarrier
};

struct alignas(64) TmaMaps {
  CUtensorMap f, g, rf, rg;  // current buffer's populations (3D) and FP16 reference planes (2D)
};


// Most tiles a fused or batched step launches over an nx x ny domain (the 32 x 8 tile, the smallest
// shape). A step with the domain-mean buoyancy writes one partial sum per tile, so the partials array
// holds at least this many; on narrow domains (nx < 4) it exceeds the 2 * ceil(N / 64) of the split step.
inline size_t fused_max_tiles(int nx, int ny) { return (size_t)((nx + 31) / 32) * (size_t)((ny + 7) / 8); }

// Fused-step tile configuration a new context starts with: 32 x 8 tiles, one node per thread, in
// persistent CTAs that stage each next tile early (the fastest measured on GB300 at 2048^2 - 8192^2 in
// FP32 and FP16).
constexpr int kDefaultFusedTile = 4;

// Device buffers of a context, carved from the caller's workspace.
struct SplitBuffers {
  void* f[2];        // populations f, post-collision layout, A/B (storage type)
  void* g[2];        // populations g
  float* ref_f[2];   // FP16 storage: per-node reference density of the stored f deviations (A/B)
  float* ref_g[2];   // FP16 storage: per-node reference temperature of the stored g deviations (A/B)
  double* wall[2] = {nullptr, nullptr};  // wall-row forces stored with f (A/B, wall_doubles(nx) each); null if y is periodic
  void* phi_prev;    // phi(t - dt), arithmetic type
  void* planes[16];  // scratch planes of the split kernels, arithmetic type
  double* partials;  // per-block (split) or per-tile (fused) partial sums: max(2 * nblocks, fused_max_tiles)
  double* scalars;   // [0] rho_ave, [1] mass, [2] heat
  long long* status; // [0] flag, [1] step, [2] x, [3] y, [4] code; [6] tile tickets of the persistent fused step
  const TmaMaps* tma[2] = {nullptr, nullptr};  // tensor maps of buffer A / B for the TMA-staged fused step
  int fused_tile = 1;  // 0: 32x16, 1: 32x8, 2: 32x16 two nodes per thread, 3: 32x32 two per thread (maps match)
};

// ev: null, or split_kernel_count(P) + 1 events recorded before the first and after each kernel.
cudaError_t split_step(const SplitBuffers& b, const DevParams& P, int prec, int cur, long long step, cudaStream_t st,
                       cudaEvent_t* ev = nullptr);
int split_kernel_count(const DevParams& P);
const char* split_kernel_name(int k);
cudaError_t split_init(const SplitBuffers& b, const DevParams& P, int prec, const double* rho, const double* T,
                       const double* ux, const double* uy, cudaStream_t st);
cudaError_t split_sums(const SplitBuffers& b, const DevParams& P, int prec, int cur, cudaStream_t st);
cudaError_t split_fields(const SplitBuffers& b, const DevParams& P, int prec, int cur, long long step, double* rho,
                         double* ux, double* uy, double* T, cudaStream_t st);
// which = 0: f, 1: g; only < 0: all 9 planes [9][N], else plane `only` into out[N].
cudaError_t split_export_pops(const SplitBuffers& b, const DevParams& P, int prec, int cur, int which, int only,
                              double* out, cudaStream_t st);
int split_nplanes();
int split_block();

// ---- batched step (lbpc_fused.cu kernels, lbpc_batch.cu host) ----
// One instance of a batch as the device sees it; S is the storage type of the batch.
template <class S> struct alignas(16) BatchInst {
  DevParams P;
  PopBuf<S> f[2], g[2];
  void* phi_prev;      // arithmetic type
  double* scalars;     // [0] rho_ave, [1] mass, [2] heat
  double* partials;    // per-tile partial sums of rho (buoyancy) and per-block sums
  long long* status;   // first non-physical node of this instance
  long long step;      // steps taken
  int cur;             // buffer holding the current state
  int active;
  int ntiles;          // tiles of this instance in the current work list
  int pad_;
};
struct BatchTile {
  int inst, x0, y0, pslot;
};
struct BatchMeta {
  const BatchTile* tiles;
  int ntiles;
  int ninst;  // instance slots (active or not)
};
// Step-kernel variants of a batch (tile shape and nodes per thread): 0 = 32x8, 1 = 32x16, 2 = 64x8
// with one node per thread; 3 = 32x16, 4 = 64x16, 5 = 32x32 with two nodes per thread.
constexpr int kBatchVariants = 6;
inline void batch_tile_shape(int v, int& tx, int& ty) {
  static const int TXS[kBatchVariants] = {32, 32, 64, 32, 64, 32}, TYS[kBatchVariants] = {8, 16, 8, 16, 16, 32};
  const int k = (v >= 0 && v < kBatchVariants) ? v : 0;
  tx = TXS[k];
  ty = TYS[k];
}
inline int batch_nodes_per_thread(int v) { return v >= 3 && v < kBatchVariants ? 2 : 1; }
// Enqueue one batched step (persistent step kernel + per-instance advance) on st.
cudaError_t batch_step_launch(int prec, int variant, int ctas, const BatchMeta* d_meta, void* d_insts, int ninst,
                              cudaStream_t st);

// Per-tile launches of a batched step (the configuration with 0 CTAs per SM): one CTA per tile, and the
// instances of a launch in its kernel parameters, so that the tile body reads every per-instance value
// and buffer pointer as a uniform operand, as the single-instance kernel does. A step is a sequence of
// such launches over the active instances (up to seg_capacity each), then the per-instance advance.
template <class S> struct ArithOf { using type = float; };  // arithmetic of a storage type in a batch
template <> struct ArithOf<double> { using type = double; };
template <class S> struct alignas(16) SegInst {
  DevParamsOf<typename ArithOf<S>::type> P;  // header and the one coefficient set the kernel reads
  PopBuf<S> fs, gs, fd, gd;  // this launch's source and destination populations
  void* phi_prev;            // arithmetic type
  double* scalars;
  double* partials;
  long long* status;
  const long long* step;     // the instance's step counter (in its device descriptor), read to report
  int tiles_x;               // tiles per row
  int first;                 // the instance's first step (its source term starts from phi itself)
};
constexpr size_t kSegParamBytes = 32000;  // within the 32,764 bytes of kernel parameters
template <class S> constexpr int seg_capacity() {
  return (int)((kSegParamBytes - 32) / (sizeof(SegInst<S>) + sizeof(int))) & ~3;
}
// Launches of few instances take a kernel with smaller parameters (measured 4 % faster on one 2048^2
// instance than the full-size parameters, which every launch copies).
constexpr int kSegSmall = 16;
template <class S, int CAP> struct SegLaunch {
  int n;      // instances of this launch
  int tiles;  // its CTAs
  int pad_[2];
  int first_tile[CAP];  // each instance's first CTA, ascending: kept together so that the search of a
                        // CTA's instance reads a few cache lines
  SegInst<S> in[CAP];
};
static_assert(sizeof(SegLaunch<double, seg_capacity<double>()>) <= kSegParamBytes &&
                  sizeof(SegLaunch<float, seg_capacity<float>()>) <= kSegParamBytes,
              "per-tile launch parameters");
// Enqueue one per-tile launch over the instances of L, a host SegLaunch<S, CAP> of the batch's storage
// type with CAP = kSegSmall (small) or seg_capacity<S>(). pdl: the launch may begin while the previous
// kernel on st drains (its instances are others).
cudaError_t batch_seg_launch(int prec, int variant, bool small, const void* L, bool pdl, cudaStream_t st);
// Enqueue the per-instance advance of a step (rho_ave, buffer parity, step count).
cudaError_t batch_advance_launch(int prec, void* d_insts, int ninst, cudaStream_t st);
// Largest resident CTAs per SM of the step kernel for (prec, variant).
int batch_max_ctas_per_sm(int prec, int variant);

// Fused single-kernel step (lbpc_fused.cu); same buffers, no scratch planes touched.
cudaError_t fused_step(const SplitBuffers& b, const DevParams& P, int prec, int cur, long long step, cudaStream_t st,
                       cudaEvent_t* ev = nullptr);
// Encode the tensor maps of one buffer (populations f, g and, for FP16, the reference planes) for the
// TMA-staged fused step; false when the layout does not allow TMA (row stride not 16-byte aligned).
bool fused_tma_encode(TmaMaps* m, int prec, int tile, void* f, void* g, float* rf, float* rg, const DevParams& P);
// rho_ave <- sum of n per-tile partials / N (fixed order), on st.
void fused_finish(const SplitBuffers& b, const DevParams& P, int n, cudaStream_t st);

}  // namespace lbpc
