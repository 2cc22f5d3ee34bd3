// Internal interfaces between the C-ABI layer (lbpc_api.cu) and the kernel files.
#pragma once

#include <cuda_runtime.h>

#include "lbpc_device.cuh"

namespace lbpc {

// Device buffers of a context, carved from the caller's workspace.
struct SplitBuffers {
  void* f[2];        // populations f, post-collision layout, A/B (storage type)
  void* g[2];        // populations g
  float* ref_f[2];   // FP16 storage: per-node reference density of the stored f deviations (A/B)
  float* ref_g[2];   // FP16 storage: per-node reference temperature of the stored g deviations (A/B)
  void* phi_prev;    // phi(t - dt), arithmetic type
  void* planes[16];  // scratch planes of the split kernels, arithmetic type
  double* partials;  // 2 * nblocks per-block partial sums
  double* scalars;   // [0] rho_ave, [1] mass, [2] heat
  long long* status; // [0] flag, [1] step, [2] x, [3] y, [4] code
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

// Fused single-kernel step (lbpc_fused.cu); same buffers, no scratch planes touched.
cudaError_t fused_step(const SplitBuffers& b, const DevParams& P, int prec, int cur, long long step, cudaStream_t st,
                       cudaEvent_t* ev = nullptr);
// rho_ave <- sum of n per-tile partials / N (fixed order), on st.
void fused_finish(const SplitBuffers& b, const DevParams& P, int n, cudaStream_t st);

}  // namespace lbpc
