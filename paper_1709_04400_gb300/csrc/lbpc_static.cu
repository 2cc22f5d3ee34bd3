// lbpc_step_static: one time step whose scratch lives in a fixed device array of the library, for
// callers that cannot allocate device memory (see include/lbpc.h). The kernels are the split step's;
// only where their scratch comes from differs.
#include <stdint.h>

#include <cuda_runtime.h>

#include "../../include/lbpc.h"
#include "lbpc_internal.h"

#define LBPC_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr long long kMaxNodes = LBPC_STATIC_MAX_NODES;
constexpr int kPlanes = 12;                      // the scratch planes of the split step
constexpr long long kPartials = 2 * ((kMaxNodes + 63) / 64);
constexpr long long kStatusDoubles = 8;
constexpr long long kDoubles = kPlanes * kMaxNodes + kPartials + kStatusDoubles;

// The scratch itself. Every GPU that loads the library holds it (about 6 MiB) until the process exits.
// In host code this name is only a host-side stand-in for the device symbol: its device address comes
// from cudaGetSymbolAddress below, in the device context current at each call.
static __device__ __align__(256) double g_scratch[kDoubles];

// Device address of the scratch in the current device context. It is looked up on every call, not
// cached: a device reset creates a new context in which the module, and with it the array, may sit at
// another address. Under lazy module loading the first lookup in a context loads the module.
cudaError_t scratch_on_current_device(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return e;
  *out = (double*)p;
  return cudaSuccess;
}

}  // namespace

namespace lbpc {
DevParams make_dev_params_public(const lbpc_params* p);
}

LBPC_API lbpc_status lbpc_step_static(const lbpc_params* p, const void* f_in, const void* g_in, void* f_out,
                                      void* g_out, const double* wall_in, double* wall_out, void* phi_prev,
                                      double* rho_ave, int64_t step, void* stream) {
  if (lbpc_check_params(p, nullptr, 0) != LBPC_OK) return LBPC_EINVAL;
  if (p->prec == LBPC_FP16DEV) return LBPC_EINVAL;  // FP16 storage needs reference planes this call does not take
  const long long N = (long long)p->nx * p->ny;
  if (N > kMaxNodes) return LBPC_ENOMEM;  // beyond the static scratch: use lbpc_create with a workspace
  if (!f_in || !g_in || !f_out || !g_out || !phi_prev || step < 0) return LBPC_EINVAL;
  if (p->buoyancy == 1 && !rho_ave) return LBPC_EINVAL;
  if (f_in == f_out || g_in == g_out) return LBPC_EINVAL;
  const bool walls = p->flow_bc[2] == LBPC_WALL || p->flow_bc[3] == LBPC_WALL;
  if (walls && (!wall_in || !wall_out || wall_in == wall_out)) return LBPC_EINVAL;
  if (lbpc::split_nplanes() > kPlanes) return LBPC_ECUDA;
  double* s = nullptr;
  if (scratch_on_current_device(&s) != cudaSuccess) return LBPC_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;

  const lbpc::DevParams dp = lbpc::make_dev_params_public(p);
  lbpc::SplitBuffers b{};
  b.f[0] = (void*)f_in;
  b.g[0] = (void*)g_in;
  b.f[1] = f_out;
  b.g[1] = g_out;
  b.wall[0] = walls ? (double*)wall_in : nullptr;  // read only: the step writes the other parity
  b.wall[1] = walls ? wall_out : nullptr;
  b.phi_prev = phi_prev;
  for (int k = 0; k < lbpc::split_nplanes() && k < kPlanes; ++k) b.planes[k] = s + (long long)k * kMaxNodes;
  b.partials = s + kPlanes * kMaxNodes;
  b.status = (long long*)(s + kPlanes * kMaxNodes + kPartials);
  b.scalars = rho_ave;  // the step reads rho_ave[0] and, with buoyancy, writes this step's mean back

  // the status word keeps the last call's contents: clear it before the step
  if (cudaMemsetAsync(b.status, 0, kStatusDoubles * sizeof(double), st) != cudaSuccess) return LBPC_ECUDA;
  if (lbpc::split_step(b, dp, p->prec, 0, (long long)step, st, nullptr) != cudaSuccess) return LBPC_ECUDA;
  long long status[5] = {0, 0, 0, 0, 0};
  if (cudaMemcpyAsync(status, b.status, sizeof status, cudaMemcpyDeviceToHost, st) != cudaSuccess) return LBPC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LBPC_ECUDA;
  return status[0] ? LBPC_ENONPHYS : LBPC_OK;
}
