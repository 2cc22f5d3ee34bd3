// FMA-throughput probe: the measured denominator of the ALU roofline of the binary64 step (and of
// binary32 work). It is not part of the method. Each thread runs eight independent FMA chains, so the
// FMA pipe and not the latency of one chain bounds the kernel; the grid fills every SM with as many
// CTAs as can be resident.
#include <stdint.h>

#include <cuda_runtime.h>

#include "../../include/lbpc.h"

#define LBPC_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ double g_probe_sink;  // written only if the chains reach an impossible value: keeps them live

template <class T> __global__ void __launch_bounds__(kThreads) k_fma_probe(int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
#pragma unroll 8
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s < T(-1)) g_probe_sink = double(s);  // the chains converge to c / (1 - b) > 0
}

template <class T> cudaError_t time_probe(int iters, cudaStream_t st, double* flop_per_s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, kThreads, 0);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  const T b = T(0.999999), c = T(1e-4);
  if (e == cudaSuccess) {
    k_fma_probe<T><<<blocks, kThreads, 0, st>>>(iters / 8 + 1, b, c);  // warm-up
    cudaEventRecord(ev[0], st);
    k_fma_probe<T><<<blocks, kThreads, 0, st>>>(iters, b, c);
    cudaEventRecord(ev[1], st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return e;
  if (!(ms > 0.f)) return cudaErrorUnknown;
  *flop_per_s = 2.0 * kChains * (double)iters * (double)blocks * kThreads / (ms * 1e-3);
  return cudaSuccess;
}

}  // namespace

LBPC_API lbpc_status lbpc_fma_rate(int32_t prec, void* stream, double* flop_per_s) {
  if (!flop_per_s) return LBPC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (prec == LBPC_FP64)
    e = time_probe<double>(8192, st, flop_per_s);  // about 30 ms at 1.2 TFLOP/s
  else if (prec == LBPC_FP32)
    e = time_probe<float>(262144, st, flop_per_s);  // about 60 ms at 70 TFLOP/s
  else
    return LBPC_EINVAL;
  return e == cudaSuccess ? LBPC_OK : LBPC_ECUDA;
}
