// cbs_probe.cu -- measurement support for the benchmark's rooflines (not part
// of the method): the FP64 fused multiply-add throughput of the device.
//
// Every thread runs kChains independent chains x <- fma(x, m, c) in
// registers (no memory traffic, enough independent work per warp to cover
// the FP64 pipe's latency); the grid fills every SM with 4 CTAs of 256
// threads.  Timed with CUDA events after a warm-up launch.
#include <cuda_runtime.h>

#include <string>

#include "cbs_plan_struct.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_probe(double* sink, int iters, double m, double c) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = fma(x[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += x[k];
  if (s == 1234.5) sink[blockIdx.x] = s;  // keeps the chains alive; never true for these m, c
}

}  // namespace

extern "C" cbs_status cbs_probe_fp64_peak(double* tflops) {
  if (!tflops) return cbs::set_error(CBS_ERR_INVALID_ARG, "null argument");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(double) * 4 * sms);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int iters = 1 << 14, blocks = 4 * sms, threads = 256;
  float ms = 0.f;
  if (e == cudaSuccess) {
    fp64_fma_probe<<<blocks, threads>>>(sink, iters, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(e0);
    fp64_fma_probe<<<blocks, threads>>>(sink, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cbs::set_error(CBS_ERR_CUDA, std::string("FP64 probe: ") + cudaGetErrorString(e));
  const double flops = 2.0 * kChains * (double)iters * blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return CBS_OK;
}
