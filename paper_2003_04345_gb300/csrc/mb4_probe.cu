// mb4_fp64_fma_rate: the FP64 FMA throughput of the current device, measured.
//
// The step's FP64 kernels are bound by the FP64 pipe, not by memory, so their
// roofline is the FP64 rate.  The nominal figure (SMs x clock x FMAs per clock)
// assumes the maximum clock; this probe measures what the device delivers at the
// clock it runs at: every thread runs independent chains of dependent FP64 FMAs
// (enough chains and warps to keep the pipe full), with no memory traffic.  The
// paper has no counterpart: this is a measurement service of the library.
#include <cuda_runtime.h>

#include <algorithm>

#include "mb4_internal.h"

namespace {

constexpr int kChains = 8;         // independent FMA chains per thread
constexpr int kProbeThreads = 256;

__device__ double g_probe_sink;    // keeps the chains' results live; written almost never

__global__ void __launch_bounds__(kProbeThreads) k_fma_chains(int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 1234.5678) g_probe_sink = s;      // never true for these inputs; the compiler cannot know
}

}  // namespace

extern "C" int mb4_fp64_fma_rate(double seconds, double* flops_per_s, double* elapsed_s) {
  if (!flops_per_s || !(seconds > 0.0) || seconds > 10.0) return MB4_ERR_INVALID_ARG;
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MB4_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MB4_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_chains, kProbeThreads, 0) != cudaSuccess || occ < 1)
    return MB4_ERR_CUDA;
  const int blocks = sms * occ;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return MB4_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MB4_ERR_CUDA;
  }
  int rc = MB4_OK;
  // b slightly below 1 and c small keep every chain near its fixed point c / (1 - b):
  // normal numbers throughout, no overflow, no denormals.
  const double b = 0.9999999, c = 1e-7;
  int iters = 64;                   // 64 x 16 x 8 FMAs per thread; grown until the launch is long enough
  float ms = 0.f;
  for (int round = 0; round < 24 && rc == MB4_OK; ++round) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kProbeThreads);
    cfg.stream = 0;
    if (cudaEventRecord(e0, 0) != cudaSuccess || cudaLaunchKernelEx(&cfg, k_fma_chains, iters, b, c) != cudaSuccess ||
        cudaEventRecord(e1, 0) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = MB4_ERR_CUDA;
      break;
    }
    if (ms >= 1e3 * seconds || iters >= (1 << 26)) break;
    const double grow = (ms > 0.f) ? (1e3 * seconds) / ms : 16.0;
    iters = (int)std::min<double>((double)(1 << 26), iters * std::min(16.0, std::max(2.0, 1.05 * grow)));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MB4_OK) return rc;
  if (!(ms > 0.f)) return MB4_ERR_CUDA;
  const double flops = 2.0 * kChains * 16.0 * (double)iters * (double)blocks * kProbeThreads;
  *flops_per_s = flops / (1e-3 * ms);
  if (elapsed_s) *elapsed_s = 1e-3 * ms;
  return MB4_OK;
}
