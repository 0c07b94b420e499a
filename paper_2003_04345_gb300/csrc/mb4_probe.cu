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

constexpr int kProbeThreads = 256;

__device__ double g_probe_sink;    // keeps the chains' results live; written almost never

// NCH independent chains per thread of a = fma(a, b, c).  b and c differ per thread, so
// they live in registers like a real kernel's operands (not uniform constants).
template <int NCH>
__global__ void __launch_bounds__(kProbeThreads) k_fma_chains(int iters, double b0, double c0) {
  const double b = b0 + 1e-18 * threadIdx.x, c = c0 * (1.0 + 1e-12 * blockIdx.x);
  double a[NCH];
#pragma unroll
  for (int j = 0; j < NCH; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 128 / NCH; ++r)
#pragma unroll
      for (int j = 0; j < NCH; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < NCH; ++j) s += a[j];
  if (s == 1234.5678) g_probe_sink = s;      // never true for these inputs; the compiler cannot know
}

// Times one chain width: the launch is lengthened until it runs for about `seconds`.
template <int NCH>
int time_chains(double seconds, double* rate, double* elapsed) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MB4_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MB4_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_chains<NCH>, kProbeThreads, 0) != cudaSuccess ||
      occ < 1)
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
  int iters = 64;                   // 64 x 128 FMAs per thread; grown until the launch is long enough
  float ms = 0.f;
  for (int round = 0; round < 24; ++round) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kProbeThreads);
    cfg.stream = 0;
    if (cudaEventRecord(e0, 0) != cudaSuccess || cudaLaunchKernelEx(&cfg, k_fma_chains<NCH>, iters, b, c) != cudaSuccess ||
        cudaEventRecord(e1, 0) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = MB4_ERR_CUDA;
      break;
    }
    if (ms >= 1e3 * seconds || iters >= (1 << 24)) break;
    const double grow = (ms > 0.f) ? (1e3 * seconds) / ms : 16.0;
    iters = (int)std::min<double>((double)(1 << 24), iters * std::min(16.0, std::max(2.0, 1.05 * grow)));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MB4_OK) return rc;
  if (!(ms > 0.f)) return MB4_ERR_CUDA;
  const double flops = 2.0 * 128.0 * (double)iters * (double)blocks * kProbeThreads;
  *rate = flops / (1e-3 * ms);
  *elapsed = 1e-3 * ms;
  return MB4_OK;
}

}  // namespace

extern "C" int mb4_fp64_fma_rate(double seconds, double* flops_per_s, double* elapsed_s) {
  if (!flops_per_s || !(seconds > 0.0) || seconds > 10.0) return MB4_ERR_INVALID_ARG;
  // two chain widths, each for half the time; the faster is the device's rate
  double r8 = 0.0, t8 = 0.0, r16 = 0.0, t16 = 0.0;
  int rc = time_chains<8>(0.5 * seconds, &r8, &t8);
  if (rc != MB4_OK) return rc;
  rc = time_chains<16>(0.5 * seconds, &r16, &t16);
  if (rc != MB4_OK) return rc;
  *flops_per_s = std::max(r8, r16);
  if (elapsed_s) *elapsed_s = (r8 >= r16) ? t8 : t16;
  return MB4_OK;
}
