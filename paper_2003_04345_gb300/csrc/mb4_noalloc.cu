// mb4_observables_noalloc: the observables reduction for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at the moment they need an energy or a
// norm: code running under a memory pool or allocator that owns all device
// memory (for example a framework's caching allocator with a fixed budget),
// code inside a region where new allocations would break its memory plan, or
// hosts that forbid the implicit synchronisation cudaMalloc/cudaFree can
// cause.  This entry point needs no context and allocates nothing: the
// per-block partial sums live in a file-scope device array that is part of
// the library image, loaded once per GPU and kept until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "mb4_internal.h"

namespace {

constexpr int kNaBlocks = 256;   // grid of the partial-sum kernel (fixed, any S)
constexpr int kNaObs = 6;        // H, U_K, U_E, U_nl, sum|u|^2, sum|u|^4
constexpr int kNaThreads = 256;

// Scratch: one (sum, compensation) pair per observable and block,
// 256 x 6 x 2 doubles = 24 KiB.  Every block overwrites its own slot on every
// call, so nothing in it has to start at zero.
static __device__ __align__(256) double g_na_scratch[kNaBlocks * kNaObs * 2];

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
void* g_na_ptr[kMaxDevices] = {};

// Device address of g_na_scratch on the current device (looked up once per device and
// kept: a cudaDeviceReset, which unloads the library image from the device, makes the
// kept address stale, so the entry point may not be used after one).
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MB4_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return MB4_ERR_CUDA;
    g_na_ptr[dev] = p;
  }
  *out = static_cast<double*>(g_na_ptr[dev]);
  return MB4_OK;
}

struct NaSum { double s, c; };

__device__ __forceinline__ void na_add(NaSum& a, double x) {   // TwoSum into (s, c)
  const double t = __dadd_rn(a.s, x);
  const double bp = __dsub_rn(t, a.s);
  const double err = __dadd_rn(__dsub_rn(a.s, __dsub_rn(t, bp)), __dsub_rn(x, bp));
  a.s = t;
  a.c = __dadd_rn(a.c, err);
}
__device__ __forceinline__ NaSum na_merge(NaSum a, NaSum b) {
  na_add(a, b.s);
  a.c = __dadd_rn(a.c, b.c);
  return a;
}

// Per-block compensated partial sums of the energy terms (Sec. 2.1: U_K = u^H K u,
// U_E = u^H V u, U_nl = (chi/2) sum |u|^4) and of sum |u|^2, sum |u|^4, reading the
// state as two planes.
__global__ void __launch_bounds__(kNaThreads) k_obs_planar(int nx, int ny, double tx, double ty, double onsite,
                                                           double chi, const double* __restrict__ re,
                                                           const double* __restrict__ im,
                                                           const double* __restrict__ V,
                                                           double* __restrict__ scratch) {
  const int S = nx * ny;
  NaSum acc[kNaObs];
#pragma unroll
  for (int o = 0; o < kNaObs; ++o) acc[o].s = acc[o].c = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S; k += gridDim.x * blockDim.x) {
    const int y = k / nx, x = k - y * nx;
    const int xm = (x == 0) ? k + nx - 1 : k - 1, xp = (x == nx - 1) ? k - nx + 1 : k + 1;
    const int ym = (y == 0) ? k + S - nx : k - nx, yp = (y == ny - 1) ? k - S + nx : k + nx;
    const double p = re[k], q = im[k];
    const double Kp = fma(-ty, re[ym] + re[yp], fma(-tx, re[xm] + re[xp], onsite * p));
    const double Kq = fma(-ty, im[ym] + im[yp], fma(-tx, im[xm] + im[xp], onsite * q));
    const double tK = fma(p, Kp, q * Kq);
    const double n = fma(p, p, q * q);
    const double tE = V[k] * n;
    const double tI = 0.5 * chi * n * n;
    na_add(acc[0], tK);
    na_add(acc[0], tE);
    na_add(acc[0], tI);
    na_add(acc[1], tK);
    na_add(acc[2], tE);
    na_add(acc[3], tI);
    na_add(acc[4], n);
    na_add(acc[5], n * n);
  }
  __shared__ NaSum red[kNaThreads / 32][kNaObs];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 0; o < kNaObs; ++o) {
    NaSum r = acc[o];
    for (int off = 16; off > 0; off >>= 1) {
      NaSum t;
      t.s = __shfl_xor_sync(0xffffffffu, r.s, off);
      t.c = __shfl_xor_sync(0xffffffffu, r.c, off);
      r = na_merge(r, t);
    }
    if (lane == 0) red[warp][o] = r;
  }
  __syncthreads();
  if (threadIdx.x < kNaObs) {
    NaSum r = red[0][threadIdx.x];
    for (int w = 1; w < kNaThreads / 32; ++w) r = na_merge(r, red[w][threadIdx.x]);
    scratch[((size_t)blockIdx.x * kNaObs + threadIdx.x) * 2 + 0] = r.s;
    scratch[((size_t)blockIdx.x * kNaObs + threadIdx.x) * 2 + 1] = r.c;
  }
}

// Sum the block partials in block order and write the six observables.
__global__ void k_obs_planar_final(const double* __restrict__ scratch, double* __restrict__ out6) {
  const int o = threadIdx.x;
  if (o >= kNaObs) return;
  NaSum r;
  r.s = r.c = 0.0;
  for (int b = 0; b < kNaBlocks; ++b) {
    NaSum t;
    t.s = scratch[((size_t)b * kNaObs + o) * 2 + 0];
    t.c = scratch[((size_t)b * kNaObs + o) * 2 + 1];
    r = na_merge(r, t);
  }
  out6[o] = r.s + r.c;
}

}  // namespace

extern "C" int mb4_observables_noalloc(int nx, int ny, double tx, double ty, double onsite, double chi,
                                       const double* re, const double* im, const double* v, double* out6,
                                       void* stream) {
  if (nx < 3 || ny < 3) return MB4_ERR_INVALID_ARG;
  if ((long long)nx * (long long)ny > (long long)MB4_NOALLOC_MAX_SITES) return MB4_ERR_INVALID_ARG;
  if (!re || !im || !v || !out6) return MB4_ERR_INVALID_ARG;
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != MB4_OK) return rc;
  // Each launch is checked through its own return code, so an error the caller left
  // pending is neither reported as this call's nor cleared.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kNaBlocks);
  cfg.blockDim = dim3(kNaThreads);
  cfg.stream = static_cast<cudaStream_t>(stream);
  if (cudaLaunchKernelEx(&cfg, k_obs_planar, nx, ny, tx, ty, onsite, chi, re, im, v, scratch) != cudaSuccess)
    return MB4_ERR_CUDA;
  cfg.gridDim = dim3(1);
  cfg.blockDim = dim3(32);
  if (cudaLaunchKernelEx(&cfg, k_obs_planar_final, (const double*)scratch, out6) != cudaSuccess) return MB4_ERR_CUDA;
  return MB4_OK;
}
