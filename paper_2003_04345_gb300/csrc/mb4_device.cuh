// Device-side helpers shared by the libmb4 kernel translation units: layouts,
// neighbour indexing, integer-pipe float/double conversions, programmatic
// dependent launch.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "mb4_internal.h"

namespace mb4 {

template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

// J coefficients at u0, pre-scaled by 1/theta: e1 = (d + chi(p^2 + 3q^2)), e2 = (d + chi(3p^2 + q^2)),
// a = 2 chi p q  (eq. JL + eq. JR with gamma = -chi).
template <typename T> struct alignas(4 * sizeof(T)) JCoef { T e1, e2, a, pad; };

struct Nbr { int xm, xp, ym, yp; };

// Programmatic dependent launch (griddepcontrol).  A kernel launched with
// programmatic stream serialisation can be scheduled once every block of its
// predecessor has called pdl_launch_dependents(); pdl_wait() then blocks until
// the predecessor grid has completed and its writes are visible.  Every kernel
// that may be launched this way calls pdl_wait() before it reads anything;
// without such a launch both calls do nothing.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch kern with programmatic stream serialisation when dep is set (the
// previous launch on the stream is a kernel whose results it waits for).
template <typename... KArgs, typename... Args>
void launch_k(bool dep, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dep ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

__device__ __forceinline__ Nbr neighbours(int k, int nx, int ny, int S) {
  int y = k / nx;
  int x = k - y * nx;
  Nbr n;
  n.xm = (x == 0) ? k + nx - 1 : k - 1;
  n.xp = (x == nx - 1) ? k - nx + 1 : k + 1;
  n.ym = (y == 0) ? k + S - nx : k - nx;
  n.yp = (y == ny - 1) ? k - S + nx : k + nx;
  return n;
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Float <-> double conversions on the integer pipe.  On this GPU the FP64 pipe
// is the scarce unit (about 1/59 of the FP32 rate) and a hardware conversion
// occupies it like several FP64 FMAs, so the kernels move values between the
// FP64 state and the FP32 Krylov solve by rearranging IEEE-754 bit fields.
//  - f2d_bits: exact for zero, normal floats, +-inf and NaN; FP32 subnormals
//    (below 1.2e-38) become +-0.
//  - d2f_trunc: rounds toward zero (relative error below 2^-23), which is
//    harmless for values that only feed the FP32 solve; magnitudes below the
//    FP32 normal range become +-0, above it +-inf; NaN stays NaN.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int sign = u & 0x80000000u;
  const unsigned int e = (u >> 23) & 0xffu;
  const unsigned int m = u & 0x7fffffu;
  unsigned int hi = sign | ((e + 896u) << 20) | (m >> 3);
  unsigned int lo = m << 29;
  if (e == 0u) { hi = sign; lo = 0u; }
  if (e == 255u) { hi = sign | 0x7ff00000u | (m ? 0x80000u : 0u); lo = 0u; }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  const unsigned int sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  unsigned int r = sign | ((unsigned int)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  if (e <= 0) r = sign;
  if (e >= 255) r = sign | 0x7f800000u;
  if ((hi & 0x7ff00000u) == 0x7ff00000u && ((hi & 0xfffffu) | lo)) r = 0x7fc00000u;
  return __uint_as_float(r);
}

// |x| of a double as a float (integer pipe, truncating): for max-norms.
__device__ __forceinline__ float absf_of(double x) {
  return d2f_trunc(__hiloint2double(__double2hiint(x) & 0x7fffffff, __double2loint(x)));
}

// A uniform constant in the Krylov precision: the host-made FP32 copy, or the FP64 value.
template <typename T> __device__ __forceinline__ T kval(double d, float f);
template <> __device__ __forceinline__ float kval<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double kval<double>(double d, float) { return d; }

template <typename T> __device__ __forceinline__ T from_double(double x);
template <> __device__ __forceinline__ float from_double<float>(double x) { return d2f_trunc(x); }
template <> __device__ __forceinline__ double from_double<double>(double x) { return x; }
template <typename T> __device__ __forceinline__ double to_double(T x);
template <> __device__ __forceinline__ double to_double<float>(float x) { return f2d_bits(x); }
template <> __device__ __forceinline__ double to_double<double>(double x) { return x; }
template <typename T> __device__ __forceinline__ float to_float(T x);
template <> __device__ __forceinline__ float to_float<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_float<double>(double x) { return d2f_trunc(x); }

// Arithmetic that the compiler never contracts or reorders: a*b + c rounded once (fma_)
// or twice (mul_ then add_).  The step's phases are inlined into two kernel forms (one
// launch per phase, or one persistent kernel); with plain expressions the compiler may fuse
// a multiply into an add in one form and not in the other, and the two would round
// differently.  Writing every product-sum explicitly makes both forms compute bit for bit
// the same.
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }

// Threads per block of the one-site-per-thread kernels: chosen per context (StepParams
// bs_*; the autotuner of the C ABI or 128), at most kSiteThreadsMax.  Their results do
// not depend on it: each site is computed alone and the only reductions are maxima.
constexpr int kSiteThreadsMax = 256;

// sum_j K_kj x_j over the off-diagonal of a general kinetic matrix in slot-major ELL
// form (nbr[e * S + k] = j or -1, w[e * S + k] = K_kj, e < deg), both parts of a
// complex plane x.
template <typename T, typename T2>
__device__ __forceinline__ T2 ell_offdiag(const int* __restrict__ nbr, const T* __restrict__ w, int deg, int S, int k,
                                          const T2* __restrict__ x) {
  T2 s;
  s.x = 0;
  s.y = 0;
  for (int e = 0; e < deg; ++e) {
    const int j = nbr[(size_t)e * S + k];
    if (j >= 0) {
      const T wv = w[(size_t)e * S + k];
      const T2 xv = x[j];
      s.x = fma_(wv, xv.x, s.x);
      s.y = fma_(wv, xv.y, s.y);
    }
  }
  return s;
}

// The same for a complex Hermitian K: w[e * S + k] = K_kj as (re, im), and the sum is
// the complex product sum_j K_kj x_j.
template <typename T, typename T2>
__device__ __forceinline__ T2 ell_offdiag_c(const int* __restrict__ nbr, const T2* __restrict__ w, int deg, int S,
                                            int k, const T2* __restrict__ x) {
  T2 s;
  s.x = 0;
  s.y = 0;
  for (int e = 0; e < deg; ++e) {
    const int j = nbr[(size_t)e * S + k];
    if (j >= 0) {
      const T2 wv = w[(size_t)e * S + k];
      const T2 xv = x[j];
      s.x = fma_(wv.x, xv.x, fma_(-wv.y, xv.y, s.x));
      s.y = fma_(wv.x, xv.y, fma_(wv.y, xv.x, s.y));
    }
  }
  return s;
}

// Offsets of instance b's data.
__device__ __forceinline__ size_t plane(int b, int S) { return (size_t)b * S; }
__device__ __forceinline__ size_t stage(int b, int m, int S) { return ((size_t)b * 3 + m) * S; }
__device__ __forceinline__ size_t level(int b, int a, int i, int s, int S) {
  return (((size_t)b * (s + 1) + a) * 3 + i) * S;
}

}  // namespace mb4
