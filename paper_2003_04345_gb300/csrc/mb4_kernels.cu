// libmb4 kernels: MB4 steps for a batch of B independent instances of one grid
// shape on the device (sm_103a).  A single context is a batch of one.
//
// Data layout: complex planes are interleaved (re, im) pairs, site k = y*nx + x;
// every per-instance array is instance-major (instance b's planes are
// contiguous).  The Newton iteration runs in the eigenbasis of E on the stage
// increments dU = T^-1 (U - e3 (x) u0) (Sec. 2.2, eq. MB4_4..MB4_6): the T and
// T^-1 mixes of Algorithm 1 then fold into constants, the linear part of the
// residual needs only one stencil per stage (T^-1 E T = Lambda), the update is
// dU += rbar, and the step is u1 = u0 + sum_n T[2][n] dU_n.  Carrying
// increments keeps the identity part of the step exact: with the constants
// rounded to FP64, u1 = sum_n T[2][n] Ubar_n would scale every step by
// T[2] . T^-1 1 = 1 - O(1e-16) and the energy would drift linearly in time.
// Each instance keeps its own Newton status; an instance that has converged
// (or failed) is masked while the others iterate.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "mb4_device.cuh"
#include "mb4_internal.h"
#include "mb4_phases.cuh"

namespace cg = cooperative_groups;

namespace mb4 {

template <typename TK, bool ELL>
__global__ void __launch_bounds__(kSiteThreadsMax) k_setup(StepParams p, const double2* __restrict__ u,
                                               const double* __restrict__ D, double2* __restrict__ S0,
                                               JCoef<TK>* __restrict__ jc, typename Vec2<TK>::type* __restrict__ v,
                                               const double2* __restrict__ dUh, double2* __restrict__ dUb,
                                               const double* __restrict__ p_chi,
                                               const InstConst* __restrict__ ic, InstStatus* is) {
  const int b = blockIdx.y;
  if (!is[b].active) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const float m = (k < p.S) ? setup_site<TK, ELL>(p, u, D, S0, jc, v, dUh, dUb, p_chi, ic[b], is[b], b, k) : 0.f;
  block_max_into(m, &is[b].u0max_bits);
}

template <typename TK>
void launch_setup(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  dim3 grid((p.S + p.bs_site - 1) / p.bs_site, p.B);
  if (p.ell)
    k_setup<TK, true><<<grid, p.bs_site, 0, s>>>(p, b.u, b.d, b.S0, (JCoef<TK>*)b.jc, (typename Vec2<TK>::type*)b.v,
                                                 b.dU_hist, b.Ubar, b.chi, b.ic, b.is);
  else
    k_setup<TK, false><<<grid, p.bs_site, 0, s>>>(p, b.u, b.d, b.S0, (JCoef<TK>*)b.jc, (typename Vec2<TK>::type*)b.v,
                                                  b.dU_hist, b.Ubar, b.chi, b.ic, b.is);
}

template <typename TO, bool CHIF, int KM>
__global__ void __launch_bounds__(kSiteThreadsMax) k_residual(StepParams p, const double2* __restrict__ u,
                                                  const double* __restrict__ D, const double2* __restrict__ S0,
                                                  const double2* __restrict__ dUb,
                                                  typename Vec2<TO>::type* __restrict__ out, long long out_stride,
                                                  int skip_first, const double* __restrict__ p_chi,
                                                  const InstConst* __restrict__ ic, const InstStatus* is) {
  pdl_wait();
  pdl_launch_dependents();
  const int b = blockIdx.y;
  if (!is[b].active) return;
  if (skip_first && is[b].newton_iter == 0 && !is[b].predicted) return;   // b^0 was written by k_setup
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.S) return;
  residual_site<TO, CHIF, KM>(p, u, D, S0, dUb, out, out_stride, p_chi, ic[b], b, k);
}

// Kinetic mode of the residual and the FP64 basis (template argument KM).
inline int kin_mode(const StepParams& p) { return p.ell ? (p.ell_cplx ? 3 : 2) : (p.kin_unit ? 1 : 0); }

template <typename TK>
void launch_residual(const StepParams& p, const DevBuffers& b, bool skip_first, cudaStream_t s) {
  dim3 grid((p.S + p.bs_residual - 1) / p.bs_residual, p.B);
  // b_i of instance b goes to its level 0: level(b, 0, i) = b*(s+1)*3*S + i*S
  typedef typename Vec2<TK>::type TK2;
  const long long os = (long long)(p.s + 1) * 3 * p.S;
  const int sf = skip_first ? 1 : 0;
  const double* D = p.kin_unit ? b.dtx : b.d;
#define MB4_RES(CF, KM)                                                                                     \
  launch_k(p.pdl != 0, k_residual<TK, CF, KM>, grid, dim3(p.bs_residual), 0, s, p, (const double2*)b.u, D,     \
           (const double2*)b.S0, (const double2*)b.Ubar, (TK2*)b.v, os, sf, (const double*)b.chi,               \
           (const InstConst*)b.ic, (const InstStatus*)b.is)
  switch (kin_mode(p)) {
    case 3: if (p.chi_field) MB4_RES(true, 3); else MB4_RES(false, 3); break;
    case 2: if (p.chi_field) MB4_RES(true, 2); else MB4_RES(false, 2); break;
    case 1: if (p.chi_field) MB4_RES(true, 1); else MB4_RES(false, 1); break;
    default: if (p.chi_field) MB4_RES(true, 0); else MB4_RES(false, 0); break;
  }
#undef MB4_RES
}

template <typename TK>
void launch_residual_out(const StepParams& p, const DevBuffers& b, double2* phibar3, cudaStream_t s) {
  dim3 grid((p.S + p.bs_residual - 1) / p.bs_residual, p.B);
  const double* D = p.kin_unit ? b.dtx : b.d;
#define MB4_RES(CF, KM) \
  k_residual<double, CF, KM><<<grid, p.bs_residual, 0, s>>>(p, b.u, D, b.S0, b.Ubar, phibar3, 3LL * p.S, 0, b.chi, \
                                                            b.ic, b.is)
  switch (kin_mode(p)) {
    case 3: if (p.chi_field) MB4_RES(true, 3); else MB4_RES(false, 3); break;
    case 2: if (p.chi_field) MB4_RES(true, 2); else MB4_RES(false, 2); break;
    case 1: if (p.chi_field) MB4_RES(true, 1); else MB4_RES(false, 1); break;
    default: if (p.chi_field) MB4_RES(true, 0); else MB4_RES(false, 0); break;
  }
#undef MB4_RES
}

template <typename TK, int KM>
__global__ void __launch_bounds__(kSiteThreadsMax) k_matvec(StepParams p, const JCoef<TK>* __restrict__ jc,
                                                typename Vec2<TK>::type* __restrict__ v, int a_in,
                                                const InstConst* __restrict__ ic, const InstStatus* is) {
  // Before the wait for the predecessor: the status and the J coefficients, which this step's
  // set-up wrote and no kernel after it changes (the predecessor of a basis launch is a
  // residual or a basis launch, and both start only after the set-up and the last loop test
  // have completed).
  const int b = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool go = is[b].active && k < p.S;
  JCoef<TK> j;
  if (go) j = jc[plane(b, p.S) + k];
  pdl_wait();
  pdl_launch_dependents();
  if (!go) return;
  matvec_site_j<TK, KM>(p, j, v, a_in, ic[b], b, k);
}

template <int SK, int TX, int TY, int FORM>
__global__ void __launch_bounds__(kPowThreads) k_powers(StepParams p, const float4* __restrict__ jc,
                                                        float2* __restrict__ v, const InstConst* __restrict__ ic,
                                                        const InstStatus* is) {
  pdl_wait();
  pdl_launch_dependents();
  const int b = blockIdx.y;
  if (!is[b].active) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if constexpr (FORM == 1) powers_tile_rows<SK, TX, TY>(p, jc, v, ic[b], b, blockIdx.x, smem_raw);
  else if constexpr (FORM == 2) powers_tile_sys<SK, TX, TY>(p, jc, v, ic[b], b, blockIdx.x, smem_raw);
  else powers_tile<SK, TX, TY>(p, jc, v, ic[b], b, blockIdx.x, smem_raw);
}

// One warp per tile (form 3): kPowWarpsPerBlock tiles per block, no shared memory.
template <int SK, int TY>
__global__ void __launch_bounds__(32 * kPowWarpsPerBlock, TY <= 4 ? 4 : 3)
    k_powers_warp(StepParams p, const float4* __restrict__ jc, float2* __restrict__ v,
                  const InstConst* __restrict__ ic, const InstStatus* is, int ntiles) {
  pdl_wait();
  pdl_launch_dependents();
  const int b = blockIdx.y;
  if (!is[b].active) return;
  const int tile = blockIdx.x * kPowWarpsPerBlock + (threadIdx.x >> 5);
  if (tile >= ntiles) return;                    // whole warps leave: the shuffles see full warps
  powers_warp<SK, TY>(p, jc, v, ic[b], b, tile);
}

template <typename TK, int SK, int CL>
__global__ void __launch_bounds__(256) k_gram_lsq(StepParams p, const typename Vec2<TK>::type* __restrict__ v,
                                                  double* __restrict__ part, double* __restrict__ coef,
                                                  const InstConst* __restrict__ ic, InstStatus* is) {
  pdl_wait();
  pdl_launch_dependents();
  const int inst = blockIdx.z;
  if (!is[inst].active) return;
  constexpr int NV = SK + 1;
  constexpr int NE = NV * (NV + 1) / 2;
  const int i = blockIdx.y;
  __shared__ double blk[NE];
  __shared__ bool is_last;
  gram_accumulate<TK, SK>(p, v, inst, i, blockIdx.x, gridDim.x, blk);
  const int nb = gridDim.x / CL;                 // partials of system i
  double* pi = part + ((size_t)inst * 3 + i) * nb * NE;
  bool leader = true;
  if (CL > 1) {
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();                              // members' blk[] complete and visible
    leader = (cluster.block_rank() == 0);
    if (leader) {
      for (int e = threadIdx.x; e < NE; e += blockDim.x) {
        double t = 0.0;
        for (int r = 0; r < CL; ++r) t += cluster.map_shared_rank(blk, r)[e];
        pi[(size_t)(blockIdx.x / CL) * NE + e] = t;
      }
    }
    cluster.sync();                              // members stay resident until read
  } else {
    for (int e = threadIdx.x; e < NE; e += blockDim.x) pi[(size_t)blockIdx.x * NE + e] = blk[e];
  }
  if (!leader) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(&is[inst].ticket_gram[i], 1u);
    is_last = (t == (unsigned int)(nb - 1));
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  gram_lsq_solve<SK>(p, part, coef, ic, is, inst, i, nb);
}

// One warp per strip of H rows (form 4).
// Two rows of loads in flight and 4 blocks (16 warps) per SM: measured at 2048^2 against
// no prefetch (126 us per launch), and against 3 blocks per SM with 2 or 3 rows ahead
// (128, 124 us): 117 us.
template <int SK, int H>
__global__ void __launch_bounds__(32 * kPowWarpsPerBlock, 4)
    k_powers_stream(StepParams p, const float4* __restrict__ jc, float2* __restrict__ v,
                    const InstConst* __restrict__ ic, const InstStatus* is, int nstrips) {
  pdl_wait();
  pdl_launch_dependents();
  const int b = blockIdx.y;
  if (!is[b].active) return;
  const int strip = blockIdx.x * kPowWarpsPerBlock + (threadIdx.x >> 5);
  if (strip >= nstrips) return;                  // whole warps leave: the shuffles see full warps
  powers_stream<SK, H, 2>(p, jc, v, ic[b], b, strip);
}

// One warp per strip, rows staged through shared memory (form 5).
template <int SK, int H>
__global__ void __launch_bounds__(32 * kPowWarpsPerBlock, 4)
    k_powers_stream_cp(StepParams p, const float4* __restrict__ jc, float2* __restrict__ v,
                       const InstConst* __restrict__ ic, const InstStatus* is, int nstrips) {
  pdl_wait();
  pdl_launch_dependents();
  const int b = blockIdx.y;
  if (!is[b].active) return;
  const int strip = blockIdx.x * kPowWarpsPerBlock + (threadIdx.x >> 5);
  if (strip >= nstrips) return;                  // whole warps leave: the shuffles see full warps
  extern __shared__ __align__(16) unsigned char smem_raw[];
  powers_stream_cp<SK, H, kPowStreamAhead>(p, jc, v, ic[b], b, strip,
                                           smem_raw + (threadIdx.x >> 5) * pow_cp_warp_bytes<kPowStreamAhead>());
}

template <int SK, int SH>
void launch_powers_shape(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  constexpr int TX = kPowShapeTX[SH], TY = kPowShapeTY[SH];
  constexpr int F = kPowShapeForm[SH];
  if constexpr (F >= 3) {
    constexpr int WX = 32 - 2 * SK;              // the warp's interior width
    const int ntiles = ((p.nx + WX - 1) / WX) * ((p.ny + TY - 1) / TY);
    dim3 grid((ntiles + kPowWarpsPerBlock - 1) / kPowWarpsPerBlock, p.B);
    if constexpr (F == 3)
      launch_k(p.pdl != 0, k_powers_warp<SK, TY>, grid, dim3(32 * kPowWarpsPerBlock), 0, s, p, (const float4*)b.jc,
               (float2*)b.v, (const InstConst*)b.ic, (const InstStatus*)b.is, ntiles);
    else if constexpr (F == 4)
      launch_k(p.pdl != 0, k_powers_stream<SK, TY>, grid, dim3(32 * kPowWarpsPerBlock), 0, s, p, (const float4*)b.jc,
               (float2*)b.v, (const InstConst*)b.ic, (const InstStatus*)b.is, ntiles);
    else
      launch_k(p.pdl != 0, k_powers_stream_cp<SK, TY>, grid, dim3(32 * kPowWarpsPerBlock),
               kPowWarpsPerBlock * pow_cp_warp_bytes<kPowStreamAhead>(), s, p, (const float4*)b.jc, (float2*)b.v,
               (const InstConst*)b.ic, (const InstStatus*)b.is, ntiles);
  } else {
    dim3 grid(((p.nx + TX - 1) / TX) * ((p.ny + TY - 1) / TY), p.B);
    launch_k(p.pdl != 0, k_powers<SK, TX, TY, F>, grid, dim3(kPowThreads),
             pow_smem_bytes<SK, TX, TY, F == 2 ? 1 : 3>(), s, p, (const float4*)b.jc, (float2*)b.v,
             (const InstConst*)b.ic, (const InstStatus*)b.is);
  }
}

template <int SK>
void launch_powers_s(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  if constexpr (SK <= kPowShapeMaxS) {
    switch (p.pow_shape) {
      case 1: launch_powers_shape<SK, 1>(p, b, s); return;
      case 2: launch_powers_shape<SK, 2>(p, b, s); return;
      case 3: launch_powers_shape<SK, 3>(p, b, s); return;
      case 4: launch_powers_shape<SK, 4>(p, b, s); return;
      case 5: launch_powers_shape<SK, 5>(p, b, s); return;
      case 6: launch_powers_shape<SK, 6>(p, b, s); return;
      case 7: launch_powers_shape<SK, 7>(p, b, s); return;
      case 8: launch_powers_shape<SK, 8>(p, b, s); return;
      case 9: launch_powers_shape<SK, 9>(p, b, s); return;
      case 10: launch_powers_shape<SK, 10>(p, b, s); return;
      case 11: launch_powers_shape<SK, 11>(p, b, s); return;
      case 12: launch_powers_shape<SK, 12>(p, b, s); return;
      case 13: launch_powers_shape<SK, 13>(p, b, s); return;
      default: break;
    }
  }
  launch_powers_shape<SK, 0>(p, b, s);
}

// Opt the matrix-powers kernels into more than 48 KB of dynamic shared memory.
template <int SK, int SH>
bool powers_attr() {
  constexpr int TX = kPowShapeTX[SH], TY = kPowShapeTY[SH];
  constexpr int F = kPowShapeForm[SH];
  if constexpr (F == 3 || F == 4) return true;   // no shared memory
  else if constexpr (F == 5)                     // the per-warp rings: under the 48 KB default
    return kPowWarpsPerBlock * pow_cp_warp_bytes<kPowStreamAhead>() <= 48 * 1024;
  else
    return cudaFuncSetAttribute(k_powers<SK, TX, TY, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pow_smem_bytes<SK, TX, TY, F == 2 ? 1 : 3>()) == cudaSuccess;
}
template <int SK>
bool powers_attrs() {
  if constexpr (SK <= kPowShapeMaxS)
    return powers_attr<SK, 0>() && powers_attr<SK, 1>() && powers_attr<SK, 2>() && powers_attr<SK, 3>() &&
           powers_attr<SK, 4>() && powers_attr<SK, 5>() && powers_attr<SK, 6>() && powers_attr<SK, 7>() &&
           powers_attr<SK, 8>() && powers_attr<SK, 9>() && powers_attr<SK, 10>() && powers_attr<SK, 11>() &&
           powers_attr<SK, 12>() && powers_attr<SK, 13>();
  else
    return powers_attr<SK, 0>();
}

int prepare_powers() {
  const bool ok = powers_attrs<1>() && powers_attrs<2>() && powers_attrs<3>() && powers_attrs<4>() &&
                  powers_attrs<5>() && powers_attrs<6>() && powers_attrs<7>() && powers_attrs<8>() &&
                  powers_attrs<9>() && powers_attrs<10>();
  return ok ? MB4_OK : MB4_ERR_CUDA;
}

#define MB4_SWITCH_S(CALL)        \
  switch (p.s) {                  \
    case 1: CALL(1); break;       \
    case 2: CALL(2); break;       \
    case 3: CALL(3); break;       \
    case 4: CALL(4); break;       \
    case 5: CALL(5); break;       \
    case 6: CALL(6); break;       \
    case 7: CALL(7); break;       \
    case 8: CALL(8); break;       \
    case 9: CALL(9); break;       \
    default: CALL(10); break;     \
  }

template <typename TK>
void launch_matvecs(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  typedef typename Vec2<TK>::type TK2;
  if (sizeof(TK) == sizeof(float) && p.use_powers && p.pow_shape != kPowLevels) {
#define MB4_CALL(N) launch_powers_s<N>(p, b, s)
    MB4_SWITCH_S(MB4_CALL)
#undef MB4_CALL
    return;
  }
  dim3 grid((p.S + p.bs_matvec - 1) / p.bs_matvec, p.B);
  auto kern = p.ell ? (p.ell_cplx ? k_matvec<TK, 3> : k_matvec<TK, 2>)
                    : (sizeof(TK) == sizeof(double) && p.mv_unit) ? k_matvec<TK, 1> : k_matvec<TK, 0>;
  for (int a = 0; a < p.s; ++a)
    launch_k(p.pdl != 0, kern, grid, dim3(p.bs_matvec), 0, s, p, (const JCoef<TK>*)b.jc, (TK2*)b.v, a,
             (const InstConst*)b.ic, (const InstStatus*)b.is);
}

template <typename TK, int SK>
void launch_gram_s(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  typedef typename Vec2<TK>::type TK2;
  const TK2* v = (const TK2*)b.v;
  // Clusters pay off for the FP32 basis, whose Gram kernel is short and tail-bound;
  // the FP64 kernel is FP64-issue-bound, and whole 8-block clusters spread less
  // evenly over the SMs than single blocks.
  if (sizeof(TK) == sizeof(float) && p.gram_blocks % kGramCluster == 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.gram_blocks, 3, p.B);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kGramCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = p.pdl ? 2 : 1;
    cudaLaunchKernelEx(&cfg, k_gram_lsq<TK, SK, kGramCluster>, p, v, b.gram_part, b.coef,
                       (const InstConst*)b.ic, b.is);
  } else {
    launch_k(p.pdl != 0, k_gram_lsq<TK, SK, 1>, dim3(p.gram_blocks, 3, p.B), dim3(256), 0, s, p, v, b.gram_part,
             b.coef, (const InstConst*)b.ic, b.is);
  }
}

template <typename TK>
void launch_gram(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
#define MB4_CALL(N) launch_gram_s<TK, N>(p, b, s)
  MB4_SWITCH_S(MB4_CALL)
#undef MB4_CALL
}

// Blocks per (instance, system) that keep the Gram kernel about one wave deep, and no
// more than one per 1024 sites: on a small grid more blocks only add partial sums for the
// last block's fixed-order reduction to read.
template <typename TK>
int gram_blocks_per_system(int s_dim, int B, int S) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
  switch (s_dim) {
#define MB4_OCC(N) case N: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_lsq<TK, N, 1>, 256, 0); break;
    MB4_OCC(1) MB4_OCC(2) MB4_OCC(3) MB4_OCC(4) MB4_OCC(5) MB4_OCC(6) MB4_OCC(7) MB4_OCC(8) MB4_OCC(9)
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_lsq<TK, 10, 1>, 256, 0); break;
#undef MB4_OCC
  }
  if (e != cudaSuccess || occ < 1 || sms < 1) return 0;
  // The FP64 kernel is bound by the FP64 pipe: one block per SM (8 warps, each with
  // the loads of 4 sites in flight) keeps it busy, spreads evenly over the SMs and
  // leaves the fewest partial sums (measured at 512x512: 54 us against 57 us with two).
  if (sizeof(TK) == sizeof(double)) occ = 1;
  long long nb = (long long)sms * occ / (3LL * (B > 0 ? B : 1));
  if (nb > kGramCap) nb = kGramCap;   // more blocks only lengthen the last block's reduction
  const long long by_sites = ((long long)S + 1023) / 1024;
  if (nb > by_sites) nb = by_sites;
  if (sizeof(TK) == sizeof(float) && nb >= kGramCluster) nb -= nb % kGramCluster;   // whole clusters
  return nb < 1 ? 1 : (int)nb;
}
template int gram_blocks_per_system<float>(int, int, int);
template int gram_blocks_per_system<double>(int, int, int);

template <typename TK>
void launch_krylov(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  if (p.precond) launch_precond_basis<TK>(p, b, s);
  else launch_matvecs<TK>(p, b, s);
  launch_gram<TK>(p, b, s);
}

template <typename TK, int SK>
__global__ void __launch_bounds__(kSiteThreadsMax) k_update(StepParams p, const typename Vec2<TK>::type* __restrict__ v,
                                                const double* __restrict__ coef, double2* __restrict__ Ubar,
                                                InstStatus* is) {
  // Before the wait for the predecessor: the status and the increments dU, which the last
  // update (or this step's set-up) wrote before the residual of this iteration started.
  const int inst = blockIdx.y;
  InstStatus& I = is[inst];
  const bool active = I.active;
  const bool first = I.newton_iter == 0 && !I.predicted;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double2 Uold[3];
  if (active && k < p.S) load_increments(Ubar, first, inst, p.S, k, Uold);
  pdl_wait();
  pdl_launch_dependents();
  if (!active) return;
  __shared__ TK cs[3][SK];
  if (threadIdx.x < 3 * SK)
    cs[threadIdx.x / SK][threadIdx.x % SK] =
        (TK)coef[((size_t)inst * 3 + threadIdx.x / SK) * kMaxS + threadIdx.x % SK];
  __syncthreads();
  float m = 0.f;
  int bad = 0;
  if (k < p.S) update_site_u<TK, SK>(p, v, cs, Uold, Ubar, first, inst, k, m, bad);
  block_update_flags(m, bad, I);
}

__global__ void k_newton_test(StepParams p, InstStatus* is, BatchCtl* bc, cudaGraphConditionalHandle h,
                              int use_cond) {
  pdl_wait();
  const int any = newton_test_all(p, is, bc);
  if (threadIdx.x == 0 && use_cond) cudaGraphSetConditional(h, any ? 1u : 0u);
}

template <typename TK>
void launch_update(const StepParams& p, const DevBuffers& b, unsigned long long h, int use_cond, cudaStream_t s) {
  dim3 grid((p.S + p.bs_update - 1) / p.bs_update, p.B);
  const void* basis = p.precond ? b.pz : b.v;      // rbar = sum_a c_a z_a when preconditioned
#define MB4_CALL(N)                                                                                      \
  launch_k(p.pdl != 0, k_update<TK, N>, grid, dim3(p.bs_update), 0, s, p, (const typename Vec2<TK>::type*)basis, \
           (const double*)b.coef, b.Ubar, b.is)
  MB4_SWITCH_S(MB4_CALL)
#undef MB4_CALL
  const int nt = p.B >= 1024 ? 1024 : ((p.B + 31) / 32) * 32;
  launch_k(p.pdl != 0, k_newton_test, dim3(1), dim3(nt), 0, s, p, b.is, b.bc, (cudaGraphConditionalHandle)h,
           use_cond);
}

// Newton start of the next step (option newton_start).  Fixed mode: extrapolate.
// Adaptive mode: record the Newton iterations this step's start took; take the start
// whose last measured cost is lower -- iterations, plus pred_cost for the extra residual
// of an extrapolated start -- and every explore_every steps the other one, so that a
// change of regime is seen.  Integer data only: the choice is reproducible.
__device__ void choose_next_start(const StepParams& p, InstStatus& I) {
  const int full_before = I.pred_count >= p.pred_order;   // this step's extrapolation used all m
  if (I.pred_count < p.pred_order) I.pred_count += 1;
  if (!p.pred_adaptive) {
    I.next_predicted = 1;
    return;
  }
  const int m = I.predicted ? 1 : 0;
  if (m == 0 || full_before) {                   // a start with less history is not representative
    I.start_iters[m] = I.newton_iter;
    if (!(I.start_known & (1 << m)) && (I.start_known | (1 << m)) == 3) I.explore_in = p.explore_every;
    I.start_known |= 1 << m;
  }
  int next;
  if (!(I.start_known & 2)) {
    next = (I.pred_count >= p.pred_order) ? 1 : 0;   // try the extrapolation once it has full history
  } else if (!(I.start_known & 1)) {
    next = 0;
  } else {
    next = (1000 * I.start_iters[1] + p.pred_cost_milli < 1000 * I.start_iters[0]) ? 1 : 0;
    if (--I.explore_in <= 0) {
      next = 1 - next;
      I.explore_in = p.explore_every;
    }
  }
  I.next_predicted = next;
}

// The end of a step of Algorithm 1 with c3 = 1: u(t+h) = U_c3 = u0 + sum_n T[2][n] dU_n, for the
// instances that took part in the step and did not fail.  Block 0 of each instance
// books the step and re-arms the instance for the next one.
__global__ void __launch_bounds__(kSiteThreadsMax) k_accept(StepParams p, double2* __restrict__ u,
                                                const double2* __restrict__ Ubar, double2* __restrict__ dUh,
                                                InstStatus* is) {
  const int inst = blockIdx.y;
  InstStatus& I = is[inst];
  const int took_part = I.in_step;
  const int failed = I.error;
  const int S = p.S;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (took_part && !failed && k < S) {
    double2 a = Ubar[stage(inst, 0, S) + k], b = Ubar[stage(inst, 1, S) + k], c = Ubar[stage(inst, 2, S) + k];
    double2 r = u[plane(inst, S) + k];
    r.x = fma(p.T[2][2], c.x, fma(p.T[2][1], b.x, fma(p.T[2][0], a.x, r.x)));
    r.y = fma(p.T[2][2], c.y, fma(p.T[2][1], b.y, fma(p.T[2][0], a.y, r.y)));
    u[plane(inst, S) + k] = r;
    if (p.pred_order > 0) {   // keep the converged increments, newest first (entries past
                              // pred_count are moved too, unread, so no block reads pred_count)
      double2* H = dUh + (size_t)inst * p.pred_order * 3 * S;
      for (int q = p.pred_order - 1; q >= 1; --q)
        for (int i = 0; i < 3; ++i) H[(size_t)(3 * q + i) * S + k] = H[(size_t)(3 * (q - 1) + i) * S + k];
      H[k] = a;
      H[(size_t)S + k] = b;
      H[(size_t)2 * S + k] = c;
    }
  }
  // Block 0 rewrites in_step and active below while other blocks of this grid may still
  // read in_step as took_part.  That is safe only because of an invariant: the host
  // changes `enabled` only between calls, and an error is only ever set during a call,
  // so when block 0 sets go = 1 the old in_step was already 1 with no error (k_arm or
  // the previous k_accept armed it), and when it sets go = 0 after a step it took part
  // in, the instance has an error and the branch above is skipped with either value.
  // A block that reads the new in_step therefore does what one that reads the old does.
  // A change to how instances are armed must keep that, or move this bookkeeping into
  // a kernel of its own.
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (took_part && !failed) {
      I.steps_done += 1;
      I.newton_total += I.newton_iter;
      if (p.pred_order > 0) choose_next_start(p, I);
    }
    I.newton_iter = 0;
    I.nonfinite = 0;
    I.rmax_bits = 0ull;
    I.u0max_bits = 0u;
    I.prev_rmax = 0.0;
    const int go = I.enabled && !I.error;
    I.in_step = go;
    I.active = go;
    I.predicted = go && p.pred_order > 0 && I.pred_count > 0 && I.next_predicted;
  }
}

void launch_accept(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  dim3 grid((p.S + p.bs_site - 1) / p.bs_site, p.B);
  k_accept<<<grid, p.bs_site, 0, s>>>(p, b.u, b.Ubar, b.dU_hist, b.is);
}

// Arms every enabled instance without an error for the next step (start of a call).
__global__ void k_arm(int B, int pred_order, InstStatus* is, BatchCtl* bc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) {
    bc->any_cont = 0;
    bc->abort = 0;                               // (the barrier slots are cleared by the host)
  }
  if (b >= B) return;
  InstStatus& I = is[b];
  I.newton_iter = 0;
  I.nonfinite = 0;
  I.rmax_bits = 0ull;
  I.u0max_bits = 0u;
  I.prev_rmax = 0.0;
  I.ticket_gram[0] = I.ticket_gram[1] = I.ticket_gram[2] = 0u;
  const int go = I.enabled && !I.error;
  I.in_step = go;
  I.active = go;
  I.predicted = go && pred_order > 0 && I.pred_count > 0 && I.next_predicted;
}

// Forget the Newton-start history of an instance (it no longer fits the state).  Every
// writer stores the same zeros, so concurrent writers need no ordering.
__device__ __forceinline__ void forget_history(InstStatus& I) {
  I.pred_count = 0;
  I.start_known = 0;
  I.explore_in = 0;
}

// set_state: pack (re, im) into the state; an instance whose state changes (any bit)
// forgets its Newton-start history.
__global__ void k_set_state(const double* __restrict__ re, const double* __restrict__ im, double2* __restrict__ z,
                            size_t n, int S, InstStatus* is) {
  const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double2 old = z[k];
  const double2 v = make_double2(re[k], im[k]);
  z[k] = v;
  if (dbits(old.x) != dbits(v.x) || dbits(old.y) != dbits(v.y)) {
    InstStatus& I = is[k / (size_t)S];
    if (*(volatile int*)&I.pred_count || *(volatile int*)&I.start_known) forget_history(I);
  }
}

__global__ void k_forget_range(InstStatus* is, int ninst) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < ninst) forget_history(is[b]);
}

void launch_forget_range(const StepParams& p, const DevBuffers& b, int first, int ninst, cudaStream_t s) {
  k_forget_range<<<(ninst + 255) / 256, 256, 0, s>>>(b.is + first, ninst);
}

void launch_set_state(const StepParams& p, const DevBuffers& b, const double* re, const double* im, int first,
                      int ninst, cudaStream_t s) {
  const size_t n = (size_t)ninst * p.S;
  if (n) k_set_state<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(re, im, b.u + (size_t)first * p.S, n, p.S,
                                                                  b.is + first);
}

void launch_arm(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  k_arm<<<(p.B + 255) / 256, 256, 0, s>>>(p.B, p.pred_order, b.is, b.bc);
}

// ---------------------------------------------------------------------------
// Observables (Sec. 2.1 energy terms, Sec. 3.2 participation ratio) per instance,
// with compensated FP64 sums (TwoSum) in a fixed order: per-thread, per-warp,
// per-block, then one block per instance over its block partials.
// ---------------------------------------------------------------------------
struct DD { double s, c; };
__device__ __forceinline__ void two_sum_add(DD& a, double x) {
  double t = __dadd_rn(a.s, x);
  double bp = __dsub_rn(t, a.s);
  double err = __dadd_rn(__dsub_rn(a.s, __dsub_rn(t, bp)), __dsub_rn(x, bp));
  a.s = t;
  a.c = __dadd_rn(a.c, err);
}
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  DD r = a;
  two_sum_add(r, b.s);
  r.c = __dadd_rn(r.c, b.c);
  return r;
}

constexpr int kObs = 6;            // H, U_K, U_E, U_nl, sum|u|^2, sum|u|^4
constexpr int kParts = 5;          // summed per site: U_K, U_E, U_nl, sum|u|^2, sum|u|^4 (H = the first three)

// Warp sums of kParts double-double values (fixed order).  Recursive halving as in
// warp_sum_f64: at o = 16, 8, 4 a lane keeps half of its live values (padded to 8)
// and adds the partner's copy; o = 2, 1 then add the one value left.  9 dd_adds
// per lane instead of 25 for a butterfly per value.  Entry e ends in the lanes
// whose bits 4, 3, 2 spell e.
__device__ __forceinline__ void warp_sum_dd(DD (&x)[8], int lane) {
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const int o = 16 >> st;
    const int h = 4 >> st;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < (4 >> st); ++j) {
      DD send = up ? x[j] : x[j + h];
      DD keep = up ? x[j + h] : x[j];
      DD t;
      t.s = __shfl_xor_sync(0xffffffffu, send.s, o);
      t.c = __shfl_xor_sync(0xffffffffu, send.c, o);
      x[j] = up ? dd_add(t, keep) : dd_add(keep, t);   // lower lane's half first, in both lanes
    }
  }
#pragma unroll
  for (int o = 2; o > 0; o >>= 1) {
    DD t;
    t.s = __shfl_xor_sync(0xffffffffu, x[0].s, o);
    t.c = __shfl_xor_sync(0xffffffffu, x[0].c, o);
    x[0] = (lane & o) ? dd_add(t, x[0]) : dd_add(x[0], t);
  }
}

template <bool ELL>
__global__ void __launch_bounds__(256) k_observables(StepParams p, const double2* __restrict__ u,
                                                     const double* __restrict__ Vp, const double* __restrict__ p_chi,
                                                     const InstConst* __restrict__ ic, double* __restrict__ part) {
  const int inst = blockIdx.y;
  const int S = p.S;
  const double half_chi = 0.5 * ic[inst].chi;
  const double2* ub = u + plane(inst, S);
  const double* vb = Vp + plane(inst, S);
  DD acc[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) acc[o].s = acc[o].c = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S; k += gridDim.x * blockDim.x) {
    const double2 c = ub[k];
    double Kx, Ky;
    if constexpr (ELL) {
      const double2 o = p.ell_cplx
                            ? ell_offdiag_c<double, double2>(p.ell_nbr, (const double2*)p.ell_w, p.ell_deg, S, k, ub)
                            : ell_offdiag<double, double2>(p.ell_nbr, (const double*)p.ell_w, p.ell_deg, S, k, ub);
      Kx = fma(p.eps0, c.x, o.x);
      Ky = fma(p.eps0, c.y, o.y);
    } else {
      Nbr n = neighbours(k, p.nx, p.ny, S);
      const double2 a = ub[n.xm], b = ub[n.xp], e = ub[n.ym], f = ub[n.yp];
      Kx = fma(-p.ty, e.x + f.x, fma(-p.tx, a.x + b.x, p.eps0 * c.x));
      Ky = fma(-p.ty, e.y + f.y, fma(-p.tx, a.y + b.y, p.eps0 * c.y));
    }
    double nn = fma(c.x, c.x, c.y * c.y);
    double n4 = nn * nn;
    two_sum_add(acc[0], fma(c.x, Kx, c.y * Ky));
    two_sum_add(acc[1], vb[k] * nn);
    two_sum_add(acc[2], (p.chi_field ? 0.5 * p_chi[plane(inst, S) + k] : half_chi) * n4);
    two_sum_add(acc[3], nn);
    two_sum_add(acc[4], n4);
  }
  __shared__ DD red[8][kParts];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  warp_sum_dd(acc, lane);
  if ((lane & 3) == 0) {
    const int e = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if (e < kParts) red[warp][e] = acc[0];
  }
  __syncthreads();
  if (threadIdx.x < kParts) {
    DD r = red[0][threadIdx.x];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = dd_add(r, red[w][threadIdx.x]);
    double* pb = part + ((size_t)inst * gridDim.x + blockIdx.x) * kParts * 2;
    pb[threadIdx.x * 2 + 0] = r.s;
    pb[threadIdx.x * 2 + 1] = r.c;
  }
}

// One block of kParts warps per instance: warp o sums part o over the block
// partials (lane l takes blocks l, l + 32, ...; then a butterfly in a fixed
// order); H = U_K + U_E + U_nl in double-double.
__global__ void k_observables_final(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  const int inst = blockIdx.x;
  const int o = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ DD tot[kParts];
  const double* pb = part + (size_t)inst * nblocks * kParts * 2;
  DD r;
  r.s = r.c = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    DD t;
    t.s = pb[((size_t)b * kParts + o) * 2 + 0];
    t.c = pb[((size_t)b * kParts + o) * 2 + 1];
    r = dd_add(r, t);
  }
  for (int off = 1; off < 32; off <<= 1) {
    DD t;
    t.s = __shfl_xor_sync(0xffffffffu, r.s, off);
    t.c = __shfl_xor_sync(0xffffffffu, r.c, off);
    r = (lane & off) ? dd_add(t, r) : dd_add(r, t);
  }
  if (lane == 0) tot[o] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    const DD H = dd_add(dd_add(tot[0], tot[1]), tot[2]);
    double* ob = out + (size_t)inst * kObs;
    ob[0] = H.s + H.c;
    for (int q = 0; q < kParts; ++q) ob[1 + q] = tot[q].s + tot[q].c;
  }
}

int obs_blocks_per_instance(int B) {
  int nb = kObsBlocksTotal / (B > 0 ? B : 1);
  if (nb > kObsBlocksMax) nb = kObsBlocksMax;
  return nb < 1 ? 1 : nb;
}

void launch_observables(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  const int nb = obs_blocks_per_instance(p.B);
  if (p.ell) k_observables<true><<<dim3(nb, p.B), 256, 0, s>>>(p, b.u, b.V, b.chi, b.ic, b.obs_part);
  else k_observables<false><<<dim3(nb, p.B), 256, 0, s>>>(p, b.u, b.V, b.chi, b.ic, b.obs_part);
  k_observables_final<<<p.B, 32 * kParts, 0, s>>>(b.obs_part, nb, b.obs_out);
}

// ---------------------------------------------------------------------------
// Packing and basis changes used by state I/O and the test entry points.
// ---------------------------------------------------------------------------
__global__ void k_pack(const double* __restrict__ re, const double* __restrict__ im, double2* __restrict__ z,
                       size_t n) {
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k < n) z[k] = make_double2(re[k], im[k]);
}
__global__ void k_unpack(const double2* __restrict__ z, double* __restrict__ re, double* __restrict__ im,
                         size_t n) {
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k < n) {
    double2 v = z[k];
    re[k] = v.x;
    im[k] = v.y;
  }
}
void launch_pack(const double* re, const double* im, double2* z, size_t n, cudaStream_t s) {
  if (n) k_pack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(re, im, z, n);
}
void launch_unpack(const double2* z, double* re, double* im, size_t n, cudaStream_t s) {
  if (n) k_unpack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(z, re, im, n);
}

// Y_j = sum_n M[j][n] X_n on three planes of S sites.
__global__ void k_mix3(int S, const double2* __restrict__ X, double2* __restrict__ Y, double m00, double m01,
                       double m02, double m10, double m11, double m12, double m20, double m21, double m22) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S) return;
  double2 a = X[k], b = X[(size_t)S + k], c = X[(size_t)2 * S + k];
  Y[k] = make_double2(m00 * a.x + m01 * b.x + m02 * c.x, m00 * a.y + m01 * b.y + m02 * c.y);
  Y[(size_t)S + k] = make_double2(m10 * a.x + m11 * b.x + m12 * c.x, m10 * a.y + m11 * b.y + m12 * c.y);
  Y[(size_t)2 * S + k] = make_double2(m20 * a.x + m21 * b.x + m22 * c.x, m20 * a.y + m21 * b.y + m22 * c.y);
}

// Z_j = Y_j + sign * x on three planes (adds or removes u0 from stage values).
__global__ void k_add_plane3(int S, double2* __restrict__ Y, const double2* __restrict__ x, double sign) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S) return;
  const double2 a = x[k];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    double2 y = Y[(size_t)j * S + k];
    y.x = fma(sign, a.x, y.x);
    y.y = fma(sign, a.y, y.y);
    Y[(size_t)j * S + k] = y;
  }
}

void launch_add_plane3(int S, double2* Y, const double2* x, double sign, cudaStream_t s) {
  k_add_plane3<<<(S + 255) / 256, 256, 0, s>>>(S, Y, x, sign);
}

void launch_mix3(int S, const double2* X, double2* Y, const double M[3][3], cudaStream_t s) {
  k_mix3<<<(S + 255) / 256, 256, 0, s>>>(S, X, Y, M[0][0], M[0][1], M[0][2], M[1][0], M[1][1], M[1][2],
                                         M[2][0], M[2][1], M[2][2]);
}

// Instance 0's level 0 <- b (3 planes), and x = sum_a c_a v_a of instance 0 -> x3.
template <typename TK>
__global__ void k_rhs_in(int S, const double2* __restrict__ b3, typename Vec2<TK>::type* __restrict__ v0) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 3 * S) return;
  double2 x = b3[k];
  typename Vec2<TK>::type y;
  y.x = (TK)x.x;
  y.y = (TK)x.y;
  v0[k] = y;
}

template <typename TK>
void launch_copy_rhs_in(const StepParams& p, const DevBuffers& b, const double2* b3, cudaStream_t s) {
  k_rhs_in<TK><<<(3 * p.S + 255) / 256, 256, 0, s>>>(p.S, b3, (typename Vec2<TK>::type*)b.v);
}

template <typename TK>
__global__ void k_solution_out(StepParams p, const typename Vec2<TK>::type* __restrict__ v,
                               const double* __restrict__ coef, double2* __restrict__ x3) {
  const int S = p.S;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S) return;
  for (int i = 0; i < 3; ++i) {
    double sx = 0, sy = 0;
    for (int a = 0; a < p.s; ++a) {
      const double c = coef[i * kMaxS + a];
      const typename Vec2<TK>::type w = v[level(0, a, i, p.s, S) + k];
      sx += c * (double)w.x;
      sy += c * (double)w.y;
    }
    x3[(size_t)i * S + k] = make_double2(sx, sy);
  }
}

template <typename TK>
void launch_copy_solution_out(const StepParams& p, const DevBuffers& b, double2* x3, cudaStream_t s) {
  const void* basis = p.precond ? b.pz : b.v;
  k_solution_out<TK><<<(p.S + 255) / 256, 256, 0, s>>>(p, (const typename Vec2<TK>::type*)basis, b.coef, x3);
}

// Explicit instantiations.
#define MB4_INST(TK)                                                                                \
  template void launch_setup<TK>(const StepParams&, const DevBuffers&, cudaStream_t);              \
  template void launch_residual<TK>(const StepParams&, const DevBuffers&, bool, cudaStream_t);     \
  template void launch_residual_out<TK>(const StepParams&, const DevBuffers&, double2*, cudaStream_t); \
  template void launch_krylov<TK>(const StepParams&, const DevBuffers&, cudaStream_t);             \
  template void launch_matvecs<TK>(const StepParams&, const DevBuffers&, cudaStream_t);            \
  template void launch_gram<TK>(const StepParams&, const DevBuffers&, cudaStream_t);               \
  template void launch_update<TK>(const StepParams&, const DevBuffers&, unsigned long long, int, cudaStream_t); \
  template void launch_copy_rhs_in<TK>(const StepParams&, const DevBuffers&, const double2*, cudaStream_t); \
  template void launch_copy_solution_out<TK>(const StepParams&, const DevBuffers&, double2*, cudaStream_t);
MB4_INST(float)
MB4_INST(double)
#undef MB4_INST

}  // namespace mb4
