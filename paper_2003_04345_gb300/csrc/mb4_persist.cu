// Persistent step kernel: one MB4 step of every instance of a batch -- the set-up and
// the whole simplified-Newton loop of Algorithm 1 -- in ONE cooperative launch, its
// phases separated by grid barriers instead of kernel boundaries (k_accept follows as
// a launch of its own, so that a step whose barrier gave up is never half accepted).
//
// Each phase runs the same device code as the one-launch-per-phase form
// (mb4_phases.cuh) over the same data: per-site phases loop over the sites of each
// instance with a grid-wide stride, the matrix-powers phase over the tiles, and the
// Gram phase over exactly the blocks (and 8-block clusters in FP32) of the Gram grid of
// the other form, in the same order, so both forms give the same results bit for bit.
// The Newton loop test runs in the last block to reach the update's barrier, before
// the others are released.
//
// Every barrier wait is bounded (StepParams::wait_limit polls).  A block whose wait
// runs out marks every instance of the step MB4_ERR_TIMEOUT, raises the batch's abort
// flag and returns; every other block returns at its next barrier (or when its own
// wait runs out), so the kernel always ends, k_accept skips the failed instances and
// their state stays at the last accepted step.  With a cooperative launch every block
// is resident, so in a healthy run no wait comes near the limit.
#include <cuda_runtime.h>

#include <algorithm>

#include "mb4_phases.cuh"

namespace mb4 {

namespace {

// A barrier over the whole grid, after which every block sees every other block's
// writes from before it.  Arrival is two-level: a block counts itself in its group's slot,
// the group's last block counts the group in slot 0, and the last group's last block --
// the last block to arrive -- runs tail() (all its threads) and then bumps every group's
// release word.  Each block polls only its own group's word.  Returns false when this
// block must stop: its wait ran out, or another block's did (abort).  Every thread of
// every block calls it.
template <typename Tail>
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, BatchCtl* bc, InstStatus* is, int B, long long limit,
                                             Tail tail) {
  __shared__ int s_state;                        // 0 stop, 1 released, 2 last to arrive
  volatile BatchCtl* vb = bc;
  const unsigned int ng = (gridDim.x + kBarGroup - 1) / kBarGroup;
  __syncthreads();
  if (threadIdx.x == 0) {
    int state = 0;
    if (!vb->abort) {
      const unsigned int g = blockIdx.x / kBarGroup;
      const unsigned int members = min((unsigned int)kBarGroup, gridDim.x - g * kBarGroup);
      unsigned int* grp = bar + (size_t)(1 + g) * kBarSlotWords;
      volatile unsigned int* rel = grp + 1;
      // the release word cannot move before this block arrives, so this is the current one
      const unsigned int gen = *rel;
      __threadfence();                           // this block's writes before the arrival
      if (atomicAdd(grp, 1u) == members - 1) {   // the group is complete: count it
        atomicExch(grp, 0u);
        __threadfence();
        if (atomicAdd(bar, 1u) == ng - 1) state = 2;
      }
      if (state != 2) {
        for (long long n = 0;; ++n) {
          if (*rel != gen) {
            state = 1;
            break;
          }
          if (vb->abort || n >= limit) break;
          __nanosleep(32);
        }
        if (state == 0 && !vb->abort) {          // this block's wait ran out: fail the step
          for (int b = 0; b < B; ++b)
            if (is[b].in_step) is[b].error = MB4_ERR_TIMEOUT;
          __threadfence();
          atomicExch(&bc->abort, 1);
        }
      }
      __threadfence();                           // the others' writes before their arrivals
    }
    s_state = state;
  }
  __syncthreads();
  const int state = s_state;
  if (state == 2) {
    tail();
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicExch(bar, 0u);                       // before the release, so no arrival at the
      __threadfence();                           // next barrier counts against this one
      for (unsigned int h = 0; h < ng; ++h) atomicAdd(bar + (size_t)(1 + h) * kBarSlotWords + 1, 1u);
    }
    __syncthreads();
    return true;
  }
  return state == 1;
}

struct NoTail {
  __device__ void operator()() const {}
};

template <typename TK, int SK, int KMR, int KMV, bool CHIF>
__global__ void __launch_bounds__(kPersistThreads, 2) k_step_persistent(StepParams p, DevBuffers d) {
  typedef typename Vec2<TK>::type TK2;
  constexpr bool MIXED = sizeof(TK) == sizeof(float);
  constexpr int NV = SK + 1;
  constexpr int NE = NV * (NV + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double blk[NE];
  __shared__ double tsum[NE];
  __shared__ TK cs[3][SK];
  __shared__ bool is_last;
  const int B = p.B, S = p.S;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gstride = gridDim.x * blockDim.x;
  InstStatus* is = d.is;
  BatchCtl* bc = d.bc;
  const long long lim = p.wait_limit;
  if (((volatile BatchCtl*)bc)->abort) return;   // an earlier step of this call gave up
  TK2* v = (TK2*)d.v;
  const double* D = KMR ? d.dtx : d.d;
  const long long os = (long long)(SK + 1) * 3 * S;

  // set-up: u0, (K+V) u0, J at u0, the first right-hand side or the extrapolated start
  for (int b = 0; b < B; ++b) {
    if (!is[b].active) continue;
    float m = 0.f;
    for (int k = gtid; k < S; k += gstride)
      m = fmaxf(m, setup_site<TK, false>(p, d.u, d.d, d.S0, (JCoef<TK>*)d.jc, v, d.dU_hist, d.Ubar, d.chi, d.ic[b],
                                         is[b], b, k));
    block_max_into(m, &is[b].u0max_bits);
  }
  if (!grid_barrier(d.bar, bc, is, B, lim, NoTail())) return;

  for (;;) {
    // residual b = -Phibar (the first one of a step from U^0 = e3 (x) u0 was written by the set-up)
    for (int b = 0; b < B; ++b) {
      if (!is[b].active || (is[b].newton_iter == 0 && !is[b].predicted)) continue;
      for (int k = gtid; k < S; k += gstride)
        residual_site<TK, CHIF, KMR>(p, d.u, D, d.S0, d.Ubar, v, os, d.chi, d.ic[b], b, k);
    }
    if (!grid_barrier(d.bar, bc, is, B, lim, NoTail())) return;

    // Krylov basis: all s levels per tile (FP32 matrix powers) or one level per phase (FP64)
    if constexpr (MIXED) {
      const int tiles = ((p.nx + kPowTX - 1) / kPowTX) * ((p.ny + kPowTY - 1) / kPowTY);
      for (int item = blockIdx.x; item < B * tiles; item += gridDim.x) {
        const int b = item / tiles;
        if (!is[b].active) continue;
        powers_tile<SK, kPowTX, kPowTY>(p, (const float4*)d.jc, (float2*)d.v, d.ic[b], b, item - b * tiles, smem_raw);
      }
      if (!grid_barrier(d.bar, bc, is, B, lim, NoTail())) return;
    } else {
      for (int a = 0; a < SK; ++a) {
        for (int b = 0; b < B; ++b) {
          if (!is[b].active) continue;
          for (int k = gtid; k < S; k += gstride) matvec_site<TK, KMV>(p, (const JCoef<TK>*)d.jc, v, a, d.ic[b], b, k);
        }
        if (!grid_barrier(d.bar, bc, is, B, lim, NoTail())) return;
      }
    }

    // Gram partials over the blocks (clusters) of the Gram grid; the last of a system solves
    const int nbx = p.gram_blocks;
    const int CL = (MIXED && nbx % kGramCluster == 0) ? kGramCluster : 1;
    const int nb = nbx / CL;
    for (int item = blockIdx.x; item < B * 3 * nb; item += gridDim.x) {
      const int inst = item / (3 * nb), rem = item - inst * 3 * nb, i = rem / nb, c = rem - i * nb;
      if (!is[inst].active) continue;
      double* pi = d.gram_part + ((size_t)inst * 3 + i) * nb * NE;
      if (CL > 1) {                              // the cluster leader's sum, in rank order
        for (int e = threadIdx.x; e < NE; e += blockDim.x) tsum[e] = 0.0;
        for (int r = 0; r < CL; ++r) {
          gram_accumulate<TK, SK>(p, v, inst, i, c * CL + r, nbx, blk);
          for (int e = threadIdx.x; e < NE; e += blockDim.x) tsum[e] += blk[e];
          __syncthreads();
        }
        for (int e = threadIdx.x; e < NE; e += blockDim.x) pi[(size_t)c * NE + e] = tsum[e];
      } else {
        gram_accumulate<TK, SK>(p, v, inst, i, c, nbx, blk);
        for (int e = threadIdx.x; e < NE; e += blockDim.x) pi[(size_t)c * NE + e] = blk[e];
      }
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) is_last = (atomicAdd(&is[inst].ticket_gram[i], 1u) == (unsigned int)(nb - 1));
      __syncthreads();
      if (is_last) {
        __threadfence();
        gram_lsq_solve<SK>(p, d.gram_part, d.coef, d.ic, is, inst, i, nb);
      }
      __syncthreads();
    }
    if (!grid_barrier(d.bar, bc, is, B, lim, NoTail())) return;

    // Newton update, then the loop test in the last block to arrive
    for (int b = 0; b < B; ++b) {
      if (!is[b].active) continue;
      if (threadIdx.x < 3 * SK)
        cs[threadIdx.x / SK][threadIdx.x % SK] = (TK)d.coef[((size_t)b * 3 + threadIdx.x / SK) * kMaxS + threadIdx.x % SK];
      const bool first = is[b].newton_iter == 0 && !is[b].predicted;
      __syncthreads();
      float m = 0.f;
      int bad = 0;
      for (int k = gtid; k < S; k += gstride) update_site<TK, SK>(p, v, cs, d.Ubar, first, b, k, m, bad);
      block_update_flags(m, bad, is[b]);
    }
    auto test = [&]() { newton_test_all(p, is, bc); };
    if (!grid_barrier(d.bar, bc, is, B, lim, test)) return;
    if (!((volatile BatchCtl*)bc)->any_cont) break;
  }
}

typedef void (*PersistKernel)(StepParams, DevBuffers);

template <typename TK, int SK>
PersistKernel pick(const StepParams& p) {
  const int kmr = p.kin_unit ? 1 : 0;
  const int kmv = (sizeof(TK) == sizeof(double) && p.mv_unit) ? 1 : 0;
  if (p.chi_field) {
    if (kmr && kmv) return k_step_persistent<TK, SK, 1, 1, true>;
    if (kmr) return k_step_persistent<TK, SK, 1, 0, true>;
    return k_step_persistent<TK, SK, 0, 0, true>;
  }
  if (kmr && kmv) return k_step_persistent<TK, SK, 1, 1, false>;
  if (kmr) return k_step_persistent<TK, SK, 1, 0, false>;
  return k_step_persistent<TK, SK, 0, 0, false>;
}

PersistKernel kernel_for(const StepParams& p, bool mixed) {
  if (mixed) return (p.s == 4) ? pick<float, 4>(p) : pick<float, 5>(p);
  return (p.s == 4) ? pick<double, 4>(p) : pick<double, 5>(p);
}

size_t dyn_smem(const StepParams& p, bool mixed) {
  if (!mixed) return 0;
  return (p.s == 4) ? pow_smem_bytes<4>() : pow_smem_bytes<5>();
}

}  // namespace

bool persistent_supported(const StepParams& p, bool mixed) {
  return !p.ell && !p.precond && (p.s == 4 || p.s == 5) && (!mixed || p.use_powers);
}

int persistent_blocks(const StepParams& p, bool mixed) {
  if (!persistent_supported(p, mixed)) return 0;
  PersistKernel k = kernel_for(p, mixed);
  const size_t smem = dyn_smem(p, mixed);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kPersistThreads, smem) != cudaSuccess || occ < 1)
    return 0;
  // no more blocks than the sites (or, in FP32, the tiles) give one thread (block) work:
  // a small problem then needs fewer arrivals per barrier
  const long long sites = (long long)p.B * p.S;
  long long want = (sites + kPersistThreads - 1) / kPersistThreads;
  if (mixed) want = std::max(want, (long long)p.B * ((p.nx + kPowTX - 1) / kPowTX) * ((p.ny + kPowTY - 1) / kPowTY));
  return (int)std::min<long long>((long long)sms * occ, std::max<long long>(want, 1));
}

cudaError_t launch_step_persistent(const StepParams& p, const DevBuffers& b, bool mixed, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.pers_blocks);
  cfg.blockDim = dim3(kPersistThreads);
  cfg.dynamicSmemBytes = dyn_smem(p, mixed);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // every block resident at once: the barriers need it
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel_for(p, mixed), p, b);
}

}  // namespace mb4
