// The step's work per site (per tile, per Gram block, per instance), as device
// functions shared by the step kernels of mb4_kernels.cu (one launch per phase, chained
// in a CUDA graph) and the persistent step kernel of mb4_persist.cu (every phase in one
// launch, separated by grid barriers).  Both forms run the same arithmetic on the same
// data, so they give the same results bit for bit.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "mb4_device.cuh"
#include "mb4_internal.h"

namespace mb4 {

// ---------------------------------------------------------------------------
// Step set-up (Algorithm 1, start of a step, and the first residual): u0 = u(t); J at u0
// as per-site coefficients; (K+V) u0; ||u0||_inf.  At U^0 = e3 (x) u0 every stage
// polynomial value equals u0, so Phi_i(U^0) = -h c_i f(u0) and the first
// right-hand side is b = -Phibar^0 = -i h (T^-1 c)_i [(K+V) u0 + chi |u0|^2 u0].
// J and b^0 only feed the Krylov solve, so they are formed in its precision TK;
// (K+V) u0 is reused by every residual and stays FP64.  The increments start at
// dU^0 = 0 (the first update writes them), or, for an instance whose step starts
// from an extrapolation (option newton_start), at the polynomial extrapolation of
// the last m converged increments (m = 1: the last; 2: 2 H0 - H1; 3: 3 H0 - 3 H1 + H2,
// H0 the newest), whose residual the first k_residual then evaluates.
// Grid: (sites / bs_site, B).
// ---------------------------------------------------------------------------
template <typename TK, bool ELL>
__device__ __forceinline__ float setup_site(const StepParams& p, const double2* __restrict__ u,
                                            const double* __restrict__ D, double2* __restrict__ S0,
                                            JCoef<TK>* __restrict__ jc, typename Vec2<TK>::type* __restrict__ v,
                                            const double2* __restrict__ dUh, double2* __restrict__ dUb,
                                            const double* __restrict__ p_chi, const InstConst& C,
                                            const InstStatus& I, int b, int k) {
  typedef typename Vec2<TK>::type TK2;
  const int S = p.S;
  const double2* ub = u + plane(b, S);
  double2 c = ub[k];
  double d = D[plane(b, S) + k];
  double2 s0;
  if constexpr (ELL) {
    const double2 o = p.ell_cplx
                          ? ell_offdiag_c<double, double2>(p.ell_nbr, (const double2*)p.ell_w, p.ell_deg, S, k, ub)
                          : ell_offdiag<double, double2>(p.ell_nbr, (const double*)p.ell_w, p.ell_deg, S, k, ub);
    s0.x = fma(d, c.x, o.x);
    s0.y = fma(d, c.y, o.y);
  } else {
    Nbr n = neighbours(k, p.nx, p.ny, S);
    double2 a = ub[n.xm], bb = ub[n.xp], e = ub[n.ym], f = ub[n.yp];
    s0.x = fma(-p.ty, e.x + f.x, fma(-p.tx, a.x + bb.x, d * c.x));
    s0.y = fma(-p.ty, e.y + f.y, fma(-p.tx, a.y + bb.y, d * c.y));
  }
  S0[plane(b, S) + k] = s0;
  const TK pk = from_double<TK>(c.x), qk = from_double<TK>(c.y);
  const TK pp = mul_(pk, pk), qq = mul_(qk, qk), nn = add_(pp, qq);
  const TK dt = mul_(from_double<TK>(d), kval<TK>(C.inv_theta, C.f_inv_theta));
  const double chik = p.chi_field ? p_chi[plane(b, S) + k] : 1.0;   // per-site chi (InstConst chi = 1)
  TK ct = kval<TK>(C.chi_theta, C.f_chi_theta);
  if (p.chi_field) ct = mul_(ct, from_double<TK>(chik));
  JCoef<TK> j;
  j.e1 = fma_(ct, fma_((TK)3, qq, pp), dt);
  j.e2 = fma_(ct, fma_((TK)3, pp, qq), dt);
  j.a = mul_(mul_(mul_((TK)2, ct), pk), qk);
  j.pad = (TK)0;
  jc[plane(b, S) + k] = j;
  if (I.predicted) {
    const int mo = min(I.pred_count, p.pred_order);
    const double w0 = (mo == 1) ? 1.0 : (mo == 2) ? 2.0 : 3.0;
    const double w1 = (mo == 2) ? -1.0 : -3.0;
    const double2* H = dUh + (size_t)b * p.pred_order * 3 * S;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double2 x = H[(size_t)i * S + k];
      if (mo >= 2) {
        const double2 y = H[(size_t)(3 + i) * S + k];
        double2 z = make_double2(0.0, 0.0);
        if (mo >= 3) z = H[(size_t)(6 + i) * S + k];
        x.x = fma(w0, x.x, fma(w1, y.x, z.x));
        x.y = fma(w0, x.y, fma(w1, y.y, z.y));
      }
      dUb[stage(b, i, S) + k] = x;
    }
  } else {
    TK cn = mul_(kval<TK>(C.chi, C.f_chi), nn);
    if (p.chi_field) cn = mul_(cn, from_double<TK>(chik));
    const TK Fx = fma_(cn, pk, from_double<TK>(s0.x)), Fy = fma_(cn, qk, from_double<TK>(s0.y));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      TK2 bi;
      const TK hc = kval<TK>(p.hTc[i], p.f_hTc[i]);
      bi.x = mul_(hc, Fy);
      bi.y = mul_(-hc, Fx);
      v[level(b, 0, i, p.s, S) + k] = bi;
    }
  }
  return fmaxf(absf_of(c.x), absf_of(c.y));
}

// The largest m over the block, merged into *target with one atomic (same-address atomics
// queue at one L2 slice, so not one per thread).  Every thread of the block calls it.
__device__ __forceinline__ void block_max_into(float m, unsigned int* target) {
  m = warp_max(m);
  __shared__ float wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float bm = wm[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) bm = fmaxf(bm, wm[w]);
    if (bm > 0.f) atomicMax(target, __float_as_uint(bm));
  }
  __syncthreads();                               // wm is reused by the next call
}

// ---------------------------------------------------------------------------
// Residual (Algorithm 1; eq. Phidefinition, eq. fKu2, eq. fIu2) in
// the eigenbasis, on the increments dU: b = -Phibar with
//   Phibar_i = dU_i + i [ h lam_i (K+V) dU_i + h (T^-1 c)_i (K+V) u0
//                         + sum_q h chi W~_iq |X_q|^2 X_q ],
//   X_q = u0 + sum_n (L T)_qn dU_n   (the stage polynomial at the 6 Gauss nodes;
// exact for the degree-11 integrand).  (The u0 terms: T^-1 E T = Lambda and
// T^-1 (E_{.0} + E 1) = T^-1 c, since the rows of E sum to c.)  All FP64.
// KM selects the kinetic term: 0 the grid stencil, 1 the grid stencil with tx factored
// out (StepParams::kin_unit), 2 the general sparse K (ELL), 3 a complex Hermitian one.
// ---------------------------------------------------------------------------
template <typename TO, bool CHIF, int KM>
__device__ __forceinline__ void residual_site(const StepParams& p, const double2* __restrict__ u,
                                              const double* __restrict__ D, const double2* __restrict__ S0,
                                              const double2* __restrict__ dUb,
                                              typename Vec2<TO>::type* __restrict__ out, long long out_stride,
                                              const double* __restrict__ p_chi, const InstConst& C, int b,
                                              int k) {
  typedef typename Vec2<TO>::type TO2;
  const int S = p.S;
  Nbr n;
  if constexpr (KM < 2) n = neighbours(k, p.nx, p.ny, S);
  const double2 u0 = u[plane(b, S) + k];
  const double2 s0 = S0[plane(b, S) + k];
  const double d = D[plane(b, S) + k];           // D / tx when KM == 1
  const double chik = CHIF ? p_chi[plane(b, S) + k] : 1.0;   // per-site chi (InstConst chi = 1)
  // b = -Phibar is accumulated directly.  With Phibar = dU + i Q,
  //   Q = h lam (K+V) dU + hTc (K+V) u0 + sum_q h chi W~_q |X_q|^2 X_q,
  // b.x = -dU.x + Q.y and b.y = -dU.y - Q.x: the dU terms ride on the first FMAs and
  // every sign is an operand modifier.
  double2 dU[3], bo[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const double2* P = dUb + stage(b, m, S);
    const double2 c = P[k];
    dU[m] = c;
    double sx, sy, hl;
    if constexpr (KM >= 2) {
      const double2 o =
          (KM == 3) ? ell_offdiag_c<double, double2>(p.ell_nbr, (const double2*)p.ell_w, p.ell_deg, S, k, P)
                    : ell_offdiag<double, double2>(p.ell_nbr, (const double*)p.ell_w, p.ell_deg, S, k, P);
      sx = fma(d, c.x, o.x);
      sy = fma(d, c.y, o.y);
      hl = p.hlam[m];
    } else if constexpr (KM == 1) {
      // (K+V) x / tx = D/tx x - (x_x- + x_x+) - (ty/tx) (x_y- + x_y+)
      const double2 a = P[n.xm], bb = P[n.xp], e = P[n.ym], f = P[n.yp];
      sx = fma(d, c.x, -fma(p.rty, e.x + f.x, a.x + bb.x));
      sy = fma(d, c.y, -fma(p.rty, e.y + f.y, a.y + bb.y));
      hl = p.hltx[m];
    } else {
      const double2 a = P[n.xm], bb = P[n.xp], e = P[n.ym], f = P[n.yp];
      sx = fma(-p.ty, e.x + f.x, fma(-p.tx, a.x + bb.x, d * c.x));
      sy = fma(-p.ty, e.y + f.y, fma(-p.tx, a.y + bb.y, d * c.y));
      hl = p.hlam[m];
    }
    bo[m].x = fma(hl, sy, fma(p.hTc[m], s0.y, -c.x));
    bo[m].y = fma(-hl, sx, fma(-p.hTc[m], s0.x, -c.y));
  }
#pragma unroll
  for (int q = 0; q < kGauss; ++q) {
    double Xx = fma(p.LT[q][0], dU[0].x, u0.x), Xy = fma(p.LT[q][0], dU[0].y, u0.y);
    Xx = fma(p.LT[q][1], dU[1].x, Xx);
    Xy = fma(p.LT[q][1], dU[1].y, Xy);
    Xx = fma(p.LT[q][2], dU[2].x, Xx);
    Xy = fma(p.LT[q][2], dU[2].y, Xy);
    double nn = fma(Xx, Xx, mul_(Xy, Xy));
    if (CHIF) nn = mul_(nn, chik);
    const double gx = mul_(nn, Xx), gy = mul_(nn, Xy);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      bo[i].x = fma(C.hchiW[i][q], gy, bo[i].x);
      bo[i].y = fma(-C.hchiW[i][q], gx, bo[i].y);
    }
  }
  TO2* ob = out + (size_t)b * (size_t)out_stride;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    TO2 o;
    o.x = from_double<TO>(bo[i].x);
    o.y = from_double<TO>(bo[i].y);
    ob[(size_t)i * S + k] = o;
  }
}


// ---------------------------------------------------------------------------
// Shifted solves (Algorithm 1; eq. MB4_5): one s-step GMRES cycle per
// system.  The Krylov space K_s(I - h lam_i J, b_i) = span{b_i, Jb_i, .., J^{s-1} b_i}
// is the same monomial space for all three shifts, so the basis
// v_{a+1} = (J/theta) v_a is built for the three right-hand sides together, and
// (I - h lam_i J) v_a = v_a - sig_i v_{a+1} with sig_i = h lam_i theta.
// ---------------------------------------------------------------------------
// v modulo n in 0 .. n - 1 (periodic grid index).
__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// (J/theta) x at one site of the grid stencil from the site's value c and its x-1, x+1,
// y-1, y+1 neighbours a, bb, e, f (every grid form of the basis uses this sequence):
//   (J x)_re = a xp + e1 xq - tx (xq_x- + xq_x+) - ty (xq_y- + xq_y+)
//   (J x)_im = -e2 xp - a xq + tx (xp_x- + xp_x+) + ty (xp_y- + xp_y+)
template <typename TK, int KM>
__device__ __forceinline__ typename Vec2<TK>::type grid_jx(const JCoef<TK>& j, const typename Vec2<TK>::type c,
                                                           const typename Vec2<TK>::type a,
                                                           const typename Vec2<TK>::type bb,
                                                           const typename Vec2<TK>::type e,
                                                           const typename Vec2<TK>::type f, TK tx, TK ty) {
  typename Vec2<TK>::type o;
  if constexpr (KM == 1) {                       // theta = tx: tx / theta = 1
    o.x = fma(j.a, c.x, fma(j.e1, c.y, -fma(ty, e.y + f.y, a.y + bb.y)));
    o.y = fma(-j.e2, c.x, fma(-j.a, c.y, fma(ty, e.x + f.x, a.x + bb.x)));
  } else {
    o.x = fma_(-ty, add_(e.y, f.y), fma_(-tx, add_(a.y, bb.y), fma_(j.e1, c.y, mul_(j.a, c.x))));
    o.y = fma_(ty, add_(e.x, f.x), fma_(tx, add_(a.x, bb.x), fma_(-j.a, c.y, mul_(-j.e2, c.x))));
  }
  return o;
}

template <typename TK, int KM>
__device__ __forceinline__ void matvec_site_j(const StepParams& p, const JCoef<TK> j,
                                              typename Vec2<TK>::type* __restrict__ v, int a_in, const InstConst& C,
                                              int b, int k) {
  typedef typename Vec2<TK>::type TK2;
  const int S = p.S;
  if constexpr (KM >= 2) {
    // (J x)_re = a xp + e1 xq + Im(sum_j (K_kj / theta) x_j), (J x)_im = -e2 xp - a xq - Re(sum_j ..):
    // with s = sum_j K_kj x_j / theta (a complex product when K is complex), the kinetic
    // part of J x is the real form of -i s (eq. JL)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const TK2* P = v + level(b, a_in, i, p.s, S);
      const TK2 c = P[k];
      const TK2 s = (KM == 3) ? ell_offdiag_c<TK, TK2>(p.ell_nbr, (const TK2*)p.ell_wt, p.ell_deg, S, k, P)
                              : ell_offdiag<TK, TK2>(p.ell_nbr, (const TK*)p.ell_wt, p.ell_deg, S, k, P);
      TK2 o;
      o.x = fma_(j.a, c.x, fma_(j.e1, c.y, s.y));
      o.y = fma_(-j.e2, c.x, fma_(-j.a, c.y, -s.x));
      v[level(b, a_in + 1, i, p.s, S) + k] = o;
    }
  } else {
    Nbr n = neighbours(k, p.nx, p.ny, S);
    const TK tx = kval<TK>(C.txt, C.f_txt), ty = kval<TK>(C.tyt, C.f_tyt);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const TK2* P = v + level(b, a_in, i, p.s, S);
      v[level(b, a_in + 1, i, p.s, S) + k] = grid_jx<TK, KM>(j, P[k], P[n.xm], P[n.xp], P[n.ym], P[n.yp], tx, ty);
    }
  }
}


// The same with the J coefficients read here (the persistent step; the launch-per-phase
// kernel reads them before it waits for its predecessor).
template <typename TK, int KM>
__device__ __forceinline__ void matvec_site(const StepParams& p, const JCoef<TK>* __restrict__ jc,
                                            typename Vec2<TK>::type* __restrict__ v, int a_in, const InstConst& C,
                                            int b, int k) {
  matvec_site_j<TK, KM>(p, jc[plane(b, p.S) + k], v, a_in, C, b, k);
}

// Matrix powers on a tile (FP32 Krylov basis): one block builds v_1..v_SK on a
// TX x TY tile from v_0 and the J coefficients loaded once, with an SK-wide
// periodic halo in shared memory; level a is valid on the tile grown by SK - a,
// so no block needs another block's result.  Replaces SK stencil launches by
// one at the price of recomputing the shrinking halo (cheap in FP32).  Each
// thread owns fixed positions of the extended tile (columns tx0 + 32 ix, rows
// ty0 + 8 iy) at every level, so their J coefficients stay in registers and
// shared memory holds only the two level buffers: 4 blocks per SM at SK = 4,
// which puts a 512 x 512 grid's 512 tiles in one wave.
constexpr int kPowTX = 32, kPowTY = 16, kPowThreads = 256;   // the default tile (shape 0)

template <int SK, int TX = kPowTX>
__host__ __device__ constexpr int pow_ext_x() { return TX + 2 * SK; }
template <int SK, int TY = kPowTY>
__host__ __device__ constexpr int pow_ext_y() { return TY + 2 * SK; }
template <int SK, int TX = kPowTX, int TY = kPowTY, int NSYS = 3>
constexpr size_t pow_smem_bytes() {
  return (size_t)pow_ext_x<SK, TX>() * pow_ext_y<SK, TY>() * (2 * NSYS * sizeof(float2));
}

// Tile shapes the launch-shape tuner chooses among (TX a multiple of 32): the results do
// not depend on the shape -- every tile computes each level at each site it holds with
// the same arithmetic from the same neighbours -- only the halo overhead, the shared
// memory per block and so the blocks per SM do.
// Forms 3 and 4 (one warp per tile or per strip: powers_warp, powers_stream) list the warp's
// extended width, 32: the interior is 32 - 2 s sites wide.
constexpr int kPowShapes = 14;      // 4, 5: rows in registers; 6, 7: one system at a time; 8, 9: one warp
                                    // per tile; 10, 11: one warp per strip; 12, 13: strips staged by cp.async
constexpr int kPowShapeTX[kPowShapes] = {32, 32, 64, 32, 32, 64, 32, 64, 32, 32, 32, 32, 32, 32};
constexpr int kPowShapeTY[kPowShapes] = {16, 32, 16, 8, 16, 16, 16, 16, 4, 8, 8, 16, 8, 16};
constexpr int kPowShapeForm[kPowShapes] = {0, 0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 5, 5};   // 0 tile, 1 rows,
                                          // 2 by system, 3 warp, 4 strip, 5 strip staged through shared memory
constexpr int kPowStreamAhead = 4;   // form 5: rows copied ahead
constexpr int kPowWarpsPerBlock = 4;   // form 3: warps (tiles) per block
constexpr int kPowShapeMaxS = 6;   // larger s: the default tile only
constexpr int kPowLevels = kPowShapes;   // pow_shape value: no tiles, one stencil launch per level

template <int SK, int TX = kPowTX, int TY = kPowTY>
__device__ __forceinline__ void powers_tile(const StepParams& p, const float4* __restrict__ jc,
                                            float2* __restrict__ v, const InstConst& C, int b, int tile,
                                            unsigned char* smem_raw) {
  static_assert(TX % 32 == 0, "tile width is a multiple of the warp");
  constexpr int EX = pow_ext_x<SK, TX>(), EY = pow_ext_y<SK, TY>(), EA = EX * EY;
  constexpr int NCX = (EX + 31) / 32, NCY = (EY + 7) / 8;      // positions per thread
  float2* buf0 = reinterpret_cast<float2*>(smem_raw);     // [3][EA]
  float2* buf1 = buf0 + 3 * EA;                           // [3][EA]
  const int S = p.S, nx = p.nx, ny = p.ny;
  const int tiles_x = (nx + TX - 1) / TX;
  const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
  const int x0 = txi * TX - SK, y0 = tyi * TY - SK;
  const float4* jb = jc + plane(b, S);
  const int tx0 = threadIdx.x & 31, ty0 = threadIdx.x >> 5;   // 32 x 8 thread layout
  float4 jr[NCY][NCX];
#pragma unroll
  for (int iy = 0; iy < NCY; ++iy) {
    const int ly = ty0 + 8 * iy;
#pragma unroll
    for (int ix = 0; ix < NCX; ++ix) {
      const int lx = tx0 + 32 * ix;
      if (ly < EY && lx < EX) {
        const int t = ly * EX + lx;
        const int g = wrap(y0 + ly, ny) * nx + wrap(x0 + lx, nx);
        jr[iy][ix] = jb[g];
#pragma unroll
        for (int i = 0; i < 3; ++i) buf0[i * EA + t] = v[level(b, 0, i, SK, S) + g];
      }
    }
  }
  __syncthreads();
  const float tx = C.f_txt, ty = C.f_tyt;
  float2* src = buf0;
  float2* dst = buf1;
#pragma unroll 1
  for (int a = 1; a <= SK; ++a) {
#pragma unroll
    for (int iy = 0; iy < NCY; ++iy) {
      const int ly = ty0 + 8 * iy;
#pragma unroll
      for (int ix = 0; ix < NCX; ++ix) {
        const int lx = tx0 + 32 * ix;
        if (ly < a || ly >= EY - a || lx < a || lx >= EX - a) continue;   // level a lives on the tile grown by SK - a
        const int c = ly * EX + lx;
        const float4 j = jr[iy][ix];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float2* P = src + i * EA;
          const float2 cc = P[c], xa = P[c - 1], xb = P[c + 1], ya = P[c - EX], yb = P[c + EX];
          float2 o;
          o.x = fma_(-ty, add_(ya.y, yb.y), fma_(-tx, add_(xa.y, xb.y), fma_(j.x, cc.y, mul_(j.z, cc.x))));
          o.y = fma_(ty, add_(ya.x, yb.x), fma_(tx, add_(xa.x, xb.x), fma_(-j.z, cc.y, mul_(-j.y, cc.x))));
          dst[i * EA + c] = o;
        }
      }
    }
    __syncthreads();
    // interior of level a to global
    for (int ly = ty0; ly < TY; ly += kPowThreads / 32) {
#pragma unroll
      for (int lx = tx0; lx < TX; lx += 32) {
        const int gx = txi * TX + lx, gy = tyi * TY + ly;
        if (gx < nx && gy < ny) {
          const int c = (ly + SK) * EX + (lx + SK);
          const size_t g = (size_t)gy * nx + gx;
#pragma unroll
          for (int i = 0; i < 3; ++i) v[level(b, a, i, SK, S) + g] = dst[i * EA + c];
        }
      }
    }
    float2* tmp = src;
    src = dst;
    dst = tmp;
  }
  __syncthreads();                               // the caller may reuse shared memory for the next tile
}

// The same tile with the three systems built one after the other through buffers for one
// system: a third of the shared memory per block, so more blocks fit an SM (the kernel is
// bound by shared-memory latency, not by its arithmetic).  Same arithmetic, same basis.
template <int SK, int TX, int TY>
__device__ __forceinline__ void powers_tile_sys(const StepParams& p, const float4* __restrict__ jc,
                                                float2* __restrict__ v, const InstConst& C, int b, int tile,
                                                unsigned char* smem_raw) {
  static_assert(TX % 32 == 0, "tile width is a multiple of the warp");
  constexpr int EX = pow_ext_x<SK, TX>(), EY = pow_ext_y<SK, TY>(), EA = EX * EY;
  constexpr int NCX = (EX + 31) / 32, NCY = (EY + 7) / 8;      // positions per thread
  float2* buf0 = reinterpret_cast<float2*>(smem_raw);     // [EA]
  float2* buf1 = buf0 + EA;                               // [EA]
  const int S = p.S, nx = p.nx, ny = p.ny;
  const int tiles_x = (nx + TX - 1) / TX;
  const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
  const int x0 = txi * TX - SK, y0 = tyi * TY - SK;
  const float4* jb = jc + plane(b, S);
  const int tx0 = threadIdx.x & 31, ty0 = threadIdx.x >> 5;   // 32 x 8 thread layout
  const float tx = C.f_txt, ty = C.f_tyt;
  float4 jr[NCY][NCX];
#pragma unroll
  for (int iy = 0; iy < NCY; ++iy)
#pragma unroll
    for (int ix = 0; ix < NCX; ++ix) {
      const int ly = ty0 + 8 * iy, lx = tx0 + 32 * ix;
      if (ly < EY && lx < EX) jr[iy][ix] = jb[wrap(y0 + ly, ny) * nx + wrap(x0 + lx, nx)];
    }
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int iy = 0; iy < NCY; ++iy)
#pragma unroll
      for (int ix = 0; ix < NCX; ++ix) {
        const int ly = ty0 + 8 * iy, lx = tx0 + 32 * ix;
        if (ly < EY && lx < EX)
          buf0[ly * EX + lx] = v[level(b, 0, i, SK, S) + wrap(y0 + ly, ny) * nx + wrap(x0 + lx, nx)];
      }
    __syncthreads();
    float2* src = buf0;
    float2* dst = buf1;
#pragma unroll 1
    for (int a = 1; a <= SK; ++a) {
#pragma unroll
      for (int iy = 0; iy < NCY; ++iy) {
        const int ly = ty0 + 8 * iy;
#pragma unroll
        for (int ix = 0; ix < NCX; ++ix) {
          const int lx = tx0 + 32 * ix;
          if (ly < a || ly >= EY - a || lx < a || lx >= EX - a) continue;   // the tile grown by SK - a
          const int c = ly * EX + lx;
          const float4 j = jr[iy][ix];
          const float2 cc = src[c], xa = src[c - 1], xb = src[c + 1], ya = src[c - EX], yb = src[c + EX];
          float2 o;
          o.x = fma_(-ty, add_(ya.y, yb.y), fma_(-tx, add_(xa.y, xb.y), fma_(j.x, cc.y, mul_(j.z, cc.x))));
          o.y = fma_(ty, add_(ya.x, yb.x), fma_(tx, add_(xa.x, xb.x), fma_(-j.z, cc.y, mul_(-j.y, cc.x))));
          dst[c] = o;
        }
      }
      __syncthreads();
      for (int ly = ty0; ly < TY; ly += kPowThreads / 32) {
#pragma unroll
        for (int lx = tx0; lx < TX; lx += 32) {
          const int gx = txi * TX + lx, gy = tyi * TY + ly;
          if (gx < nx && gy < ny) v[level(b, a, i, SK, S) + (size_t)gy * nx + gx] = dst[(ly + SK) * EX + (lx + SK)];
        }
      }
      float2* tmp = src;
      src = dst;
      dst = tmp;
    }
    __syncthreads();                             // before the next system overwrites the buffers
  }
}

// The same tile with each warp owning a band of NR consecutive rows (lane = column):
// a thread keeps its own positions' values of the previous level in registers, so the
// centre and the y neighbours inside its band need no shared-memory read; only the x
// neighbours (other lanes) and the rows just outside the band come from shared memory.
// Same arithmetic on the same values as powers_tile, so the same basis bit for bit.
template <int SK, int TX, int TY>
__device__ __forceinline__ void powers_tile_rows(const StepParams& p, const float4* __restrict__ jc,
                                                 float2* __restrict__ v, const InstConst& C, int b, int tile,
                                                 unsigned char* smem_raw) {
  static_assert(TX % 32 == 0, "tile width is a multiple of the warp");
  constexpr int EX = pow_ext_x<SK, TX>(), EY = pow_ext_y<SK, TY>(), EA = EX * EY;
  constexpr int NCX = (EX + 31) / 32, NR = (EY + 7) / 8;       // columns and rows per thread
  float2* buf0 = reinterpret_cast<float2*>(smem_raw);     // [3][EA]
  float2* buf1 = buf0 + 3 * EA;                           // [3][EA]
  const int S = p.S, nx = p.nx, ny = p.ny;
  const int tiles_x = (nx + TX - 1) / TX;
  const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
  const int x0 = txi * TX - SK, y0 = tyi * TY - SK;
  const float4* jb = jc + plane(b, S);
  const int tx0 = threadIdx.x & 31, ly0 = (threadIdx.x >> 5) * NR;   // lane = column, warp = band of rows
  float4 jr[NR][NCX];
  float2 own[NR][NCX][3];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int ly = ly0 + r;
#pragma unroll
    for (int ix = 0; ix < NCX; ++ix) {
      const int lx = tx0 + 32 * ix;
      if (ly < EY && lx < EX) {
        const int t = ly * EX + lx;
        const int g = wrap(y0 + ly, ny) * nx + wrap(x0 + lx, nx);
        jr[r][ix] = jb[g];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          own[r][ix][i] = v[level(b, 0, i, SK, S) + g];
          buf0[i * EA + t] = own[r][ix][i];
        }
      }
    }
  }
  __syncthreads();
  const float tx = C.f_txt, ty = C.f_tyt;
  float2* src = buf0;
  float2* dst = buf1;
#pragma unroll 1
  for (int a = 1; a <= SK; ++a) {
    float2 above[NCX][3];                        // the previous row's level a-1 values
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int ly = ly0 + r;
#pragma unroll
      for (int ix = 0; ix < NCX; ++ix) {
        const int lx = tx0 + 32 * ix;
        const bool live = !(ly < a || ly >= EY - a || lx < a || lx >= EX - a);   // the tile grown by SK - a
        const int c = ly * EX + lx;
        const float4 j = jr[r][ix];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float2 cc = own[r][ix][i];
          if (live) {
            const float2* P = src + i * EA;
            const float2 xa = P[c - 1], xb = P[c + 1];
            const float2 ya = (r > 0) ? above[ix][i] : P[c - EX];
            const float2 yb = (r < NR - 1) ? own[r + 1][ix][i] : P[c + EX];
            float2 o;
            o.x = fma_(-ty, add_(ya.y, yb.y), fma_(-tx, add_(xa.y, xb.y), fma_(j.x, cc.y, mul_(j.z, cc.x))));
            o.y = fma_(ty, add_(ya.x, yb.x), fma_(tx, add_(xa.x, xb.x), fma_(-j.z, cc.y, mul_(-j.y, cc.x))));
            dst[i * EA + c] = o;
            own[r][ix][i] = o;
          }
          above[ix][i] = cc;
        }
      }
    }
    // interior of level a to global, from the registers
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int ly = ly0 + r - SK;
#pragma unroll
      for (int ix = 0; ix < NCX; ++ix) {
        const int lx = tx0 + 32 * ix - SK;
        const int gx = txi * TX + lx, gy = tyi * TY + ly;
        if (ly >= 0 && ly < TY && lx >= 0 && lx < TX && gx < nx && gy < ny) {
          const size_t g = (size_t)gy * nx + gx;
#pragma unroll
          for (int i = 0; i < 3; ++i) v[level(b, a, i, SK, S) + g] = own[r][ix][i];
        }
      }
    }
    __syncthreads();
    float2* tmp = src;
    src = dst;
    dst = tmp;
  }
}

// A store issued where it stands: the compiler may not sink it below later arithmetic.
// (Plain stores of each level's interior were all held back to the end of the tile,
// which kept every level's values live and doubled the registers of powers_warp.)
__device__ __forceinline__ void st_global_now(float2* p, float2 x) {
  asm volatile("st.global.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(x.x), "f"(x.y) : "memory");
}

// The same levels built by one warp per tile, in registers: lane l holds column l of a
// 32-wide extended tile (an interior 32 - 2 SK wide) over TY + 2 SK rows, one system at a
// time.  The x neighbours come from the adjacent lanes by shuffles and the y neighbours
// from the thread's own registers, so the form uses no shared memory and no block barrier;
// warps run their tiles independently.  Level a is valid on lanes and rows a .. end - a;
// the values outside (from the wrapped shuffles at lanes 0 and 31, or rows not updated)
// never reach the interior.  Same arithmetic on the same values as powers_tile, so the
// same basis bit for bit.
template <int SK, int TY>
__device__ __forceinline__ void powers_warp(const StepParams& p, const float4* __restrict__ jc,
                                            float2* __restrict__ v, const InstConst& C, int b, int tile) {
  constexpr int TX = 32 - 2 * SK, EY = TY + 2 * SK;
  static_assert(TX >= 1, "the warp's interior is 32 - 2 SK columns");
  const int S = p.S, nx = p.nx, ny = p.ny;
  const int tiles_x = (nx + TX - 1) / TX;
  const int tyi = tile / tiles_x, txi = tile - tyi * tiles_x;
  const int lane = threadIdx.x & 31;
  const int gx = txi * TX - SK + lane;           // this lane's column, before wrapping
  const int gxw = wrap(gx, nx);
  const int y0w = wrap(tyi * TY - SK, ny);       // the first row, wrapped
  const bool store_lane = lane >= SK && lane < SK + TX && gx < nx;
  const float4* jb = jc + plane(b, S);
  float jx[EY], jy[EY], jz[EY];
  {
    int yw = y0w;
#pragma unroll
    for (int r = 0; r < EY; ++r) {
      const float4 j = jb[yw * nx + gxw];          // S < 2^31: a plane's index fits an int
      jx[r] = j.x;
      jy[r] = j.y;
      jz[r] = j.z;
      yw = (yw + 1 == ny) ? 0 : yw + 1;
    }
  }
  const float tx = C.f_txt, ty = C.f_tyt;
#pragma unroll 1
  for (int i = 0; i < 3; ++i) {
    float2 u[EY];
    {
      const float2* v0 = v + level(b, 0, i, SK, S);
      int yw = y0w;
#pragma unroll
      for (int r = 0; r < EY; ++r) {
        u[r] = v0[yw * nx + gxw];
        yw = (yw + 1 == ny) ? 0 : yw + 1;
      }
    }
#pragma unroll
    for (int a = 1; a <= SK; ++a) {
      float2 ya = u[a - 1];                      // row r - 1 at level a - 1
#pragma unroll
      for (int r = a; r < EY - a; ++r) {
        const float2 cc = u[r], yb = u[r + 1];
        float2 xa, xb;
        xa.x = __shfl_up_sync(0xffffffffu, cc.x, 1);
        xa.y = __shfl_up_sync(0xffffffffu, cc.y, 1);
        xb.x = __shfl_down_sync(0xffffffffu, cc.x, 1);
        xb.y = __shfl_down_sync(0xffffffffu, cc.y, 1);
        float2 o;
        o.x = fma_(-ty, add_(ya.y, yb.y), fma_(-tx, add_(xa.y, xb.y), fma_(jx[r], cc.y, mul_(jz[r], cc.x))));
        o.y = fma_(ty, add_(ya.x, yb.x), fma_(tx, add_(xa.x, xb.x), fma_(-jz[r], cc.y, mul_(-jy[r], cc.x))));
        ya = cc;
        u[r] = o;
      }
      if (store_lane) {
        float2* va = v + level(b, a, i, SK, S) + (tyi * TY * nx + gx);
#pragma unroll
        for (int r = 0; r < TY; ++r)
          if (tyi * TY + r < ny) st_global_now(va + r * nx, u[SK + r]);
      }
    }
  }
}

// The same levels built by one warp walking down a strip of H rows (form 4), for the three
// systems together: lane l holds column l of a 32-wide strip (an interior 32 - 2 SK wide).
// At each row t of level 0 read, level a is formed at row t - a from level a - 1 at rows
// t - a - 1 .. t - a + 1, so each level keeps a window of three rows in registers and the
// y halo (SK rows above and below the strip) is computed once per strip instead of once
// per tile.  Row t + PD of level 0 and of J is loaded before row t is used, so PD rows of
// loads are in flight while the warp computes.  x neighbours come by shuffles, as in
// powers_warp.  Same arithmetic on the same values as powers_tile, so the same basis bit
// for bit.
template <int SK, int H, int PD>
__device__ __forceinline__ void powers_stream(const StepParams& p, const float4* __restrict__ jc,
                                              float2* __restrict__ v, const InstConst& C, int b, int strip) {
  constexpr int TX = 32 - 2 * SK, NR = H + 2 * SK;
  constexpr int RJ = SK + 1 + PD, R0 = 3 + PD;    // ring sizes: J rows, level-0 rows
  static_assert(TX >= 1, "the warp's interior is 32 - 2 SK columns");
  const int S = p.S, nx = p.nx, ny = p.ny;
  const int tiles_x = (nx + TX - 1) / TX;
  const int syi = strip / tiles_x, sxi = strip - syi * tiles_x;
  const int lane = threadIdx.x & 31;
  const int gx = sxi * TX - SK + lane;           // this lane's column, before wrapping
  const int gxw = wrap(gx, nx);
  const int gy0 = syi * H;                       // the strip's first interior row
  const bool store_lane = lane >= SK && lane < SK + TX && gx < nx;
  const float4* jb = jc + plane(b, S);
  const float2* v0 = v + level(b, 0, 0, SK, S);
  const float tx = C.f_txt, ty = C.f_tyt;
  float2 w0[3][R0];                              // level 0: [system][row mod R0]
  float2 w[3][SK > 1 ? SK - 1 : 1][3];           // levels 1 .. SK - 1: [system][level - 1][row mod 3]
  float jx[RJ], jy[RJ], jz[RJ];                  // J coefficients: row mod RJ
  int yw = wrap(gy0 - SK, ny);                   // the next level-0 row to load, wrapped
  auto load_row = [&](int t) {
    const int off = yw * nx + gxw;               // S < 2^31: a plane's index fits an int
    const float4 j = jb[off];
    jx[t % RJ] = j.x;
    jy[t % RJ] = j.y;
    jz[t % RJ] = j.z;
#pragma unroll
    for (int i = 0; i < 3; ++i) w0[i][t % R0] = v0[(size_t)i * S + off];
    yw = (yw + 1 == ny) ? 0 : yw + 1;
  };
#pragma unroll
  for (int t = 0; t < PD; ++t) load_row(t);
#pragma unroll
  for (int t = 0; t < NR; ++t) {
    if (t + PD < NR) load_row(t + PD);
#pragma unroll
    for (int a = 1; a <= SK; ++a) {
      const int r = t - a;                       // the row level a is formed at
      if (t < 2 * a) continue;                   // level a starts SK - a rows above the strip
      const int q = r % RJ;
      const bool st = r >= SK && r < SK + H && store_lane && gy0 + r - SK < ny;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float2 cc, ya, yb;
        if (a == 1) {
          cc = w0[i][r % R0];
          ya = w0[i][(r - 1) % R0];
          yb = w0[i][(r + 1) % R0];
        } else {
          cc = w[i][a - 2][r % 3];
          ya = w[i][a - 2][(r + 2) % 3];
          yb = w[i][a - 2][(r + 1) % 3];
        }
        float2 xa, xb;
        xa.x = __shfl_up_sync(0xffffffffu, cc.x, 1);
        xa.y = __shfl_up_sync(0xffffffffu, cc.y, 1);
        xb.x = __shfl_down_sync(0xffffffffu, cc.x, 1);
        xb.y = __shfl_down_sync(0xffffffffu, cc.y, 1);
        float2 o;
        o.x = fma_(-ty, add_(ya.y, yb.y), fma_(-tx, add_(xa.y, xb.y), fma_(jx[q], cc.y, mul_(jz[q], cc.x))));
        o.y = fma_(ty, add_(ya.x, yb.x), fma_(tx, add_(xa.x, xb.x), fma_(-jz[q], cc.y, mul_(-jy[q], cc.x))));
        if (a < SK) w[i][a - 1][r % 3] = o;
        if (st) st_global_now(v + level(b, a, i, SK, S) + ((size_t)(gy0 + r - SK) * nx + gx), o);
      }
    }
  }
}

// Asynchronous copies global -> shared (cp.async): each lane copies its own words, so a
// lane that waits for its own groups sees its own data without a warp barrier.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
               "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
               "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared memory of one warp of powers_stream_cp: rings of PD + 1 rows of J and of level 0.
template <int PD>
__host__ __device__ constexpr int pow_cp_warp_bytes() {
  return (PD + 1) * 32 * ((int)sizeof(float4) + 3 * (int)sizeof(float2));
}

// powers_stream with the rows staged through shared memory (form 5): row t + PD of J and
// of level 0 is copied asynchronously (cp.async) into a per-warp ring before row t is
// used, so PD rows of loads are in flight without holding registers.  Row t then moves
// from the ring into the same register windows as in powers_stream, and the levels are
// formed by the same code: the same basis bit for bit.
template <int SK, int H, int PD>
__device__ __forceinline__ void powers_stream_cp(const StepParams& p, const float4* __restrict__ jc,
                                                 float2* __restrict__ v, const InstConst& C, int b, int strip,
                                                 unsigned char* wsmem) {
  constexpr int TX = 32 - 2 * SK, NR = H + 2 * SK;
  constexpr int RS = PD + 1;                      // ring slots (rows t .. t + PD)
  static_assert(TX >= 1, "the warp's interior is 32 - 2 SK columns");
  const int S = p.S, nx = p.nx, ny = p.ny;
  const int tiles_x = (nx + TX - 1) / TX;
  const int syi = strip / tiles_x, sxi = strip - syi * tiles_x;
  const int lane = threadIdx.x & 31;
  const int gx = sxi * TX - SK + lane;
  const int gxw = wrap(gx, nx);
  const int gy0 = syi * H;
  const bool store_lane = lane >= SK && lane < SK + TX && gx < nx;
  const float4* jb = jc + plane(b, S);
  const float2* v0 = v + level(b, 0, 0, SK, S);
  float4* sj = reinterpret_cast<float4*>(wsmem);                     // [RS][32]
  float2* sv = reinterpret_cast<float2*>(wsmem + RS * 32 * sizeof(float4));   // [RS][3][32]
  const float tx = C.f_txt, ty = C.f_tyt;
  float2 w0[3][3];                                // level 0: [system][row mod 3]
  float2 w[3][SK > 1 ? SK - 1 : 1][3];            // levels 1 .. SK - 1
  float jx[SK + 1], jy[SK + 1], jz[SK + 1];       // J of rows t - SK .. t: row mod SK + 1
  int yw = wrap(gy0 - SK, ny);                    // the next row to copy, wrapped
  auto copy_row = [&](int t) {                    // row t into ring slot t mod RS, one group
    if (t < NR) {
      const int off = yw * nx + gxw;
      cp_async16(&sj[(t % RS) * 32 + lane], jb + off);
#pragma unroll
      for (int i = 0; i < 3; ++i) cp_async8(&sv[((t % RS) * 3 + i) * 32 + lane], v0 + (size_t)i * S + off);
      yw = (yw + 1 == ny) ? 0 : yw + 1;
    }
    cp_async_commit();                            // (empty past the last row: the count stays uniform)
  };
#pragma unroll
  for (int t = 0; t < PD; ++t) copy_row(t);
#pragma unroll
  for (int t = 0; t < NR; ++t) {
    copy_row(t + PD);
    cp_async_wait<PD>();                          // this lane's groups up to row t are complete
    {
      const float4 j = sj[(t % RS) * 32 + lane];
      jx[t % (SK + 1)] = j.x;
      jy[t % (SK + 1)] = j.y;
      jz[t % (SK + 1)] = j.z;
#pragma unroll
      for (int i = 0; i < 3; ++i) w0[i][t % 3] = sv[((t % RS) * 3 + i) * 32 + lane];
    }
#pragma unroll
    for (int a = 1; a <= SK; ++a) {
      const int r = t - a;
      if (t < 2 * a) continue;
      const int q = r % (SK + 1);
      const bool st = r >= SK && r < SK + H && store_lane && gy0 + r - SK < ny;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float2 cc, ya, yb;
        if (a == 1) {
          cc = w0[i][r % 3];
          ya = w0[i][(r + 2) % 3];
          yb = w0[i][(r + 1) % 3];
        } else {
          cc = w[i][a - 2][r % 3];
          ya = w[i][a - 2][(r + 2) % 3];
          yb = w[i][a - 2][(r + 1) % 3];
        }
        float2 xa, xb;
        xa.x = __shfl_up_sync(0xffffffffu, cc.x, 1);
        xa.y = __shfl_up_sync(0xffffffffu, cc.y, 1);
        xb.x = __shfl_down_sync(0xffffffffu, cc.x, 1);
        xb.y = __shfl_down_sync(0xffffffffu, cc.y, 1);
        float2 o;
        o.x = fma_(-ty, add_(ya.y, yb.y), fma_(-tx, add_(xa.y, xb.y), fma_(jx[q], cc.y, mul_(jz[q], cc.x))));
        o.y = fma_(ty, add_(ya.x, yb.x), fma_(tx, add_(xa.x, xb.x), fma_(-jz[q], cc.y, mul_(-jy[q], cc.x))));
        if (a < SK) w[i][a - 1][r % 3] = o;
        if (st) st_global_now(v + level(b, a, i, SK, S) + ((size_t)(gy0 + r - SK) * nx + gx), o);
      }
    }
  }
  cp_async_wait<0>();                             // nothing left in flight into this warp's ring
}

// Gram accumulators.  FP32 mode: products and per-thread sums in FP32, a
// pairwise (shuffle-tree) warp sum per entry, then FP64 across warps and blocks.
// For the monomial bases met here (s <= 10, ||J/theta|| <= 1) the normal
// equations are well enough conditioned that this gives the same least-squares
// residual as exact sums of the FP32 products; the FP32 basis vectors themselves
// set the accuracy of the inner solve.  FP64 mode: see warp_sum_f64.
template <typename TK> struct GramAcc;
template <> struct GramAcc<float> {
  float v;
  __device__ void zero() { v = 0.f; }
  __device__ void add(float2 a, float2 b) { v = fmaf(a.x, b.x, v); v = fmaf(a.y, b.y, v); }
};
template <> struct GramAcc<double> {
  double v;
  __device__ void zero() { v = 0.0; }
  __device__ void add(double2 a, double2 b) { v = fma(a.x, b.x, v); v = fma(a.y, b.y, v); }
};

// Warp sums of NE per-lane FP64 values, written to out[0..NE).  A butterfly per
// entry would cost 5 NE adds per lane on the FP64 pipe -- the pipe that bounds
// the Gram kernel.  Recursive halving instead: at offset o = 16, 8, 4, 2 each lane
// keeps the half of its live values picked by lane bit o and adds the partner's
// copy of that half; after four steps a lane holds P/16 entries (P = NE padded
// to a multiple of 16), which the o = 1 partner holds too.  About P adds per lane.
template <int NE>
__device__ __forceinline__ void warp_sum_f64(const GramAcc<double> (&acc)[NE], double* out, int lane) {
  constexpr int P = ((NE + 15) / 16) * 16;
  double x[P];
#pragma unroll
  for (int j = 0; j < P; ++j) x[j] = (j < NE) ? acc[j].v : 0.0;
  int base = 0;
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    const int o = 16 >> st;
    const int h = P >> (st + 1);
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < (P >> (st + 1)); ++j) {
      const double send = up ? x[j] : x[j + h];
      const double keep = up ? x[j + h] : x[j];
      x[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    if (up) base += h;
  }
#pragma unroll
  for (int j = 0; j < P / 16; ++j) x[j] += __shfl_xor_sync(0xffffffffu, x[j], 1);
  if ((lane & 1) == 0) {
#pragma unroll
    for (int j = 0; j < P / 16; ++j)
      if (base + j < NE) out[base + j] = x[j];
  }
}

template <int NE>
__device__ __forceinline__ void warp_sums(const GramAcc<float> (&acc)[NE], double* out, int lane) {
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    float r = acc[e].v;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) out[e] = f2d_bits(r);
  }
}
template <int NE>
__device__ __forceinline__ void warp_sums(const GramAcc<double> (&acc)[NE], double* out, int lane) {
  warp_sum_f64<NE>(acc, out, lane);
}

// Gram matrices G_ab = <v_a, v_b> (real inner product of the [p; q] form),
// a <= b <= s, of system i = blockIdx.y of instance blockIdx.z.  With CL > 1 the
// blocks form clusters of CL along x: each cluster's rank-0 block adds its
// members' block sums from their shared memory (distributed shared memory, in
// rank order) and writes one partial per cluster to
// part[((inst * 3 + i) * (gridDim.x / CL) + cluster) * NE + e].  The last
// cluster of system i to finish then
//  1. reduces that system's partials in a fixed order (so results do not depend
//     on which block finishes last),
//  2. forms the normal equations of the least-squares problem
//     min_c || b - (I - h lam_i J) sum_a c_a v_a ||:
//       (B^T G B) c = B^T G e_0,  B = [I; 0] - sig_i [0; I]  (s x s),
//  3. factors them with one warp (right-looking Cholesky; the basis is truncated
//     at the first pivot below trunc_rel times the larger of the leading one and
//     its own diagonal entry before elimination, a numerically exhausted Krylov
//     space whatever the scale of the levels; b = 0 gives c = 0) and solves.
// The three systems finish on three different blocks, in parallel.
// The Gram partial sums of one launch block of the Gram grid -- block bx of nbx, 256
// threads, system i of instance inst -- into blk[0..NE) (shared memory), complete and
// visible to the whole block on return.  Every thread of the block calls it.
template <typename TK, int SK>
__device__ __forceinline__ void gram_accumulate(const StepParams& p, const typename Vec2<TK>::type* __restrict__ v,
                                                int inst, int i, int bx, int nbx, double* blk) {
  typedef typename Vec2<TK>::type TK2;
  constexpr int NV = SK + 1;
  constexpr int NE = NV * (NV + 1) / 2;
  constexpr int U = 4;                          // sites whose loads are in flight together
  const int S = p.S;
  GramAcc<TK> acc[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) acc[e].zero();
  const int stride = nbx * blockDim.x;
  const TK2* vi = v + level(inst, 0, i, SK, S);
  const size_t lstride = (size_t)3 * S;         // from level a to level a+1 of the same system
  int k = bx * blockDim.x + threadIdx.x;
  for (; k + (U - 1) * stride < S; k += U * stride) {
    TK2 x[U][NV];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int a = 0; a < NV; ++a) x[u][a] = vi[(size_t)a * lstride + k + u * stride];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int e = 0;
#pragma unroll
      for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int c = a; c < NV; ++c) acc[e++].add(x[u][a], x[u][c]);
    }
  }
  for (; k < S; k += stride) {
    TK2 x[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) x[a] = vi[(size_t)a * lstride + k];
    int e = 0;
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int c = a; c < NV; ++c) acc[e++].add(x[a], x[c]);
  }
  __shared__ double red[8][NE];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  warp_sums<NE>(acc, red[warp], lane);
  __syncthreads();
  for (int e = threadIdx.x; e < NE; e += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][e];
    blk[e] = t;
  }
  __syncthreads();
}

// The last block of system i (by ticket) of instance inst: the fixed-order reduction of the
// nb partials, the normal equations and their Cholesky solve -> coef.  Every thread of
// the block calls it.
template <int SK>
__device__ void gram_lsq_solve(const StepParams& p, const double* __restrict__ part, double* __restrict__ coef,
                               const InstConst* __restrict__ ic, InstStatus* is, int inst, int i, int nb) {
  constexpr int NV = SK + 1;
  constexpr int NE = NV * (NV + 1) / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* pi = part + ((size_t)inst * 3 + i) * nb * NE;
  // 1. fixed-order reduction: thread t takes entry t % NE and partial slice t / NE.
  constexpr int SLICES = (256 / NE) > 0 ? (256 / NE) : 1;
  __shared__ double slice[SLICES][NE];
  __shared__ double G[NE];
  __shared__ double Nm[SK][SK + 1];             // [.., SK] holds the right-hand side
  __shared__ double rinv[SK];
  __shared__ double Ndiag[SK];                  // diagonal of the normal matrix before elimination
  for (int t = threadIdx.x; t < SLICES * NE; t += blockDim.x) {
    const int sl = t / NE, e = t - sl * NE;
    const int b0 = sl * nb / SLICES, b1 = (sl + 1) * nb / SLICES;
    const double* pp = pi + e;
    double q[4] = {0, 0, 0, 0};
    int bb = b0;
    for (; bb + 4 <= b1; bb += 4) {
      double w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = __ldcg(pp + (size_t)(bb + j) * NE);
#pragma unroll
      for (int j = 0; j < 4; ++j) q[j] += w[j];
    }
    for (int j = 0; bb < b1; ++bb, ++j) q[j] += __ldcg(pp + (size_t)bb * NE);
    slice[sl][e] = (q[0] + q[1]) + (q[2] + q[3]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NE; e += blockDim.x) {
    double sum = 0.0;
    for (int sl = 0; sl < SLICES; ++sl) sum += slice[sl][e];
    G[e] = sum;
  }
  __syncthreads();
  // 2. normal equations, all entries in parallel
  auto g = [&](int a, int c) -> double {
    if (a > c) { int t = a; a = c; c = t; }
    return G[a * NV - a * (a - 1) / 2 + (c - a)];
  };
  const double sg = p.precond ? -1.0 : ic[inst].sig[i];   // preconditioned: A z_a = v_a + v_{a+1}
  for (int t = threadIdx.x; t < SK * (SK + 1); t += blockDim.x) {
    const int a = t / (SK + 1), c = t - a * (SK + 1);
    Nm[a][c] = (c < SK) ? fma_(mul_(sg, sg), g(a + 1, c + 1), fma_(-sg, add_(g(a + 1, c), g(a, c + 1)), g(a, c)))
                        : fma_(-sg, g(a + 1, 0), g(a, 0));
    if (c == a) Ndiag[a] = Nm[a][c];
  }
  __syncthreads();
  // 3. one warp: Cholesky in place (lower triangle), then the two triangular solves,
  // with one reciprocal square root per pivot (kept in rinv) and no divisions.
  if (warp == 0) {
    int dim = (G[0] > 0.0) ? SK : 0;
    const double lead = Nm[0][0];
    for (int a = 0; a < dim; ++a) {
      const double dg = Nm[a][a];
      if (!(dg > (double)p.trunc_rel * fmax(lead, Ndiag[a]))) { dim = a; break; }
      const double il = rsqrt(dg);
      __syncwarp();
      for (int b2 = a + 1 + lane; b2 < SK; b2 += 32) Nm[b2][a] *= il;
      if (lane == 0) { Nm[a][a] = dg * il; rinv[a] = il; }
      __syncwarp();
      const int m = SK - a - 1;
      for (int idx = lane; idx < m * m; idx += 32) {
        const int b2 = a + 1 + idx / m, c = a + 1 + idx % m;
        if (c <= b2) Nm[b2][c] = fma_(-Nm[b2][a], Nm[c][a], Nm[b2][c]);
      }
      __syncwarp();
    }
    if (lane == 0) {
      double y[SK], cc[SK];
      for (int a = 0; a < dim; ++a) {
        double t = Nm[a][SK];
        for (int b2 = 0; b2 < a; ++b2) t = fma_(-Nm[a][b2], y[b2], t);
        y[a] = t * rinv[a];
      }
      for (int a = dim - 1; a >= 0; --a) {
        double t = y[a];
        for (int b2 = a + 1; b2 < dim; ++b2) t = fma_(-Nm[b2][a], cc[b2], t);
        cc[a] = t * rinv[a];
      }
      for (int a = 0; a < SK; ++a) coef[((size_t)inst * 3 + i) * kMaxS + a] = (a < dim) ? cc[a] : 0.0;
      is[inst].ticket_gram[i] = 0u;
    }
  }
}


// Newton update (Algorithm 1): rbar_i = sum_a c_ia v_a,i; dU_i += rbar_i in FP64 (from
// dU^0 = 0 the first iteration writes rbar); ||r||_inf with r = (T (x) I) rbar, merged over
// the blocks with an atomic max; NaN/Inf flagged.  No block waits for another: the loop
// test runs in k_newton_test once the whole grid has finished.  Grid: (sites / bs_update, B).
template <typename TK, int SK>
__device__ __forceinline__ void update_site_u(const StepParams& p, const typename Vec2<TK>::type* __restrict__ v,
                                              const TK (&cs)[3][SK], const double2 (&Uold)[3],
                                              double2* __restrict__ Ubar, bool first, int inst, int k, float& m,
                                              int& bad) {
  typedef typename Vec2<TK>::type TK2;
  const int S = p.S;
  TK2 x[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    TK sx = 0, sy = 0;
#pragma unroll
    for (int a = 0; a < SK; ++a) {
      const TK2 w = v[level(inst, a, i, SK, S) + k];
      sx = fma_(cs[i][a], w.x, sx);
      sy = fma_(cs[i][a], w.y, sy);
    }
    x[i].x = sx;
    x[i].y = sy;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double2 U;
    if (first) {
      U.x = to_double(x[i].x);
      U.y = to_double(x[i].y);
    } else {
      U = Uold[i];
      U.x += to_double(x[i].x);
      U.y += to_double(x[i].y);
    }
    Ubar[stage(inst, i, S) + k] = U;
  }
  // ||r||_inf with r = T rbar, in FP32: it only decides whether to iterate again.
  float xf[3][2];
#pragma unroll
  for (int i = 0; i < 3; ++i) { xf[i][0] = to_float(x[i].x); xf[i][1] = to_float(x[i].y); }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float t0 = p.fT[j][0], t1 = p.fT[j][1], t2 = p.fT[j][2];
    const float rx = fma_(t2, xf[2][0], fma_(t1, xf[1][0], mul_(t0, xf[0][0])));
    const float ry = fma_(t2, xf[2][1], fma_(t1, xf[1][1], mul_(t0, xf[0][1])));
    bad |= !(isfinite(rx) && isfinite(ry));
    m = fmaxf(m, fmaxf(fabsf(rx), fabsf(ry)));
  }
}

// dU of the site before the update (unread on the first iteration, which writes dU).
__device__ __forceinline__ void load_increments(const double2* __restrict__ Ubar, bool first, int inst, int S, int k,
                                                double2 (&Uold)[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) Uold[i] = first ? make_double2(0.0, 0.0) : Ubar[stage(inst, i, S) + k];
}

template <typename TK, int SK>
__device__ __forceinline__ void update_site(const StepParams& p, const typename Vec2<TK>::type* __restrict__ v,
                                            const TK (&cs)[3][SK], double2* __restrict__ Ubar, bool first,
                                            int inst, int k, float& m, int& bad) {
  double2 Uold[3];
  load_increments(Ubar, first, inst, p.S, k, Uold);
  update_site_u<TK, SK>(p, v, cs, Uold, Ubar, first, inst, k, m, bad);
}

// Merges the block's largest |r| and non-finite flag into instance I (one atomic each).
// Every thread of the block calls it.
__device__ __forceinline__ void block_update_flags(float m, int bad, InstStatus& I) {
  __shared__ float wmax[32];
  __shared__ int wbad[32];
  m = warp_max(m);
  bad = __any_sync(0xffffffffu, bad);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { wmax[warp] = m; wbad[warp] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float bm = wmax[0];
    int bb = wbad[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { bm = fmaxf(bm, wmax[w]); bb |= wbad[w]; }
    if (bm > 0.f) atomicMax(&I.rmax_bits, dbits((double)bm));
    if (bb) atomicOr(&I.nonfinite, 1);
  }
  __syncthreads();
}

// The loop test of a Newton iteration (failure rule of Sec. 2.2), one thread per instance
// that iterated: continue while ||r^l||_inf > rtol ||u0||_inf (and, when enabled, while the
// predicted remaining error is above newton_predict ||u0||_inf), for at most newton_max
// iterations.  The block then sets the WHILE condition: continue while any instance
// continues.  One block of up to 1024 threads.
// The test for every instance, by the threads of one block; returns (in every thread)
// whether any instance continues, and stores that in bc->any_cont.
static __device__ int newton_test_all(const StepParams& p, InstStatus* is, BatchCtl* bc) {
  int any = 0;
  for (int b = threadIdx.x; b < p.B; b += blockDim.x) {
    InstStatus& I = is[b];
    if (!I.active) continue;
    int cont = 0;
    const int it = I.newton_iter;                // iteration index l of this update
    const double r = __longlong_as_double((long long)I.rmax_bits);
    const double u0n = (double)__uint_as_float(I.u0max_bits);
    if (it < 8) I.hist[it] = r;
    I.last_rmax = r;
    I.last_u0max = u0n;
    I.newton_iter = it + 1;
    if (I.nonfinite || !isfinite(r)) {
      I.error = MB4_ERR_NONFINITE;
    } else if (r <= p.newton_rtol * u0n) {
      cont = 0;
    } else if (p.newton_predict > 0.0 && it >= 1 && r < 0.5 * I.prev_rmax &&
               (r / I.prev_rmax) / (1.0 - r / I.prev_rmax) * r <= p.newton_predict * u0n) {
      cont = 0;
    } else if (it + 1 >= p.newton_max) {
      I.error = MB4_ERR_NEWTON_NOT_CONVERGED;
    } else {
      cont = 1;
    }
    I.prev_rmax = r;
    I.last_newton_iters = it + 1;
    I.rmax_bits = 0ull;
    if (!cont) I.active = 0;
    any |= cont;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) bc->any_cont = any;
  return any;
}


}  // namespace mb4
