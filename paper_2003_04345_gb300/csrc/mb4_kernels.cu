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

namespace cg = cooperative_groups;

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
__global__ void __launch_bounds__(kSiteThreadsMax) k_setup(StepParams p, const double2* __restrict__ u,
                                               const double* __restrict__ D, double2* __restrict__ S0,
                                               JCoef<TK>* __restrict__ jc, typename Vec2<TK>::type* __restrict__ v,
                                               const double2* __restrict__ dUh, double2* __restrict__ dUb,
                                               const double* __restrict__ p_chi,
                                               const InstConst* __restrict__ ic, InstStatus* is) {
  const int b = blockIdx.y;
  if (!is[b].active) return;
  typedef typename Vec2<TK>::type TK2;
  const int S = p.S;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const InstConst& C = ic[b];
  float m = 0.f;
  if (k < S) {
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
    const TK pp = pk * pk, qq = qk * qk, nn = pp + qq;
    const TK dt = from_double<TK>(d) * kval<TK>(C.inv_theta, C.f_inv_theta);
    const double chik = p.chi_field ? p_chi[plane(b, S) + k] : 1.0;   // per-site chi (InstConst chi = 1)
    TK ct = kval<TK>(C.chi_theta, C.f_chi_theta);
    if (p.chi_field) ct *= from_double<TK>(chik);
    JCoef<TK> j;
    j.e1 = dt + ct * (pp + (TK)3 * qq);
    j.e2 = dt + ct * ((TK)3 * pp + qq);
    j.a = (TK)2 * ct * pk * qk;
    j.pad = (TK)0;
    jc[plane(b, S) + k] = j;
    if (is[b].predicted) {
      const int mo = min(is[b].pred_count, p.pred_order);
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
      TK cn = kval<TK>(C.chi, C.f_chi) * nn;
      if (p.chi_field) cn *= from_double<TK>(chik);
      const TK Fx = from_double<TK>(s0.x) + cn * pk, Fy = from_double<TK>(s0.y) + cn * qk;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        TK2 bi;
        const TK hc = kval<TK>(p.hTc[i], p.f_hTc[i]);
        bi.x = hc * Fy;
        bi.y = -hc * Fx;
        v[level(b, 0, i, p.s, S) + k] = bi;
      }
    }
    m = fmaxf(absf_of(c.x), absf_of(c.y));
  }
  // one atomic per block: same-address atomics queue at one L2 slice
  m = warp_max(m);
  __shared__ float wm[kSiteThreadsMax / 32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float bm = wm[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) bm = fmaxf(bm, wm[w]);
    if (bm > 0.f) atomicMax(&is[b].u0max_bits, __float_as_uint(bm));
  }
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
  typedef typename Vec2<TO>::type TO2;
  const int S = p.S;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S) return;
  const InstConst& C = ic[b];
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
    double nn = fma(Xx, Xx, Xy * Xy);
    if (CHIF) nn *= chik;
    const double gx = nn * Xx, gy = nn * Xy;
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

// ---------------------------------------------------------------------------
// Shifted solves (Algorithm 1; eq. MB4_5): one s-step GMRES cycle per
// system.  The Krylov space K_s(I - h lam_i J, b_i) = span{b_i, Jb_i, .., J^{s-1} b_i}
// is the same monomial space for all three shifts, so the basis
// v_{a+1} = (J/theta) v_a is built for the three right-hand sides together, and
// (I - h lam_i J) v_a = v_a - sig_i v_{a+1} with sig_i = h lam_i theta.
// ---------------------------------------------------------------------------
template <typename TK, int KM>
__global__ void __launch_bounds__(kSiteThreadsMax) k_matvec(StepParams p, const JCoef<TK>* __restrict__ jc,
                                                typename Vec2<TK>::type* __restrict__ v, int a_in,
                                                const InstConst* __restrict__ ic, const InstStatus* is) {
  pdl_wait();
  pdl_launch_dependents();
  const int b = blockIdx.y;
  if (!is[b].active) return;
  typedef typename Vec2<TK>::type TK2;
  const int S = p.S;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S) return;
  const JCoef<TK> j = jc[plane(b, S) + k];
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
      o.x = j.a * c.x + j.e1 * c.y + s.y;
      o.y = -j.e2 * c.x - j.a * c.y - s.x;
      v[level(b, a_in + 1, i, p.s, S) + k] = o;
    }
  } else {
    Nbr n = neighbours(k, p.nx, p.ny, S);
    const TK tx = kval<TK>(ic[b].txt, ic[b].f_txt), ty = kval<TK>(ic[b].tyt, ic[b].f_tyt);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const TK2* P = v + level(b, a_in, i, p.s, S);
      TK2 c = P[k], a = P[n.xm], bb = P[n.xp], e = P[n.ym], f = P[n.yp];
      TK2 o;
      // (J x)_re = a xp + e1 xq - tx (xq_x- + xq_x+) - ty (xq_y- + xq_y+)
      // (J x)_im = -e2 xp - a xq + tx (xp_x- + xp_x+) + ty (xp_y- + xp_y+)
      if constexpr (KM == 1) {                 // theta = tx: tx / theta = 1
        o.x = fma(j.a, c.x, fma(j.e1, c.y, -fma(ty, e.y + f.y, a.y + bb.y)));
        o.y = fma(-j.e2, c.x, fma(-j.a, c.y, fma(ty, e.x + f.x, a.x + bb.x)));
      } else {
        o.x = j.a * c.x + j.e1 * c.y - tx * (a.y + bb.y) - ty * (e.y + f.y);
        o.y = -j.e2 * c.x - j.a * c.y + tx * (a.x + bb.x) + ty * (e.x + f.x);
      }
      v[level(b, a_in + 1, i, p.s, S) + k] = o;
    }
  }
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
constexpr int kPowTX = 32, kPowTY = 16, kPowThreads = 256;

template <int SK>
__host__ __device__ constexpr int pow_ext_x() { return kPowTX + 2 * SK; }
template <int SK>
__host__ __device__ constexpr int pow_ext_y() { return kPowTY + 2 * SK; }
template <int SK>
constexpr size_t pow_smem_bytes() {
  return (size_t)pow_ext_x<SK>() * pow_ext_y<SK>() * (2 * 3 * sizeof(float2));
}

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

template <int SK>
__global__ void __launch_bounds__(kPowThreads) k_powers(StepParams p, const float4* __restrict__ jc,
                                                        float2* __restrict__ v, const InstConst* __restrict__ ic,
                                                        const InstStatus* is) {
  pdl_wait();
  pdl_launch_dependents();
  const int b = blockIdx.y;
  if (!is[b].active) return;
  constexpr int EX = pow_ext_x<SK>(), EY = pow_ext_y<SK>(), EA = EX * EY;
  constexpr int NCX = (EX + 31) / 32, NCY = (EY + 7) / 8;      // positions per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf0 = reinterpret_cast<float2*>(smem_raw);     // [3][EA]
  float2* buf1 = buf0 + 3 * EA;                           // [3][EA]
  const int S = p.S, nx = p.nx, ny = p.ny;
  const int tiles_x = (nx + kPowTX - 1) / kPowTX;
  const int tyi = blockIdx.x / tiles_x, txi = blockIdx.x - tyi * tiles_x;
  const int x0 = txi * kPowTX - SK, y0 = tyi * kPowTY - SK;
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
  const float tx = ic[b].f_txt, ty = ic[b].f_tyt;
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
          o.x = j.z * cc.x + j.x * cc.y - tx * (xa.y + xb.y) - ty * (ya.y + yb.y);
          o.y = -j.y * cc.x - j.z * cc.y + tx * (xa.x + xb.x) + ty * (ya.x + yb.x);
          dst[i * EA + c] = o;
        }
      }
    }
    __syncthreads();
    // interior of level a to global
    for (int ly = ty0; ly < kPowTY; ly += kPowThreads / 32) {
      const int lx = tx0;
      const int gx = txi * kPowTX + lx, gy = tyi * kPowTY + ly;
      if (gx < nx && gy < ny) {
        const int c = (ly + SK) * EX + (lx + SK);
        const size_t g = (size_t)gy * nx + gx;
#pragma unroll
        for (int i = 0; i < 3; ++i) v[level(b, a, i, SK, S) + g] = dst[i * EA + c];
      }
    }
    float2* tmp = src;
    src = dst;
    dst = tmp;
  }
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
template <typename TK, int SK, int CL>
__global__ void __launch_bounds__(256) k_gram_lsq(StepParams p, const typename Vec2<TK>::type* __restrict__ v,
                                                  double* __restrict__ part, double* __restrict__ coef,
                                                  const InstConst* __restrict__ ic, InstStatus* is) {
  pdl_wait();
  pdl_launch_dependents();
  const int inst = blockIdx.z;
  if (!is[inst].active) return;
  typedef typename Vec2<TK>::type TK2;
  constexpr int NV = SK + 1;
  constexpr int NE = NV * (NV + 1) / 2;
  constexpr int U = 4;                          // sites whose loads are in flight together
  const int S = p.S;
  const int i = blockIdx.y;
  GramAcc<TK> acc[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) acc[e].zero();
  const int stride = gridDim.x * blockDim.x;
  const TK2* vi = v + level(inst, 0, i, SK, S);
  const size_t lstride = (size_t)3 * S;         // from level a to level a+1 of the same system
  int k = blockIdx.x * blockDim.x + threadIdx.x;
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
  __shared__ double blk[NE];
  __shared__ bool is_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  warp_sums<NE>(acc, red[warp], lane);
  __syncthreads();
  for (int e = threadIdx.x; e < NE; e += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][e];
    blk[e] = t;
  }
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
    __syncthreads();
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
    Nm[a][c] = (c < SK) ? g(a, c) - sg * (g(a + 1, c) + g(a, c + 1)) + sg * sg * g(a + 1, c + 1)
                        : g(a, 0) - sg * g(a + 1, 0);
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
        if (c <= b2) Nm[b2][c] -= Nm[b2][a] * Nm[c][a];
      }
      __syncwarp();
    }
    if (lane == 0) {
      double y[SK], cc[SK];
      for (int a = 0; a < dim; ++a) {
        double t = Nm[a][SK];
        for (int b2 = 0; b2 < a; ++b2) t -= Nm[a][b2] * y[b2];
        y[a] = t * rinv[a];
      }
      for (int a = dim - 1; a >= 0; --a) {
        double t = y[a];
        for (int b2 = a + 1; b2 < dim; ++b2) t -= Nm[b2][a] * cc[b2];
        cc[a] = t * rinv[a];
      }
      for (int a = 0; a < SK; ++a) coef[((size_t)inst * 3 + i) * kMaxS + a] = (a < dim) ? cc[a] : 0.0;
      is[inst].ticket_gram[i] = 0u;
    }
  }
}

template <int SK>
void launch_powers_s(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  dim3 grid(((p.nx + kPowTX - 1) / kPowTX) * ((p.ny + kPowTY - 1) / kPowTY), p.B);
  launch_k(p.pdl != 0, k_powers<SK>, grid, dim3(kPowThreads), pow_smem_bytes<SK>(), s, p, (const float4*)b.jc,
           (float2*)b.v, (const InstConst*)b.ic, (const InstStatus*)b.is);
}

// Opt the matrix-powers kernels into more than 48 KB of dynamic shared memory.
int prepare_powers() {
#define MB4_ATTR(N)                                                                               \
  if (cudaFuncSetAttribute(k_powers<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                           (int)pow_smem_bytes<N>()) != cudaSuccess)                              \
    return MB4_ERR_CUDA;
  MB4_ATTR(1) MB4_ATTR(2) MB4_ATTR(3) MB4_ATTR(4) MB4_ATTR(5) MB4_ATTR(6) MB4_ATTR(7) MB4_ATTR(8) MB4_ATTR(9)
  MB4_ATTR(10)
#undef MB4_ATTR
  return MB4_OK;
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
  if (sizeof(TK) == sizeof(float) && p.use_powers) {
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

// Blocks per (instance, system) that keep the Gram kernel about one wave deep.
template <typename TK>
int gram_blocks_per_system(int s_dim, int B) {
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
  if (sizeof(TK) == sizeof(float) && nb >= kGramCluster) nb -= nb % kGramCluster;   // whole clusters
  return nb < 1 ? 1 : (int)nb;
}
template int gram_blocks_per_system<float>(int, int);
template int gram_blocks_per_system<double>(int, int);

template <typename TK>
void launch_krylov(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  if (p.precond) launch_precond_basis<TK>(p, b, s);
  else launch_matvecs<TK>(p, b, s);
  launch_gram<TK>(p, b, s);
}

// Newton update (Algorithm 1): rbar_i = sum_a c_ia v_a,i; dU_i += rbar_i in FP64 (from
// dU^0 = 0 the first iteration writes rbar); ||r||_inf with r = (T (x) I) rbar, merged over
// the blocks with an atomic max; NaN/Inf flagged.  No block waits for another: the loop
// test runs in k_newton_test once the whole grid has finished.  Grid: (sites / bs_update, B).
template <typename TK, int SK>
__global__ void __launch_bounds__(kSiteThreadsMax) k_update(StepParams p, const typename Vec2<TK>::type* __restrict__ v,
                                                const double* __restrict__ coef, double2* __restrict__ Ubar,
                                                InstStatus* is) {
  pdl_wait();
  pdl_launch_dependents();
  const int inst = blockIdx.y;
  InstStatus& I = is[inst];
  if (!I.active) return;
  typedef typename Vec2<TK>::type TK2;
  __shared__ TK cs[3][SK];
  __shared__ float wmax[8];
  __shared__ int wbad[8];
  if (threadIdx.x < 3 * SK)
    cs[threadIdx.x / SK][threadIdx.x % SK] =
        (TK)coef[((size_t)inst * 3 + threadIdx.x / SK) * kMaxS + threadIdx.x % SK];
  const bool first = I.newton_iter == 0 && !I.predicted;
  __syncthreads();
  const int S = p.S;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  float m = 0.f;
  int bad = 0;
  if (k < S) {
    TK2 x[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      TK sx = 0, sy = 0;
#pragma unroll
      for (int a = 0; a < SK; ++a) {
        const TK2 w = v[level(inst, a, i, SK, S) + k];
        sx += cs[i][a] * w.x;
        sy += cs[i][a] * w.y;
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
        U = Ubar[stage(inst, i, S) + k];
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
      const float rx = t0 * xf[0][0] + t1 * xf[1][0] + t2 * xf[2][0];
      const float ry = t0 * xf[0][1] + t1 * xf[1][1] + t2 * xf[2][1];
      bad |= !(isfinite(rx) && isfinite(ry));
      m = fmaxf(m, fmaxf(fabsf(rx), fabsf(ry)));
    }
  }
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
}

// The loop test of a Newton iteration (failure rule of Sec. 2.2), one thread per instance
// that iterated: continue while ||r^l||_inf > rtol ||u0||_inf (and, when enabled, while the
// predicted remaining error is above newton_predict ||u0||_inf), for at most newton_max
// iterations.  The block then sets the WHILE condition: continue while any instance
// continues.  One block of up to 1024 threads.
__global__ void k_newton_test(StepParams p, InstStatus* is, BatchCtl* bc, cudaGraphConditionalHandle h,
                              int use_cond) {
  pdl_wait();
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
  if (threadIdx.x == 0) {
    bc->any_cont = any;
    if (use_cond) cudaGraphSetConditional(h, any ? 1u : 0u);
  }
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
  if (b == 0) bc->any_cont = 0;
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
