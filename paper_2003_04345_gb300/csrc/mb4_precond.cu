// Spectrally preconditioned shifted solves (option precondition = 1).
//
// For stiff kinetic terms (the paper's own setup: K = -Laplacian with hx = 2 pi / 70,
// so h ||K|| ~ 10) the monomial Krylov basis of J cannot resolve the shifted systems
// (I - h lam_i J) x = b_i (Algorithm 1, the shifted solves) in a few vectors.  The constant-
// coefficient part of J is diagonal in Fourier space: with the on-site term replaced
// by its grid mean e and the cubic term's Jacobian dropped, J_c z = -i (K z + e z),
// so A_i ~ I + i h lam_i (K + e) has the per-mode multiplier
//   m_i(k) = 1 + i h lam_i (e - 2 tx cos(2 pi kx / nx) - 2 ty cos(2 pi ky / ny)),
// and P_i = (that operator)^-1 is applied by a 2D DFT, a pointwise division, and the
// inverse DFT.  Each system then takes the right-preconditioned Krylov space of
// A_i P_i in the shifted basis
//   z_a = P_i v_a,   v_{a+1} = A_i z_a - v_a = (A_i P_i - I) v_a,
// in which A_i z_a = v_a + v_{a+1}: the least squares over the Gram matrix of
// v_0..v_s is the one of the unpreconditioned path with sigma = -1, and the
// correction is rbar_i = sum_a c_a z_a (flexible form: the z_a are stored, so the
// rounding of P does not enter the relation).  The root of the step does not change.
//
// The DFTs are mixed-radix FFTs in the Krylov precision TK (self-sorting Stockham form:
// each stage of radix R maps sub-transforms of length Ns to length Ns R, with the
// twiddles exp(-2 pi i m / n) from one table), one block per grid line with the line, a
// scratch line and the twiddles in shared memory (at most 3 x 1024 x 16 B = 48 KB).
// A stage of radix R costs R complex multiply-adds per element: 14 for n = 70 (2, 5, 7),
// 20 for n = 1024 (4^5), n for a prime n.  Sides up to MB4_MAX_PRECOND_SIDE.
#include <cuda_runtime.h>

#include <cmath>
#include <initializer_list>
#include <vector>

#include "mb4_device.cuh"
#include "mb4_internal.h"

namespace mb4 {

template <typename TK>
__device__ __forceinline__ typename Vec2<TK>::type cmul(typename Vec2<TK>::type a, typename Vec2<TK>::type b) {
  typename Vec2<TK>::type r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// Radices of an FFT of length n (host): 4s first, then 2, 3, 5, 7, then the other primes.
int fft_radices(int n, int* rad) {
  int k = 0;
  for (int r : {4, 2, 3, 5, 7})
    while (n > 1 && n % r == 0) {
      rad[k++] = r;
      n /= r;
    }
  for (int r = 11; n > 1; r += 2)
    while (n % r == 0) {
      rad[k++] = r;
      n /= r;
    }
  return k;
}

// FFT of one line of n values in shared memory, out_k = sum_j a_j w^(j k) with the
// twiddles w[m] = exp(-2 pi i m / n) (conjugated when inverse).  Stage q of radix R
// (Ns = product of the earlier radices): output (j, t), j < n/R, t < R, k = j mod Ns, is
//   sum_s a[j + s n/R] exp(-2 pi i s (k / (Ns R) + t / R)),
// written to (j / Ns) Ns R + k + t Ns.  a and b alternate as input and output; returns
// the buffer holding the result.  Every thread of the block takes part (stages sync).
template <typename TK>
__device__ typename Vec2<TK>::type* fft_line(typename Vec2<TK>::type* a, typename Vec2<TK>::type* b,
                                             const typename Vec2<TK>::type* w, int n, const int* rad, int nrad,
                                             bool inverse) {
  typedef typename Vec2<TK>::type TK2;
  int Ns = 1;
  for (int q = 0; q < nrad; ++q) {
    const int R = rad[q], nb = n / R, tw = n / (Ns * R);
    for (int o = threadIdx.x; o < n; o += blockDim.x) {
      const int t = o / nb, j = o - t * nb, k = j % Ns;
      int e = k * tw + t * nb;                   // < 2n
      if (e >= n) e -= n;
      TK sx = 0, sy = 0;
      int m = 0;                                 // (s e) mod n
      for (int s = 0; s < R; ++s) {
        TK2 c = w[m];
        if (inverse) c.y = -c.y;
        const TK2 x = a[j + s * nb];
        sx += x.x * c.x - x.y * c.y;
        sy += x.x * c.y + x.y * c.x;
        m += e;
        if (m >= n) m -= n;
      }
      TK2 r;
      r.x = sx;
      r.y = sy;
      b[(j / Ns) * Ns * R + k + t * Ns] = r;
    }
    __syncthreads();
    TK2* tmp = a;
    a = b;
    b = tmp;
    Ns *= R;
  }
  return a;
}

// Row pass: src level (rows of nx) -> dst, forward or inverse (inverse scales by scale).
// Grid (ny, 3, B); dynamic shared memory 3 * nx TK2.
template <typename TK>
__global__ void k_dft_rows(StepParams p, const typename Vec2<TK>::type* __restrict__ src, size_t src_inst_stride,
                           typename Vec2<TK>::type* __restrict__ dst, size_t dst_inst_stride,
                           const typename Vec2<TK>::type* __restrict__ wx, int inverse, TK scale,
                           const InstStatus* is) {
  pdl_wait();
  pdl_launch_dependents();
  typedef typename Vec2<TK>::type TK2;
  const int y = blockIdx.x, i = blockIdx.y, b = blockIdx.z;
  if (!is[b].active) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TK2* line = reinterpret_cast<TK2*>(smem_raw);
  TK2* w = line + p.nx;
  TK2* scratch = w + p.nx;
  const size_t off_s = (size_t)b * src_inst_stride + (size_t)i * p.S + (size_t)y * p.nx;
  const size_t off_d = (size_t)b * dst_inst_stride + (size_t)i * p.S + (size_t)y * p.nx;
  for (int x = threadIdx.x; x < p.nx; x += blockDim.x) {
    line[x] = src[off_s + x];
    w[x] = wx[x];
  }
  __syncthreads();
  const TK2* r = fft_line<TK>(line, scratch, w, p.nx, p.fft_rx, p.fft_nrx, inverse != 0);
  for (int x = threadIdx.x; x < p.nx; x += blockDim.x) {
    TK2 o = r[x];
    o.x *= scale;
    o.y *= scale;
    dst[off_d + x] = o;
  }
}

// Column pass on buf (in place): forward FFT along y, multiply by 1 / m_i(kx, ky),
// inverse FFT along y.  Grid (nx, 3, B); dynamic shared memory 3 * ny TK2.
template <typename TK>
__global__ void k_dft_cols_apply(StepParams p, typename Vec2<TK>::type* __restrict__ buf, size_t inst_stride,
                                 const typename Vec2<TK>::type* __restrict__ wy,
                                 const typename Vec2<TK>::type* __restrict__ minv, const InstStatus* is) {
  pdl_wait();
  pdl_launch_dependents();
  typedef typename Vec2<TK>::type TK2;
  const int x = blockIdx.x, i = blockIdx.y, b = blockIdx.z;
  if (!is[b].active) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TK2* line = reinterpret_cast<TK2*>(smem_raw);
  TK2* w = line + p.ny;
  TK2* tmp = w + p.ny;
  TK2* col = buf + (size_t)b * inst_stride + (size_t)i * p.S + x;
  const TK2* mi = minv + ((size_t)b * 3 + i) * p.S + x;
  for (int y = threadIdx.x; y < p.ny; y += blockDim.x) {
    line[y] = col[(size_t)y * p.nx];
    w[y] = wy[y];
  }
  __syncthreads();
  TK2* f = fft_line<TK>(line, tmp, w, p.ny, p.fft_ry, p.fft_nry, false);
  for (int k = threadIdx.x; k < p.ny; k += blockDim.x) f[k] = cmul<TK>(f[k], mi[(size_t)k * p.nx]);
  __syncthreads();
  const TK2* r = fft_line<TK>(f, f == line ? tmp : line, w, p.ny, p.fft_ry, p.fft_nry, true);
  for (int y = threadIdx.x; y < p.ny; y += blockDim.x) col[(size_t)y * p.nx] = r[y];
}

// v_{a+1} = A_i z_a - v_a = z_a - sig_i (J/theta) z_a - v_a, J/theta from the per-site
// coefficients of k_setup.  Grid (sites / bs_matvec, B).
template <typename TK>
__global__ void __launch_bounds__(kSiteThreadsMax) k_pmatvec(StepParams p, const JCoef<TK>* __restrict__ jc,
                                                             typename Vec2<TK>::type* __restrict__ v,
                                                             const typename Vec2<TK>::type* __restrict__ z, int a,
                                                             const InstConst* __restrict__ ic, const InstStatus* is) {
  pdl_wait();
  pdl_launch_dependents();
  typedef typename Vec2<TK>::type TK2;
  const int b = blockIdx.y;
  if (!is[b].active) return;
  const int S = p.S;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= S) return;
  Nbr n = neighbours(k, p.nx, p.ny, S);
  const JCoef<TK> j = jc[plane(b, S) + k];
  const TK tx = kval<TK>(ic[b].txt, ic[b].f_txt), ty = kval<TK>(ic[b].tyt, ic[b].f_tyt);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const TK2* Z = z + level(b, a, i, p.s, S);
    const TK2 c = Z[k], l = Z[n.xm], r = Z[n.xp], d = Z[n.ym], u = Z[n.yp];
    const TK jx = j.a * c.x + j.e1 * c.y - tx * (l.y + r.y) - ty * (d.y + u.y);
    const TK jy = -j.e2 * c.x - j.a * c.y + tx * (l.x + r.x) + ty * (d.x + u.x);
    const TK sg = (TK)ic[b].sig[i];
    const TK2 va = v[level(b, a, i, p.s, S) + k];
    TK2 o;
    o.x = c.x - sg * jx - va.x;
    o.y = c.y - sg * jy - va.y;
    v[level(b, a + 1, i, p.s, S) + k] = o;
  }
}

template <typename TK>
void launch_precond_basis(const StepParams& p, const DevBuffers& b, cudaStream_t s) {
  typedef typename Vec2<TK>::type TK2;
  TK2* v = (TK2*)b.v;
  TK2* z = (TK2*)b.pz;
  TK2* t = (TK2*)b.ptmp;
  const size_t vstride = (size_t)(p.s + 1) * 3 * p.S;    // per instance, v and z
  const size_t tstride = (size_t)3 * p.S;
  const int rows_threads = p.nx < 256 ? ((p.nx + 31) / 32) * 32 : 256;
  const int cols_threads = p.ny < 256 ? ((p.ny + 31) / 32) * 32 : 256;
  const TK scale = (TK)(1.0 / ((double)p.nx * (double)p.ny));
  const dim3 gsite((p.S + p.bs_matvec - 1) / p.bs_matvec, p.B);
  for (int a = 0; a < p.s; ++a) {
    const size_t lev = (size_t)a * 3 * p.S;
    // z_a = P v_a: rows forward (v_a -> t), columns forward / 1/m / inverse (t), rows inverse (t -> z_a)
    launch_k(p.pdl != 0, k_dft_rows<TK>, dim3(p.ny, 3, p.B), dim3(rows_threads), 3 * p.nx * sizeof(TK2), s, p,
             (const TK2*)(v + lev), vstride, t, tstride, (const TK2*)b.pwx, 0, (TK)1, (const InstStatus*)b.is);
    launch_k(p.pdl != 0, k_dft_cols_apply<TK>, dim3(p.nx, 3, p.B), dim3(cols_threads), 3 * p.ny * sizeof(TK2), s, p,
             t, tstride, (const TK2*)b.pwy, (const TK2*)b.pminv, (const InstStatus*)b.is);
    launch_k(p.pdl != 0, k_dft_rows<TK>, dim3(p.ny, 3, p.B), dim3(rows_threads), 3 * p.nx * sizeof(TK2), s, p,
             (const TK2*)t, tstride, z + lev, vstride, (const TK2*)b.pwx, 1, scale, (const InstStatus*)b.is);
    launch_k(p.pdl != 0, k_pmatvec<TK>, gsite, dim3(p.bs_matvec), 0, s, p, (const JCoef<TK>*)b.jc, v,
             (const TK2*)z, a, (const InstConst*)b.ic, (const InstStatus*)b.is);
  }
}

// Twiddles exp(-2 pi i m / n), m < n, and the per-mode inverses 1 / m_i(k) of every
// instance and system, on the host in double and stored in TK.
template <typename TK>
int precond_tables(const StepParams& p, const double* ebar, const double* hlam_i, void* wx, void* wy, void* minv,
                   cudaStream_t s) {
  typedef typename Vec2<TK>::type TK2;
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<TK2> hx(p.nx), hy(p.ny);
  for (int m = 0; m < p.nx; ++m) {
    hx[m].x = (TK)std::cos(two_pi * m / p.nx);
    hx[m].y = (TK)-std::sin(two_pi * m / p.nx);
  }
  for (int m = 0; m < p.ny; ++m) {
    hy[m].x = (TK)std::cos(two_pi * m / p.ny);
    hy[m].y = (TK)-std::sin(two_pi * m / p.ny);
  }
  std::vector<TK2> hm((size_t)p.B * 3 * p.S);
  for (int b = 0; b < p.B; ++b)
    for (int i = 0; i < 3; ++i)
      for (int ky = 0; ky < p.ny; ++ky)
        for (int kx = 0; kx < p.nx; ++kx) {
          const double khat = ebar[b] - 2.0 * p.tx * std::cos(two_pi * kx / p.nx) -
                              2.0 * p.ty * std::cos(two_pi * ky / p.ny);
          const double im = hlam_i[i] * khat;    // m = 1 + i im, 1/m = (1 - i im) / (1 + im^2)
          const double den = 1.0 + im * im;
          TK2 q;
          q.x = (TK)(1.0 / den);
          q.y = (TK)(-im / den);
          hm[(((size_t)b * 3 + i) * p.ny + ky) * p.nx + kx] = q;
        }
  if (cudaMemcpyAsync(wx, hx.data(), hx.size() * sizeof(TK2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(wy, hy.data(), hy.size() * sizeof(TK2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(minv, hm.data(), hm.size() * sizeof(TK2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MB4_ERR_CUDA;
  return MB4_OK;
}

template void launch_precond_basis<float>(const StepParams&, const DevBuffers&, cudaStream_t);
template void launch_precond_basis<double>(const StepParams&, const DevBuffers&, cudaStream_t);
template int precond_tables<float>(const StepParams&, const double*, const double*, void*, void*, void*,
                                   cudaStream_t);
template int precond_tables<double>(const StepParams&, const double*, const double*, void*, void*, void*,
                                    cudaStream_t);

}  // namespace mb4
