// Internal declarations shared by the libmb4 translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/mb4.h"

namespace mb4 {

constexpr int kGauss = 6;          // Gauss-Legendre nodes: exact for the degree-11 integrand of eq. (fIu2)
constexpr int kMaxS = MB4_MAX_KRYLOV_S;
constexpr int kGramCap = 152;      // Gram blocks per (instance, system), at most
constexpr int kGramCluster = 8;    // thread-block cluster size of the Gram reduction
constexpr int kObsBlocksTotal = 152;   // observables: blocks over the whole batch
constexpr int kObsBlocksMax = 152;     // ... and per instance, at most
constexpr double kUnitGrowthMax = 4096.0;   // mv_unit: largest Gershgorin bound / |tx| accepted
constexpr int kUnrolledNewton = 2;  // Newton iterations of a step graph before its WHILE node
constexpr int kMaxFftStages = 12;  // radices of one FFT length <= MB4_MAX_PRECOND_SIDE (1024 = 4^5)

// MB4 constants in FP64, computed on the host (mb4_consts.cpp).
struct Constants {
  double alpha1, c[3];
  double E[3][4];        // E[i][j], i = 1..3 -> 0..2, j = 0..3 (j = 0: E_i0)
  double lam[3];         // eigenvalues of E(1:3,1:3), ascending
  double T[3][3];        // E3 = T diag(lam) Tinv, unit columns
  double Tinv[3][3];
  double gx[kGauss], gw[kGauss];   // Gauss-Legendre on [0, 1]
  double lag[4][4];      // l_j(zeta) = sum_p lag[j][p] zeta^p on nodes (0, c1, c2, c3)
  double Acoef[3][3];    // A_{c_i, zeta} = sum_b Acoef[i][b] zeta^b  (eq. Adefinition)
};

// Returns 0 or an MB4_ERR_* code (alpha1 out of range, bad nodes).
int compute_constants(double alpha1, double c1, double c2, Constants* out);

// Constants shared by every instance of a batch (one grid shape and h), passed
// by value in kernel parameter space.
struct StepParams {
  int nx, ny, S, B;
  int s;                   // Krylov subspace dimension
  int gram_blocks;         // Gram blocks per (instance, system)
  int use_powers;          // FP32 basis: one tiled matrix-powers launch instead of s stencil launches
  int pow_shape;           // its tile shape (kPowShapeTX/TY index; the tuner's choice, 0 = 32 x 16)
  int pdl;                 // programmatic dependent launch inside the Newton loop
  int precond;             // spectral preconditioning of the shifted solves (mb4_precond.cu)
  // radices of the preconditioner's FFTs along x and y (product nx, ny; none for 1)
  int fft_nrx, fft_nry;
  int fft_rx[kMaxFftStages], fft_ry[kMaxFftStages];
  int chi_field;           // chi per site (DevBuffers::chi); InstConst then holds chi = 1
  // general kinetic matrix (mb4_create_sparse) instead of the grid stencil: K = onsite I + T,
  // T's off-diagonal in slot-major ELL form, nbr[e * S + k] = j or -1, w = K_kj (FP64) and
  // wt = K_kj / theta in the Krylov precision, e < ell_deg
  int ell, ell_deg;
  int ell_cplx;            // complex Hermitian K: ell_w holds double2 (re, im), ell_wt Vec2<TK>
  // grid stencil with the x hopping factored out (tx != 0): the residual reads D / tx
  // (DevBuffers::dtx) and forms h lam_i tx (D/tx x - (x_x- + x_x+) - (ty/tx)(x_y- + x_y+)),
  // one FP64 instruction less per component than h lam_i (D x - tx (..) - ty (..))
  int kin_unit;
  // FP64 basis built from J / tx (theta = tx): the x neighbours' coefficient is then 1
  // and the matvec spends 5 FP64 instructions per component instead of 6
  int mv_unit;
  const int* ell_nbr;
  const void* ell_w;       // double (real K) or double2 (complex K)
  const void* ell_wt;
  int persistent;          // the step as one persistent kernel with grid barriers (mb4_persist.cu)
  int pers_blocks;         // its grid: co-resident blocks of kPersistThreads
  long long wait_limit;    // polls of a grid-barrier wait before it gives up (MB4_ERR_TIMEOUT)
  int bs_site, bs_residual, bs_matvec, bs_update;   // threads per block of the per-site kernels
                                                    // (bs_site: k_setup, k_accept)
  int pred_order;          // Newton start: 0 = e3 (x) u0; m = extrapolate the last m increments
  int pred_adaptive;       // choose per instance between the two starts by measured cost
  int pred_cost_milli;     // the extrapolated start's extra residual, in 1/1000 Newton iterations
  int explore_every;       // steps between tries of the start not currently preferred
  double tx, ty, eps0, h;
  // residual in the eigenbasis of E on the increments dU = Tinv (U - e3 (x) u0)
  double hlam[3];          // h * lambda_i
  double hltx[3];          // h * lambda_i * tx (kin_unit)
  double rty;              // ty / tx (kin_unit)
  double hTc[3];           // h * (Tinv c)_i : the (K+V) u0 coefficient, and Phibar^0 = i hTc_i f(u0)-part
  double LT[kGauss][3];    // sum_m l_m(zeta_q) T[m][n]:  X_q = u0 + sum_n LT[q][n] dU_n
  double T[3][3];          // r = T rbar ;  u1 = u0 + sum_n T[2][n] dU_n
  double newton_rtol;
  double newton_predict;   // 0: off; else Hairer-Wanner predicted-error stop
  int newton_max;
  float trunc_rel;         // relative pivot threshold of the Gram Cholesky
  // FP32 copies of uniform constants (no per-thread conversions on the FP64 pipe)
  float fT[3][3];
  float f_hTc[3];
};

// Per-instance constants (device array of B).  theta scales the monomial basis,
// v_{a+1} = (J/theta) v_a.  By default it bounds the spectral radius of J
// (Gershgorin: max|onsite + V| + 2|tx| + 2|ty|), so that the vectors stay O(1); with
// mv_unit it is tx, and level a grows by at most (Gershgorin bound / |tx|)^a, a factor
// kept below kUnitGrowthMax per level.
struct InstConst {
  double hchiW[3][kGauss]; // h chi (Tinv W)_iq, W_jq = w_q A_{c_j}(zeta_q)
  double chi, chi_theta;
  double inv_theta;        // 1 / theta
  double txt, tyt;         // tx / theta, ty / theta
  double sig[3];           // h lambda_i theta
  float f_chi, f_chi_theta, f_inv_theta, f_txt, f_tyt;
};

// Per-instance Newton status (device array of B).
struct InstStatus {
  int error;                         // MB4_OK or MB4_ERR_*
  int enabled;                       // set by the host: step this instance
  int in_step;                       // takes part in the current step
  int active;                        // still iterating in the current step
  int newton_iter;                   // iterations of the current step
  int nonfinite;                     // set by update kernels
  int last_newton_iters;
  unsigned int u0max_bits;           // ||u0||_inf of the current step (float bits, >= 0)
  unsigned int ticket_gram[3];       // last-block tickets, one per shifted system (reset by the last block)
  int pred_count;                    // converged increments kept for the Newton start (<= pred_order)
  int predicted;                     // the current step started from an extrapolation
  int next_predicted;                // start chosen for the next step (adaptive mode)
  int start_known;                   // bit m: start_iters[m] holds a measurement
  int start_iters[2];                // Newton iterations of the last step with start m (0: e3 (x) u0)
  int explore_in;                    // steps until the other start is tried again
  unsigned long long rmax_bits;      // max |r| of the current iteration (double bits, >= 0)
  long long steps_done;              // accepted steps since the last reset
  long long newton_total;
  double prev_rmax;                  // ||r^(l-1)||_inf
  double last_rmax;
  double last_u0max;
  double hist[8];                    // ||r^l||_inf of the current step
};

// Batch-wide loop control.
struct BatchCtl {
  int any_cont;                      // some instance continues its Newton loop (k_newton_test)
  int abort;                         // persistent step: a block's bounded barrier wait ran out
                                     // (every instance of the step then carries MB4_ERR_TIMEOUT)
  int pad[2];
};

// Grid barrier of the persistent step kernel: blocks arrive in groups of kBarGroup, each
// group with its own counter and release word in a slot of its own 128-byte line (slot 0
// counts the groups), so no cache line sees more than kBarGroup arrivals or pollers.
constexpr int kBarGroup = 16;
constexpr int kBarSlotWords = 32;    // unsigned ints per slot: [0] arrivals, [1] generation

// Device buffers of one batch.
struct DevBuffers {
  double2* u;        // state, B*S
  double* V;         // potential, B*S
  double* d;         // onsite + V, B*S
  double* dtx;       // (onsite + V) / tx, B*S (kin_unit only)
  double2* S0;       // (K+V) u0, B*S
  double2* Ubar;     // transformed stage increments dU, B*3*S
  double2* dU_hist;  // converged dU of the last pred_order steps, newest first: B*pred_order*3*S (or null)
  void* jc;          // J coefficients {e1, e2, a, 0} (TK4), B*S
  void* v;           // Krylov basis, B*(s+1)*3*S of TK2; level 0 = right-hand side b
  double* gram_part; // B*3*gram_blocks*nent (per-cluster partials use the first part)
  double* coef;      // B*3*kMaxS least-squares coefficients
  double* obs_part;  // observables partial sums
  double* obs_out;   // B*6
  double* chi;       // per-site chi, B*S (chi_field only)
  // spectral preconditioner (precond only): z_a = P v_a (layout of v), a DFT work plane
  // triple per instance, twiddles along x and y, per-mode inverse multipliers B*3*S (TK2)
  void* pz;
  void* ptmp;
  void* pwx;
  void* pwy;
  void* pminv;
  InstConst* ic;     // B
  InstStatus* is;    // B
  BatchCtl* bc;
  unsigned int* bar; // persistent step only: (1 + groups) x kBarSlotWords barrier slots
};

// The observables of every instance of a batch, enqueued on the batch's stream and copied
// to host_out (batch x 6 doubles; page-locked memory for the copy to be asynchronous)
// without waiting (mb4_capi.cu).  For the serving loop, which reads them once a later
// event on that stream has completed.
int batch_observables_async(mb4_batch* b, double* host_out);

// Host launchers (mb4_kernels.cu).  TK = float (mixed) or double (fp64).
template <typename TK> void launch_setup(const StepParams& p, const DevBuffers& b, cudaStream_t st);
template <typename TK> void launch_residual(const StepParams& p, const DevBuffers& b, bool skip_first,
                                            cudaStream_t st);
template <typename TK> void launch_krylov(const StepParams& p, const DevBuffers& b, cudaStream_t st);
// the two parts of launch_krylov, for profiling
template <typename TK> void launch_matvecs(const StepParams& p, const DevBuffers& b, cudaStream_t st);
template <typename TK> void launch_gram(const StepParams& p, const DevBuffers& b, cudaStream_t st);
// Raise the dynamic shared-memory limit of the matrix-powers kernels (once per process/device).
int prepare_powers();
// Blocks per (instance, system) that make the Gram kernel about one wave (0 on error).
template <typename TK> int gram_blocks_per_system(int s_dim, int B, int S);
// Newton update and loop test; cond_handle drives the graph's WHILE node when use_cond.
template <typename TK> void launch_update(const StepParams& p, const DevBuffers& b, unsigned long long cond_handle,
                                          int use_cond, cudaStream_t st);
void launch_accept(const StepParams& p, const DevBuffers& b, cudaStream_t st);
void launch_arm(const StepParams& p, const DevBuffers& b, cudaStream_t st);
// Persistent step (mb4_persist.cu): set-up and the whole Newton loop of one step of every
// instance in one cooperative launch; launch_accept follows it.  persistent_supported tells
// whether this (precision, s, kinetic form, chi field) has a persistent kernel;
// persistent_blocks returns its co-resident grid (0 on error) and sets its attributes.
constexpr int kPersistThreads = 256;
bool persistent_supported(const StepParams& p, bool mixed);
int persistent_blocks(const StepParams& p, bool mixed);
cudaError_t launch_step_persistent(const StepParams& p, const DevBuffers& b, bool mixed, cudaStream_t st);
// Write n = ninst * S sites of state from re/im into u starting at instance first; an
// instance whose state changes (any bit) forgets its Newton-start history.
void launch_set_state(const StepParams& p, const DevBuffers& b, const double* re, const double* im, int first,
                      int ninst, cudaStream_t st);
// Drop the Newton-start history of instances first .. first + ninst - 1.
void launch_forget_range(const StepParams& p, const DevBuffers& b, int first, int ninst, cudaStream_t st);
int obs_blocks_per_instance(int B);
void launch_observables(const StepParams& p, const DevBuffers& b, cudaStream_t st);
// Y_j += sign * x on three complex planes of S sites.
void launch_add_plane3(int S, double2* Y, const double2* x, double sign, cudaStream_t st);
// Y_j = sum_n M[j][n] X_n on three complex planes of S sites.
void launch_mix3(int S, const double2* X, double2* Y, const double M[3][3], cudaStream_t st);
template <typename TK> void launch_copy_rhs_in(const StepParams& p, const DevBuffers& b, const double2* b3,
                                               cudaStream_t st);
template <typename TK> void launch_copy_solution_out(const StepParams& p, const DevBuffers& b,
                                                     double2* x3, cudaStream_t st);
template <typename TK> void launch_residual_out(const StepParams& p, const DevBuffers& b, double2* phibar3,
                                                cudaStream_t st);
void launch_pack(const double* re, const double* im, double2* z, size_t n, cudaStream_t st);
// Preconditioned Krylov basis (mb4_precond.cu): z_a = P_i v_a, v_{a+1} = A_i z_a - v_a, a < s.
template <typename TK> void launch_precond_basis(const StepParams& p, const DevBuffers& b, cudaStream_t st);
// Radices of an FFT of length n: 4s, then 2, 3, 5, 7, then any other prime factor.
int fft_radices(int n, int* rad);
// Twiddles and per-mode inverse multipliers 1 / (1 + i h lam_i (ebar_b + Khat(k))) (host-made).
template <typename TK>
int precond_tables(const StepParams& p, const double* ebar, const double* hlam_i, void* wx, void* wy, void* minv,
                   cudaStream_t st);
void launch_unpack(const double2* z, double* re, double* im, size_t n, cudaStream_t st);

}  // namespace mb4
