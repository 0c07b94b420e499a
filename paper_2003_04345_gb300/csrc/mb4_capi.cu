// libmb4 C ABI: batches and single contexts, device buffers, the step graph
// and the entry points declared in include/mb4.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "mb4_internal.h"
#include "mb4_phases.cuh"

using namespace mb4;

struct mb4_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  int precision = MB4_FP64;
  int use_graph = 1;
  int B = 1;
  Constants k{};
  StepParams p{};
  DevBuffers b{};
  size_t tk = 8;                  // sizeof(TK)
  // step graph (one launch = one MB4 step of every instance)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle handle = 0;
  // scratch for state I/O and the test entry points (allocated on first use)
  double2* tmp3a = nullptr;
  double2* tmp3b = nullptr;
  double* io = nullptr;           // 6*max(B*S, S) doubles
  std::vector<void*> allocs;
  std::vector<InstStatus> host_status;
  bool err_seen = false;          // a wait saw an instance error that clear_errors has not cleared
  // device step counters at the last wait: stats report the steps since then
  std::vector<long long> base_steps, base_newton;
  std::vector<double> ebar;       // per instance: mean of onsite + V (spectral preconditioner)
  int* ell_nbr = nullptr;         // general kinetic matrix (mb4_create_sparse), device
  void* ell_w = nullptr;          // double, or double2 for a complex K
  void* ell_wt = nullptr;
  bool forced_tile = false;       // option powers_tile set: the tuner keeps it
};

struct mb4_ctx : mb4_batch {};

namespace {

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return MB4_OK;
  if (e == cudaErrorMemoryAllocation) return MB4_ERR_OUT_OF_MEMORY;
  return MB4_ERR_CUDA;
}

#define MB4_TRY(call)                        \
  do {                                       \
    int _rc = cuda_rc(call);                 \
    if (_rc != MB4_OK) return _rc;           \
  } while (0)

#define MB4_CHECK(call)                      \
  do {                                       \
    int _rc = (call);                        \
    if (_rc != MB4_OK) return _rc;           \
  } while (0)

size_t round256(size_t bytes) { return (bytes + 255) & ~size_t(255); }

int dalloc(mb4_batch* c, void** ptr, size_t bytes) {
  // 256-byte aligned by cudaMalloc; sizes rounded up so every array keeps that alignment.
  cudaError_t e = cudaMalloc(ptr, round256(bytes));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return cuda_rc(e);
  }
  c->allocs.push_back(*ptr);
  return MB4_OK;
}

int validate_options(const mb4_options* in, mb4_options* o) {
  if (in) *o = *in;
  else mb4_default_options(o);
  if (o->precision != MB4_FP64 && o->precision != MB4_MIXED) return MB4_ERR_INVALID_ARG;
  if (!(o->newton_predict >= 0.0)) return MB4_ERR_INVALID_ARG;
  // Measured on GB300 at 512x512: with the update test alone the Newton loop takes
  // 4 iterations for s >= 4, so s = 4 is cheapest; the predicted-error test cuts
  // it to 3 from s = 5 on.
  if (o->krylov_s == 0) o->krylov_s = (o->newton_predict > 0.0) ? 5 : 4;
  if (o->krylov_s < 1 || o->krylov_s > MB4_MAX_KRYLOV_S) return MB4_ERR_INVALID_ARG;
  if (!(o->newton_rtol > 0.0) || o->newton_max < 1) return MB4_ERR_INVALID_ARG;
  if (o->overlap_launches != 0 && o->overlap_launches != 1) return MB4_ERR_INVALID_ARG;
  if (o->newton_start < 0 || o->newton_start > MB4_MAX_NEWTON_START) return MB4_ERR_INVALID_ARG;
  if (o->newton_start_adaptive != 0 && o->newton_start_adaptive != 1) return MB4_ERR_INVALID_ARG;
  if (o->autotune != 0 && o->autotune != 1) return MB4_ERR_INVALID_ARG;
  if (o->site_threads != 0 && o->site_threads != 64 && o->site_threads != 128 && o->site_threads != 256)
    return MB4_ERR_INVALID_ARG;
  if (o->precondition != 0 && o->precondition != 1) return MB4_ERR_INVALID_ARG;
  if (o->site_chi != 0 && o->site_chi != 1) return MB4_ERR_INVALID_ARG;
  if (o->persistent != 0 && o->persistent != 1) return MB4_ERR_INVALID_ARG;
  if (o->wait_limit < 0) return MB4_ERR_INVALID_ARG;
  if (o->powers_tile < 0 || o->powers_tile > kPowShapes + 1) return MB4_ERR_INVALID_ARG;
  if (o->powers_tile > 1 && o->powers_tile <= kPowShapes && o->krylov_s > kPowShapeMaxS) return MB4_ERR_INVALID_ARG;
  return MB4_OK;
}

int validate_grid(const mb4_grid* grid, int B) {
  if (!grid || B < 1) return MB4_ERR_INVALID_ARG;
  if (grid->nx < 3 || grid->ny < 3) return MB4_ERR_INVALID_ARG;
  if ((long long)grid->nx * grid->ny > (1LL << 30)) return MB4_ERR_INVALID_ARG;
  if ((long long)grid->nx * grid->ny * B > (1LL << 34)) return MB4_ERR_INVALID_ARG;
  if (!std::isfinite(grid->tx) || !std::isfinite(grid->ty) || !std::isfinite(grid->onsite))
    return MB4_ERR_INVALID_ARG;
  return MB4_OK;
}

// theta for one instance: a Gershgorin bound on the spectral radius of J (onsite+V part).
double instance_theta(const StepParams& p, const double* V, size_t S) {
  double vmax = 0.0;
  for (size_t k = 0; k < S; ++k) vmax = std::fmax(vmax, std::fabs(p.eps0 + V[k]));
  double theta = vmax + 2.0 * std::fabs(p.tx) + 2.0 * std::fabs(p.ty);
  return (theta > 0.0) ? theta : 1.0;
}

// D / tx for the residual's factored stencil (kin_unit); false if a ratio overflows.
bool fill_dtx(const StepParams& p, const double* D, size_t n, std::vector<double>* out) {
  out->resize(n);
  for (size_t k = 0; k < n; ++k) {
    (*out)[k] = D[k] / p.tx;
    if (!std::isfinite((*out)[k])) return false;
  }
  return true;
}

// The basis scale of an instance: tx with mv_unit (refused, -1, when the Gershgorin
// bound exceeds kUnitGrowthMax |tx|), else the Gershgorin bound.
double basis_theta(const StepParams& p, const double* V, size_t S) {
  const double g = instance_theta(p, V, S);
  if (!p.mv_unit) return g;
  return (g <= kUnitGrowthMax * std::fabs(p.tx)) ? p.tx : -1.0;
}

void fill_inst_const(const mb4_batch* c, double chi, double theta, InstConst* out) {
  const Constants& K = c->k;
  std::memset(out, 0, sizeof(*out));
  for (int q = 0; q < kGauss; ++q) {
    const double z = K.gx[q];
    double W[3];
    for (int j = 0; j < 3; ++j) W[j] = K.gw[q] * ((K.Acoef[j][2] * z + K.Acoef[j][1]) * z + K.Acoef[j][0]);
    for (int i = 0; i < 3; ++i) {
      double s = 0;
      for (int j = 0; j < 3; ++j) s += K.Tinv[i][j] * W[j];
      out->hchiW[i][q] = c->p.h * chi * s;
    }
  }
  out->chi = chi;
  out->chi_theta = chi / theta;
  out->inv_theta = 1.0 / theta;
  out->txt = c->p.tx / theta;
  out->tyt = c->p.ty / theta;
  for (int i = 0; i < 3; ++i) out->sig[i] = c->p.h * K.lam[i] * theta;
  out->f_chi = (float)chi;
  out->f_chi_theta = (float)(chi / theta);
  out->f_inv_theta = (float)(1.0 / theta);
  out->f_txt = (float)(c->p.tx / theta);
  out->f_tyt = (float)(c->p.ty / theta);
}

void fill_params(mb4_batch* c, const mb4_grid* grid, double h, const mb4_options& o) {
  StepParams& p = c->p;
  const Constants& K = c->k;
  p.nx = grid->nx;
  p.ny = grid->ny;
  p.S = grid->nx * grid->ny;
  p.B = c->B;
  p.s = o.krylov_s;
  p.pdl = o.overlap_launches;
  p.precond = o.precondition;
  p.chi_field = o.site_chi;
  p.bs_site = p.bs_residual = p.bs_matvec = p.bs_update = o.site_threads > 0 ? o.site_threads : 128;
  p.pred_order = o.newton_start;
  p.persistent = o.persistent;
  p.pow_shape = o.powers_tile > 0 ? o.powers_tile - 1 : 0;
  p.wait_limit = o.wait_limit;
  p.pred_adaptive = o.newton_start_adaptive;
  // Cost of the extra residual of an extrapolated start, in Newton iterations (1/1000):
  // measured at 512x512, s = 4: residual 78 us of a 239 us FP64 iteration, of a 134 us
  // mixed one.
  p.pred_cost_milli = (o.precision == MB4_MIXED) ? 580 : 330;
  p.explore_every = 32;
  p.tx = grid->tx;
  p.ty = grid->ty;
  p.eps0 = grid->onsite;
  p.h = h;
  p.rty = (grid->tx != 0.0) ? grid->ty / grid->tx : 0.0;
  for (int i = 0; i < 3; ++i) {
    p.hlam[i] = h * K.lam[i];
    p.hltx[i] = p.hlam[i] * grid->tx;
    double tc = 0;
    for (int j = 0; j < 3; ++j) tc += K.Tinv[i][j] * K.c[j];
    p.hTc[i] = h * tc;
    for (int j = 0; j < 3; ++j) p.T[i][j] = K.T[i][j];
  }
  for (int q = 0; q < kGauss; ++q) {
    const double z = K.gx[q];
    double l[4];
    for (int j = 0; j < 4; ++j) l[j] = ((K.lag[j][3] * z + K.lag[j][2]) * z + K.lag[j][1]) * z + K.lag[j][0];
    for (int n = 0; n < 3; ++n) {
      double s = 0;
      for (int m = 0; m < 3; ++m) s += l[m + 1] * K.T[m][n];
      p.LT[q][n] = s;
    }
  }
  p.newton_rtol = o.newton_rtol;
  p.newton_predict = o.newton_predict;
  p.newton_max = o.newton_max;
  p.trunc_rel = (o.precision == MB4_MIXED) ? 1e-12f : 1e-26f;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) p.fT[i][j] = (float)p.T[i][j];
    p.f_hTc[i] = (float)p.hTc[i];
  }
}

template <typename TK>
void enqueue_newton_body(mb4_batch* c, cudaStream_t s, unsigned long long handle, int use_cond) {
  launch_residual<TK>(c->p, c->b, true, s);
  launch_krylov<TK>(c->p, c->b, s);
  launch_update<TK>(c->p, c->b, handle, use_cond, s);
}

void enqueue_body(mb4_batch* c, cudaStream_t s, unsigned long long handle, int use_cond) {
  if (c->precision == MB4_MIXED) enqueue_newton_body<float>(c, s, handle, use_cond);
  else enqueue_newton_body<double>(c, s, handle, use_cond);
}

void enqueue_setup(mb4_batch* c, cudaStream_t s) {
  if (c->precision == MB4_MIXED) launch_setup<float>(c->p, c->b, s);
  else launch_setup<double>(c->p, c->b, s);
}

// One MB4 step as a graph: setup -> kUnrolledNewton x {residual, basis, gram+lsq, update,
// test} -> WHILE(any instance continues){the same} -> accept.
int build_graph(mb4_batch* c) {
  cudaStream_t cap;
  MB4_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  int rc = MB4_OK;
  cudaGraph_t g = nullptr;
  do {
    if ((rc = cuda_rc(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal))) != MB4_OK) break;
    enqueue_setup(c, cap);
    cudaStreamCaptureStatus cs;
    cudaGraph_t capg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if ((rc = cuda_rc(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &capg, &deps, nullptr, &ndeps))) != MB4_OK) {
      cudaStreamEndCapture(cap, &g);
      break;
    }
    cudaGraphConditionalHandle h;
    if ((rc = cuda_rc(cudaGraphConditionalHandleCreate(&h, capg, 1, cudaGraphCondAssignDefault))) != MB4_OK) {
      cudaStreamEndCapture(cap, &g);
      break;
    }
    // The first Newton iterations are unrolled into the step graph, so their kernels chain by
    // programmatic dependent launch; their loop tests set the WHILE node's condition.  An
    // instance that has already converged makes them no-ops (every kernel skips it).
    for (int u = 0; u < kUnrolledNewton; ++u) enqueue_body(c, cap, (unsigned long long)h, 1);
    if ((rc = cuda_rc(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &capg, &deps, nullptr, &ndeps))) != MB4_OK) {
      cudaStreamEndCapture(cap, &g);
      break;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    if ((rc = cuda_rc(cudaGraphAddNode(&cnode, capg, deps, nullptr, ndeps, &cp))) != MB4_OK) {
      cudaStreamEndCapture(cap, &g);
      break;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((rc = cuda_rc(cudaStreamUpdateCaptureDependencies(cap, &cnode, nullptr, 1,
                                                          cudaStreamSetCaptureDependencies))) != MB4_OK) {
      cudaStreamEndCapture(cap, &g);
      break;
    }
    launch_accept(c->p, c->b, cap);
    if ((rc = cuda_rc(cudaStreamEndCapture(cap, &g))) != MB4_OK) break;
    if ((rc = cuda_rc(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0,
                                                    cudaStreamCaptureModeThreadLocal))) != MB4_OK)
      break;
    enqueue_body(c, cap, (unsigned long long)h, 1);
    cudaGraph_t body_out = nullptr;
    if ((rc = cuda_rc(cudaStreamEndCapture(cap, &body_out))) != MB4_OK) break;
    if ((rc = cuda_rc(cudaGraphInstantiate(&c->exec, g, 0))) != MB4_OK) break;
    c->graph = g;
    c->handle = h;
    g = nullptr;
  } while (0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  return rc;
}

// Barrier slots of the persistent step: slot 0 and one per group of kBarGroup blocks.
size_t bar_bytes(const StepParams& p) {
  return (size_t)(1 + (p.pers_blocks + kBarGroup - 1) / kBarGroup) * kBarSlotWords * sizeof(unsigned int);
}

int ensure_scratch(mb4_batch* c) {
  if (c->io) return MB4_OK;
  const size_t S = (size_t)c->p.S, BS = (size_t)c->B * S;
  MB4_CHECK(dalloc(c, (void**)&c->tmp3a, 3 * S * sizeof(double2)));
  MB4_CHECK(dalloc(c, (void**)&c->tmp3b, 3 * S * sizeof(double2)));
  MB4_CHECK(dalloc(c, (void**)&c->io, 6 * std::max(BS, S) * sizeof(double)));
  return MB4_OK;
}

// The device address of a host buffer that is page-locked and mapped (cudaHostAlloc,
// cudaMallocHost, or cudaHostRegister with mapping: with unified addressing every
// page-locked buffer is), else null.  Kernels then read or write such a buffer in
// place over the host link, with no staging copy.
template <typename T>
T* mapped_host(T* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();                          // clear the error of an unknown pointer
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? static_cast<T*>(a.devicePointer) : nullptr;
}

// Bring n (re, im) doubles onto the device, planar: device and mapped host buffers are
// used in place, other host data is staged through c->io.
int stage_in(mb4_batch* c, const double* re, const double* im, size_t n, int on_device, const double** dre,
             const double** dim) {
  if (on_device) {
    *dre = re;
    *dim = im;
    return MB4_OK;
  }
  const double* mre = mapped_host(re);
  const double* mim = mapped_host(im);
  if (mre && mim) {                              // the pack kernel reads the host buffers in place
    *dre = mre;
    *dim = mim;
    return MB4_OK;
  }
  MB4_TRY(cudaMemcpyAsync(c->io, re, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  MB4_TRY(cudaMemcpyAsync(c->io + n, im, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  *dre = c->io;
  *dim = c->io + n;
  return MB4_OK;
}

// Unpack n complex values to (re, im) and synchronise: device and mapped host buffers are
// written in place, other host buffers through c->io.
int stage_out(mb4_batch* c, const double2* z, double* re, double* im, size_t n, int on_device) {
  if (on_device) {
    launch_unpack(z, re, im, n, c->stream);
    MB4_TRY(cudaGetLastError());
    MB4_TRY(cudaStreamSynchronize(c->stream));
    return MB4_OK;
  }
  double* mre = mapped_host(re);
  double* mim = mapped_host(im);
  if (mre && mim) {                              // the unpack kernel writes the host buffers in place
    launch_unpack(z, mre, mim, n, c->stream);
    MB4_TRY(cudaGetLastError());
    MB4_TRY(cudaStreamSynchronize(c->stream));
    return MB4_OK;
  }
  launch_unpack(z, c->io, c->io + n, n, c->stream);
  MB4_TRY(cudaGetLastError());
  MB4_TRY(cudaMemcpyAsync(re, c->io, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MB4_TRY(cudaMemcpyAsync(im, c->io + n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  MB4_TRY(cudaStreamSynchronize(c->stream));
  return MB4_OK;
}

int read_status(mb4_batch* c) {
  c->host_status.resize(c->B);
  MB4_TRY(cudaMemcpyAsync(c->host_status.data(), c->b.is, sizeof(InstStatus) * c->B, cudaMemcpyDeviceToHost,
                          c->stream));
  MB4_TRY(cudaStreamSynchronize(c->stream));
  return MB4_OK;
}

int write_status(mb4_batch* c) {
  MB4_TRY(cudaMemcpyAsync(c->b.is, c->host_status.data(), sizeof(InstStatus) * c->B, cudaMemcpyHostToDevice,
                          c->stream));
  MB4_TRY(cudaStreamSynchronize(c->stream));
  return MB4_OK;
}

void fill_stats(const InstStatus& s, mb4_stats* st) {
  std::memset(st, 0, sizeof(*st));
  st->steps_done = s.steps_done;
  st->newton_iters_total = s.newton_total;
  st->newton_iters_last = s.last_newton_iters;
  st->last_update_inf = s.last_rmax;
  st->u0_inf = s.last_u0max;
  for (int l = 0; l < 8; ++l) st->update_hist[l] = (l < s.last_newton_iters) ? s.hist[l] : 0.0;
}

long long batch_bytes(int nx, int ny, int B, const mb4_options& o) {
  const size_t S = (size_t)nx * ny, BS = S * B;
  const size_t tk = (o.precision == MB4_MIXED) ? 4 : 8;
  const int nent = (o.krylov_s + 1) * (o.krylov_s + 2) / 2;
  size_t t = 0;
  // u, V, onsite + V, D/tx (grids with tx != 0; counted always), (K+V) u0, dU
  t += round256(BS * 16) + 3 * round256(BS * 8) + round256(BS * 16) + round256(3 * BS * 16);
  t += round256(BS * 4 * tk) + round256((size_t)(o.krylov_s + 1) * 3 * BS * 2 * tk);
  t += round256((size_t)B * 3 * kGramCap * nent * 8) + round256((size_t)B * 3 * kMaxS * 8);
  t += round256((size_t)B * kObsBlocksMax * 12 * 8) + round256((size_t)B * 6 * 8);
  t += round256(B * sizeof(InstConst)) + round256(B * sizeof(InstStatus)) + round256(sizeof(BatchCtl));
  t += 2 * round256(3 * S * 16) + round256(6 * std::max(BS, S) * 8);   // I/O scratch
  if (o.newton_start > 0) t += round256((size_t)o.newton_start * 3 * BS * 16);
  if (o.precondition)
    t += round256((size_t)(o.krylov_s + 1) * 3 * BS * 2 * tk) + 2 * round256((size_t)3 * BS * 2 * tk) +
         round256((size_t)nx * 2 * tk) + round256((size_t)ny * 2 * tk);
  if (o.site_chi) t += round256(BS * 8);
  return (long long)t;
}

// ---- launch-shape autotuner ------------------------------------------------
// The per-site kernels (residual, FP64 Krylov basis, update) are timed with 64, 128
// and 256 threads per block on the batch's own buffers (10 launches each after a
// warm-up), and the fastest kept: 128 unless another is faster by more than 5%, a
// margin above the launch-to-launch noise of these 10-80 us kernels.  Set-up and
// accept take the residual's shape.  None of this changes results: those kernels
// compute each site alone.  (A grid-stride form one wave deep was tried as a further
// candidate: its loop made the default launch 5% slower, so it is not offered.)
typedef std::tuple<int, int, int, int, int, int, int> TuneKey;   // device, precision, nx, ny, B, s, precond
std::mutex g_tune_mu;
std::map<TuneKey, std::array<int, 5>> g_tune;   // threads of the four per-site groups, the FP32 basis form

// which: 0 residual, 1 FP64 stencil basis, 2 update (bs = threads per block), 3 FP32 matrix
// powers (bs = tile shape index).
int time_site_kernel(mb4_batch* c, int which, int bs, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  if (which == 1 && (c->precision == MB4_MIXED || c->p.precond)) return MB4_ERR_INVALID_ARG;   // FP64 buffers only
  if (which == 3 && !(c->precision == MB4_MIXED && c->p.use_powers)) return MB4_ERR_INVALID_ARG;
  StepParams p = c->p;
  if (which == 0) p.bs_residual = bs;
  else if (which == 1) p.bs_matvec = bs;
  else if (which == 2) p.bs_update = bs;
  else p.pow_shape = bs;
  const bool mixed = (c->precision == MB4_MIXED);
  float total = 0.f;
  for (int r = 0; r < 11; ++r) {
    launch_arm(p, c->b, c->stream);                // active, Newton iteration 0
    MB4_TRY(cudaEventRecord(e0, c->stream));
    if (which == 0) {
      if (mixed) launch_residual<float>(p, c->b, false, c->stream);
      else launch_residual<double>(p, c->b, false, c->stream);
    } else if (which == 1) {
      launch_matvecs<double>(p, c->b, c->stream);
    } else if (which == 3) {
      launch_matvecs<float>(p, c->b, c->stream);
    } else {
      if (mixed) launch_update<float>(p, c->b, 0ull, 0, c->stream);
      else launch_update<double>(p, c->b, 0ull, 0, c->stream);
    }
    MB4_TRY(cudaEventRecord(e1, c->stream));
    MB4_TRY(cudaEventSynchronize(e1));
    float t = 0.f;
    MB4_TRY(cudaEventElapsedTime(&t, e0, e1));
    if (r > 0) total += t;                         // the first launch warms up
  }
  *ms = total / 10.f;
  return MB4_OK;
}

// The fastest of n timed candidates, unless it is within 5% of the default: the margin is
// above the launch-to-launch noise, and the default is what a run without tuning uses.
int pick_fastest(const float* t, int n, int dflt) {
  int best = 0;
  for (int k = 1; k < n; ++k)
    if (t[k] < t[best]) best = k;
  return (t[best] < 0.95f * t[dflt]) ? best : dflt;
}

void apply_shape(StepParams& p, const std::array<int, 5>& t) {
  p.bs_site = t[0];
  p.bs_residual = t[1];
  p.bs_matvec = t[2];
  p.bs_update = t[3];
  p.pow_shape = t[4];
}

int autotune_launch_shapes(mb4_batch* c, const mb4_grid* grid) {
  const int mixed = (c->precision == MB4_MIXED);
  const TuneKey key(c->device, c->precision, grid->nx, grid->ny, c->B, c->p.s, c->p.precond);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end() && !c->forced_tile) {  // (a forced tile is neither taken from nor put in the cache)
      apply_shape(c->p, it->second);
      return MB4_OK;
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MB4_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MB4_ERR_CUDA;
  }
  const int cand[3] = {64, 128, 256};
  int chosen[3] = {128, 128, 128};
  int rc = MB4_OK;
  for (int which = 0; which < 3 && rc == MB4_OK; ++which) {
    // the FP64 stencil basis is timed only where it is the basis in use: not in mixed
    // mode (FP32 buffers, matrix powers) nor with the preconditioner (DFT basis)
    if (which == 1 && (mixed || c->p.precond)) continue;
    float t[3];
    for (int k = 0; k < 3 && rc == MB4_OK; ++k) rc = time_site_kernel(c, which, cand[k], e0, e1, &t[k]);
    if (rc != MB4_OK) break;
    chosen[which] = cand[pick_fastest(t, 3, 1)];  // 128 unless another is clearly faster
  }
  // FP32 matrix-powers tile: the default 32 x 16 unless another shape is clearly faster
  int shape = c->p.pow_shape;                    // a forced tile (option powers_tile) stays
  if (rc == MB4_OK && mixed && c->p.use_powers && c->p.s <= kPowShapeMaxS && !c->forced_tile) {
    float t[kPowShapes + 1];                       // the tile forms, then one launch per level
    for (int k = 0; k <= kPowShapes && rc == MB4_OK; ++k) rc = time_site_kernel(c, 3, k, e0, e1, &t[k]);
    if (rc == MB4_OK) shape = pick_fastest(t, kPowShapes + 1, 0);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MB4_OK) return rc;
  const std::array<int, 5> t = {chosen[0], chosen[0], chosen[1], chosen[2], shape};
  apply_shape(c->p, t);
  // the timing launches wrote scratch, the increments and the status: start clean
  MB4_TRY(cudaMemsetAsync(c->b.Ubar, 0, (size_t)3 * c->B * c->p.S * sizeof(double2), c->stream));
  MB4_TRY(cudaMemsetAsync(c->b.bc, 0, sizeof(BatchCtl), c->stream));
  MB4_CHECK(write_status(c));
  if (c->forced_tile) return MB4_OK;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = t;
  return MB4_OK;
}

// Spectral preconditioner tables from the instances' mean on-site terms.
int upload_precond_tables(mb4_batch* c) {
  if (!c->p.precond) return MB4_OK;
  if (c->precision == MB4_MIXED)
    return precond_tables<float>(c->p, c->ebar.data(), c->p.hlam, c->b.pwx, c->b.pwy, c->b.pminv, c->stream);
  return precond_tables<double>(c->p, c->ebar.data(), c->p.hlam, c->b.pwx, c->b.pwy, c->b.pminv, c->stream);
}

double mean_of(const double* x, size_t n) {
  long double s = 0.0L;
  for (size_t k = 0; k < n; ++k) s += x[k];
  return (double)(s / (long double)n);
}

// Create a batch of B instances; V is host B*S doubles, chi host B doubles.
// A general kinetic matrix for make_batch: its off-diagonal in slot-major ELL form.
struct EllHost {
  int deg = 0;
  bool cplx = false;         // complex Hermitian K
  std::vector<int> nbr;      // deg * S, nbr[e * S + k] = j or -1
  std::vector<double> w;     // deg * S, Re K_kj
  std::vector<double> wi;    // deg * S, Im K_kj (cplx only)
};

int make_batch(mb4_batch* c, const mb4_grid* grid, int B, const double* V, const double* chi, double h,
               const mb4_options& o, const EllHost* ell = nullptr) {
  MB4_CHECK(compute_constants(o.alpha1, o.c1, o.c2, &c->k));
  c->precision = o.precision;
  c->use_graph = o.use_graph ? 1 : 0;
  c->forced_tile = o.powers_tile > 0;
  c->stream = (cudaStream_t)o.stream;
  c->tk = (o.precision == MB4_MIXED) ? sizeof(float) : sizeof(double);
  c->B = B;
  MB4_TRY(cudaGetDevice(&c->device));
  const size_t S = (size_t)grid->nx * grid->ny, BS = S * B;
  std::vector<double> D(BS);
  for (size_t k = 0; k < BS; ++k) {
    if (!std::isfinite(V[k])) return MB4_ERR_INVALID_ARG;
    D[k] = grid->onsite + V[k];
  }
  for (int b = 0; b < B; ++b)
    if (!std::isfinite(chi[b])) return MB4_ERR_INVALID_ARG;
  fill_params(c, grid, h, o);
  StepParams& p = c->p;
  if (ell) {
    if (B != 1 || p.precond) return MB4_ERR_INVALID_ARG;   // one instance; no spectral preconditioner
    p.ell = 1;
    p.ell_deg = ell->deg;
    p.ell_cplx = ell->cplx ? 1 : 0;
  }
  p.gram_blocks = (o.precision == MB4_MIXED) ? gram_blocks_per_system<float>(p.s, B, p.S)
                                              : gram_blocks_per_system<double>(p.s, B, p.S);
  if (p.gram_blocks < 1) return MB4_ERR_CUDA;
  if (p.precond && (grid->nx > MB4_MAX_PRECOND_SIDE || grid->ny > MB4_MAX_PRECOND_SIDE)) return MB4_ERR_INVALID_ARG;
  if (p.precond) {
    p.fft_nrx = fft_radices(grid->nx, p.fft_rx);
    p.fft_nry = fft_radices(grid->ny, p.fft_ry);
  }
  p.use_powers = (o.precision == MB4_MIXED && !p.precond && !p.ell) ? 1 : 0;
  if (p.use_powers) MB4_CHECK(prepare_powers());
  std::vector<double> Dtx;
  p.kin_unit = (!p.ell && grid->tx != 0.0 && std::isfinite(p.rty) && fill_dtx(p, D.data(), BS, &Dtx)) ? 1 : 0;
  p.mv_unit = 0;
  if (p.kin_unit && o.precision == MB4_FP64 && !p.precond) {
    p.mv_unit = 1;
    for (int b = 0; b < B && p.mv_unit; ++b)
      if (basis_theta(p, V + (size_t)b * S, S) < 0.0) p.mv_unit = 0;
  }

  DevBuffers& d = c->b;
  const size_t tk = c->tk;
  const int nent = (p.s + 1) * (p.s + 2) / 2;
  MB4_CHECK(dalloc(c, (void**)&d.u, BS * sizeof(double2)));
  MB4_CHECK(dalloc(c, (void**)&d.V, BS * sizeof(double)));
  MB4_CHECK(dalloc(c, (void**)&d.d, BS * sizeof(double)));
  if (p.kin_unit) MB4_CHECK(dalloc(c, (void**)&d.dtx, BS * sizeof(double)));
  MB4_CHECK(dalloc(c, (void**)&d.S0, BS * sizeof(double2)));
  MB4_CHECK(dalloc(c, (void**)&d.Ubar, 3 * BS * sizeof(double2)));
  if (p.pred_order > 0) MB4_CHECK(dalloc(c, (void**)&d.dU_hist, (size_t)p.pred_order * 3 * BS * sizeof(double2)));
  if (p.precond) {
    MB4_CHECK(dalloc(c, &d.pz, (size_t)(p.s + 1) * 3 * BS * 2 * tk));
    MB4_CHECK(dalloc(c, &d.ptmp, (size_t)3 * BS * 2 * tk));
    MB4_CHECK(dalloc(c, &d.pwx, (size_t)grid->nx * 2 * tk));
    MB4_CHECK(dalloc(c, &d.pwy, (size_t)grid->ny * 2 * tk));
    MB4_CHECK(dalloc(c, &d.pminv, (size_t)3 * BS * 2 * tk));
  }
  MB4_CHECK(dalloc(c, &d.jc, BS * 4 * tk));
  MB4_CHECK(dalloc(c, &d.v, (size_t)(p.s + 1) * 3 * BS * 2 * tk));
  MB4_CHECK(dalloc(c, (void**)&d.gram_part, (size_t)B * 3 * p.gram_blocks * nent * sizeof(double)));
  MB4_CHECK(dalloc(c, (void**)&d.coef, (size_t)B * 3 * kMaxS * sizeof(double)));
  MB4_CHECK(dalloc(c, (void**)&d.obs_part, (size_t)B * obs_blocks_per_instance(B) * 12 * sizeof(double)));
  MB4_CHECK(dalloc(c, (void**)&d.obs_out, (size_t)B * 6 * sizeof(double)));
  MB4_CHECK(dalloc(c, (void**)&d.ic, (size_t)B * sizeof(InstConst)));
  MB4_CHECK(dalloc(c, (void**)&d.is, (size_t)B * sizeof(InstStatus)));
  MB4_CHECK(dalloc(c, (void**)&d.bc, sizeof(BatchCtl)));
  std::vector<InstConst> ic(B);
  // with a chi field the per-instance constants carry chi = 1 and the kernels scale by chi_k
  for (int b = 0; b < B; ++b) {
    double theta = basis_theta(c->p, V + (size_t)b * S, S);
    if (ell) {                                  // Gershgorin: max_k |d_k| + sum_j |K_kj|
      theta = 0.0;
      for (size_t k = 0; k < S; ++k) {
        double r = std::fabs(D[k]);
        for (int e = 0; e < ell->deg; ++e)
          if (ell->nbr[(size_t)e * S + k] >= 0)
            r += ell->cplx ? std::hypot(ell->w[(size_t)e * S + k], ell->wi[(size_t)e * S + k])
                           : std::fabs(ell->w[(size_t)e * S + k]);
        theta = std::fmax(theta, r);
      }
      if (!(theta > 0.0)) theta = 1.0;
    }
    fill_inst_const(c, p.chi_field ? 1.0 : chi[b], theta, &ic[b]);
  }
  if (ell) {                                    // off-diagonal in FP64 and, scaled by 1/theta, in TK
    const size_t n = (size_t)ell->deg * S;
    const int nc = ell->cplx ? 2 : 1;            // (re, im) pairs for a complex K
    MB4_CHECK(dalloc(c, (void**)&c->ell_nbr, n * sizeof(int)));
    MB4_CHECK(dalloc(c, &c->ell_w, n * nc * sizeof(double)));
    MB4_CHECK(dalloc(c, &c->ell_wt, n * nc * tk));
    MB4_TRY(cudaMemcpy(c->ell_nbr, ell->nbr.data(), n * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<double> w(n * nc);
    for (size_t q = 0; q < n; ++q) {
      w[q * nc] = ell->w[q];
      if (ell->cplx) w[q * nc + 1] = ell->wi[q];
    }
    MB4_TRY(cudaMemcpy(c->ell_w, w.data(), n * nc * sizeof(double), cudaMemcpyHostToDevice));
    if (tk == sizeof(float)) {
      std::vector<float> wt(n * nc);
      for (size_t q = 0; q < n * nc; ++q) wt[q] = (float)(w[q] * ic[0].inv_theta);
      MB4_TRY(cudaMemcpy(c->ell_wt, wt.data(), n * nc * sizeof(float), cudaMemcpyHostToDevice));
    } else {
      std::vector<double> wt(n * nc);
      for (size_t q = 0; q < n * nc; ++q) wt[q] = w[q] * ic[0].inv_theta;
      MB4_TRY(cudaMemcpy(c->ell_wt, wt.data(), n * nc * sizeof(double), cudaMemcpyHostToDevice));
    }
    p.ell_nbr = c->ell_nbr;
    p.ell_w = c->ell_w;
    p.ell_wt = c->ell_wt;
  }
  if (p.chi_field) {
    MB4_CHECK(dalloc(c, (void**)&d.chi, BS * sizeof(double)));
    std::vector<double> field(BS);
    for (int b = 0; b < B; ++b) std::fill(field.begin() + (size_t)b * S, field.begin() + (size_t)(b + 1) * S, chi[b]);
    MB4_TRY(cudaMemcpy(d.chi, field.data(), BS * sizeof(double), cudaMemcpyHostToDevice));
  }
  c->host_status.assign(B, InstStatus{});
  for (int b = 0; b < B; ++b) c->host_status[b].enabled = 1;
  c->base_steps.assign(B, 0);
  c->base_newton.assign(B, 0);
  c->ebar.assign(B, 0.0);
  for (int b = 0; b < B; ++b) c->ebar[b] = mean_of(D.data() + (size_t)b * S, S);
  MB4_CHECK(upload_precond_tables(c));
  MB4_TRY(cudaMemcpyAsync(d.V, V, BS * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  MB4_TRY(cudaMemcpyAsync(d.d, D.data(), BS * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (p.kin_unit)
    MB4_TRY(cudaMemcpyAsync(d.dtx, Dtx.data(), BS * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  MB4_TRY(cudaMemcpyAsync(d.ic, ic.data(), B * sizeof(InstConst), cudaMemcpyHostToDevice, c->stream));
  MB4_TRY(cudaMemsetAsync(d.u, 0, BS * sizeof(double2), c->stream));
  MB4_TRY(cudaMemsetAsync(d.Ubar, 0, 3 * BS * sizeof(double2), c->stream));
  MB4_TRY(cudaMemsetAsync(d.coef, 0, (size_t)B * 3 * kMaxS * sizeof(double), c->stream));
  MB4_TRY(cudaMemsetAsync(d.bc, 0, sizeof(BatchCtl), c->stream));
  MB4_CHECK(write_status(c));
  if (o.autotune && o.site_threads == 0) MB4_CHECK(autotune_launch_shapes(c, grid));
  if (p.persistent) {
    if (!persistent_supported(p, c->precision == MB4_MIXED)) return MB4_ERR_INVALID_ARG;
    p.pers_blocks = persistent_blocks(p, c->precision == MB4_MIXED);
    if (p.pers_blocks < 1) return MB4_ERR_CUDA;
    MB4_CHECK(dalloc(c, (void**)&d.bar, bar_bytes(p)));
    MB4_TRY(cudaMemsetAsync(d.bar, 0, bar_bytes(p), c->stream));
  } else if (c->use_graph) {
    MB4_CHECK(build_graph(c));
  }
  return MB4_OK;
}

int potential_to_host(const mb4_potential* pot, size_t n, std::vector<double>* V) {
  if (!pot || !pot->v) return MB4_ERR_INVALID_ARG;
  V->resize(n);
  if (pot->on_device) {
    MB4_TRY(cudaMemcpy(V->data(), pot->v, n * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(V->data(), pot->v, n * sizeof(double));
  }
  return MB4_OK;
}

int step_async(mb4_batch* c, int nsteps) {
  launch_arm(c->p, c->b, c->stream);
  if (c->p.persistent) {
    // arrival counts start at zero (a call whose barrier gave up may have left some)
    MB4_TRY(cudaMemsetAsync(c->b.bar, 0, bar_bytes(c->p), c->stream));
    // one cooperative launch per step, then the accept (kept outside, so that a step whose
    // barrier gave up is never half accepted)
    for (int n = 0; n < nsteps; ++n) {
      MB4_TRY(launch_step_persistent(c->p, c->b, c->precision == MB4_MIXED, c->stream));
      launch_accept(c->p, c->b, c->stream);
    }
  } else if (c->use_graph) {
    for (int n = 0; n < nsteps; ++n) MB4_TRY(cudaGraphLaunch(c->exec, c->stream));
  } else {
    for (int n = 0; n < nsteps; ++n) {
      enqueue_setup(c, c->stream);
      for (;;) {
        enqueue_body(c, c->stream, 0ull, 0);
        MB4_TRY(cudaGetLastError());
        BatchCtl bc;
        MB4_TRY(cudaMemcpyAsync(&bc, c->b.bc, sizeof(bc), cudaMemcpyDeviceToHost, c->stream));
        MB4_TRY(cudaStreamSynchronize(c->stream));
        if (!bc.any_cont) break;
      }
      launch_accept(c->p, c->b, c->stream);
    }
  }
  MB4_TRY(cudaGetLastError());
  return MB4_OK;
}

int wait_batch(mb4_batch* c, mb4_stats* stats, int* status) {
  MB4_CHECK(read_status(c));
  int first = MB4_OK;
  for (int b = 0; b < c->B; ++b) {
    InstStatus s = c->host_status[b];
    s.steps_done -= c->base_steps[b];
    s.newton_total -= c->base_newton[b];
    c->base_steps[b] = c->host_status[b].steps_done;
    c->base_newton[b] = c->host_status[b].newton_total;
    if (stats) fill_stats(s, stats + b);
    if (status) status[b] = s.error;
    if (first == MB4_OK && s.error) first = s.error;
  }
  if (first != MB4_OK) c->err_seen = true;
  return first;
}

int clear_errors(mb4_batch* c) {
  MB4_CHECK(read_status(c));
  for (auto& s : c->host_status) {
    s.error = MB4_OK;
    s.steps_done = 0;
    s.newton_total = 0;
  }
  std::fill(c->base_steps.begin(), c->base_steps.end(), 0LL);
  std::fill(c->base_newton.begin(), c->base_newton.end(), 0LL);
  c->err_seen = false;
  return write_status(c);
}

int check_instance(const mb4_batch* c, int instance, bool allow_all) {
  if (!c) return MB4_ERR_INVALID_ARG;
  if (instance == -1 && allow_all) return MB4_OK;
  if (instance < 0 || instance >= c->B) return MB4_ERR_INVALID_ARG;
  return MB4_OK;
}

}  // namespace

extern "C" {

int mb4_default_options(mb4_options* o) {
  if (!o) return MB4_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->newton_rtol = 1e-13;
  o->newton_max = 30;
  o->krylov_s = 0;
  o->precision = MB4_FP64;
  o->alpha1 = -300.0 * 19.0 / 8.0;
  o->c1 = 1.0 / 3.0;
  o->c2 = 2.0 / 3.0;
  o->stream = nullptr;
  o->use_graph = 1;
  o->newton_predict = 0.0;
  o->overlap_launches = 1;
  o->newton_start = 2;
  o->newton_start_adaptive = 1;
  o->autotune = 1;
  o->persistent = 0;
  o->wait_limit = 1LL << 22;
  return MB4_OK;
}

const char* mb4_version(void) { return "libmb4 0.2 (sm_103a)"; }

const char* mb4_status_string(int s) {
  switch (s) {
    case MB4_OK: return "ok";
    case MB4_ERR_INVALID_ARG: return "invalid argument";
    case MB4_ERR_OUT_OF_MEMORY: return "out of device memory";
    case MB4_ERR_CUDA: return "CUDA runtime error";
    case MB4_ERR_NEWTON_NOT_CONVERGED: return "simplified Newton iteration did not converge (reduce h)";
    case MB4_ERR_KRYLOV_BREAKDOWN: return "Krylov least-squares breakdown";
    case MB4_ERR_NONFINITE: return "non-finite value in a Newton update";
    case MB4_ERR_TIMEOUT: return "bounded device wait timed out";
    case MB4_ERR_ADMISSION_REJECTED: return "admission rejected: no slot or memory budget";
    default: return "unknown status";
  }
}

// ---- batches ---------------------------------------------------------------

void mb4_batch_destroy(mb4_batch* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  for (void* p : c->allocs) cudaFree(p);
  delete c;
}

long long mb4_batch_bytes(int nx, int ny, int batch, const mb4_options* opt) {
  mb4_options o;
  if (nx < 3 || ny < 3 || batch < 1 || validate_options(opt, &o) != MB4_OK) return -1;
  return batch_bytes(nx, ny, batch, o);
}

int mb4_batch_create(const mb4_grid* grid, int batch, const mb4_potential* pot, const double* chi, double h,
                     const mb4_options* opt, mb4_batch** out) {
  if (!out) return MB4_ERR_INVALID_ARG;
  *out = nullptr;
  MB4_CHECK(validate_grid(grid, batch));
  if (!chi || !std::isfinite(h) || h == 0.0) return MB4_ERR_INVALID_ARG;
  mb4_options o;
  MB4_CHECK(validate_options(opt, &o));
  std::vector<double> V;
  MB4_CHECK(potential_to_host(pot, (size_t)grid->nx * grid->ny * batch, &V));
  mb4_batch* c = new (std::nothrow) mb4_batch();
  if (!c) return MB4_ERR_OUT_OF_MEMORY;
  int rc = make_batch(c, grid, batch, V.data(), chi, h, o);
  if (rc != MB4_OK) {
    mb4_batch_destroy(c);
    return rc;
  }
  *out = c;
  return MB4_OK;
}

int mb4_batch_set_state(mb4_batch* c, int instance, const double* re, const double* im, int on_device) {
  MB4_CHECK(check_instance(c, instance, true));
  if (!re || !im) return MB4_ERR_INVALID_ARG;
  MB4_CHECK(ensure_scratch(c));
  const size_t S = (size_t)c->p.S;
  const size_t n = (instance < 0) ? S * c->B : S;
  const double *dre, *dim;
  MB4_CHECK(stage_in(c, re, im, n, on_device, &dre, &dim));
  launch_set_state(c->p, c->b, dre, dim, instance < 0 ? 0 : instance, instance < 0 ? c->B : 1, c->stream);
  MB4_TRY(cudaGetLastError());
  MB4_TRY(cudaStreamSynchronize(c->stream));
  return MB4_OK;
}

int mb4_batch_get_state(const mb4_batch* cc, int instance, double* re, double* im, int on_device) {
  mb4_batch* c = const_cast<mb4_batch*>(cc);
  MB4_CHECK(check_instance(c, instance, true));
  if (!re || !im) return MB4_ERR_INVALID_ARG;
  MB4_CHECK(ensure_scratch(c));
  const size_t S = (size_t)c->p.S;
  const size_t n = (instance < 0) ? S * c->B : S;
  const double2* src = c->b.u + ((instance < 0) ? 0 : (size_t)instance * S);
  return stage_out(c, src, re, im, n, on_device);
}

int mb4_batch_load(mb4_batch* c, int instance, const double* v, double chi, const double* re, const double* im,
                   int on_device) {
  MB4_CHECK(check_instance(c, instance, false));
  if (!v || !re || !im || !std::isfinite(chi)) return MB4_ERR_INVALID_ARG;
  const size_t S = (size_t)c->p.S;
  std::vector<double> V(S), D(S);
  if (on_device) {
    MB4_TRY(cudaMemcpy(V.data(), v, S * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(V.data(), v, S * sizeof(double));
  }
  for (size_t k = 0; k < S; ++k) {
    if (!std::isfinite(V[k])) return MB4_ERR_INVALID_ARG;
    D[k] = c->p.eps0 + V[k];
  }
  std::vector<double> Dtx;
  if (c->p.kin_unit && !fill_dtx(c->p, D.data(), S, &Dtx)) return MB4_ERR_INVALID_ARG;
  const double theta = basis_theta(c->p, V.data(), S);
  if (c->p.mv_unit && theta < 0.0) return MB4_ERR_INVALID_ARG;   // outside the batch's basis scaling
  InstConst ic;
  fill_inst_const(c, c->p.chi_field ? 1.0 : chi, theta, &ic);
  if (c->p.chi_field) {
    const std::vector<double> field(S, chi);
    MB4_TRY(cudaMemcpy(c->b.chi + (size_t)instance * S, field.data(), S * sizeof(double), cudaMemcpyHostToDevice));
  }
  MB4_TRY(cudaMemcpyAsync(c->b.V + (size_t)instance * S, V.data(), S * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
  MB4_TRY(cudaMemcpyAsync(c->b.d + (size_t)instance * S, D.data(), S * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
  if (c->p.kin_unit)
    MB4_TRY(cudaMemcpyAsync(c->b.dtx + (size_t)instance * S, Dtx.data(), S * sizeof(double),
                            cudaMemcpyHostToDevice, c->stream));
  MB4_TRY(cudaMemcpyAsync(c->b.ic + instance, &ic, sizeof(ic), cudaMemcpyHostToDevice, c->stream));
  c->ebar[instance] = mean_of(D.data(), S);
  MB4_CHECK(upload_precond_tables(c));
  MB4_CHECK(mb4_batch_set_state(c, instance, re, im, on_device));
  MB4_CHECK(read_status(c));
  InstStatus fresh{};
  fresh.enabled = 1;
  c->host_status[instance] = fresh;
  c->base_steps[instance] = 0;
  c->base_newton[instance] = 0;
  return write_status(c);
}

int mb4_batch_enable(mb4_batch* c, int instance, int enabled) {
  MB4_CHECK(check_instance(c, instance, true));
  MB4_CHECK(read_status(c));
  for (int b = 0; b < c->B; ++b)
    if (instance < 0 || b == instance) c->host_status[b].enabled = enabled ? 1 : 0;
  return write_status(c);
}

int mb4_batch_step_async(mb4_batch* c, int nsteps) {
  if (!c || nsteps < 0) return MB4_ERR_INVALID_ARG;
  return step_async(c, nsteps);
}

int mb4_batch_wait(mb4_batch* c, mb4_stats* stats, int* status) {
  if (!c) return MB4_ERR_INVALID_ARG;
  return wait_batch(c, stats, status);
}

int mb4_batch_step(mb4_batch* c, int nsteps, mb4_stats* stats, int* status) {
  if (!c || nsteps < 0) return MB4_ERR_INVALID_ARG;
  MB4_CHECK(step_async(c, nsteps));
  return wait_batch(c, stats, status);
}

}  // extern "C"

int mb4::batch_observables_async(mb4_batch* c, double* host_out) {
  if (!c || !host_out) return MB4_ERR_INVALID_ARG;
  launch_observables(c->p, c->b, c->stream);
  MB4_TRY(cudaGetLastError());
  MB4_TRY(cudaMemcpyAsync(host_out, c->b.obs_out, (size_t)c->B * 6 * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  return MB4_OK;
}

extern "C" {

int mb4_batch_observables(const mb4_batch* cc, double* out) {
  mb4_batch* c = const_cast<mb4_batch*>(cc);
  if (!c || !out) return MB4_ERR_INVALID_ARG;
  launch_observables(c->p, c->b, c->stream);
  MB4_TRY(cudaGetLastError());
  MB4_TRY(cudaMemcpyAsync(out, c->b.obs_out, (size_t)c->B * 6 * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
  MB4_TRY(cudaStreamSynchronize(c->stream));
  return MB4_OK;
}

int mb4_batch_clear_errors(mb4_batch* c) {
  if (!c) return MB4_ERR_INVALID_ARG;
  return clear_errors(c);
}

int mb4_batch_set_chi_field(mb4_batch* c, int instance, const double* chi, int on_device) {
  MB4_CHECK(check_instance(c, instance, false));
  if (!chi || !c->p.chi_field) return MB4_ERR_INVALID_ARG;
  const size_t S = (size_t)c->p.S;
  std::vector<double> h(S);
  if (on_device) {
    MB4_TRY(cudaMemcpy(h.data(), chi, S * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(h.data(), chi, S * sizeof(double));
  }
  for (size_t k = 0; k < S; ++k)
    if (!std::isfinite(h[k])) return MB4_ERR_INVALID_ARG;
  MB4_TRY(cudaMemcpyAsync(c->b.chi + (size_t)instance * S, h.data(), S * sizeof(double), cudaMemcpyHostToDevice,
                          c->stream));
  launch_forget_range(c->p, c->b, instance, 1, c->stream);   // another flow: the increments no longer fit
  MB4_TRY(cudaGetLastError());
  MB4_TRY(cudaStreamSynchronize(c->stream));
  return MB4_OK;
}

int mb4_set_chi_field(mb4_ctx* c, const double* chi, int on_device) {
  return mb4_batch_set_chi_field(c, 0, chi, on_device);
}

int mb4_batch_get_launch_shape(const mb4_batch* c, int* shape8) {
  if (!c || !shape8) return MB4_ERR_INVALID_ARG;
  const int bs[4] = {c->p.bs_site, c->p.bs_residual, c->p.bs_matvec, c->p.bs_update};
  for (int i = 0; i < 4; ++i) {
    shape8[i] = bs[i];
    shape8[4 + i] = (c->p.S + bs[i] - 1) / bs[i];
  }
  return MB4_OK;
}

int mb4_get_launch_shape(const mb4_ctx* c, int* shape8) { return mb4_batch_get_launch_shape(c, shape8); }

int mb4_batch_get_tile_shape(const mb4_batch* c, int* tx, int* ty) {
  if (!c || !tx || !ty) return MB4_ERR_INVALID_ARG;
  const bool powers = c->precision == MB4_MIXED && c->p.use_powers && c->p.pow_shape != kPowLevels;
  *tx = !powers ? 0 : kPowShapeForm[c->p.pow_shape] >= 3 ? 32 - 2 * c->p.s : kPowShapeTX[c->p.pow_shape];
  *ty = powers ? kPowShapeTY[c->p.pow_shape] : 0;
  return MB4_OK;
}

// ---- single contexts: a batch of one -------------------------------------

void mb4_destroy(mb4_ctx* c) { mb4_batch_destroy(c); }

int mb4_create(const mb4_grid* grid, const mb4_potential* pot, const mb4_nonlinearity* nl, double h,
               const mb4_options* opt_in, mb4_ctx** out) {
  if (!out) return MB4_ERR_INVALID_ARG;
  *out = nullptr;
  if (!nl || !std::isfinite(nl->chi)) return MB4_ERR_INVALID_ARG;
  MB4_CHECK(validate_grid(grid, 1));
  if (!std::isfinite(h) || h == 0.0) return MB4_ERR_INVALID_ARG;
  mb4_options o;
  MB4_CHECK(validate_options(opt_in, &o));
  std::vector<double> V;
  MB4_CHECK(potential_to_host(pot, (size_t)grid->nx * grid->ny, &V));
  mb4_ctx* c = new (std::nothrow) mb4_ctx();
  if (!c) return MB4_ERR_OUT_OF_MEMORY;
  const double chi = nl->chi;
  int rc = make_batch(c, grid, 1, V.data(), &chi, h, o);
  if (rc != MB4_OK) {
    mb4_batch_destroy(c);
    return rc;
  }
  *out = c;
  return MB4_OK;
}

int mb4_create_sparse(const mb4_sparse_kinetic* K, const mb4_potential* pot, const mb4_nonlinearity* nl, double h,
                      const mb4_options* opt_in, mb4_ctx** out) {
  if (!out) return MB4_ERR_INVALID_ARG;
  *out = nullptr;
  if (!K || K->S < 1 || K->S > (1 << 30) || K->max_degree < 1 || K->max_degree > MB4_MAX_DEGREE || !K->nbr ||
      !K->t || !std::isfinite(K->onsite))
    return MB4_ERR_INVALID_ARG;
  if (!nl || !std::isfinite(nl->chi) || !std::isfinite(h) || h == 0.0) return MB4_ERR_INVALID_ARG;
  mb4_options o;
  MB4_CHECK(validate_options(opt_in, &o));
  if (o.precondition) return MB4_ERR_INVALID_ARG;
  const size_t S = (size_t)K->S;
  const int deg = K->max_degree;
  // row-major input -> slot-major ELL; entries in range, no self links, finite, Hermitian
  EllHost ell;
  ell.deg = deg;
  ell.cplx = (K->t_im != nullptr);
  ell.nbr.assign((size_t)deg * S, -1);
  ell.w.assign((size_t)deg * S, 0.0);
  if (ell.cplx) ell.wi.assign((size_t)deg * S, 0.0);
  for (size_t k = 0; k < S; ++k)
    for (int e = 0; e < deg; ++e) {
      const int j = K->nbr[k * deg + e];
      if (j < -1 || j >= K->S || j == (int)k) return MB4_ERR_INVALID_ARG;
      if (j < 0) continue;
      const double w = K->t[k * deg + e];
      const double wi = ell.cplx ? K->t_im[k * deg + e] : 0.0;
      if (!std::isfinite(w) || !std::isfinite(wi)) return MB4_ERR_INVALID_ARG;
      int found = 0;                             // K_jk = conj(K_kj)
      for (int f = 0; f < deg; ++f)
        if (K->nbr[(size_t)j * deg + f] == (int)k && K->t[(size_t)j * deg + f] == w &&
            (!ell.cplx || K->t_im[(size_t)j * deg + f] == -wi))
          found = 1;
      if (!found) return MB4_ERR_INVALID_ARG;   // K must be Hermitian
      ell.nbr[(size_t)e * S + k] = j;
      ell.w[(size_t)e * S + k] = w;
      if (ell.cplx) ell.wi[(size_t)e * S + k] = wi;
    }
  std::vector<double> V;
  MB4_CHECK(potential_to_host(pot, S, &V));
  mb4_ctx* c = new (std::nothrow) mb4_ctx();
  if (!c) return MB4_ERR_OUT_OF_MEMORY;
  const mb4_grid g = {K->S, 1, 0.0, 0.0, K->onsite};
  const double chi = nl->chi;
  int rc = make_batch(c, &g, 1, V.data(), &chi, h, o, &ell);
  if (rc != MB4_OK) {
    mb4_batch_destroy(c);
    return rc;
  }
  *out = c;
  return MB4_OK;
}

int mb4_set_state(mb4_ctx* c, const double* re, const double* im, int on_device) {
  return mb4_batch_set_state(c, 0, re, im, on_device);
}

int mb4_get_state(const mb4_ctx* c, double* re, double* im, int on_device) {
  return mb4_batch_get_state(c, 0, re, im, on_device);
}

int mb4_get_stages(const mb4_ctx* cc, double* re3, double* im3, int on_device) {
  mb4_ctx* c = const_cast<mb4_ctx*>(cc);
  if (!c || !re3 || !im3) return MB4_ERR_INVALID_ARG;
  MB4_CHECK(ensure_scratch(c));
  // U_j = u0 + sum_n T[j][n] dU_n and u1 = u0 + sum_n T[2][n] dU_n, so U_j = u1 + sum_n (T[j][n] - T[2][n]) dU_n
  double M[3][3];
  for (int j = 0; j < 3; ++j)
    for (int n = 0; n < 3; ++n) M[j][n] = c->k.T[j][n] - c->k.T[2][n];
  launch_mix3(c->p.S, c->b.Ubar, c->tmp3a, M, c->stream);
  launch_add_plane3(c->p.S, c->tmp3a, c->b.u, 1.0, c->stream);
  MB4_TRY(cudaGetLastError());
  return stage_out(c, c->tmp3a, re3, im3, 3 * (size_t)c->p.S, on_device);
}

int mb4_step(mb4_ctx* c, int nsteps, mb4_stats* stats) {
  if (!c || nsteps < 0) return MB4_ERR_INVALID_ARG;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  // every call starts from the last accepted state: clear an error a previous call left
  // (the status round trip is skipped when there is none to clear)
  if (c->err_seen) MB4_CHECK(clear_errors(c));
  MB4_CHECK(step_async(c, nsteps));
  return wait_batch(c, stats, nullptr);
}

int mb4_step_async(mb4_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return MB4_ERR_INVALID_ARG;
  return step_async(c, nsteps);
}

int mb4_wait(mb4_ctx* c, mb4_stats* stats) {
  if (!c) return MB4_ERR_INVALID_ARG;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  const int rc = wait_batch(c, stats, nullptr);
  if (rc != MB4_OK && c->host_status[0].error != MB4_OK)
    MB4_CHECK(clear_errors(c));   // the next steps start from the last accepted state
  return rc;
}

int mb4_observables(const mb4_ctx* c, double* out6) { return mb4_batch_observables(c, out6); }

int mb4_energy(const mb4_ctx* c, double* H, double* parts3) {
  if (!c || !H) return MB4_ERR_INVALID_ARG;
  double o[6];
  MB4_CHECK(mb4_observables(c, o));
  *H = o[0];
  if (parts3) {
    parts3[0] = o[1];
    parts3[1] = o[2];
    parts3[2] = o[3];
  }
  return MB4_OK;
}

int mb4_norm(const mb4_ctx* c, double* norm2) {
  if (!c || !norm2) return MB4_ERR_INVALID_ARG;
  double o[6];
  MB4_CHECK(mb4_observables(c, o));
  *norm2 = o[4];
  return MB4_OK;
}

int mb4_residual(mb4_ctx* c, const double* u0_re, const double* u0_im, const double* U_re3, const double* U_im3,
                 double* phi_re3, double* phi_im3, int on_device) {
  if (!c || !u0_re || !u0_im || !U_re3 || !U_im3 || !phi_re3 || !phi_im3) return MB4_ERR_INVALID_ARG;
  MB4_CHECK(mb4_set_state(c, u0_re, u0_im, on_device));
  MB4_CHECK(clear_errors(c));
  const size_t S = (size_t)c->p.S;
  launch_arm(c->p, c->b, c->stream);
  enqueue_setup(c, c->stream);
  const double *dre, *dim;
  MB4_CHECK(stage_in(c, U_re3, U_im3, 3 * S, on_device, &dre, &dim));
  launch_pack(dre, dim, c->tmp3a, 3 * S, c->stream);
  launch_add_plane3((int)S, c->tmp3a, c->b.u, -1.0, c->stream);   // U_j - u0
  launch_mix3((int)S, c->tmp3a, c->b.Ubar, c->k.Tinv, c->stream);
  if (c->precision == MB4_MIXED) launch_residual_out<float>(c->p, c->b, c->tmp3b, c->stream);
  else launch_residual_out<double>(c->p, c->b, c->tmp3b, c->stream);
  // Phi = T Phibar = -T b
  double mT[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) mT[i][j] = -c->k.T[i][j];
  launch_mix3((int)S, c->tmp3b, c->tmp3a, mT, c->stream);
  MB4_TRY(cudaGetLastError());
  return stage_out(c, c->tmp3a, phi_re3, phi_im3, 3 * S, on_device);
}

int mb4_solve_shifted(mb4_ctx* c, const double* u0_re, const double* u0_im, const double* b_re3,
                      const double* b_im3, double* x_re3, double* x_im3, int on_device) {
  if (!c || !u0_re || !u0_im || !b_re3 || !b_im3 || !x_re3 || !x_im3) return MB4_ERR_INVALID_ARG;
  MB4_CHECK(mb4_set_state(c, u0_re, u0_im, on_device));
  MB4_CHECK(clear_errors(c));
  const size_t S = (size_t)c->p.S;
  launch_arm(c->p, c->b, c->stream);
  enqueue_setup(c, c->stream);
  const double *dre, *dim;
  MB4_CHECK(stage_in(c, b_re3, b_im3, 3 * S, on_device, &dre, &dim));
  launch_pack(dre, dim, c->tmp3a, 3 * S, c->stream);
  if (c->precision == MB4_MIXED) {
    launch_copy_rhs_in<float>(c->p, c->b, c->tmp3a, c->stream);
    launch_krylov<float>(c->p, c->b, c->stream);
    launch_copy_solution_out<float>(c->p, c->b, c->tmp3b, c->stream);
  } else {
    launch_copy_rhs_in<double>(c->p, c->b, c->tmp3a, c->stream);
    launch_krylov<double>(c->p, c->b, c->stream);
    launch_copy_solution_out<double>(c->p, c->b, c->tmp3b, c->stream);
  }
  MB4_TRY(cudaGetLastError());
  return stage_out(c, c->tmp3b, x_re3, x_im3, 3 * S, on_device);
}

}  // extern "C"

// ---- profiling: the step with an event pair around every launch -----------

namespace {

struct Prof {
  cudaStream_t s;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> open;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  double ms[MB4_K_COUNT] = {0};
  long long n[MB4_K_COUNT] = {0};
  double sites[MB4_K_COUNT] = {0};
  cudaEvent_t ev() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  // work: sites the launch(es) compute (instances that take part x sites per instance)
  template <typename F> void run(int cls, int count, double work, F f) {
    cudaEvent_t a = ev(), b = ev();
    cudaEventRecord(a, s);
    f();
    cudaEventRecord(b, s);
    open.push_back({cls, {a, b}});
    n[cls] += count;
    sites[cls] += work;
  }
  void harvest() {  // stream must be synchronised
    for (auto& o : open) {
      float t = 0.f;
      cudaEventElapsedTime(&t, o.second.first, o.second.second);
      ms[o.first] += t;
    }
    open.clear();
    used = 0;
  }
  ~Prof() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// Instances that a launch works on, read from the device status (the stream is idle).
struct Work {
  double active = 0, residual = 0, accept = 0;
};

int count_work(mb4_batch* c, bool first_iteration, Work* w) {
  MB4_CHECK(read_status(c));
  *w = Work{};
  const double S = (double)c->p.S;
  for (const InstStatus& I : c->host_status) {
    if (I.active) {
      w->active += S;
      // the first residual of a step from U^0 = e3 (x) u0 returns at once: k_setup wrote b^0
      if (!first_iteration || I.predicted) w->residual += S;
    }
    if (I.in_step && !I.error) w->accept += S;
  }
  return MB4_OK;
}

template <typename TK>
int profiled_steps(mb4_batch* c, int nsteps, Prof& P) {
  cudaStream_t s = c->stream;
  launch_arm(c->p, c->b, s);
  // the FP32 grid basis is one matrix-powers launch for all s levels
  const bool powers = sizeof(TK) == sizeof(float) && c->p.use_powers && !c->p.precond && c->p.pow_shape != kPowLevels;
  Work w;
  for (int n = 0; n < nsteps; ++n) {
    MB4_CHECK(count_work(c, true, &w));
    P.run(MB4_K_SETUP, 1, w.active, [&] { launch_setup<TK>(c->p, c->b, s); });
    for (int it = 0;; ++it) {
      if (it > 0) MB4_CHECK(count_work(c, false, &w));
      P.run(MB4_K_RESIDUAL, 1, w.residual, [&] { launch_residual<TK>(c->p, c->b, true, s); });
      P.run(MB4_K_MATVEC, powers ? 1 : c->p.s, w.active * (powers ? 1 : c->p.s), [&] {
        if (c->p.precond) launch_precond_basis<TK>(c->p, c->b, s);
        else launch_matvecs<TK>(c->p, c->b, s);
      });
      P.run(MB4_K_GRAM, 1, w.active, [&] { launch_gram<TK>(c->p, c->b, s); });
      P.run(MB4_K_UPDATE, 1, w.active, [&] { launch_update<TK>(c->p, c->b, 0ull, 0, s); });
      MB4_TRY(cudaGetLastError());
      BatchCtl bc;
      MB4_TRY(cudaMemcpyAsync(&bc, c->b.bc, sizeof(bc), cudaMemcpyDeviceToHost, s));
      MB4_TRY(cudaStreamSynchronize(s));
      P.harvest();
      if (!bc.any_cont) break;
    }
    MB4_CHECK(count_work(c, false, &w));
    P.run(MB4_K_ACCEPT, 1, w.accept, [&] { launch_accept(c->p, c->b, s); });
  }
  MB4_TRY(cudaStreamSynchronize(s));
  P.harvest();
  return MB4_OK;
}

int profiled(mb4_batch* c, int nsteps, double* ms, long long* launches, double* sites) {
  Prof P;
  P.s = c->stream;
  MB4_CHECK((c->precision == MB4_MIXED) ? profiled_steps<float>(c, nsteps, P) : profiled_steps<double>(c, nsteps, P));
  for (int k = 0; k < MB4_K_COUNT; ++k) {
    if (ms) ms[k] += P.ms[k];
    if (launches) launches[k] += P.n[k];
    if (sites) sites[k] += P.sites[k];
  }
  return MB4_OK;
}

}  // namespace

extern "C" int mb4_step_profiled(mb4_ctx* c, int nsteps, mb4_stats* stats, double* ms, long long* launches,
                                 double* sites) {
  if (!c || nsteps < 0) return MB4_ERR_INVALID_ARG;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  MB4_CHECK(clear_errors(c));
  MB4_CHECK(profiled(c, nsteps, ms, launches, sites));
  return wait_batch(c, stats, nullptr);
}

extern "C" int mb4_batch_step_profiled(mb4_batch* c, int nsteps, mb4_stats* stats, int* status, double* ms,
                                       long long* launches, double* sites) {
  if (!c || nsteps < 0) return MB4_ERR_INVALID_ARG;
  MB4_CHECK(profiled(c, nsteps, ms, launches, sites));
  return wait_batch(c, stats, status);
}
