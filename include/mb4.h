/*
 * mb4.h -- C ABI of libmb4: one time step of the MB4 energy-preserving
 * integrator (a fourth-order continuous-stage Runge-Kutta method) for the
 * 2D-grid nonlinear Schroedinger-type system, on one NVIDIA GB300 (sm_103a).
 *
 * Source of the method: T. Sakai, S. Kudo, H. Imachi, Y. Miyatake, T. Hoshi,
 * Y. Yamamoto, "A parallelizable energy-preserving integrator MB4 and its
 * application to quantum-mechanical wavepacket dynamics", arXiv:2003.04345.
 *
 * The system (Sec. 2.1, eq. dNLS, with chi = -gamma):
 *     i dpsi/dt = (K + V) psi + chi |psi|^2 psi
 * on an nx x ny periodic grid, site k = y*nx + x (x fastest).  K is the
 * 5-point operator of eq. (Kdefinition) generalised to hoppings tx, ty and an
 * on-site shift:  (K psi)_k = onsite*psi_k - tx (psi_{x-1} + psi_{x+1})
 *                                        - ty (psi_{y-1} + psi_{y+1}).
 * The paper's Laplacian is tx = 1/hx^2, ty = 1/hy^2, onsite = 2tx + 2ty.
 * The conserved energy is H = psi^H K psi + psi^H V psi + (chi/2) sum |psi|^4.
 *
 * One step (Algorithm 1, one pass of its time loop): the stage equations
 * Phi(U) = 0 (eq. Phidefinition) are solved by the simplified Newton
 * iteration (eq. Newton1) with the Jacobian frozen at u0 (eq. Jacobian2),
 * decoupled through E = T Lambda T^-1 into three independent shifted systems
 * (I - h lambda_i J) rbar_i = -Phibar_i (eq. Newton3, eq. MB4_4..MB4_6), each
 * solved matrix-free by an s-step GMRES cycle; u1 = U_c3 (c3 = 1, Sec. 2.2).
 *
 * Conventions for every entry point:
 *   - Return value: MB4_OK (0) or a negative MB4_ERR_* code; mb4_status_string
 *     gives a message.  Nothing aborts or prints.
 *   - Pointers are borrowed: the library copies what it needs before the call
 *     returns (device-to-device or host-to-device) and keeps no reference.
 *     `on_device` = 1 means the pointer is CUDA device memory of the current
 *     device, 0 means host memory.
 *   - A context owns all of its device memory (allocated in mb4_create,
 *     released in mb4_destroy) and its CUDA stream binding; it is not
 *     thread-safe.  Calls are asynchronous with respect to the host only where
 *     stated; every call that returns data synchronises the context's stream.
 *   - Arrays of S = nx*ny doubles are row-major, k = y*nx + x.  Stage arrays
 *     hold 3*S doubles, stage i (i = 1..3) at offset (i-1)*S.
 */
#ifndef MB4_H
#define MB4_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define MB4_OK                        0
#define MB4_ERR_INVALID_ARG          -1  /* a size, pointer or option is out of range            */
#define MB4_ERR_OUT_OF_MEMORY        -2  /* cudaMalloc failed                                     */
#define MB4_ERR_CUDA                 -3  /* any other CUDA runtime error (no GPU, launch failure) */
#define MB4_ERR_NEWTON_NOT_CONVERGED -4  /* ||r||_inf still above tolerance after newton_max
                                            iterations (Sec. 2.2: decrease h and redo)          */
#define MB4_ERR_KRYLOV_BREAKDOWN     -5  /* reserved: not returned by this build (the least squares
                                            truncates a numerically dependent Krylov basis)      */
#define MB4_ERR_NONFINITE            -6  /* NaN or Inf met in a Newton update                     */
#define MB4_ERR_TIMEOUT              -7  /* a bounded device-side wait ran out (the persistent
                                            step's grid barriers, option wait_limit)            */
#define MB4_ERR_ADMISSION_REJECTED   -8  /* a batch slot or memory budget is exhausted            */

/* ---- precision modes --------------------------------------------------- */
#define MB4_FP64   0   /* every step of the path in FP64                                        */
#define MB4_MIXED  1   /* shifted-system Krylov solves in FP32; residual, state, update and the
                          energy/norm reductions in FP64 (simplified Newton refines the result) */

typedef struct mb4_ctx mb4_ctx;   /* opaque */

/* Grid and kinetic operator (eq. Kdefinition, generalised; see above). nx, ny >= 3. */
typedef struct {
    int nx, ny;
    double tx, ty;     /* hoppings along x and y                           */
    double onsite;     /* diagonal of K                                    */
} mb4_grid;

/* External potential V: S doubles (diagonal of V, Sec. 2.1). Copied at create. */
typedef struct {
    const double* v;
    int on_device;
} mb4_potential;

/* Nonlinearity: chi = -gamma of eq. (dNLS); Table 2 of the paper calls it eps. */
typedef struct {
    double chi;
} mb4_nonlinearity;

typedef struct {
    double newton_rtol;  /* stop when ||r^l||_inf <= newton_rtol * ||u0||_inf (Algorithm 1's
                            test on the Newton update, made relative); default 1e-13           */
    int    newton_max;   /* Newton iteration cap per step, then MB4_ERR_NEWTON_NOT_CONVERGED;
                            default 30                                                          */
    int    krylov_s;     /* Krylov subspace dimension of the one s-step GMRES cycle per Newton
                            iteration, 1..MB4_MAX_KRYLOV_S; 0 = default: 4, or 5 when
                            newton_predict > 0                                                  */
    int    precision;    /* MB4_FP64 or MB4_MIXED; default MB4_FP64                            */
    double alpha1;       /* eq. (Adefinition); must be < -300*0.7770503941; default -712.5    */
    double c1, c2;       /* interior Lagrange nodes, 0 < c1 < c2 < 1; c3 = 1; default 1/3, 2/3 */
    void*  stream;       /* cudaStream_t to run on; NULL = the legacy default stream            */
    int    use_graph;    /* 1 (default): each step is one CUDA-graph launch whose Newton loop is
                            a device-side conditional WHILE node; 0: host-driven Newton loop    */
    double newton_predict; /* 0 (default): only the test above.  > 0: also stop after iteration
                            l >= 1 when the predicted remaining error theta/(1-theta)*||r^l||_inf,
                            theta = ||r^l||/||r^(l-1)|| < 1, is <= newton_predict*||u0||_inf
                            (Hairer-Wanner's stopping test for simplified Newton, Solving ODEs II
                            Sec. IV.8); the iterate is then accurate to that bound, so a value at
                            the rounding level (1e-16) skips only an iteration that changes U by
                            less than rounding                                                */
    int    overlap_launches; /* 1 (default): the kernels inside the Newton loop use programmatic
                            dependent launch, so each one's blocks are resident while its
                            predecessor drains (they wait for its completion before reading
                            its results; same arithmetic, same results); 0: plain launches    */
    int    newton_start; /* 0: every step starts at U^0 = e3 (x) u0 (Algorithm 1).
                            1..MB4_MAX_NEWTON_START: start from the previous steps' converged
                            stage increments U - e3 (x) u0, extrapolated in time with a
                            polynomial through the last newton_start of them (fewer steps of
                            history just after mb4_create / set_state use fewer).  The Newton
                            loop and its stopping test are unchanged, so the step solves the
                            same equations to the same tolerance; only the start moves.  Not
                            in the paper.  Keeps newton_start x 3 extra complex planes.
                            Default 2 (linear extrapolation): at 512x512, h = 0.005 it takes
                            the loop from 4 iterations to 3.                                  */
    int    newton_start_adaptive; /* with newton_start > 0: 1 (default) = each instance takes,
                            step by step, whichever of the two starts (U^0 = e3 (x) u0, or the
                            extrapolation) its recent steps show to be cheaper -- Newton
                            iterations taken, plus one residual evaluation that only the
                            extrapolated start needs -- and tries the other start every 32
                            steps; the choice depends only on iteration counts, so runs repeat
                            bit for bit.  0 = always extrapolate once history exists.        */
    int    autotune;     /* 1 (default): at create, time the one-site-per-thread kernels
                            (residual, Krylov basis, update; set-up and accept follow the
                            residual) with 64, 128 and 256 threads per block, and in mixed
                            mode the matrix-powers kernel in each form of option
                            powers_tile, on the context's own buffers, and keep
                            the fastest (the default unless another is faster by more than
                            5%); the choice is cached per device, precision, grid, batch size
                            and s.  Every choice gives the same results bit for bit.  0: 128
                            threads and the 32 x 16 tile everywhere.                          */
    int    site_threads; /* 0 (default): as autotune says.  64, 128 or 256: that many threads per
                            block for every per-site kernel, no tuning.                       */
    int    precondition; /* 0 (default): the shifted solves use the monomial Krylov basis of J.
                            1: right-precondition each shifted system with the inverse of its
                            constant-coefficient part, I + i h lam_i (K + mean(onsite + V)),
                            applied by 2D FFTs (hand-written mixed-radix; a side with a large
                            prime factor p costs O(p) per site and pass; nx, ny <=
                            MB4_MAX_PRECOND_SIDE).  For stiff kinetic terms such as
                            the paper's Laplacian (h ||K|| ~ 10 on its 70 x 70 grid, Sec. 3),
                            where the plain basis cannot reduce the residual in s vectors.
                            The root of each step is the same.                                */
    int    site_chi;     /* 0 (default): chi is one value per context (per instance in a batch).
                            1: chi is a per-site field (the m-site model of the paper's
                            appendix, U_I = -(1/2) sum_i gamma_i n_i^2), set with
                            mb4_set_chi_field / mb4_batch_set_chi_field and initialised to
                            the scalar chi; costs S more doubles per instance.                */
    int    persistent;   /* 0 (default): each step is the CUDA graph described under use_graph
                            (one launch per phase of the Newton loop).  1: each step is ONE
                            persistent cooperative kernel -- set-up and the whole Newton loop,
                            its phases separated by grid barriers -- followed by the accept
                            launch: no kernel boundary inside a step.  Same arithmetic, same
                            results bit for bit.  Grid problems (mb4_create, mb4_batch_create)
                            without the preconditioner, krylov_s 4 or 5; else
                            MB4_ERR_INVALID_ARG at create.                                     */
    int    powers_tile;  /* mixed mode, matrix-powers basis: 0 (default) = the tuner's choice
                            (32 x 16 when autotune = 0); 1, 2, 3, 4 = a tile of 32 x 16,
                            32 x 32, 64 x 16 or 32 x 8 sites; 5, 6 = 32 x 16 or 64 x 16 with
                            each warp's band of rows kept in registers (fewer shared-memory
                            reads); 7, 8 = 32 x 16 or 64 x 16 building the three systems one
                            after the other (a third of the shared memory per block); 9, 10 =
                            one warp per tile in registers, (32 - 2 krylov_s) x 4 or x 8
                            sites (neighbours by shuffles, no shared memory); 11, 12 = one
                            warp walking down a strip of (32 - 2 krylov_s) x 8 or x 16 sites,
                            three rows per level in registers; 13, 14 = the same strips with
                            the rows copied ahead through shared memory (cp.async); 2..14
                            need krylov_s <= 6; 15 = no tiles: one stencil launch per level.
                            Every form gives the same basis bit for bit.                      */
    long long wait_limit; /* persistent = 1: polls (each followed by a short sleep) that a
                            grid-barrier wait makes before it gives up; the step then fails
                            with MB4_ERR_TIMEOUT and the state stays at the last accepted step.
                            Default 1 << 22 (a fraction of a second; a healthy wait takes
                            microseconds).  0 gives up at the first poll (for tests).         */
} mb4_options;

#define MB4_MAX_PRECOND_SIDE 1024

#define MB4_MAX_NEWTON_START 3

#define MB4_MAX_KRYLOV_S 10

typedef struct {
    long long steps_done;         /* steps accepted by this call                               */
    long long newton_iters_total; /* Newton iterations over those steps                        */
    int       newton_iters_last;  /* Newton iterations of the last step attempted              */
    double    last_update_inf;    /* ||r^l||_inf of the last Newton iteration                  */
    double    u0_inf;             /* ||u0||_inf of the last step attempted                     */
    double    update_hist[8];     /* ||r^l||_inf, l = 0..7, of the last step attempted (0 if not run) */
} mb4_stats;

/* Fill *opt with the defaults listed above.  Never fails for a non-NULL pointer. */
int mb4_default_options(mb4_options* opt);

/* Create a context on the current CUDA device: validates the arguments,
 * computes the MB4 constants (E, E_i0, Lambda, T, T^-1 -- the set-up of Algorithm 1,
 * Sec. 2.2 -- and a 6-node Gauss-Legendre rule that integrates the degree-11
 * stage integrand of eq. (fIu2) exactly), allocates every device buffer and,
 * with use_graph, builds the step graph.  h may be negative (MB4 is symmetric).
 * The state starts at zero; set it with mb4_set_state.  opt may be NULL. */
int mb4_create(const mb4_grid* grid, const mb4_potential* pot, const mb4_nonlinearity* nl,
               double h, const mb4_options* opt, mb4_ctx** out);

/* A general kinetic matrix in place of the grid stencil: the m-site model of the
 * paper's appendix, where K_kj is the transfer between neighbouring sites (molecules).
 * K = onsite * I + T with T Hermitian (Sec. 2.1 asks only that K be Hermitian), at most
 * max_degree nonzeros per row, given row-major: nbr[k * max_degree + e] is a neighbour of
 * site k (or -1 for an unused slot), t[k * max_degree + e] the real part of the matching
 * K_kj and t_im[k * max_degree + e] its imaginary part (complex transfer integrals, e.g.
 * Peierls phases; t_im = NULL for a real symmetric T).  All arrays are host memory,
 * copied. */
#define MB4_MAX_DEGREE 16
typedef struct {
    int S;                /* sites, >= 1                                              */
    int max_degree;       /* 1..MB4_MAX_DEGREE                                        */
    const int* nbr;       /* S * max_degree, values in -1..S-1, no self links          */
    const double* t;      /* S * max_degree, finite; t(k,j) = t(j,k)                   */
    double onsite;        /* diagonal of K (V adds to it)                             */
    const double* t_im;   /* NULL, or S * max_degree, finite; t_im(k,j) = -t_im(j,k),
                             so that K_jk = conj(K_kj) (Hermitian)                    */
} mb4_sparse_kinetic;

/* mb4_create for a general kinetic matrix (one instance).  Rejects a T that is not
 * Hermitian (bit for bit: t(j,k) == t(k,j) and t_im(j,k) == -t_im(k,j)), out-of-range or
 * self-linked neighbours, and precondition = 1 (the spectral preconditioner needs the
 * grid).  With a complex T the state, stages and Krylov vectors are unchanged in form;
 * the kinetic term is a complex sparse product, and J's kinetic block is the real form
 * of -i K (eq. JL with K complex).  The FP32 path builds its Krylov basis one level per
 * launch (no matrix-powers tiles).  Every other entry point of a context applies. */
int mb4_create_sparse(const mb4_sparse_kinetic* K, const mb4_potential* pot, const mb4_nonlinearity* nl,
                      double h, const mb4_options* opt, mb4_ctx** out);

void mb4_destroy(mb4_ctx* ctx);

/* Copy psi = re + i im (S doubles each) into the context's state.  If any bit of
 * the state changes, the history that newton_start extrapolates is dropped. */
int mb4_set_state(mb4_ctx* ctx, const double* re, const double* im, int on_device);

/* Copy the state out (S doubles each).  Synchronises the context's stream. */
int mb4_get_state(const mb4_ctx* ctx, double* re, double* im, int on_device);

/* Copy out the converged stage values U_c1, U_c2, U_c3 (eq. Lagrange) of the last
 * accepted step, 3*S doubles each (untransformed, i.e. T applied).  Synchronises. */
int mb4_get_stages(const mb4_ctx* ctx, double* re3, double* im3, int on_device);

/* Advance nsteps MB4 steps (Algorithm 1's time loop).  On success returns MB4_OK.
 * On a Newton failure (Sec. 2.2, last paragraph) or a non-finite update the
 * state stays at the last accepted step and the code is returned; stats
 * (nullable) reports what was done.  Synchronises the context's stream. */
int mb4_step(mb4_ctx* ctx, int nsteps, mb4_stats* stats);

/* Enqueues nsteps MB4 steps on the context's stream and returns at once: no
 * host synchronisation, no read-back.  Several calls queue back to back with any
 * other work on the stream.  A step that fails stops the context where mb4_step
 * would; the queued steps after it do nothing.  Not part of the paper's method:
 * the asynchronous form of mb4_step for callers that overlap their own work. */
int mb4_step_async(mb4_ctx* ctx, int nsteps);

/* Waits for the context's queued steps.  stats (nullable) covers every step
 * since the previous mb4_wait / mb4_step; returns the code of a failed step (and
 * then clears it, so that later steps start from the last accepted state). */
int mb4_wait(mb4_ctx* ctx, mb4_stats* stats);

/* Kernel classes reported by mb4_step_profiled. */
#define MB4_K_SETUP        0   /* u0, (K+V)u0, J coefficients, first right-hand side          */
#define MB4_K_RESIDUAL     1   /* stage residual Phi (FP64)                                    */
#define MB4_K_MATVEC       2   /* Krylov basis v_{a+1} = (J/theta) v_a, three systems (one
                                  launch per level; the FP32 grid basis is one matrix-powers
                                  launch for all s levels)                                      */
#define MB4_K_GRAM         3   /* Gram matrix, its fixed-order reduction and least squares     */
#define MB4_K_UPDATE       4   /* Newton update Ubar += rbar, ||r||_inf, Newton loop test      */
#define MB4_K_ACCEPT       5   /* u1 = U_c3                                                    */
#define MB4_K_COUNT        6

/* mb4_step with a host-driven Newton loop and a CUDA event pair around every
 * kernel launch, for profiling.  Same arithmetic and results as mb4_step (bit
 * for bit).  Adds to ms[MB4_K_COUNT] the summed device time of each kernel
 * class, to launches[MB4_K_COUNT] its launch count and to sites[MB4_K_COUNT] the
 * sites its launches computed (all three nullable): an instance that has
 * converged, or the first residual of a step that starts at U^0 = e3 (x) u0
 * (whose right-hand side the set-up wrote), is skipped by a launch and not
 * counted, so sites / time is the rate of the work actually done.  The status
 * is read back between launches. */
int mb4_step_profiled(mb4_ctx* ctx, int nsteps, mb4_stats* stats, double* ms, long long* launches,
                      double* sites);

/* Per-site nonlinearity chi_k = -gamma_k (S doubles, finite), for a context created
 * with site_chi = 1 (else MB4_ERR_INVALID_ARG).  The energy becomes
 * H = psi^H (K+V) psi + (1/2) sum_k chi_k |psi_k|^4 and the step its Hamiltonian flow;
 * the history of newton_start is dropped.  Synchronises. */
int mb4_set_chi_field(mb4_ctx* ctx, const double* chi, int on_device);

/* Launch shape of the context's per-site kernels, shape8[8]: threads per block of
 * {set-up and accept, residual, Krylov basis (FP64 stencil), update}, then blocks per
 * instance of the same four (one site per thread). */
int mb4_get_launch_shape(const mb4_ctx* ctx, int* shape8);

/* Energy H = U_K + U_E + U_nl of the current state (Sec. 2.1: U_K = u^H K u,
 * U_E = u^H V u, U_nl = -(gamma/2)||n||^2 = (chi/2) sum |u|^4), with compensated
 * FP64 sums in a fixed order.  parts3 (nullable) receives U_K, U_E, U_nl. */
int mb4_energy(const mb4_ctx* ctx, double* H, double* parts3);

/* Norm sum |u|^2 (the total probability of Sec. 3.1), compensated FP64. */
int mb4_norm(const mb4_ctx* ctx, double* norm2);

/* All observables in one sweep: out[6] = {H, U_K, U_E, U_nl, sum|u|^2, sum|u|^4}
 * (the last is the participation ratio of Sec. 3.2). */
int mb4_observables(const mb4_ctx* ctx, double* out6);

/* Stage residual Phi(U) of eq. (Phidefinition) evaluated by the step's FP64
 * residual kernel for a given u0 (S complex) and stages U (3*S complex), all
 * untransformed; writes Phi (3*S complex).  For testing the kernel on its own;
 * it overwrites the context's state with u0 and its stage buffers.  Synchronises. */
int mb4_residual(mb4_ctx* ctx, const double* u0_re, const double* u0_im,
                 const double* U_re3, const double* U_im3,
                 double* phi_re3, double* phi_im3, int on_device);

/* One s-step GMRES cycle on each decoupled system (I - h lambda_i J) x_i = b_i
 * (eq. MB4_5), J frozen at u0 (eq. JL, eq. JR), in the context's precision.
 * b and x are in the eigenbasis of E (3*S complex each).  Overwrites the
 * context's state with u0.  Synchronises. */
int mb4_solve_shifted(mb4_ctx* ctx, const double* u0_re, const double* u0_im,
                      const double* b_re3, const double* b_im3,
                      double* x_re3, double* x_im3, int on_device);

/* ---- batches: many independent instances of one grid shape per launch -----
 * A batch holds `batch` instances that share the grid (nx, ny, tx, ty, onsite),
 * h and the options; each has its own potential, nonlinearity chi, state and
 * Newton status.  Every kernel of a step covers all instances in one launch;
 * an instance whose Newton iteration has converged (or failed) is masked while
 * the others continue, so one slow or failing instance neither blocks nor
 * corrupts the rest.  Instance-major arrays: instance b's S values start at
 * offset b*S.  A single context (mb4_create) is a batch of one. */
typedef struct mb4_batch mb4_batch;

/* Create a batch.  pot->v holds batch*S doubles (instance-major); chi is a host
 * array of batch values.  All instances start enabled with a zero state. */
int mb4_batch_create(const mb4_grid* grid, int batch, const mb4_potential* pot, const double* chi, double h,
                     const mb4_options* opt, mb4_batch** out);

void mb4_batch_destroy(mb4_batch* b);

/* State of one instance (instance >= 0: S doubles each) or of all of them
 * (instance = -1: batch*S doubles each).  As mb4_set_state, per instance. */
int mb4_batch_set_state(mb4_batch* b, int instance, const double* re, const double* im, int on_device);
int mb4_batch_get_state(const mb4_batch* b, int instance, double* re, double* im, int on_device);

/* Reuse one slot: new potential (S doubles), chi and state; clears the
 * instance's error and counters and enables it.  MB4_ERR_INVALID_ARG for a
 * non-finite input and, in an FP64 batch without preconditioning on a grid with
 * tx != 0 (whose Krylov basis is scaled by tx), for a potential whose Gershgorin
 * bound max|onsite + V| + 2|tx| + 2|ty| exceeds 4096 |tx|. */
int mb4_batch_load(mb4_batch* b, int instance, const double* v, double chi, const double* re, const double* im,
                   int on_device);

/* Enable (1) or disable (0) stepping of one instance (instance = -1: all); a
 * disabled instance keeps its state and takes no part in later steps. */
int mb4_batch_enable(mb4_batch* b, int instance, int enabled);

/* Enqueue nsteps MB4 steps for every enabled instance without an error, on the
 * batch's stream, without waiting.  Counters restart at zero. */
int mb4_batch_step_async(mb4_batch* b, int nsteps);

/* Wait for the batch's stream; per-instance stats (`batch` entries) and status
 * codes (MB4_OK or the instance's error) for the steps enqueued since the last
 * mb4_batch_step_async.  Either pointer may be NULL.  Returns MB4_OK if every
 * enabled instance is error-free, else the first instance error. */
int mb4_batch_wait(mb4_batch* b, mb4_stats* stats, int* status);

/* mb4_batch_step_async followed by mb4_batch_wait. */
int mb4_batch_step(mb4_batch* b, int nsteps, mb4_stats* stats, int* status);

/* Observables of every instance: out[b*6 + k], k as in mb4_observables. */
int mb4_batch_observables(const mb4_batch* b, double* out);

/* Clear the error of every instance (the state is the last accepted one). */
int mb4_batch_clear_errors(mb4_batch* b);

/* As mb4_set_chi_field, for one instance of a batch (instance >= 0). */
int mb4_batch_set_chi_field(mb4_batch* b, int instance, const double* chi, int on_device);

/* As mb4_get_launch_shape, for a batch. */
int mb4_batch_get_launch_shape(const mb4_batch* b, int* shape8);

/* The tile (*tx x *ty sites) of the FP32 matrix-powers Krylov basis that the tuner chose
 * for this batch or context (cast an mb4_ctx* to mb4_batch*: a context is a batch of one),
 * or 0 x 0 where that kernel is not used (FP64 mode, the preconditioner, a general K, or a
 * basis built by one stencil launch per level, option powers_tile = 15 or the tuner's choice).
 * Every tile gives the same basis bit for bit. */
int mb4_batch_get_tile_shape(const mb4_batch* b, int* tx, int* ty);

/* As mb4_step_profiled, for a batch: nsteps steps of every enabled instance with a
 * host-driven Newton loop and an event pair around every launch; adds the summed
 * device time of each kernel class to ms[MB4_K_COUNT], its launch count to
 * launches[MB4_K_COUNT] and the sites computed to sites[MB4_K_COUNT] (all
 * nullable); stats and status as mb4_batch_wait. */
int mb4_batch_step_profiled(mb4_batch* b, int nsteps, mb4_stats* stats, int* status, double* ms,
                            long long* launches, double* sites);

/* Device bytes a batch of this shape and options would allocate (for admission). */
long long mb4_batch_bytes(int nx, int ny, int batch, const mb4_options* opt);

/* ---- serving: continuous batching of simulation requests ------------------
 * A server keeps one batch per shape class (nx, ny, tx, ty, onsite, h), each on
 * its own CUDA stream, inside an HBM budget.  Requests carry their own grid,
 * potential, chi, initial state, step count and arrival time.  The serving loop
 * admits every request that has arrived into a free slot of its class (creating
 * the class's batch when the budget allows, and releasing idle batches when it
 * does not), advances all classes concurrently (their kernels overlap on the
 * GPU), and retires each request after exactly its step count, freeing the slot
 * for the next.  States stay on the GPU from admission to completion.  Latency
 * is completion time minus arrival time on the server's clock. */
typedef struct mb4_server mb4_server;

typedef struct {
    mb4_grid grid;
    double h;
    double chi;
    int nsteps;               /* MB4 steps to run (>= 1)                                        */
    const double* v;          /* host, S doubles, copied at submit                             */
    const double* re;         /* host, S doubles: initial state, copied at submit              */
    const double* im;
    double arrival;           /* seconds on the server clock; not admitted before this time    */
} mb4_request;

typedef struct {
    int status;               /* MB4_OK, or the error that stopped the request                  */
    int done;                 /* 1 once completed (or failed)                                   */
    long long steps_done;
    long long newton_iters_total;
    double arrival, admitted, completed;   /* server clock, seconds                           */
    double energy_start, energy_end;       /* H at admission and at completion               */
} mb4_result;

/* hbm_budget_bytes: device memory the server's batches may hold together;
 * max_slots: instances per class batch, at most; keep_states: 1 to keep each
 * final state for mb4_server_result.  opt applies to every batch, except that the
 * server's batches skip the launch-shape tuner (its timings would run behind the
 * other classes' kernels and delay the admitted request). */
int mb4_server_create(long long hbm_budget_bytes, int max_slots, int keep_states, const mb4_options* opt,
                      mb4_server** out);
void mb4_server_destroy(mb4_server* s);

/* Queue a request; *id receives its index (0, 1, ...).  MB4_ERR_ADMISSION_REJECTED
 * if a single instance of its class cannot fit the budget at all; MB4_ERR_INVALID_ARG
 * for a bad grid, h, chi or step count, or a non-finite v, re or im. */
int mb4_server_submit(mb4_server* s, const mb4_request* req, long long* id);

/* Run the serving loop until every submitted request is done or the server clock
 * reaches `until` seconds; *n_done (nullable) receives the number done so far.  A
 * request that its class batch refuses at admission (mb4_batch_load) is done with that
 * status and no steps; the others go on. */
int mb4_server_run(mb4_server* s, double until, long long* n_done);

/* Result of request id; re/im (nullable, S doubles each, host) receive the final
 * state when the server keeps states. */
int mb4_server_result(const mb4_server* s, long long id, mb4_result* out, double* re, double* im);

/* Seconds on the server clock (0 at creation). */
double mb4_server_clock(const mb4_server* s);

/* Host-only: the MB4 constants the library computes for (alpha1, c1, c2), c3 = 1.
 * E34: 12 doubles, row-major E[i][j], i = 1..3, j = 0..3 (j = 0 is E_i0, eq. Ei0).
 * lam3: eigenvalues of E(1:3,1:3), ascending.  T9, Tinv9: row-major 3x3.
 * gauss_x6, gauss_w6: the 6-node Gauss-Legendre rule on [0, 1].
 * Any output pointer may be NULL.  Needs no GPU. */
int mb4_constants(double alpha1, double c1, double c2, double* E34, double* lam3,
                  double* T9, double* Tinv9, double* gauss_x6, double* gauss_w6);

/* Largest grid (nx*ny sites) that mb4_observables_noalloc accepts. */
#define MB4_NOALLOC_MAX_SITES (1 << 30)

/* The six observables of mb4_observables for a state given directly as device
 * planes, for callers that cannot allocate device memory: code that runs under
 * an allocator or memory pool owning all device memory, or where a cudaMalloc
 * (and the synchronisation it may cause) is not allowed at that moment.  The
 * paper has no counterpart: this is a service entry point of the library.
 *
 * It needs no context and allocates nothing.  re, im, v (S = nx*ny doubles
 * each, row-major) and out6 (6 doubles: H, U_K, U_E, U_nl, sum|u|^2, sum|u|^4)
 * are device memory of the current device, supplied by the caller; the call
 * only enqueues two kernels on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and returns; synchronise the stream before reading out6.  Its scratch
 * is a fixed 24 KiB array of block partial sums inside the library image,
 * which every GPU that loads the library holds until the process exits.  The
 * first call on a device looks up that array's device address (once per device,
 * with the device current), so make the first call before any stream capture.
 * That address is kept for the life of the process: after a cudaDeviceReset of
 * the device (which unloads the library image from it) this entry point must not
 * be called again.  All calls share the array: calls that overlap on the GPU (different streams,
 * other host threads) race and give wrong results; serialise them.  Every call
 * overwrites the whole part of the array it reads, so no clearing is needed.
 * Returns MB4_ERR_INVALID_ARG for nx or ny < 3, nx*ny > MB4_NOALLOC_MAX_SITES
 * or a NULL pointer, MB4_ERR_CUDA if the set-up or a launch fails (judged by the
 * launches' own return codes: an error left pending by earlier work of the caller
 * is neither reported nor cleared). */
int mb4_observables_noalloc(int nx, int ny, double tx, double ty, double onsite, double chi,
                            const double* re, const double* im, const double* v, double* out6,
                            void* stream);

/* The FP64 FMA throughput of the current device, measured: independent chains of
 * dependent FP64 FMAs in every thread of a grid that fills the device, with no memory
 * traffic, timed with CUDA events; the launch is lengthened until it runs for about
 * `seconds` (0 < seconds <= 10).  *flops_per_s receives 2 x FMAs per second;
 * *elapsed_s (nullable) the duration of the timed launch.  It is the ceiling of the
 * step's FP64-bound kernels at the clock the device runs at.  Runs on the legacy
 * default stream and synchronises it.  The paper has no counterpart: a measurement
 * service of the library.  MB4_ERR_INVALID_ARG for a NULL output or seconds out of
 * range, MB4_ERR_CUDA on a launch or event failure. */
int mb4_fp64_fma_rate(double seconds, double* flops_per_s, double* elapsed_s);

const char* mb4_status_string(int status);

/* Library version, for diagnostics. */
const char* mb4_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MB4_H */
